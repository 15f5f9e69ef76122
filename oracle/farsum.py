"""Loader for the oracle's C far-sum and correction-sum routines (test
infrastructure only).

Compiles oracle/csrc/farsum.c with gcc (-O2 -fopenmp) into oracle/_build on
first use, or when the source is newer than the library.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "csrc", "farsum.c")
_LIB = os.path.join(_HERE, "_build", "liboracle_far.so")
_lib = None


def build(force: bool = False) -> str:
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c99",
                               "-ffp-contract=off", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        lib.oracle_far_sums.restype = ctypes.c_int
        lib.oracle_far_sums.argtypes = [
            ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
            ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_int64,
            ctypes.c_void_p, ctypes.c_void_p]
        lib.oracle_far_sums_src.restype = ctypes.c_int
        lib.oracle_far_sums_src.argtypes = [
            ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
            ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
            ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
            ctypes.c_void_p]
        lib.oracle_near_apply.restype = ctypes.c_int
        lib.oracle_near_apply.argtypes = [
            ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
            ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p]
        _lib = lib
    return _lib


def near_sums(geo, near_ptr, near_patch, vals, sigma, targets=None) -> np.ndarray:
    """Correction sums of all four kernels from the block CSR: [nrhs, 4, ntargets]."""
    lib = _load()
    sig = np.ascontiguousarray(np.atleast_2d(sigma), dtype=np.float64)
    nrhs = sig.shape[0]
    if targets is None:
        targets = np.arange(geo.N, dtype=np.int64)
    targets = np.ascontiguousarray(targets, dtype=np.int64)
    ptr = np.ascontiguousarray(near_ptr, dtype=np.int64)
    pl = np.ascontiguousarray(near_patch, dtype=np.int32)
    v = np.ascontiguousarray(vals, dtype=np.float64)
    if v.shape != (len(pl), 4, geo.np_) or len(ptr) != geo.N + 1:
        raise ValueError("correction arrays do not match the geometry")
    out = np.zeros((nrhs, 4, len(targets)))
    lib.oracle_near_apply(geo.N, geo.np_, ptr.ctypes.data, pl.ctypes.data, v.ctypes.data, nrhs,
                          sig.ctypes.data, len(targets), targets.ctypes.data, out.ctypes.data)
    return out


def far_sums(geo, near_ptr, near_patch, sigma, targets=None, far=None) -> np.ndarray:
    """Far sums of all four kernels: [nrhs, 4, ntargets] (kernel order S, D, S', S''+D').

    far (a geometry.FarRule) replaces the nodes as sources by the oversampled
    rule's points, with the densities interpolated to them (Section 4)."""
    lib = _load()
    if far is not None:
        sig = np.ascontiguousarray(far.densities(sigma), dtype=np.float64)
        nrhs = sig.shape[0]
        if targets is None:
            targets = np.arange(geo.N, dtype=np.int64)
        targets = np.ascontiguousarray(targets, dtype=np.int64)
        X = np.ascontiguousarray(geo.X)
        n = np.ascontiguousarray(geo.n)
        Y = np.ascontiguousarray(far.Y)
        ny = np.ascontiguousarray(far.n)
        wy = np.ascontiguousarray(far.w)
        ptr = np.ascontiguousarray(near_ptr, dtype=np.int64)
        pl = np.ascontiguousarray(near_patch, dtype=np.int32)
        out = np.zeros((nrhs, 4, len(targets)))
        rc = lib.oracle_far_sums_src(geo.N, X.ctypes.data, n.ctypes.data, ptr.ctypes.data, pl.ctypes.data,
                                     geo.npatch, Y.shape[0], far.nps, Y.ctypes.data, ny.ctypes.data,
                                     wy.ctypes.data, nrhs, sig.ctypes.data, len(targets), targets.ctypes.data,
                                     out.ctypes.data)
        if rc != 0:
            raise MemoryError("oracle far sum could not allocate its work arrays")
        return out
    sig = np.ascontiguousarray(np.atleast_2d(sigma), dtype=np.float64)
    nrhs = sig.shape[0]
    if targets is None:
        targets = np.arange(geo.N, dtype=np.int64)
    targets = np.ascontiguousarray(targets, dtype=np.int64)
    X = np.ascontiguousarray(geo.X)
    n = np.ascontiguousarray(geo.n)
    w = np.ascontiguousarray(geo.w)
    ptr = np.ascontiguousarray(near_ptr, dtype=np.int64)
    pl = np.ascontiguousarray(near_patch, dtype=np.int32)
    out = np.zeros((nrhs, 4, len(targets)))
    rc = lib.oracle_far_sums(geo.N, geo.np_, X.ctypes.data, n.ctypes.data, w.ctypes.data,
                             ptr.ctypes.data, pl.ctypes.data, nrhs, sig.ctypes.data,
                             len(targets), targets.ctypes.data, out.ctypes.data)
    if rc != 0:
        raise MemoryError("oracle far sum could not allocate its work arrays")
    return out
