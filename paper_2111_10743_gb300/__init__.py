"""Python binding of the GB300 Laplace-Beltrami layer-potential library.

Argument marshalling only: every computation runs in the CUDA library
(_build/libgblb.so, built by build.py).  The names mirror the C ABI in
include/gblb.h.  Arrays may be numpy arrays (host) or torch tensors (host or
CUDA); they must be contiguous float64 (int64 / int32 for index arrays).
Device tensors are passed by pointer; the library copies host arrays through
its own device buffers.  Importing this package fails loudly when the shared
library has not been built; there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import checkpoint as _checkpoint
from .checkpoint import CheckpointError

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libgblb.so")

LB_OK, LB_EINVAL, LB_ENOMEM, LB_ECUDA, LB_ENOTCONVERGED, LB_ETIMEOUT, LB_EGEOM, LB_ESTATE = 0, -1, -2, -3, -4, -5, -6, -7
LB_FP64, LB_FP32, LB_FP32_REFINED, LB_DF64 = 0, 1, 2, 3
LB_A1, LB_A2, LB_A3 = 1, 2, 3
LB_K_S, LB_K_D, LB_K_SP, LB_K_SPPDP = 0, 1, 2, 3
NKERNELS = 4
_STATUS = {0: "LB_OK", -1: "LB_EINVAL", -2: "LB_ENOMEM", -3: "LB_ECUDA", -4: "LB_ENOTCONVERGED",
           -5: "LB_ETIMEOUT", -6: "LB_EGEOM", -7: "LB_ESTATE"}


class lb_params(ctypes.Structure):
    _fields_ = [("eps_quad", ctypes.c_double), ("near_factor", ctypes.c_double),
                ("precision", ctypes.c_int), ("formulation", ctypes.c_int),
                ("max_iter", ctypes.c_int), ("tol", ctypes.c_double),
                ("inner_tol", ctypes.c_double), ("max_refine", ctypes.c_int),
                ("graphs", ctypes.c_int)]


class lb_solve_info(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int32), ("refinements", ctypes.c_int32),
                ("converged", ctypes.c_int32), ("applies_fp64", ctypes.c_int32),
                ("applies_fp32", ctypes.c_int32), ("nrhs", ctypes.c_int32),
                ("rel_residual", ctypes.c_double), ("removed_mean", ctypes.c_double),
                ("history", ctypes.c_double * 128), ("history_len", ctypes.c_int32),
                ("pairs", ctypes.c_int64), ("graph_iterations", ctypes.c_int32)]

    def as_dict(self):
        return {"iterations": self.iterations, "refinements": self.refinements,
                "converged": bool(self.converged), "applies_fp64": self.applies_fp64,
                "applies_fp32": self.applies_fp32, "nrhs": self.nrhs,
                "rel_residual": self.rel_residual, "removed_mean": self.removed_mean,
                "history": list(self.history[:self.history_len]), "pairs": self.pairs,
                "graph_iterations": self.graph_iterations}


class lb_geom_info(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int64), ("npatch", ctypes.c_int64), ("np", ctypes.c_int32),
                ("order", ctypes.c_int32), ("nnzb", ctypes.c_int64), ("area", ctypes.c_double),
                ("sm_count", ctypes.c_int32), ("corrections", ctypes.c_int32)]


PROF_NCAT = 16
PROF_NAMES = {0: "far32_k1", 1: "far32_kall", 2: "far32_k2", 3: "far32_k4", 4: "far64_k1", 5: "far64_kall",
              6: "far64_k2", 7: "far64_k4", 8: "epilogue_spmv", 9: "quad", 10: "fardf_k1", 11: "fardf_kall",
              12: "fardf_k2", 13: "fardf_k4", 14: "shape_grad"}


class lb_profile(ctypes.Structure):
    _fields_ = [("ms", ctypes.c_double * PROF_NCAT), ("calls", ctypes.c_int64 * PROF_NCAT),
                ("launches", ctypes.c_int64), ("pairs", ctypes.c_int64 * PROF_NCAT)]


class LBError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{_STATUS.get(code, code)}: {msg}")
        self.code = code


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(
            f"CUDA library not built: {LIB_PATH} is missing; run "
            "`python -c 'import __graft_entry__ as g; g.build()'` (needs nvcc) first")
    lib = ctypes.CDLL(LIB_PATH)
    P = ctypes.c_void_p
    sig = {
        "lb_default_params": [P], "lb_create": [P, ctypes.c_int, P], "lb_destroy": [P],
        "lb_set_params": [P, P], "lb_get_params": [P, P], "lb_set_stream": [P, P],
        "lb_upload_geometry": [P, ctypes.c_int64, ctypes.c_int, P, P, P, P, P],
        "lb_get_geometry": [P, P, P, P], "lb_geometry_info": [P, P], "lb_build_near": [P],
        "lb_build_corrections": [P], "lb_load_corrections": [P, ctypes.c_int64, P, P, P],
        "lb_get_corrections": [P, P, P, P], "lb_far_sums": [P, ctypes.c_int, ctypes.c_int, P, P],
        "lb_apply_S": [P, ctypes.c_int, P, P], "lb_apply_Sp": [P, ctypes.c_int, P, P],
        "lb_apply_D": [P, ctypes.c_int, P, P], "lb_apply_SppDp": [P, ctypes.c_int, P, P],
        "lb_apply_gradS": [P, ctypes.c_int, P, P], "lb_apply_A": [P, ctypes.c_int, P, P],
        "lb_solve_lb": [P, ctypes.c_int, P, P, P], "lb_harmonic_fields": [P, ctypes.c_int, P, P, P],
        "lb_surface_div": [P, ctypes.c_int, P, P],
        "lb_set_profiling": [P, ctypes.c_int], "lb_get_profile": [P, P], "lb_get_tuning": [P, P],
        "lb_apply_St": [P, ctypes.c_int, P, P], "lb_apply_At": [P, ctypes.c_int, P, P],
        "lb_solve_lb_adjoint": [P, ctypes.c_int, P, P, P],
        "lb_shape_gradient": [P, ctypes.c_int, P, P, P, P],
        "lb_far_sums_noalloc": [ctypes.c_int64, ctypes.c_int, P, P, P, P, P, P, P, P],
        "lb_fmm_plan_create": [ctypes.c_int64, P, ctypes.c_double, ctypes.c_int, P],
        "lb_fmm_plan_info": [P, P],
        "lb_fmm_plan_arrays": [P, P, P, P, P, P, P, P, P, P],
        "lb_fmm_plan_destroy": [P],
        "lb_debug_fail_alloc": [P, ctypes.c_int64],
        "lb_debug_set_variant": [P, ctypes.c_int, ctypes.c_int],
        "lb_set_far_rule": [P, ctypes.c_int, P, P],
        "lb_geometry_gradient": [P, ctypes.c_int, P, P, P, P, P, P],
    }
    for name, args in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = ctypes.c_int
    lib.lb_last_error.argtypes = [P]
    lib.lb_last_error.restype = ctypes.c_char_p
    return lib


_lib = _load()
lib = _lib


def default_params(**kw) -> lb_params:
    p = lb_params()
    _lib.lb_default_params(ctypes.byref(p))
    for k, v in kw.items():
        if not hasattr(p, k):
            raise TypeError(f"unknown parameter {k}")
        setattr(p, k, v)
    return p


def _ptr(a, dtype):
    """(pointer, keep-alive) for a numpy array or torch tensor."""
    if a is None:
        return None, None
    try:
        import torch
        if isinstance(a, torch.Tensor):
            want = {np.float64: torch.float64, np.int64: torch.int64, np.int32: torch.int32}[dtype]
            if a.dtype != want or not a.is_contiguous():
                raise TypeError(f"tensor must be contiguous {want}")
            return ctypes.c_void_p(a.data_ptr()), a
    except ImportError:  # pragma: no cover
        pass
    arr = np.ascontiguousarray(a, dtype=dtype)
    return ctypes.c_void_p(arr.ctypes.data), arr


def _out(a, dtype, shape):
    if a is None:
        arr = np.empty(shape, dtype=dtype)
        return ctypes.c_void_p(arr.ctypes.data), arr
    p, keep = _ptr(a, dtype)
    if isinstance(keep, np.ndarray) and keep is not a:
        raise TypeError("output array must be contiguous of the right dtype")
    return p, keep


class Context:
    """One library context on one CUDA device (lb_create / lb_destroy)."""

    def __init__(self, device: int = 0, params: lb_params | None = None, stream=None):
        self._h = ctypes.c_void_p()
        rc = _lib.lb_create(ctypes.byref(self._h), int(device),
                            ctypes.byref(params) if params is not None else None)
        if rc != LB_OK:
            raise LBError(rc, _lib.lb_last_error(None).decode())
        self.N = 0
        if stream is not None:
            self.set_stream(stream)

    def _check(self, rc, allow=()):
        if rc != LB_OK and rc not in allow:
            raise LBError(rc, _lib.lb_last_error(self._h).decode())
        return rc

    def close(self):
        if self._h:
            _lib.lb_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # --- configuration -------------------------------------------------
    def set_params(self, p: lb_params):
        self._check(_lib.lb_set_params(self._h, ctypes.byref(p)))

    def get_params(self) -> lb_params:
        p = lb_params()
        self._check(_lib.lb_get_params(self._h, ctypes.byref(p)))
        return p

    def set_stream(self, stream):
        """stream: a torch.cuda.Stream, an int handle, or None for the default."""
        h = getattr(stream, "cuda_stream", stream)
        self._check(_lib.lb_set_stream(self._h, ctypes.c_void_p(h or 0)))

    def debug_fail_alloc(self, after: int = 0):
        """Make the device allocation `after` allocations from now fail as out
        of memory (test hook; after < 0 disarms)."""
        self._check(_lib.lb_debug_fail_alloc(self._h, int(after)))

    def debug_set_variant(self, kind: int, variant: int):
        """Use launch variant `variant` for pass `kind` on this surface
        instead of the timed choice (test hook).  kind: float32 0 K1, 1 all
        four kernels, 2 A3 pass 2, 3 A2 pass 2; double-float symmetric 4 K1,
        5 A3 pass 2."""
        self._check(_lib.lb_debug_set_variant(self._h, int(kind), int(variant)))

    def set_profiling(self, on: bool = True):
        self._check(_lib.lb_set_profiling(self._h, 1 if on else 0))

    def get_tuning(self) -> dict:
        """Launch shapes picked by the batched passes' tuner (-1: not tuned)."""
        a = (ctypes.c_int * 14)()
        self._check(_lib.lb_get_tuning(self._h, a))
        names = {0: "128x64", 1: "128x128", 2: "256x64", -1: None}
        out = {}
        for p, pn in enumerate(("far32", "fardf")):
            for k, kn in enumerate(("k1", "k2")):
                for r, rn in enumerate(("rc4", "rc8")):
                    out[f"{pn}_{kn}_{rn}"] = names[a[p * 4 + k * 2 + r]]
        sym = ("symmetric", "symmetric_packed", "symmetric_nt2", "symmetric_packed_nt2")
        pk = ("packed_nt4", "packed_nt4_3blocks", "packed_nt2") + sym
        single = {0: ("scalar_nt4", "packed_nt4", "scalar_nt8") + sym, 1: pk, 2: pk, 3: pk}
        for kind, kn in enumerate(("k1", "kall", "k2", "k4")):
            v = a[8 + kind]
            out[f"far32_single_{kn}"] = single[kind][v] if v >= 0 else None
        for p, kn in enumerate(("k1", "k2")):
            v = a[12 + p]
            out[f"fardf_sym_{kn}"] = ("nt1", "nt2")[v] if v >= 0 else None
        return out

    def get_profile(self) -> dict:
        p = lb_profile()
        self._check(_lib.lb_get_profile(self._h, ctypes.byref(p)))
        out = {"launches": p.launches}
        for k, name in PROF_NAMES.items():
            if p.calls[k]:
                out[name] = {"ms": p.ms[k], "calls": p.calls[k], "pairs": p.pairs[k]}
        return out

    # --- geometry ------------------------------------------------------
    def upload_geometry(self, npatch, order, ref_uv, ref_w, X, Xu, Xv):
        args = [_ptr(a, np.float64) for a in (ref_uv, ref_w, X, Xu, Xv)]
        self._check(_lib.lb_upload_geometry(self._h, int(npatch), int(order), *[a[0] for a in args]))
        self.N = self.info()["N"]
        host = [a.detach().cpu().numpy() if hasattr(a, "detach") else a for a in (ref_uv, ref_w, X, Xu, Xv)]
        self._digest = _checkpoint.geometry_digest(npatch, order, *host)
        # host copies of the uploaded surface, for check_geometry
        self._geom_host = {k: np.array(v, dtype=np.float64).reshape(-1, 3)
                           for k, v in zip(("X", "Xu", "Xv"), host[2:])}

    def check_geometry(self, **arrays):
        """Raise ValueError unless every given array (X=, Xu=, Xv=; numpy or
        torch, host or device) equals the uploaded one exactly."""
        if getattr(self, "_geom_host", None) is None:
            raise LBError(LB_ESTATE, "no geometry uploaded")
        for k, a in arrays.items():
            if a is None:
                continue
            h = a.detach().cpu().numpy() if hasattr(a, "detach") else np.asarray(a)
            ref = self._geom_host[k]
            if h.size != ref.size or not np.array_equal(h.reshape(-1, 3), ref):
                raise ValueError(f"{k} differs from the uploaded surface: upload it (and rebuild or load the "
                                 f"corrections) before solving")

    def upload_surface(self, surf):
        """Convenience: upload a workloads.surfaces.Surface-like object."""
        self.upload_geometry(surf.npatch, surf.order, surf.uv, surf.wref, surf.X, surf.Xu, surf.Xv)

    def info(self) -> dict:
        g = lb_geom_info()
        self._check(_lib.lb_geometry_info(self._h, ctypes.byref(g)))
        return {f: getattr(g, f) for f, _ in g._fields_}

    def get_geometry(self):
        N = self.N
        n, w, H = np.empty((N, 3)), np.empty(N), np.empty(N)
        self._check(_lib.lb_get_geometry(self._h, ctypes.c_void_p(n.ctypes.data), ctypes.c_void_p(w.ctypes.data),
                                         ctypes.c_void_p(H.ctypes.data)))
        return n, w, H

    def set_far_rule(self, order: int = 0, uv=None, w=None):
        """Oversampled far-field rule (lb_set_far_rule): a node rule of total
        degree `order` on T0 (uv [nps, 2], w [nps]); order 0 restores the
        node rule."""
        if order == 0:
            self._check(_lib.lb_set_far_rule(self._h, 0, None, None))
            return
        a, b = _ptr(uv, np.float64), _ptr(w, np.float64)
        self._check(_lib.lb_set_far_rule(self._h, int(order), a[0], b[0]))

    def build_near(self):
        self._check(_lib.lb_build_near(self._h))

    def build_corrections(self):
        return self._check(_lib.lb_build_corrections(self._h), allow=(LB_EGEOM,))

    def load_corrections(self, row_ptr, patch, vals):
        """Near lists and correction blocks computed elsewhere: row_ptr [N+1]
        int64, patch [nnzb] int32 (ascending per row), vals [nnzb, 4, n_p]
        float64.  Host arrays are checked here; the library checks the list
        structure again on the device (LB_EINVAL on any violation)."""
        info = self.info()
        nnzb = int(np.asarray(patch).shape[0]) if not hasattr(patch, "shape") else int(patch.shape[0])
        if tuple(row_ptr.shape) != (info["N"] + 1,) or len(patch.shape) != 1 or \
                tuple(vals.shape) != (nnzb, NKERNELS, info["np"]):
            raise ValueError(f"correction arrays must be row_ptr [{info['N'] + 1}], patch [nnzb], "
                             f"vals [nnzb, {NKERNELS}, {info['np']}]")
        if all(isinstance(a, np.ndarray) for a in (row_ptr, patch, vals)):
            try:
                _checkpoint._check_csr(row_ptr, patch, vals, info["N"], info["npatch"], info["np"])
            except CheckpointError as e:
                raise LBError(LB_EINVAL, str(e)) from None
        a = _ptr(row_ptr, np.int64)
        b = _ptr(patch, np.int32)
        c = _ptr(vals, np.float64)
        self._check(_lib.lb_load_corrections(self._h, nnzb, a[0], b[0], c[0]))

    def get_corrections(self, with_vals=True):
        info = self.info()
        N, nnzb, npn = info["N"], info["nnzb"], info["np"]
        rp = np.empty(N + 1, dtype=np.int64)
        pa = np.empty(nnzb, dtype=np.int32)
        vals = np.empty((nnzb, NKERNELS, npn)) if with_vals else None
        self._check(_lib.lb_get_corrections(self._h, ctypes.c_void_p(rp.ctypes.data),
                                            ctypes.c_void_p(pa.ctypes.data),
                                            ctypes.c_void_p(vals.ctypes.data) if with_vals else None))
        return rp, pa, vals

    def geometry_digest(self) -> str:
        """SHA-256 of the geometry inputs, taken when they were uploaded."""
        if getattr(self, "_digest", None) is None:
            raise LBError(LB_EINVAL, "no geometry uploaded")
        return self._digest

    def save_corrections(self, path):
        """Write the corrections with the geometry digest and parameters (.npz)."""
        p = self.get_params()
        rp, pa, vals = self.get_corrections()
        _checkpoint.save(path, self.geometry_digest(), p.near_factor, p.eps_quad, rp, pa, vals)

    def load_corrections_file(self, path):
        """Load corrections saved for this geometry and these parameters,
        in place of build_corrections; CheckpointError on any mismatch."""
        p = self.get_params()
        rp, pa, vals = _checkpoint.load(path, self.geometry_digest(), p.near_factor, p.eps_quad)
        self.load_corrections(rp, pa, vals)

    # --- applies -------------------------------------------------------
    def _nrhs(self, x, per=1):
        n = int(np.prod(x.shape)) // (self.N * per)
        if n * self.N * per != int(np.prod(x.shape)):
            raise ValueError("array size is not a multiple of N")
        return n

    def far_sums(self, sigma, precision=LB_FP64, out=None):
        nrhs = self._nrhs(sigma)
        p, keep = _ptr(sigma, np.float64)
        o, res = _out(out, np.float64, (nrhs, NKERNELS, self.N))
        self._check(_lib.lb_far_sums(self._h, int(precision), nrhs, p, o))
        return res

    def _apply(self, fn, sigma, out, per_out=1):
        nrhs = self._nrhs(sigma)
        p, keep = _ptr(sigma, np.float64)
        shape = (nrhs, self.N) if per_out == 1 else (nrhs, self.N, per_out)
        o, res = _out(out, np.float64, shape)
        self._check(fn(self._h, nrhs, p, o))
        return res

    def apply_S(self, sigma, out=None):
        return self._apply(_lib.lb_apply_S, sigma, out)

    def apply_Sp(self, sigma, out=None):
        return self._apply(_lib.lb_apply_Sp, sigma, out)

    def apply_D(self, sigma, out=None):
        return self._apply(_lib.lb_apply_D, sigma, out)

    def apply_SppDp(self, sigma, out=None):
        return self._apply(_lib.lb_apply_SppDp, sigma, out)

    def apply_gradS(self, sigma, out=None):
        return self._apply(_lib.lb_apply_gradS, sigma, out, per_out=3)

    def apply_A(self, tau, out=None):
        return self._apply(_lib.lb_apply_A, tau, out)

    def surface_div(self, F, out=None):
        nrhs = self._nrhs(F, 3)
        p, keep = _ptr(F, np.float64)
        o, res = _out(out, np.float64, (nrhs, self.N))
        self._check(_lib.lb_surface_div(self._h, nrhs, p, o))
        return res

    # --- solves --------------------------------------------------------
    def solve_lb(self, f, out=None, allow_unconverged=False):
        nrhs = self._nrhs(f)
        p, keep = _ptr(f, np.float64)
        o, res = _out(out, np.float64, (nrhs, self.N))
        info = lb_solve_info()
        self._check(_lib.lb_solve_lb(self._h, nrhs, p, o, ctypes.byref(info)),
                    allow=(LB_ENOTCONVERGED,) if allow_unconverged else ())
        return res, info.as_dict()

    def apply_St(self, y, out=None):
        """S^T y (the transpose of the discrete single-layer matrix)."""
        return self._apply(_lib.lb_apply_St, y, out)

    def apply_At(self, y, out=None):
        """A^T y (the transpose of the discrete A3 or A2 operator)."""
        return self._apply(_lib.lb_apply_At, y, out)

    def solve_lb_adjoint(self, gu, out=None, allow_unconverged=False):
        """Gradient with respect to f of a loss whose gradient with respect
        to u = solve_lb(f) is gu (A3 or A2 formulation)."""
        nrhs = self._nrhs(gu)
        p, keep = _ptr(gu, np.float64)
        o, res = _out(out, np.float64, (nrhs, self.N))
        info = lb_solve_info()
        self._check(_lib.lb_solve_lb_adjoint(self._h, nrhs, p, o, ctypes.byref(info)),
                    allow=(LB_ENOTCONVERGED,) if allow_unconverged else ())
        return res, info.as_dict()

    def shape_gradient(self, f, gu, out=None, allow_unconverged=False):
        """Gradient [nrhs, N, 3] with respect to the node positions of a loss
        whose gradient with respect to u = solve_lb(f) is gu (A3, corrections
        held fixed)."""
        nrhs = self._nrhs(f)
        if self._nrhs(gu) != nrhs:
            raise ValueError("f and gu need the same number of right-hand sides")
        p, keep = _ptr(f, np.float64)
        q, keep2 = _ptr(gu, np.float64)
        o, res = _out(out, np.float64, (nrhs, self.N, 3))
        info = lb_solve_info()
        self._check(_lib.lb_shape_gradient(self._h, nrhs, p, q, o, ctypes.byref(info)),
                    allow=(LB_ENOTCONVERGED,) if allow_unconverged else ())
        return res, info.as_dict()

    def geometry_gradient(self, f, gu, want_x=True, want_tangents=True, out=None, allow_unconverged=False):
        """Gradients [nrhs, N, 3] of a loss of the A3 solve with respect to
        the node positions X and the chart tangents X_u, X_v (corrections and
        near lists held fixed), given g_u = dL/du.  Returns (gX or None, gXu
        or None, gXv or None, info); out = (gX, gXu, gXv) buffers, optional."""
        nrhs = self._nrhs(f)
        if self._nrhs(gu) != nrhs:
            raise ValueError("f and gu need the same number of right-hand sides")
        p, keep = _ptr(f, np.float64)
        q, keep2 = _ptr(gu, np.float64)
        outs = out if out is not None else (None, None, None)
        ptrs, res = [], []
        for want, o in zip((want_x, want_tangents, want_tangents), outs):
            if want:
                pp, rr = _out(o, np.float64, (nrhs, self.N, 3))
            else:
                pp, rr = None, None
            ptrs.append(pp)
            res.append(rr)
        info = lb_solve_info()
        self._check(_lib.lb_geometry_gradient(self._h, nrhs, p, q, *ptrs, ctypes.byref(info)),
                    allow=(LB_ENOTCONVERGED,) if allow_unconverged else ())
        return res[0], res[1], res[2], info.as_dict()

    def harmonic_fields(self, F, out=None):
        nF = self._nrhs(F, 3)
        p, keep = _ptr(F, np.float64)
        o, res = _out(out, np.float64, (2 * nF, self.N, 3))
        info = lb_solve_info()
        self._check(_lib.lb_harmonic_fields(self._h, nF, p, o, ctypes.byref(info)))
        return res, info.as_dict()


class lb_fmm_info(ctypes.Structure):
    _fields_ = [("depth", ctypes.c_int32), ("n", ctypes.c_int64), ("nbox", ctypes.c_int64),
                ("nleaf", ctypes.c_int64), ("nu", ctypes.c_int64), ("nv", ctypes.c_int64),
                ("lo", ctypes.c_double * 3), ("side", ctypes.c_double)]


def fmm_plan(X, min_leaf_side: float, max_depth: int = 20) -> dict:
    """Octree plan of the nodes X [n, 3] (lb_fmm_plan_create; host only).

    Returns depth, the cube (lo, side) and the arrays perm, level_ptr,
    box_key, box_parent, node_ptr, u_ptr, u_idx, v_ptr, v_idx."""
    X = np.ascontiguousarray(X, dtype=np.float64).reshape(-1, 3)
    h = ctypes.c_void_p()
    rc = _lib.lb_fmm_plan_create(X.shape[0], ctypes.c_void_p(X.ctypes.data), float(min_leaf_side),
                                 int(max_depth), ctypes.byref(h))
    if rc != LB_OK:
        raise LBError(rc, _lib.lb_last_error(None).decode())
    try:
        inf = lb_fmm_info()
        _lib.lb_fmm_plan_info(h, ctypes.byref(inf))
        d = inf.depth
        out = {"depth": d, "lo": np.array(inf.lo[:]), "side": inf.side,
               "perm": np.empty(inf.n, np.int64), "level_ptr": np.empty(d + 2, np.int64),
               "box_key": np.empty(inf.nbox, np.int64), "box_parent": np.empty(inf.nbox, np.int64),
               "node_ptr": np.empty(inf.nleaf + 1, np.int64), "u_ptr": np.empty(inf.nleaf + 1, np.int64),
               "u_idx": np.empty(inf.nu, np.int64), "v_ptr": np.empty(inf.nbox + 1, np.int64),
               "v_idx": np.empty(inf.nv, np.int64)}
        names = ("perm", "level_ptr", "box_key", "box_parent", "node_ptr", "u_ptr", "u_idx", "v_ptr", "v_idx")
        _lib.lb_fmm_plan_arrays(h, *[ctypes.c_void_p(out[k].ctypes.data) for k in names])
        return out
    finally:
        _lib.lb_fmm_plan_destroy(h)


# --- autograd ---------------------------------------------------------------
def _torch_fns():
    import torch

    class SolveLB(torch.autograd.Function):
        """u = solve_lb(f) with its density gradient (the adjoint solve).

        f: float64 CUDA tensor [nrhs, N]; ctx_lb: a Context with the A3
        formulation and corrections.  The backward pass is the library's
        adjoint solve (transposed applies and GMRES on A3^T)."""

        @staticmethod
        def forward(ctx, f, ctx_lb):
            u = torch.empty_like(f)
            ctx_lb.solve_lb(f.detach().contiguous(), out=u)
            ctx.ctx_lb = ctx_lb
            return u

        @staticmethod
        def backward(ctx, gu):
            gf = torch.empty_like(gu)
            ctx.ctx_lb.solve_lb_adjoint(gu.contiguous(), out=gf)
            return gf, None

    class SolveLBShape(torch.autograd.Function):
        """u = solve_lb(f) differentiable in f and in the surface inputs X,
        X_u, X_v of the upload (each may be None: not differentiated).

        The given arrays must equal the uploaded ones (checked; ValueError
        otherwise).  Their gradients are the library's geometry gradients
        (A3; correction blocks and near lists held fixed), summed over the
        right-hand sides."""

        @staticmethod
        def forward(ctx, f, X, Xu, Xv, ctx_lb):
            ctx_lb.check_geometry(X=X, Xu=Xu, Xv=Xv)
            u = torch.empty_like(f)
            fd = f.detach().contiguous()
            ctx_lb.solve_lb(fd, out=u)
            ctx.ctx_lb = ctx_lb
            ctx.save_for_backward(fd)
            ctx.shapes = tuple(None if a is None else a.shape for a in (X, Xu, Xv))
            return u

        @staticmethod
        def backward(ctx, gu):
            (f,) = ctx.saved_tensors
            gu = gu.contiguous()
            gf = None
            if ctx.needs_input_grad[0]:
                gf = torch.empty_like(gu)
                ctx.ctx_lb.solve_lb_adjoint(gu, out=gf)
            want_x = ctx.needs_input_grad[1]
            want_t = ctx.needs_input_grad[2] or ctx.needs_input_grad[3]
            grads = [None, None, None]
            if want_x or want_t:
                bufs = tuple(torch.empty(gu.shape + (3,), dtype=gu.dtype, device=gu.device) if w else None
                             for w in (want_x, want_t, want_t))
                ctx.ctx_lb.geometry_gradient(f, gu, want_x, want_t, out=bufs)
                for k in range(3):
                    if ctx.needs_input_grad[1 + k]:
                        grads[k] = bufs[k].sum(dim=0).reshape(ctx.shapes[k])
            return (gf, *grads, None)

    class ApplyA(torch.autograd.Function):
        """y = A tau with gradient A^T g_y."""

        @staticmethod
        def forward(ctx, tau, ctx_lb):
            y = torch.empty_like(tau)
            ctx_lb.apply_A(tau.detach().contiguous(), out=y)
            ctx.ctx_lb = ctx_lb
            return y

        @staticmethod
        def backward(ctx, gy):
            gt = torch.empty_like(gy)
            ctx.ctx_lb.apply_At(gy.contiguous(), out=gt)
            return gt, None

    return SolveLB, ApplyA, SolveLBShape


def solve_lb_autograd(f, ctx_lb, X=None, Xu=None, Xv=None):
    """Differentiable mean-zero Laplace-Beltrami solve (A3 or A2): u = solve(f).

    With X, Xu or Xv (tensors [N, 3] equal to the uploaded node positions and
    chart tangents; checked) the solve is also differentiable in them (A3;
    correction blocks and near lists held fixed)."""
    if X is None and Xu is None and Xv is None:
        return _torch_fns()[0].apply(f, ctx_lb)
    return _torch_fns()[2].apply(f, X, Xu, Xv, ctx_lb)


def apply_A_autograd(tau, ctx_lb):
    """Differentiable apply of the context's operator (A3 or A2)."""
    return _torch_fns()[1].apply(tau, ctx_lb)
