"""Saving and reloading the near-field corrections (host-side, numpy only).

The correction build is the set-up cost of the method (the paper's t_q,
Section 6); a saved block-CSR lets a later run skip it for the same surface
and parameters.  A checkpoint is an .npz holding a format version, a SHA-256
digest of the geometry it was built for (node rule, order, X, X_u, X_v, in
float64), the near factor and quadrature tolerance, and the CSR itself
(row_ptr [N+1] int64, patch [nnzb] int32, vals [nnzb][4][n_p] float64).
Loading checks all of these before anything reaches the library.
"""
from __future__ import annotations

import hashlib

import numpy as np

VERSION = 1


def geometry_digest(npatch, order, ref_uv, ref_w, X, Xu, Xv) -> str:
    """SHA-256 over the geometry inputs as contiguous float64, with their shapes."""
    h = hashlib.sha256()
    h.update(f"lbgeom/{int(npatch)}/{int(order)}".encode())
    for a in (ref_uv, ref_w, X, Xu, Xv):
        a = np.ascontiguousarray(a, dtype=np.float64)
        h.update(str(a.shape).encode())
        h.update(a.tobytes())
    return h.hexdigest()


class CheckpointError(ValueError):
    pass


def save(path, digest: str, near_factor: float, eps_quad: float, row_ptr, patch, vals) -> None:
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int64)
    patch = np.ascontiguousarray(patch, dtype=np.int32)
    vals = np.ascontiguousarray(vals, dtype=np.float64)
    _check_csr(row_ptr, patch, vals)
    with open(path, "wb") as fh:
        np.savez(fh, version=np.int64(VERSION), digest=np.array(digest), near_factor=np.float64(near_factor),
                 eps_quad=np.float64(eps_quad), row_ptr=row_ptr, patch=patch, vals=vals)


def load(path, digest: str, near_factor: float, eps_quad: float):
    """(row_ptr, patch, vals) after checking the version, the geometry digest
    and the parameters against the caller's; CheckpointError otherwise."""
    with np.load(path, allow_pickle=False) as z:
        if int(z["version"]) != VERSION:
            raise CheckpointError(f"checkpoint format {int(z['version'])}, expected {VERSION}")
        if str(z["digest"]) != digest:
            raise CheckpointError("checkpoint was built for another geometry")
        if float(z["near_factor"]) != float(near_factor) or float(z["eps_quad"]) != float(eps_quad):
            raise CheckpointError(
                f"checkpoint parameters (near_factor {float(z['near_factor'])}, eps_quad {float(z['eps_quad'])}) "
                f"differ from the context's ({near_factor}, {eps_quad})")
        row_ptr, patch, vals = z["row_ptr"], z["patch"], z["vals"]
    _check_csr(row_ptr, patch, vals)
    return row_ptr, patch, vals


def _check_csr(row_ptr, patch, vals, N=None, npatch=None, np_=None):
    """Structure of a correction CSR; N, npatch and np_ (when given) are the
    surface's node, patch and per-patch node counts."""
    row_ptr = np.asarray(row_ptr)
    patch = np.asarray(patch)
    if row_ptr.ndim != 1 or len(row_ptr) < 2 or row_ptr[0] != 0 or np.any(np.diff(row_ptr) < 0) \
            or row_ptr[-1] != len(patch):
        raise CheckpointError("row_ptr is not a CSR row pointer for the patch list")
    if N is not None and len(row_ptr) != N + 1:
        raise CheckpointError(f"row_ptr has {len(row_ptr)} entries, the surface needs N + 1 = {N + 1}")
    if vals is not None:
        if vals.ndim != 3 or vals.shape[0] != len(patch) or vals.shape[1] != 4 \
                or (np_ is not None and vals.shape[2] != np_):
            raise CheckpointError("vals must be [nnzb][4][n_p]")
        if not np.isfinite(vals).all():
            raise CheckpointError("vals hold non-finite entries")
    if len(patch) and (patch.min() < 0 or (npatch is not None and patch.max() >= npatch)):
        raise CheckpointError("a near patch index lies outside [0, npatch)")
    # strictly ascending within each row: a step down or a repeat may only
    # happen where a new row starts
    if len(patch) > 1:
        starts = np.zeros(len(patch), dtype=bool)
        starts[row_ptr[:-1][row_ptr[:-1] < len(patch)]] = True
        if np.any((np.diff(patch.astype(np.int64)) <= 0) & ~starts[1:]):
            raise CheckpointError("near patches of a row must be strictly ascending")
