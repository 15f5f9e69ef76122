"""Locally corrected near-field quadrature weights (oracle, FP64).

Test infrastructure only (see oracle/__init__.py).

For every target x_i and every patch P in Near(i) this computes the row block
W^K_{i,P}[q] = int_{Gamma_P} K(x_i, y) l_q(y) da(y),  q = 1..n_p,
for the kernels K in {S, D, S', S''+D'} (Section 4, the corrected weights
w~_ij of the locally corrected Nystrom scheme, composed with the implicit
polynomial interpolation of the density on P).  The full integral over each
near patch is produced here; the far sum skips near patches entirely.

Integration follows Section 4's split:
  * self patch (x_i is a node of P): T0 is cut at the target's preimage
    (u_i, v_i) into three triangles, each mapped from the unit square with
    the Duffy map (s, t) -> a + s (b - a) + s t (c - b), whose Jacobian s
    cancels the 1/r singularity; the square is integrated adaptively
    (quadtree, tensor Gauss-Legendre per cell);
  * other near patches: adaptive 1 -> 4 midpoint subdivision of T0 with the
    collapsed Gauss-Legendre rule on each triangle.
A cell is accepted when its four children change its estimate by at most
max(tol, floor) in every entry, and the children's sum is kept.  Here
tol = eps_q * A_P / (4 pi R_P) (A_P the patch area, R_P its radius) and
floor = 64 eps_mach sum_cell omega J max_q |l_q| rho bounds the rounding of
the numerators n.d (each weighted by the largest interpolation weight at the
point), below which refinement cannot improve the estimate.  On other
patches d = x - y carries eps (|x| + 2 R_P) rounding, rho = (|x| + 2 R_P) /
(4 pi r^3).  On the self patch d = y(a) - y(p) is formed from basis
differences phi_b(p) - phi_b(a) carried through the basis recurrences, so it
keeps full relative accuracy next to the target, and rho = 1 / (4 pi r^2).  A cell whose children sum is below tol in every entry is also
accepted: its whole contribution is within the tolerance (this ends the
refinement of the vanishing cells next to the Duffy apex).  At most
max_cells cells per pair are refined (the rest are accepted and counted).

Every quadrature point y is on the interpolated chart y = sum_q X_q l_q
(Section 4).  Its tangents are the derivatives of that same polynomial, which
give the normal n_y = y_u x y_v / |y_u x y_v| and the area element
|y_u x y_v|; the target normal n_x is likewise the normal of the position
interpolant of the target's own patch at its node.  (Reading: the sampled
tangents X_u, X_v are not the derivatives of the position interpolant; their
mismatch, of the size of the interpolation error, adds an odd 1/r^2 term to
S', D and S''+D' on the self patch whose integral over the Duffy triangles
does not converge.  Near-field integrals therefore use the tangent plane of
the surface they integrate over.  The far field keeps the sampled normals and
weights.)

Kernels, with d = x - y, r = |d| and G = 1/(4 pi r) (Section 3):
  S      : 1/(4 pi r)
  D      : n_y . d / (4 pi r^3)            (n_y . grad_y G)
  S'     : -n_x . d / (4 pi r^3)           (n_x . grad_x G)
  S''+D' : [3 (n_x.d)((n_x - n_y).d)/r^2 - (1 - n_x.n_y)] / (4 pi r^3)
           (n_x . grad_x grad_x G . n_x + n_x . grad_x grad_y G . n_y, combined
           pointwise; each part is hypersingular, the sum is O(1/r))
"""
from __future__ import annotations

import numpy as np
from scipy.special import roots_legendre

from .basis import eval_basis, eval_basis_diff
from .geometry import Geometry

KERNELS = ("S", "D", "Sp", "SppDp")
FOUR_PI = 4.0 * np.pi


def kernel_values(x, nx, y, ny):
    """All four kernels for target/source pairs; inputs broadcast to [..., 3]."""
    return kernel_values_d(x - y, nx, ny)


def kernel_values_d(d, nx, ny):
    """All four kernels from d = x - y; returns (K [..., 4], 1/(4 pi r^3))."""
    r2 = np.sum(d * d, axis=-1)
    r = np.sqrt(r2)
    inv4pir = 1.0 / (FOUR_PI * r)
    inv4pir3 = inv4pir / r2
    nxd = np.sum(nx * d, axis=-1)
    nyd = np.sum(ny * d, axis=-1)
    kS = inv4pir
    kD = nyd * inv4pir3
    kSp = -nxd * inv4pir3
    dn = nx - ny
    # 1 - n_x.n_y = |n_x - n_y|^2 / 2 for unit normals (no cancellation)
    kSD = (3.0 * nxd * (nxd - nyd) / r2 - 0.5 * np.sum(dn * dn, axis=-1)) * inv4pir3
    return np.stack([kS, kD, kSp, kSD], axis=-1), inv4pir3


def interpolant_normals(geo: Geometry) -> np.ndarray:
    """Unit normals of the position interpolant at every node: (D_u X) x (D_v X)."""
    if getattr(geo, "_interp_n", None) is None:
        Xp = geo.X.reshape(geo.npatch, geo.np_, 3)
        yu = np.einsum("ab,pbc->pac", geo.basis.Du, Xp).reshape(-1, 3)
        yv = np.einsum("ab,pbc->pac", geo.basis.Dv, Xp).reshape(-1, 3)
        c = np.cross(yu, yv)
        geo._interp_n = c / np.linalg.norm(c, axis=1, keepdims=True)
    return geo._interp_n


class _PatchChart:
    """Interpolated chart of one patch: coefficients in the orthonormal basis."""

    def __init__(self, geo: Geometry, P: int):
        sl = slice(P * geo.np_, (P + 1) * geo.np_)
        Vinv = geo.basis.Vinv
        self.k = geo.order
        self.Vinv = Vinv
        self.cX = Vinv @ geo.X[sl]

    def at(self, u, v):
        phi, phu, phv = eval_basis(self.k, u, v, derivs=True)
        y = phi @ self.cX
        c = np.cross(phu @ self.cX, phv @ self.cX)
        J = np.linalg.norm(c, axis=-1)
        return y, c / J[:, None], J, phi @ self.Vinv

    def at_offset(self, ua, va, du, dv):
        """Chart at p = a + (du, dv) with y(a) - y(p) from basis differences."""
        phi, phu, phv, dphi = eval_basis_diff(self.k, ua, va, du, dv)
        d = -(dphi @ self.cX)
        c = np.cross(phu @ self.cX, phv @ self.cX)
        J = np.linalg.norm(c, axis=-1)
        return d, c / J[:, None], J, phi @ self.Vinv


class NearQuadrature:
    def __init__(self, geo: Geometry, eps_q: float = 1e-12, m: int = 8, max_depth: int = 30,
                 max_cells: int = 200000):
        self.geo = geo
        self.eps_q = eps_q
        self.max_depth = max_depth
        self.max_cells = max_cells
        g, gw = roots_legendre(m)
        self.gx = 0.5 * (g + 1.0)
        self.gw = 0.5 * gw
        self.depth_hits = 0

    # --- cells -----------------------------------------------------------
    # a cell: target slot, triangle (a, b, c) in T0, rectangle [s0,s1]x[t0,t1]
    # of the Duffy square; point = a + s (b - a) + s t (c - b)
    def _integrate(self, chart, tx, tn, cells, scale=None, offset=False):
        tgt, A, B, C, R = cells
        m = len(self.gx)
        s = R[:, 0:1] + (R[:, 1:2] - R[:, 0:1]) * self.gx[None, :]           # [nc, m]
        t = R[:, 2:3] + (R[:, 3:4] - R[:, 2:3]) * self.gx[None, :]
        ws = (R[:, 1:2] - R[:, 0:1]) * self.gw[None, :]
        wt = (R[:, 3:4] - R[:, 2:3]) * self.gw[None, :]
        S_ = np.repeat(s, m, axis=1)                                          # [nc, m*m]
        T_ = np.tile(t, (1, m))
        W_ = np.repeat(ws, m, axis=1) * np.tile(wt, (1, m))
        e1 = B - A
        e2 = C - B
        det = np.abs(e1[:, 0] * e2[:, 1] - e1[:, 1] * e2[:, 0])
        du = S_ * e1[:, 0:1] + S_ * T_ * e2[:, 0:1]
        dv = S_ * e1[:, 1:2] + S_ * T_ * e2[:, 1:2]
        omega = (W_ * S_ * det[:, None]).ravel()
        nc = len(tgt)
        nt = np.repeat(tn[tgt], m * m, axis=0)
        if offset:
            # self patch: every cell shares the apex a = the target's node
            d, ny, J, lag = chart.at_offset(A[0, 0], A[0, 1], du.ravel(), dv.ravel())
        else:
            y, ny, J, lag = chart.at((A[:, 0:1] + du).ravel(), (A[:, 1:2] + dv).ravel())
            d = np.repeat(tx[tgt], m * m, axis=0) - y
        K, r3 = kernel_values_d(d, nt, ny)                                    # [P, 4]
        wJ = (omega * J).reshape(nc, m * m)
        f = np.einsum("cp,cpk,cpq->ckq", wJ, K.reshape(nc, m * m, 4),
                      lag.reshape(nc, m * m, -1), optimize=True)
        lmax = np.abs(lag).max(axis=1).reshape(nc, m * m)
        if offset:
            # d is accurate to eps |d|: numerators carry eps |d| r rounding
            r2inv = (r3 * np.sqrt(np.sum(d * d, axis=1))).reshape(nc, m * m)
            rnd = (wJ * r2inv * lmax).sum(axis=1)
        else:
            sc = 1.0 if scale is None else np.repeat(scale[tgt], 1)
            rnd = (wJ * r3.reshape(nc, m * m) * lmax).sum(axis=1) * sc
        return f, rnd

    def _integrate_chunked(self, chart, tx, tn, cells, scale=None, offset=False, chunk=1024):
        n = len(cells[0])
        outs, rnds = [], []
        for a in range(0, n, chunk):
            o, r = self._integrate(chart, tx, tn, tuple(c[a:a + chunk] for c in cells), scale, offset)
            outs.append(o)
            rnds.append(r)
        return np.concatenate(outs), np.concatenate(rnds)

    @staticmethod
    def _split_triangles(cells):
        tgt, A, B, C, R = cells
        AB, BC, CA = 0.5 * (A + B), 0.5 * (B + C), 0.5 * (C + A)
        kids = [(A, AB, CA), (AB, B, BC), (CA, BC, C), (AB, BC, CA)]
        return (np.repeat(tgt, 4),
                np.stack([k[0] for k in kids], 1).reshape(-1, 2),
                np.stack([k[1] for k in kids], 1).reshape(-1, 2),
                np.stack([k[2] for k in kids], 1).reshape(-1, 2),
                np.repeat(R, 4, axis=0))

    @staticmethod
    def _split_rectangles(cells):
        tgt, A, B, C, R = cells
        sm = 0.5 * (R[:, 0] + R[:, 1])
        tm = 0.5 * (R[:, 2] + R[:, 3])
        kids = [np.stack([R[:, 0], sm, R[:, 2], tm], 1), np.stack([sm, R[:, 1], R[:, 2], tm], 1),
                np.stack([R[:, 0], sm, tm, R[:, 3]], 1), np.stack([sm, R[:, 1], tm, R[:, 3]], 1)]
        return (np.repeat(tgt, 4), np.repeat(A, 4, axis=0), np.repeat(B, 4, axis=0),
                np.repeat(C, 4, axis=0), np.stack(kids, 1).reshape(-1, 4))

    def _adaptive(self, chart, tx, tn, roots, ntgt, tol, split, scale, offset=False):
        out = np.zeros((ntgt, 4, self.geo.np_))
        cells = roots
        est, _ = self._integrate_chunked(chart, tx, tn, cells, scale, offset)
        depth = 0
        ncells = 0
        eps = np.finfo(np.float64).eps
        while len(cells[0]):
            kids = split(cells)
            kid_est, kid_rnd = self._integrate_chunked(chart, tx, tn, kids, scale, offset)
            nc = len(cells[0])
            ksum = kid_est.reshape(nc, 4, 4, -1).sum(axis=1)
            floor = 64.0 * eps * kid_rnd.reshape(nc, 4).sum(axis=1)
            err = np.max(np.abs(ksum - est), axis=(1, 2))
            depth += 1
            done = (err <= np.maximum(tol, floor)) | (np.max(np.abs(ksum), axis=(1, 2)) <= tol)
            ncells += 4 * nc
            if depth >= self.max_depth or ncells > self.max_cells * ntgt:
                self.depth_hits += int(np.count_nonzero(~done))
                done[:] = True
            np.add.at(out, cells[0][done], ksum[done])
            keep = np.repeat(~done, 4)
            cells = tuple(c[keep] for c in kids)
            est = kid_est[keep]
        return out

    def patch_blocks(self, P: int, targets: np.ndarray) -> np.ndarray:
        """Row blocks W[k, q] for the given targets (all with P in Near(i)).

        Returns [len(targets), 4, n_p] in kernel order (S, D, S', S''+D').
        """
        geo = self.geo
        chart = _PatchChart(geo, P)
        sl = slice(P * geo.np_, (P + 1) * geo.np_)
        area = geo.w[sl].sum()
        tol = self.eps_q * area / (FOUR_PI * geo.radius[P])
        tx = geo.X[targets]
        tn = interpolant_normals(geo)[targets]
        scale = np.linalg.norm(tx, axis=1) + 2.0 * geo.radius[P]
        res = np.zeros((len(targets), 4, geo.np_))
        own = (targets // geo.np_) == P
        # other near patches: root triangle T0
        idx = np.nonzero(~own)[0]
        if len(idx):
            z = np.zeros((len(idx), 2))
            roots = (np.arange(len(idx)), z, z + [1.0, 0.0], z + [0.0, 1.0],
                     np.tile([0.0, 1.0, 0.0, 1.0], (len(idx), 1)))
            res[idx] = self._adaptive(chart, tx[idx], tn[idx], roots, len(idx), tol,
                                      self._split_triangles, scale[idx])
        # self patch: three Duffy triangles with apex at the target's preimage
        verts = np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0]])
        for i in np.nonzero(own)[0]:
            apex = geo.basis.uv[targets[i] % geo.np_]
            roots = (np.zeros(3, dtype=np.int64), np.tile(apex, (3, 1)), verts[[0, 1, 2]], verts[[1, 2, 0]],
                     np.tile([0.0, 1.0, 0.0, 1.0], (3, 1)))
            res[i] = self._adaptive(chart, tx[[i]], tn[[i]], roots, 1, tol, self._split_rectangles,
                                    scale[[i]], offset=True)[0]
        return res


_WORKER_GEO = None


def _init_worker(geo):
    global _WORKER_GEO
    _WORKER_GEO = geo


def _patch_job(args):
    eps_q, m, P, targets = args
    q = NearQuadrature(_WORKER_GEO, eps_q=eps_q, m=m)
    return P, q.patch_blocks(P, targets), q.depth_hits


def build_corrections(geo: Geometry, near_ptr, near_patch, eps_q: float = 1e-12,
                      rows=None, m: int = 8, workers: int = 1, blocks=None):
    """Near-field weights as block CSR.

    Returns (vals [nnzb, 4, n_p] aligned with near_patch, depth_hits): block b
    belongs to row i with near_ptr[i] <= b < near_ptr[i+1].  If rows and/or
    blocks (a boolean mask over the nnzb blocks) are given, only the blocks of
    those rows and the selected blocks are filled (the rest stay zero).
    workers > 1 spreads patches over a spawn-started process pool.
    """
    nnzb = len(near_patch)
    vals = np.zeros((nnzb, 4, geo.np_))
    row_of = np.repeat(np.arange(geo.N), np.diff(near_ptr))
    sel = np.ones(nnzb, dtype=bool)
    if rows is not None or blocks is not None:
        sel = np.zeros(nnzb, dtype=bool)
        if rows is not None:
            sel |= np.isin(row_of, np.asarray(rows))
        if blocks is not None:
            sel |= np.asarray(blocks, dtype=bool)
    jobs = []
    for P in range(geo.npatch):
        blocks = np.nonzero(sel & (near_patch == P))[0]
        # split a patch's targets into pieces so that pool workers stay busy
        for part in np.array_split(blocks, max(1, len(blocks) // 64)):
            if len(part):
                jobs.append((part, (eps_q, m, P, row_of[part])))
    hits = 0
    if workers > 1 and len(jobs) > 1:
        import multiprocessing as mp
        from concurrent.futures import ProcessPoolExecutor
        import os
        keys = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")
        saved = {k: os.environ.get(k) for k in keys}
        os.environ.update({k: "1" for k in keys})   # one BLAS thread per worker
        try:
            with ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn"),
                                     initializer=_init_worker, initargs=(geo,)) as ex:
                results = list(ex.map(_patch_job, [j[1] for j in jobs]))
        finally:
            for k, v in saved.items():
                if v is None:
                    os.environ.pop(k, None)
                else:
                    os.environ[k] = v
    else:
        _init_worker(geo)
        results = [_patch_job(j[1]) for j in jobs]
    for (part, _), (P, blk, h) in zip(jobs, results):
        vals[part] = blk
        hits += h
    return vals, hits
