"""Surface geometry at the discretisation nodes (oracle, FP64).

Test infrastructure only (see oracle/__init__.py).

From the samples X, X_u, X_v of every patch chart (Section 4) this computes:
  * unit normal n = X_u x X_v / |X_u x X_v|                     (Section 2)
  * first fundamental form g and its inverse                       (Section 2)
  * smooth quadrature weights w_i = w_ref_q |X_u x X_v|             (Section 4)
  * mean curvature H = -1/2 tr(g^-1 L), L_ab = X_ab . n, with the second
    derivatives X_uu = D_u X_u, X_vv = D_v X_v and
    X_uv = (D_v X_u + D_u X_v)/2 from nodal differentiation of the sampled
    tangents (Section 4: only first derivatives are stored and H comes from
    spectral differentiation).  With outward n this gives H = +1 on the unit
    sphere.
  * patch centroid c_P (mean of its nodes), radius R_P (largest node distance
    from c_P), and the near lists Near(i) = {P : |x_i - c_P| < eta R_P}
    (Section 4, the Near/Far split; the criterion's form is this
    implementation's reading of "O(1) patches").
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from .basis import NodalBasis


@dataclass
class Geometry:
    order: int
    npatch: int
    np_: int
    basis: NodalBasis
    wref: np.ndarray
    X: np.ndarray      # [N, 3]
    Xu: np.ndarray
    Xv: np.ndarray
    n: np.ndarray      # [N, 3]
    J: np.ndarray      # [N]  |X_u x X_v|
    w: np.ndarray      # [N]  smooth quadrature weights
    H: np.ndarray      # [N]  mean curvature
    ginv: np.ndarray   # [N, 2, 2]
    centroid: np.ndarray  # [npatch, 3]
    radius: np.ndarray    # [npatch]

    @property
    def N(self) -> int:
        return self.X.shape[0]

    def patch_of(self, i: int) -> int:
        return i // self.np_


def build_geometry(order: int, uv, wref, X, Xu, Xv) -> Geometry:
    X = np.asarray(X, dtype=np.float64)
    Xu = np.asarray(Xu, dtype=np.float64)
    Xv = np.asarray(Xv, dtype=np.float64)
    B = NodalBasis(order, uv)
    npn = B.np_
    N = X.shape[0]
    npatch = N // npn
    c = np.cross(Xu, Xv)
    J = np.linalg.norm(c, axis=1)
    n = c / J[:, None]
    w = np.tile(np.asarray(wref, dtype=np.float64), npatch) * J
    guu = np.einsum("ij,ij->i", Xu, Xu)
    guv = np.einsum("ij,ij->i", Xu, Xv)
    gvv = np.einsum("ij,ij->i", Xv, Xv)
    det = guu * gvv - guv * guv
    ginv = np.empty((N, 2, 2))
    ginv[:, 0, 0] = gvv / det
    ginv[:, 0, 1] = -guv / det
    ginv[:, 1, 0] = -guv / det
    ginv[:, 1, 1] = guu / det
    # second derivatives by nodal differentiation, patch by patch
    Xu_p = Xu.reshape(npatch, npn, 3)
    Xv_p = Xv.reshape(npatch, npn, 3)
    Xuu = np.einsum("ab,pbc->pac", B.Du, Xu_p).reshape(N, 3)
    Xvv = np.einsum("ab,pbc->pac", B.Dv, Xv_p).reshape(N, 3)
    Xuv = 0.5 * (np.einsum("ab,pbc->pac", B.Dv, Xu_p)
                 + np.einsum("ab,pbc->pac", B.Du, Xv_p)).reshape(N, 3)
    Luu = np.einsum("ij,ij->i", Xuu, n)
    Luv = np.einsum("ij,ij->i", Xuv, n)
    Lvv = np.einsum("ij,ij->i", Xvv, n)
    H = -0.5 * (ginv[:, 0, 0] * Luu + 2.0 * ginv[:, 0, 1] * Luv + ginv[:, 1, 1] * Lvv)
    Xp = X.reshape(npatch, npn, 3)
    cen = Xp.mean(axis=1)
    rad = np.max(np.linalg.norm(Xp - cen[:, None, :], axis=2), axis=1)
    return Geometry(order, npatch, npn, B, np.asarray(wref, dtype=np.float64), X, Xu, Xv,
                    n, J, w, H, ginv, cen, rad)


def near_lists(geo: Geometry, eta: float):
    """Near(i) as CSR: (row_ptr [N+1], patches [nnzb]) with ascending patch ids.

    Patch P is near target i when |x_i - c_P| < eta * R_P (strict).
    """
    rows = []
    for i in range(geo.N):
        d = np.linalg.norm(geo.centroid - geo.X[i][None, :], axis=1)
        rows.append(np.nonzero(d < eta * geo.radius)[0].astype(np.int32))
    ptr = np.zeros(geo.N + 1, dtype=np.int64)
    ptr[1:] = np.cumsum([len(r) for r in rows])
    return ptr, (np.concatenate(rows) if rows else np.zeros(0, dtype=np.int32))


def surface_gradient(geo: Geometry, f: np.ndarray) -> np.ndarray:
    """grad_Gamma f = (g^11 f_u + g^12 f_v) X_u + (g^21 f_u + g^22 f_v) X_v (Section 2).

    f [N] or [N, r]; f_u, f_v by nodal differentiation within each patch.
    Returns [N, 3] or [N, r, 3].
    """
    squeeze = f.ndim == 1
    F = f.reshape(geo.N, -1)
    Fp = F.reshape(geo.npatch, geo.np_, -1)
    fu = np.einsum("ab,pbr->par", geo.basis.Du, Fp).reshape(geo.N, -1)
    fv = np.einsum("ab,pbr->par", geo.basis.Dv, Fp).reshape(geo.N, -1)
    a = geo.ginv[:, 0, 0][:, None] * fu + geo.ginv[:, 0, 1][:, None] * fv
    b = geo.ginv[:, 1, 0][:, None] * fu + geo.ginv[:, 1, 1][:, None] * fv
    G = a[:, :, None] * geo.Xu[:, None, :] + b[:, :, None] * geo.Xv[:, None, :]
    return G[:, 0, :] if squeeze else G


def surface_divergence(geo: Geometry, F: np.ndarray) -> np.ndarray:
    """div_Gamma F = |g|^-1/2 (d_u(|g|^1/2 F1) + d_v(|g|^1/2 F2)) (Section 2).

    F is a tangential field [N, 3]; its components F1, F2 in the basis
    (X_u, X_v) are (F.X_u, F.X_v) contracted with g^-1.  sqrt|g| = |X_u x X_v|.
    """
    a = np.einsum("ij,ij->i", F, geo.Xu)
    b = np.einsum("ij,ij->i", F, geo.Xv)
    F1 = geo.ginv[:, 0, 0] * a + geo.ginv[:, 0, 1] * b
    F2 = geo.ginv[:, 1, 0] * a + geo.ginv[:, 1, 1] * b
    P1 = (geo.J * F1).reshape(geo.npatch, geo.np_)
    P2 = (geo.J * F2).reshape(geo.npatch, geo.np_)
    d = (np.einsum("ab,pb->pa", geo.basis.Du, P1) + np.einsum("ab,pb->pa", geo.basis.Dv, P2))
    return d.reshape(geo.N) / geo.J


@dataclass
class FarRule:
    """Oversampled far-field sources (Section 4): on every patch, the patch
    interpolants of X, X_u and X_v evaluated at the nodes of a finer rule
    (uv_o, w_o) on T0.  Source s lies on patch s // nps; its normal is
    X_u x X_v / |X_u x X_v| and its weight w_o |X_u x X_v| of the interpolated
    tangents, and its density the interpolant of the nodal density."""
    nps: int
    I: np.ndarray   # [n_o, n_p] base-rule Lagrange basis at the fine nodes
    Y: np.ndarray   # [npatch * n_o, 3]
    n: np.ndarray   # [npatch * n_o, 3]
    w: np.ndarray   # [npatch * n_o]

    def densities(self, sigma: np.ndarray) -> np.ndarray:
        """Nodal densities [nrhs, N] -> source densities [nrhs, npatch * n_o]."""
        sig = np.atleast_2d(sigma)
        npatch = self.Y.shape[0] // self.nps
        s = sig.reshape(sig.shape[0], npatch, self.I.shape[1])
        return np.einsum("qb,rpb->rpq", self.I, s).reshape(sig.shape[0], -1)


def oversample(geo: Geometry, uv_o, w_o) -> FarRule:
    uv_o = np.asarray(uv_o, dtype=np.float64)
    w_o = np.asarray(w_o, dtype=np.float64)
    I = geo.basis.lagrange(uv_o[:, 0], uv_o[:, 1])
    shape = (geo.npatch, geo.np_, 3)
    Y = np.einsum("qb,pbk->pqk", I, geo.X.reshape(shape)).reshape(-1, 3)
    Xu = np.einsum("qb,pbk->pqk", I, geo.Xu.reshape(shape)).reshape(-1, 3)
    Xv = np.einsum("qb,pbk->pqk", I, geo.Xv.reshape(shape)).reshape(-1, 3)
    c = np.cross(Xu, Xv)
    J = np.linalg.norm(c, axis=1)
    w = np.tile(w_o, geo.npatch) * J
    return FarRule(len(w_o), I, Y, c / J[:, None], w)
