"""Gradient of a loss of the A3 solve with respect to the node positions (oracle, FP64).

Test infrastructure only (see oracle/__init__.py).

The node positions X enter the discrete A3 operator only through the far
field: the pair sums sum_j w_j K(x_i, x_j) sigma_j over the far pairs.  The
correction blocks, the near lists, the weights w, the normals n and the mean
curvature H are held fixed: they come from the tangents X_u, X_v and the
near-field quadrature.  That is the proposed reading for node-coordinate
gradients, which freezes the corrections.

With u = S S sigma, A3 sigma = P f and g_u = dL/du:
  dL = g_u . dS(S sigma) + (S^T g_u) . dS(sigma) - z . (dA3 sigma),
  z = A3^-T S^T S^T g_u,
  dA3 sigma = dS'(mu1) + S'(dS' sigma) - d(S''+D')(mu2) - (S''+D')(dS sigma)
              - 2H dS'(mu2) - 2H S'(dS sigma) + W dS(mu2) + W S(dS sigma),
with mu1 = S' sigma and mu2 = S sigma.  Every term has the form
a . dK(b) = sum over far pairs of a_i b_j w_j grad_d K(x_i, x_j) . (dx_i - dx_j),
d = x_i - x_j, with the normals held fixed in K.  Dense matrices throughout:
for small surfaces only.
"""
from __future__ import annotations

import numpy as np

from .gmres import dense_matrix
from .layers import K_S, K_SD, K_SP


def _pair_arrays(disc):
    g = disc.geo
    N = g.N
    near = np.zeros((N, g.npatch), bool)
    for i in range(N):
        near[i, disc.near_patch[disc.near_ptr[i]:disc.near_ptr[i + 1]]] = True
    far = ~near[:, np.arange(N) // g.np_]              # [i, j]: patch(j) not in Near(i)
    d = g.X[:, None, :] - g.X[None, :, :]
    r2 = np.einsum("ijk,ijk->ij", d, d)
    np.fill_diagonal(r2, 1.0)
    return far, d, r2


def kernel_gradients(disc):
    """w_j grad_d K(x_i, x_j) on the far pairs, [N, N, 3] for K = S, S', S''+D'."""
    g = disc.geo
    far, d, r2 = _pair_arrays(disc)
    r = np.sqrt(r2)
    c = (far * g.w[None, :] / (4.0 * np.pi))[:, :, None]
    nx = g.n[:, None, :]
    e = g.n[:, None, :] - g.n[None, :, :]
    a = np.einsum("ik,ijk->ij", g.n, d)[:, :, None]    # n_x . d
    b = np.einsum("ijk,ijk->ij", e, d)[:, :, None]     # (n_x - n_y) . d
    e2 = np.einsum("ijk,ijk->ij", e, e)[:, :, None]
    R2, R3, R5 = r2[:, :, None], (r * r2)[:, :, None], (r2 * r2 * r)[:, :, None]
    gS = -d / R3
    gSp = (-nx * R2 + 3.0 * a * d) / R5
    gSD = (3.0 * (b * nx + a * e) / R2 - 6.0 * a * b * d / (R2 * R2)) / R3 \
        - 3.0 * (3.0 * a * b / R2 - 0.5 * e2) * d / R5
    return c * gS, c * gSp, c * gSD


def _contract(GK, a, b):
    """Gradient of a . K b with respect to the positions, [N, 3]."""
    gi = a[:, None] * np.einsum("ijk,j->ik", GK, b)
    gj = -b[:, None] * np.einsum("ijk,i->jk", GK, a)
    return gi + gj


def shape_gradient_A3(disc, f, gu):
    """dL/dX [N, 3] for L(u), u = the A3 solve of f, given g_u = dL/du [N]."""
    g = disc.geo
    N = g.N
    Smat = dense_matrix(lambda x: disc.potentials(x)[:, K_S], N)
    Spmat = dense_matrix(lambda x: disc.potentials(x)[:, K_SP], N)
    SDmat = dense_matrix(lambda x: disc.potentials(x)[:, K_SD], N)
    Amat = dense_matrix(lambda x: disc.apply("A3", x), N)
    b = disc.rhs("A3", f)[0]
    sigma = np.linalg.solve(Amat, b)
    mu1, mu2 = Spmat @ sigma, Smat @ sigma
    q1 = Smat.T @ gu
    z = np.linalg.solve(Amat.T, Smat.T @ (Smat.T @ gu))
    Wz = g.w * z.sum() / g.w.sum()                     # W^T z, W = 1 w^T / |Gamma|
    H2 = 2.0 * g.H
    GS, GSp, GSD = kernel_gradients(disc)
    grad = _contract(GS, gu, mu2) + _contract(GS, q1, sigma)
    # - z . dA3 sigma, term by term
    grad -= _contract(GSp, z, mu1) + _contract(GSp, Spmat.T @ z, sigma)
    grad += _contract(GSD, z, mu2) + _contract(GS, SDmat.T @ z, sigma)
    grad += _contract(GSp, H2 * z, mu2) + _contract(GS, Spmat.T @ (H2 * z), sigma)
    grad -= _contract(GS, Wz, mu2) + _contract(GS, Smat.T @ Wz, sigma)
    return grad


# ---------------------------------------------------------------------------
# Gradient with respect to the chart tangents X_u, X_v (input model: the
# upload's X, X_u, X_v are independent inputs; the correction blocks and the
# near lists stay fixed).  X_u and X_v enter A3 through
#   * the unit normals n = X_u x X_v / |X_u x X_v| in the far kernels
#     (target normal in S' and S''+D', source normal in S''+D'),
#   * the weights w = w_ref |X_u x X_v| in every far sum, in the mean W and in
#     the projection P f = f - W f,
#   * the mean curvature H = -1/2 tr(g^-1 L), L_ab = X_ab . n, with
#     X_uu = D_u X_u, X_vv = D_v X_v, X_uv = (D_v X_u + D_u X_v)/2 per patch
#     and g the metric of X_u, X_v (Section 2).
# With the six bilinear terms a_m . K_m b_m of shape_gradient_A3 (same a_m, b_m):
#   dL/dw_j = sum_m b_m,j sum_{i far} a_m,i K_m(i, j)
#             - (sum z / |Gamma|) [(S mu2)_j - W S mu2 + f_j - W f],
#   dL/dn_i = sum_{m: S', S''+D'} a_m,i sum_{j far} w_j b_m,j dK_m/dn_x,
#   dL/dn_j += w_j mu2_j sum_{i far} z_i d(S''+D')/dn_y,
#   dL/dH_i = 2 z_i (S' mu2)_i,
# and the chain rule through n, |X_u x X_v| and H.

def _far_kernels(disc):
    """K_m(i, j) (far pairs, no weight, 1/(4 pi) included) and the normal
    derivatives of S' and S''+D': (KS, KSp, KSD, dSp_dnx, dSD_dnx, dSD_dny)."""
    g = disc.geo
    far, d, r2 = _pair_arrays(disc)
    r = np.sqrt(r2)
    f4 = far / (4.0 * np.pi)
    nx = g.n[:, None, :]
    ny = g.n[None, :, :]
    e = nx - ny
    a = np.einsum("ik,ijk->ij", g.n, d)                   # n_x . d
    b = np.einsum("ijk,ijk->ij", e, d)                    # (n_x - n_y) . d
    e2 = np.einsum("ijk,ijk->ij", e, e)
    r3 = r * r2
    KS = f4 / r
    KSp = -f4 * a / r3
    KSD = f4 * (3.0 * a * b / r2 - 0.5 * e2) / r3
    dSp = -(f4 / r3)[:, :, None] * d                      # d K_S' / d n_x
    dSDx = (f4 / r3)[:, :, None] * (3.0 * ((a + b) / r2)[:, :, None] * d - e)
    dSDy = (f4 / r3)[:, :, None] * (-3.0 * (a / r2)[:, :, None] * d + e)
    return KS, KSp, KSD, dSp, dSDx, dSDy


def tangent_gradient_A3(disc, f, gu):
    """(dL/dX_u, dL/dX_v) [N, 3] each, for L(u), u = the A3 solve of f,
    given g_u = dL/du [N]; corrections, near lists and X held fixed."""
    g = disc.geo
    N = g.N
    Smat = dense_matrix(lambda x: disc.potentials(x)[:, K_S], N)
    Spmat = dense_matrix(lambda x: disc.potentials(x)[:, K_SP], N)
    SDmat = dense_matrix(lambda x: disc.potentials(x)[:, K_SD], N)
    Amat = dense_matrix(lambda x: disc.apply("A3", x), N)
    area = g.w.sum()
    f = np.asarray(f, dtype=np.float64)
    Wf = np.dot(g.w, f) / area
    b = f - Wf
    sigma = np.linalg.solve(Amat, b)
    mu1, mu2 = Spmat @ sigma, Smat @ sigma
    z = np.linalg.solve(Amat.T, Smat.T @ (Smat.T @ gu))
    eta_z = z.sum() / area
    Smu2 = Smat @ mu2
    eta = np.dot(g.w, Smu2) / area
    H2z = 2.0 * g.H * z
    a0 = Smat.T @ gu + SDmat.T @ z + Spmat.T @ H2z - eta_z * (Smat.T @ g.w)
    a1 = gu - eta_z * g.w
    terms_S = ((a0, sigma), (a1, mu2))
    terms_Sp = ((-z, mu1), (-(Spmat.T @ z), sigma), (H2z, mu2))
    terms_SD = ((z, mu2),)
    KS, KSp, KSD, dSp, dSDx, dSDy = _far_kernels(disc)
    # weights
    gw = np.zeros(N)
    for K, terms in ((KS, terms_S), (KSp, terms_Sp), (KSD, terms_SD)):
        for am, bm in terms:
            gw += bm * (am @ K)
    gw -= eta_z * (Smu2 - eta + f - Wf)
    # normals: target side from S' and S''+D', source side from S''+D'
    gn = np.zeros((N, 3))
    for am, bm in terms_Sp:
        gn += am[:, None] * np.einsum("ijk,j->ik", dSp, g.w * bm)
    gn += z[:, None] * np.einsum("ijk,j->ik", dSDx, g.w * mu2)
    gn += (g.w * mu2)[:, None] * np.einsum("ijk,i->jk", dSDy, z)
    # mean curvature: A3 holds -2 H S' mu2
    gH = 2.0 * z * (Spmat @ mu2)
    return _tangent_chain(g, gn, gw, gH)


def _tangent_chain(g, gn, gw, gH):
    """Chain rule from (dL/dn, dL/dw, dL/dH) at the nodes to (dL/dX_u, dL/dX_v)."""
    N, npn, npatch = g.N, g.np_, g.npatch
    Xu, Xv, n = g.Xu, g.Xv, g.n
    Xu_p = Xu.reshape(npatch, npn, 3)
    Xv_p = Xv.reshape(npatch, npn, 3)
    Du, Dv = g.basis.Du, g.basis.Dv
    Xuu = np.einsum("ab,pbc->pac", Du, Xu_p).reshape(N, 3)
    Xvv = np.einsum("ab,pbc->pac", Dv, Xv_p).reshape(N, 3)
    Xuv = 0.5 * (np.einsum("ab,pbc->pac", Dv, Xu_p) + np.einsum("ab,pbc->pac", Du, Xv_p)).reshape(N, 3)
    G = g.ginv                                                   # [N, 2, 2]
    L = np.empty((N, 2, 2))
    L[:, 0, 0] = np.einsum("ij,ij->i", Xuu, n)
    L[:, 0, 1] = L[:, 1, 0] = np.einsum("ij,ij->i", Xuv, n)
    L[:, 1, 1] = np.einsum("ij,ij->i", Xvv, n)
    gXu = np.zeros((N, 3))
    gXv = np.zeros((N, 3))
    # H = -1/2 (G11 L11 + 2 G12 L12 + G22 L22)
    gXuu = (-0.5 * gH * G[:, 0, 0])[:, None] * n
    gXvv = (-0.5 * gH * G[:, 1, 1])[:, None] * n
    gXuv = (-gH * G[:, 0, 1])[:, None] * n
    gn = gn + (-0.5 * gH)[:, None] * (G[:, 0, 0, None] * Xuu + 2.0 * G[:, 0, 1, None] * Xuv
                                        + G[:, 1, 1, None] * Xvv)
    # through g^-1: dH = tr(M dg), M = 1/2 G L G
    M = 0.5 * np.einsum("iab,ibc,icd->iad", G, L, G)
    gXu += gH[:, None] * (2.0 * M[:, 0, 0, None] * Xu + 2.0 * M[:, 0, 1, None] * Xv)
    gXv += gH[:, None] * (2.0 * M[:, 1, 1, None] * Xv + 2.0 * M[:, 0, 1, None] * Xu)
    # through the nodal derivatives
    sh = (npatch, npn, 3)
    gXu += (np.einsum("ab,pac->pbc", Du, gXuu.reshape(sh))
            + 0.5 * np.einsum("ab,pac->pbc", Dv, gXuv.reshape(sh))).reshape(N, 3)
    gXv += (np.einsum("ab,pac->pbc", Dv, gXvv.reshape(sh))
            + 0.5 * np.einsum("ab,pac->pbc", Du, gXuv.reshape(sh))).reshape(N, 3)
    # n = c / |c|, w = w_ref |c|, c = X_u x X_v
    c = np.cross(Xu, Xv)
    J = np.linalg.norm(c, axis=1)
    gJ = np.tile(g.wref, npatch) * gw
    gc = (gn - np.einsum("ij,ij->i", gn, n)[:, None] * n) / J[:, None] + gJ[:, None] * n
    gXu += np.cross(Xv, gc)
    gXv += np.cross(gc, Xu)
    return gXu, gXv
