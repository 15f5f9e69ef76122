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
