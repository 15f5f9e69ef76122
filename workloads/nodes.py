"""Reference-triangle node rule: interpolation nodes and smooth quadrature weights.

A patch chart is sampled at n_p = (k+1)(k+2)/2 nodes on the standard simplex
T0 = {u, v >= 0, u + v <= 1} (Section 4, "order p discretization"; the paper's
p is total degree < p, so k = p - 1 here).  The paper uses Vioreanu-Rokhlin
nodes: points obtained as the spectrum of the operator "multiply by z = x + iy"
compressed onto the polynomials of total degree <= k.  That construction is
restated here from its definition:

1. an orthonormal basis of P_k on T0 (collapsed-coordinate Jacobi products);
2. the compressed multiplication matrix M_ij = <phi_i, z phi_j> on the
   equilateral image of T0 (so that the node set inherits the triangle's
   full symmetry group);
3. the eigenvalues of M, mapped back to T0, are the nodes;
4. the weights are interpolatory: exact for every polynomial of degree <= k.

The tabulated, further-optimised rules of the paper's software are not
reproduced; only the eigenvalue step above is.  This module is an input
generator (a mesh ingredient shared by every consumer) and holds no layer
potential arithmetic.
"""
from __future__ import annotations

import functools

import numpy as np
from scipy.special import eval_jacobi, roots_legendre

SQ3 = np.sqrt(3.0)


def n_nodes(order: int) -> int:
    """Number of nodes for total degree <= order."""
    return (order + 1) * (order + 2) // 2


def _collapsed_gauss(m: int):
    """Tensor Gauss-Legendre rule on T0 through the collapsed map.

    (a, b) in [0,1]^2 -> u = a (1 - b), v = b, Jacobian (1 - b).  Exact for
    polynomials of total degree <= 2m - 2 on T0.
    """
    x, w = roots_legendre(m)
    x = 0.5 * (x + 1.0)
    w = 0.5 * w
    a, b = np.meshgrid(x, x, indexing="ij")
    wa, wb = np.meshgrid(w, w, indexing="ij")
    u = (a * (1.0 - b)).ravel()
    v = b.ravel()
    ww = (wa * wb * (1.0 - b)).ravel()
    return u, v, ww


def _basis_raw(order: int, u: np.ndarray, v: np.ndarray) -> np.ndarray:
    """Orthogonal (unnormalised) basis of P_order on T0, shape [npts, n_p].

    phi_{n,m}(u, v) = (1-v)^n P_n(2u/(1-v) - 1) * P_m^{(2n+1,0)}(2v - 1).
    The first factor is evaluated as a homogeneous polynomial so v -> 1 is safe.
    """
    u = np.asarray(u, dtype=np.float64)
    v = np.asarray(v, dtype=np.float64)
    s = 1.0 - v
    cols = []
    for n in range(order + 1):
        # (1-v)^n P_n(2u/(1-v) - 1) = sum over the Legendre coefficients of
        # P_n(t) with t = (2u - s)/s, times s^n: use the three-term recurrence
        # in homogeneous form  q_{j+1} = ((2j+1) (2u - s) q_j - j s^2 q_{j-1})/(j+1)
        q_prev = np.ones_like(u)
        q = (2.0 * u - s)
        if n == 0:
            hom = q_prev
        else:
            for j in range(1, n):
                q_prev, q = q, ((2 * j + 1) * (2.0 * u - s) * q - j * s * s * q_prev) / (j + 1)
            hom = q
        for m in range(order + 1 - n):
            cols.append(hom * eval_jacobi(m, 2 * n + 1, 0, 2.0 * v - 1.0))
    return np.stack(cols, axis=-1)


@functools.lru_cache(maxsize=None)
def _orthonormal(order: int):
    """Normalisation factors making _basis_raw orthonormal on T0."""
    u, v, w = _collapsed_gauss(order + 3)
    P = _basis_raw(order, u, v)
    nrm = np.sqrt(np.einsum("qi,qi,q->i", P, P, w))
    return 1.0 / nrm


def basis(order: int, u, v) -> np.ndarray:
    """Orthonormal basis of P_order on T0 at points (u, v): [npts, n_p]."""
    return _basis_raw(order, u, v) * _orthonormal(order)[None, :]


@functools.lru_cache(maxsize=None)
def node_rule(order: int):
    """Nodes (u, v) and weights on T0 for total degree <= order.

    Returns (uv [n_p, 2], w [n_p]) with sum(w) = 1/2 (the area of T0).
    Nodes are sorted lexicographically by (v, u) after rounding so that the
    ordering is reproducible.
    """
    n = n_nodes(order)
    if order == 0:
        return np.array([[1.0 / 3.0, 1.0 / 3.0]]), np.array([0.5])
    u, v, w = _collapsed_gauss(order + 3)
    Phi = basis(order, u, v)
    # equilateral image of T0: (u, v) -> (u + v/2, v sqrt(3)/2)
    z = (u + 0.5 * v) + 1j * (0.5 * SQ3 * v)
    M = np.einsum("qi,q,qj,q->ij", Phi, z, Phi, w)
    lam = np.linalg.eigvals(M)
    vv = lam.imag * 2.0 / SQ3
    uu = lam.real - 0.5 * vv
    uv = np.stack([uu, vv], axis=1)
    key = np.lexsort((np.round(uv[:, 0], 12), np.round(uv[:, 1], 12)))
    uv = uv[key]
    # interpolatory weights: sum_q w_q phi_b(x_q) = int_T0 phi_b
    V = basis(order, uv[:, 0], uv[:, 1])
    mom = np.einsum("qi,q->i", Phi, w)
    wts = np.linalg.solve(V.T, mom)
    assert uv.shape == (n, 2)
    return uv, wts
