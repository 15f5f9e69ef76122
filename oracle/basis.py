"""Polynomial spaces on the reference triangle T0 (oracle, FP64).

The oracle is test infrastructure: only tests, the smoke check and the CPU
baseline leg of the benchmark may import it.  It shares no code with the
CUDA library.

A chart component, its tangents and every density are represented on a patch
by their samples at the n_p = (k+1)(k+2)/2 nodes, i.e. by the unique
polynomial of total degree <= k through them (Section 4, order-p
discretisation).  This module provides an orthonormal basis of that space
(the collapsed-coordinate Jacobi products of Koornwinder/Dubiner) with
analytic first derivatives, and from it:

  * the Vandermonde matrix V_qb = phi_b(node_q) and its inverse,
  * Lagrange values l_q(p) = sum_b phi_b(p) (V^-1)_bq at any point p,
  * nodal differentiation matrices D_u = V_u V^-1, D_v = V_v V^-1 (the
    "spectral differentiation" used for second derivatives of the chart,
    Section 4, and for surface gradients / divergences, Section 2).
"""
from __future__ import annotations

import numpy as np


def jacobi_table(mmax: int, alpha: int, x: np.ndarray):
    """P_m^{(alpha,0)}(x) and d/dx for m = 0..mmax by the three-term recurrence.

    2m(m+a)(2m+a-2) P_m = (2m+a-1)[(2m+a)(2m+a-2) x + a^2] P_{m-1}
                          - 2(m+a-1)(m-1)(2m+a) P_{m-2}      (beta = 0),
    differentiated term by term for the derivative.  Returns two lists.
    """
    a = float(alpha)
    P = [np.ones_like(x)]
    dP = [np.zeros_like(x)]
    if mmax >= 1:
        P.append(0.5 * ((a + 2.0) * x + a))
        dP.append(np.full_like(x, 0.5 * (a + 2.0)))
    for m in range(2, mmax + 1):
        c0 = 2.0 * m * (m + a) * (2 * m + a - 2)
        c1 = (2 * m + a - 1) * (2 * m + a) * (2 * m + a - 2)
        c2 = (2 * m + a - 1) * a * a
        c3 = 2.0 * (m + a - 1) * (m - 1) * (2 * m + a)
        P.append(((c1 * x + c2) * P[m - 1] - c3 * P[m - 2]) / c0)
        dP.append((c1 * P[m - 1] + (c1 * x + c2) * dP[m - 1] - c3 * dP[m - 2]) / c0)
    return P, dP


def eval_basis(k: int, u, v, derivs: bool = False):
    """Orthonormal basis of P_k on T0 at points (u, v).

    phi_{n,m} = c_{n,m} * A_n(u, v) * B_{n,m}(v), n + m <= k, where
      A_n = (1-v)^n P_n((2u - (1-v))/(1-v))  (a polynomial of degree n),
      B_{n,m} = P_m^{(2n+1,0)}(2v - 1),
      c_{n,m} = sqrt(2 (2n+1) (n+m+1))  (so that int_T0 phi^2 = 1).
    A_n obeys the homogeneous Legendre recurrence
      A_{j+1} = ((2j+1) A_1 A_j - j s^2 A_{j-1}) / (j+1),  s = 1 - v,
    which is differentiated term by term.  Returns phi [P, n_p] and, if
    derivs, (phi, phi_u, phi_v).  Column order: n outer, m inner.
    """
    u = np.asarray(u, dtype=np.float64)
    v = np.asarray(v, dtype=np.float64)
    s = 1.0 - v
    A1 = 2.0 * u - s
    A = [np.ones_like(u), A1]
    Au = [np.zeros_like(u), np.full_like(u, 2.0)]
    Av = [np.zeros_like(u), np.ones_like(u)]
    for j in range(1, k):
        A.append(((2 * j + 1) * A1 * A[j] - j * s * s * A[j - 1]) / (j + 1))
        Au.append(((2 * j + 1) * (2.0 * A[j] + A1 * Au[j]) - j * s * s * Au[j - 1]) / (j + 1))
        Av.append(((2 * j + 1) * (A[j] + A1 * Av[j])
                   - j * (-2.0 * s * A[j - 1] + s * s * Av[j - 1])) / (j + 1))
    x = 2.0 * v - 1.0
    nb = (k + 1) * (k + 2) // 2
    # filled column by column in a [n_p, ...] buffer, returned as a [..., n_p] view
    phi = np.empty((nb,) + u.shape)
    if derivs:
        phu = np.empty_like(phi)
        phv = np.empty_like(phi)
    col = 0
    for n in range(k + 1):
        B, dB = jacobi_table(k - n, 2 * n + 1, x)
        for m in range(k + 1 - n):
            c = np.sqrt(2.0 * (2 * n + 1) * (n + m + 1))
            np.multiply(c * A[n], B[m], out=phi[col])
            if derivs:
                np.multiply(c * Au[n], B[m], out=phu[col])
                phv[col] = c * (Av[n] * B[m] + A[n] * 2.0 * dB[m])
            col += 1
    phi = np.moveaxis(phi, 0, -1)
    if not derivs:
        return phi
    return phi, np.moveaxis(phu, 0, -1), np.moveaxis(phv, 0, -1)


def eval_basis_diff(k: int, ua: float, va: float, du, dv):
    """Basis at p = a + (du, dv) together with phi_b(p) - phi_b(a), free of cancellation.

    The differences are carried through the same recurrences with the product
    rule  D(PQ) = DP Q(p) + P(a) DQ, starting from D u = du, D v = dv, so that
    they keep full relative accuracy when p is close to a.  Returns
    (phi(p), phi_u(p), phi_v(p), dphi) with shapes [P, n_p].
    """
    du = np.asarray(du, dtype=np.float64)
    dv = np.asarray(dv, dtype=np.float64)
    u = ua + du
    v = va + dv
    phi, phu, phv = eval_basis(k, u, v, derivs=True)
    # values at a (scalars) and differences (arrays)
    sa, sp = 1.0 - va, 1.0 - v
    ds = -dv
    A1a, A1p, dA1 = 2.0 * ua - sa, 2.0 * u - sp, 2.0 * du + dv
    Aa = [1.0, A1a]
    Ap = [np.ones_like(u), A1p]
    dA = [np.zeros_like(u), dA1]
    ds2 = ds * (sp + sa)
    for j in range(1, k):
        c1, c2 = 2 * j + 1, j
        Aa.append((c1 * A1a * Aa[j] - c2 * sa * sa * Aa[j - 1]) / (j + 1))
        Ap.append((c1 * A1p * Ap[j] - c2 * sp * sp * Ap[j - 1]) / (j + 1))
        d_prod = dA1 * Ap[j] + A1a * dA[j]
        d_s2A = ds2 * Ap[j - 1] + sa * sa * dA[j - 1]
        dA.append((c1 * d_prod - c2 * d_s2A) / (j + 1))
    xa, xp, dx = 2.0 * va - 1.0, 2.0 * v - 1.0, 2.0 * dv
    out = np.empty(u.shape + ((k + 1) * (k + 2) // 2,))
    col = 0
    for n in range(k + 1):
        al = 2.0 * n + 1.0
        Pa = [1.0, 0.5 * ((al + 2.0) * xa + al)]
        Pp = [np.ones_like(u), 0.5 * ((al + 2.0) * xp + al)]
        dP = [np.zeros_like(u), 0.5 * (al + 2.0) * dx]
        for m in range(2, k - n + 1):
            c0 = 2.0 * m * (m + al) * (2 * m + al - 2)
            ca = (2 * m + al - 1) * (2 * m + al) * (2 * m + al - 2)
            cb = (2 * m + al - 1) * al * al
            cc = 2.0 * (m + al - 1) * (m - 1) * (2 * m + al)
            Pa.append(((ca * xa + cb) * Pa[m - 1] - cc * Pa[m - 2]) / c0)
            Pp.append(((ca * xp + cb) * Pp[m - 1] - cc * Pp[m - 2]) / c0)
            dP.append((ca * dx * Pp[m - 1] + (ca * xa + cb) * dP[m - 1] - cc * dP[m - 2]) / c0)
        for m in range(k + 1 - n):
            c = np.sqrt(2.0 * (2 * n + 1) * (n + m + 1))
            out[..., col] = c * (dA[n] * Pp[m] + Aa[n] * dP[m])
            col += 1
    return phi, phu, phv, out


class NodalBasis:
    """Interpolation and differentiation on T0 for a given node set."""

    def __init__(self, k: int, uv: np.ndarray):
        self.k = k
        self.uv = np.asarray(uv, dtype=np.float64)
        self.np_ = self.uv.shape[0]
        if self.np_ != (k + 1) * (k + 2) // 2:
            raise ValueError("node count does not match the order")
        V, Vu, Vv = eval_basis(k, self.uv[:, 0], self.uv[:, 1], derivs=True)
        self.V = V
        self.Vinv = np.linalg.inv(V)
        self.Du = Vu @ self.Vinv
        self.Dv = Vv @ self.Vinv

    def lagrange(self, u, v) -> np.ndarray:
        """Lagrange basis values [P, n_p] at points (u, v)."""
        return eval_basis(self.k, u, v) @ self.Vinv
