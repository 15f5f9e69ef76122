"""Discrete layer potentials and the Laplace-Beltrami operators (oracle, FP64).

Test infrastructure only (see oracle/__init__.py).

A discretised potential at node i is the far sum over sources outside
Near(i) plus the near-field correction sum over the patches in Near(i)
(Section 4, the corrected Nystrom form):
    K[sigma]_i = sum_{far j} w_j K(x_i, x_j) sigma_j + sum_{P in Near(i)} sum_q W^K_{i,P}[q] sigma_{P,q}.

Operators (Section 3, Section 4.2 / 4.3), W[f] = sum_j w_j f_j / sum_j w_j:
  A3 tau = -tau/4 + S'[mu1] - (S''+D')[mu2] - 2 H S'[mu2] + W S[mu2],
           mu1 = S' tau, mu2 = S tau;             solve A3 sigma = f,  u = S[S[sigma]]
  A2 tau = -tau/4 + D[mu1] + S[mu2],
           mu1 = D tau, mu2 = -(S''+D') tau - 2 H S' tau + W S tau;
                                                 solve A2 sigma = S[f], u = S[sigma]
(The printed A2 combination carries "- D[mu1]"; since the operator contains
+D^2 this implementation reads it as + D[mu1].  The A2 right-hand side is
S[f], as in the equation the operator comes from.)
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import farsum
from .geometry import Geometry, near_lists, surface_gradient
from .quadrature import build_corrections

K_S, K_D, K_SP, K_SD = 0, 1, 2, 3


@dataclass
class Discretisation:
    geo: Geometry
    near_ptr: np.ndarray
    near_patch: np.ndarray
    vals: np.ndarray        # [nnzb, 4, n_p] near-field weights
    eta: float
    eps_q: float
    far: object = None      # geometry.FarRule: oversampled far-field sources (Section 4), or None

    def near_apply(self, sigma: np.ndarray, targets=None) -> np.ndarray:
        """Correction sums [nrhs, 4, ntargets] from the block CSR: for target
        i, sum over its blocks b of vals[b] (4 x n_p) times the density on
        patch near_patch[b] (a plain loop in the oracle's C helper)."""
        return farsum.near_sums(self.geo, self.near_ptr, self.near_patch, self.vals, sigma, targets)

    def potentials(self, sigma: np.ndarray, targets=None) -> np.ndarray:
        """All four discretised potentials: [nrhs, 4, ntargets]."""
        return farsum.far_sums(self.geo, self.near_ptr, self.near_patch, sigma, targets, far=self.far) + \
            self.near_apply(sigma, targets)

    def wmean(self, f: np.ndarray) -> np.ndarray:
        """W[f] = sum w f / sum w for each row of f [nrhs, N]."""
        return np.atleast_2d(f) @ self.geo.w / self.geo.w.sum()

    # --- operators ------------------------------------------------------
    def apply_A3(self, tau: np.ndarray) -> np.ndarray:
        tau = np.atleast_2d(tau)
        p1 = self.potentials(tau)
        mu1 = p1[:, K_SP]
        mu2 = p1[:, K_S]
        q1 = self.potentials(mu1)
        q2 = self.potentials(mu2)
        H = self.geo.H[None, :]
        eta = self.wmean(q2[:, K_S])[:, None]
        return -0.25 * tau + q1[:, K_SP] - q2[:, K_SD] - 2.0 * H * q2[:, K_SP] + eta

    def apply_A2(self, tau: np.ndarray) -> np.ndarray:
        tau = np.atleast_2d(tau)
        p = self.potentials(tau)
        H = self.geo.H[None, :]
        mu1 = p[:, K_D]
        mu2 = -p[:, K_SD] - 2.0 * H * p[:, K_SP] + self.wmean(p[:, K_S])[:, None]
        q1 = self.potentials(mu1)
        q2 = self.potentials(mu2)
        return -0.25 * tau + q1[:, K_D] + q2[:, K_S]

    def apply_A1(self, tau: np.ndarray) -> np.ndarray:
        """A1 = div S grad_Gamma S + S W S (Section 4.1, eq. ie-dis0), applied
        right to left: s = S[tau]; mu = grad_Gamma s; the divergence of the
        vector single layer of mu, sum_l d_l S[mu_l], with the principal-value
        gradient d_l S[sigma] = n_l S'[sigma] + (grad_Gamma S[sigma])_l; plus
        W[s] S[1]."""
        tau = np.atleast_2d(tau)
        geo = self.geo
        nr = tau.shape[0]
        s = self.S(tau)                                        # [r, N]
        mu = surface_gradient(geo, s.T)                        # [N, r, 3]
        P = self.potentials(mu.transpose(1, 2, 0).reshape(nr * 3, geo.N))   # [r*3, 4, N]
        g = surface_gradient(geo, P[:, K_S].T).reshape(geo.N, nr, 3, 3)     # [N, r, l, 3]
        Sp = P[:, K_SP].reshape(nr, 3, geo.N)
        out = np.zeros_like(tau)
        for l in range(3):
            out += geo.n[None, :, l] * Sp[:, l] + g[:, :, l, l].T
        one = self.S(np.ones(geo.N))[0]
        return out + self.wmean(s)[:, None] * one[None, :]

    def apply(self, formulation: str, tau):
        if formulation == "A1":
            return self.apply_A1(tau)
        return self.apply_A3(tau) if formulation == "A3" else self.apply_A2(tau)

    def S(self, sigma):
        return self.potentials(sigma)[:, K_S]

    def project_mean_zero(self, f):
        f = np.atleast_2d(f)
        return f - self.wmean(f)[:, None]

    def rhs(self, formulation: str, f):
        f0 = self.project_mean_zero(f)
        return f0 if formulation == "A3" else self.S(f0)   # A1 and A2 take S[f]

    def solution(self, formulation: str, sigma):
        s = self.S(sigma)
        return self.S(s) if formulation == "A3" else s


def discretise(order, uv, wref, X, Xu, Xv, eta: float = 2.0, eps_q: float = 1e-12,
               workers: int = 1, geo: Geometry | None = None) -> Discretisation:
    from .geometry import build_geometry
    if geo is None:
        geo = build_geometry(order, uv, wref, X, Xu, Xv)
    ptr, pl = near_lists(geo, eta)
    vals, _ = build_corrections(geo, ptr, pl, eps_q=eps_q, workers=workers)
    return Discretisation(geo, ptr, pl, vals, eta, eps_q)
