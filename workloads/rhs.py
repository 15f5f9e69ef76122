"""Seeded right-hand sides sampled at surface nodes (inputs only).

Every generator takes node positions and a numpy Generator; none of them
projects to mean zero or applies any layer potential (that is the solver's
job, Lemma 1 / Section 3).
"""
from __future__ import annotations

import numpy as np
from scipy.special import eval_legendre


def y32(X: np.ndarray) -> np.ndarray:
    """Real spherical harmonic of degree 3, order 2: (x^2 - y^2) z, normalised.

    On the unit sphere Delta_Gamma Y = -3*4 Y = -12 Y, so the mean-zero
    solution of Delta_Gamma u = Y is u = -Y/12 (Section 6.1, the analytic
    solution u = -c Y/(n(n+1)) with a single mode).
    """
    x, y, z = X[:, 0], X[:, 1], X[:, 2]
    return 0.25 * np.sqrt(105.0 / np.pi) * (x * x - y * y) * z


def gaussian_bumps(X: np.ndarray, rng: np.random.Generator, count: int = 8,
                   width2: float = 0.1) -> np.ndarray:
    """sum_i a_i exp(-|x - c_i|^2 / width2), a_i ~ N(0,1), c_i = distinct nodes."""
    a = rng.standard_normal(count)
    idx = rng.choice(X.shape[0], size=count, replace=False)
    C = X[idx]
    d2 = np.sum((X[:, None, :] - C[None, :, :]) ** 2, axis=-1)
    return np.exp(-d2 / width2) @ a


def legendre_field(X: np.ndarray, rng: np.random.Generator, degree: int, L: float,
                   ncomp: int = 1) -> np.ndarray:
    """Random scaled tensor-product Legendre polynomial(s) (Section 5).

    Each component is sum_{l+m+n <= degree} c_lmn P_l(x/2L) P_m(y/2L) P_n(z/2L)
    with c_lmn ~ N(0,1).  Returns [N] for ncomp == 1 else [N, ncomp].
    """
    s = X / (2.0 * L)
    Px = [eval_legendre(l, s[:, 0]) for l in range(degree + 1)]
    Py = [eval_legendre(l, s[:, 1]) for l in range(degree + 1)]
    Pz = [eval_legendre(l, s[:, 2]) for l in range(degree + 1)]
    out = np.zeros((X.shape[0], ncomp))
    for c in range(ncomp):
        for l in range(degree + 1):
            for m in range(degree + 1 - l):
                for n in range(degree + 1 - l - m):
                    out[:, c] += rng.standard_normal() * Px[l] * Py[m] * Pz[n]
    return out[:, 0] if ncomp == 1 else out


def current_source_field(X: np.ndarray, x0=(0.2, 0.2, 0.2), ell=(0.0, 1.0, 1.0)) -> np.ndarray:
    """V = ell x (x - x0)/|x - x0|^3, the point current of Section 6.3: [N, 3]."""
    d = X - np.asarray(x0)[None, :]
    r3 = np.sum(d * d, axis=1) ** 1.5
    return np.cross(np.asarray(ell, dtype=np.float64)[None, :], d) / r3[:, None]
