"""GMRES and dense solves for the discretised operators (oracle, FP64).

Test infrastructure only (see oracle/__init__.py).

GMRES (Saad & Schultz) as used in Section 6: x0 = 0, Arnoldi with modified
Gram-Schmidt, Givens rotations on the Hessenberg matrix, no restart, stop
when the estimated relative residual |b - A x|_2 / |b|_2 drops below tol or
after max_iter iterations (the paper caps at 100).  Euclidean inner product.
"""
from __future__ import annotations

import numpy as np


def gmres(apply, b: np.ndarray, tol: float = 1e-10, max_iter: int = 100):
    """Solve A x = b for one right-hand side; returns (x, iterations, residual history)."""
    b = np.asarray(b, dtype=np.float64)
    beta = np.linalg.norm(b)
    if beta == 0.0:
        return np.zeros_like(b), 0, [0.0]
    n = b.shape[0]
    V = np.zeros((max_iter + 1, n))
    Hm = np.zeros((max_iter + 1, max_iter))
    cs = np.zeros(max_iter)
    sn = np.zeros(max_iter)
    g = np.zeros(max_iter + 1)
    g[0] = beta
    V[0] = b / beta
    hist = [1.0]
    k = 0
    for j in range(max_iter):
        w = apply(V[j])
        for i in range(j + 1):                       # modified Gram-Schmidt
            Hm[i, j] = np.dot(V[i], w)
            w = w - Hm[i, j] * V[i]
        Hm[j + 1, j] = np.linalg.norm(w)
        if Hm[j + 1, j] > 0.0:
            V[j + 1] = w / Hm[j + 1, j]
        for i in range(j):                           # previous rotations
            t = cs[i] * Hm[i, j] + sn[i] * Hm[i + 1, j]
            Hm[i + 1, j] = -sn[i] * Hm[i, j] + cs[i] * Hm[i + 1, j]
            Hm[i, j] = t
        r = np.hypot(Hm[j, j], Hm[j + 1, j])         # new rotation
        cs[j] = Hm[j, j] / r
        sn[j] = Hm[j + 1, j] / r
        Hm[j, j] = r
        Hm[j + 1, j] = 0.0
        g[j + 1] = -sn[j] * g[j]
        g[j] = cs[j] * g[j]
        k = j + 1
        hist.append(abs(g[j + 1]) / beta)
        if hist[-1] < tol or Hm[j + 1, j] == 0.0 and r == 0.0:
            break
    y = np.linalg.solve(np.triu(Hm[:k, :k]), g[:k])
    x = V[:k].T @ y
    return x, k, hist


def dense_matrix(apply, n: int) -> np.ndarray:
    """Assemble the matrix of a linear operator column by column."""
    A = np.zeros((n, n))
    eye = np.eye(n)
    for c in range(0, n, 64):
        cols = apply(eye[c:c + 64])
        A[:, c:c + cols.shape[0]] = cols.T
    return A


def solve_lb(disc, f, formulation: str = "A3", tol: float = 1e-10, max_iter: int = 100):
    """Mean-zero Laplace-Beltrami solve through A2 or A3 (Section 3, Table 2).

    f is projected to weighted mean zero first (Lemma 1).  Returns
    (u, sigma, iterations, residual history).
    """
    b = disc.rhs(formulation, f)[0]
    sigma, it, hist = gmres(lambda x: disc.apply(formulation, x)[0], b, tol, max_iter)
    u = disc.solution(formulation, sigma)[0]
    return u, sigma, it, hist
