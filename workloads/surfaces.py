"""Analytic surface charts sampled at the node rule: X, dX/du, dX/dv per node.

Each surface is a disjoint union of triangular patches Gamma_j, each with a
chart X^j : T0 -> Gamma_j (Section 4).  The library and the oracle receive the
samples (X, Xu, Xv) at the nodes of every patch, patch-major
(node index = patch * n_p + q), plus the reference rule (uv, w); everything
derived from them (normals, weights, curvature, quadrature) is theirs to
compute.  Charts are oriented so that Xu x Xv points out of the enclosed
volume.

Surfaces:
  * icosphere(level): icosahedron, each face split 4**level times (midpoints
    pushed to the sphere), every flat face radially projected onto the unit
    sphere; level 0 is the 20-face projected icosahedron;
  * ellipsoid(abc, level): the icosphere chart composed with diag(a, b, c);
  * torus(R, r, n_theta, n_phi): (theta, phi) grid, two triangles per cell;
  * twisted_torus(n_u, n_v): the doubly periodic trigonometric surface of
    Section 6.3 with its seven nonzero delta coefficients.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from .nodes import node_rule


@dataclass
class Surface:
    name: str
    order: int
    npatch: int
    uv: np.ndarray   # [n_p, 2] reference nodes on T0
    wref: np.ndarray  # [n_p] reference weights (sum 1/2)
    X: np.ndarray    # [npatch * n_p, 3]
    Xu: np.ndarray   # [npatch * n_p, 3]
    Xv: np.ndarray   # [npatch * n_p, 3]

    @property
    def np_(self) -> int:
        return self.uv.shape[0]

    @property
    def N(self) -> int:
        return self.X.shape[0]


def _icosahedron():
    t = (1.0 + np.sqrt(5.0)) / 2.0
    V = np.array([[-1, t, 0], [1, t, 0], [-1, -t, 0], [1, -t, 0],
                  [0, -1, t], [0, 1, t], [0, -1, -t], [0, 1, -t],
                  [t, 0, -1], [t, 0, 1], [-t, 0, -1], [-t, 0, 1]], dtype=np.float64)
    V /= np.linalg.norm(V, axis=1, keepdims=True)
    F = np.array([[0, 11, 5], [0, 5, 1], [0, 1, 7], [0, 7, 10], [0, 10, 11],
                  [1, 5, 9], [5, 11, 4], [11, 10, 2], [10, 7, 6], [7, 1, 8],
                  [3, 9, 4], [3, 4, 2], [3, 2, 6], [3, 6, 8], [3, 8, 9],
                  [4, 9, 5], [2, 4, 11], [6, 2, 10], [8, 6, 7], [9, 8, 1]], dtype=np.int64)
    return V, F


def icosphere_faces(level: int):
    """Vertices on the unit sphere and outward-oriented triangles."""
    V, F = _icosahedron()
    V = [v for v in V]
    for _ in range(level):
        cache = {}
        newF = []

        def mid(a, b):
            key = (min(a, b), max(a, b))
            if key not in cache:
                m = V[a] + V[b]
                V.append(m / np.linalg.norm(m))
                cache[key] = len(V) - 1
            return cache[key]

        for a, b, c in F:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            newF += [[a, ab, ca], [b, bc, ab], [c, ca, bc], [ab, bc, ca]]
        F = np.array(newF, dtype=np.int64)
    V = np.array(V)
    # orient outward
    A, B, C = V[F[:, 0]], V[F[:, 1]], V[F[:, 2]]
    nrm = np.cross(B - A, C - A)
    flip = np.einsum("ij,ij->i", nrm, A + B + C) < 0
    F[flip] = F[flip][:, [0, 2, 1]]
    return V, F


def _sphere_chart(A, B, C, uv):
    """Radial projection of the flat triangle ABC: samples of X, Xu, Xv."""
    u = uv[:, 0][None, :, None]
    v = uv[:, 1][None, :, None]
    e1 = (B - A)[:, None, :]
    e2 = (C - A)[:, None, :]
    P = A[:, None, :] + u * e1 + v * e2
    rho = np.linalg.norm(P, axis=-1, keepdims=True)
    X = P / rho
    Xu = (e1 - X * np.sum(X * e1, axis=-1, keepdims=True)) / rho
    Xv = (e2 - X * np.sum(X * e2, axis=-1, keepdims=True)) / rho
    return X.reshape(-1, 3), Xu.reshape(-1, 3), Xv.reshape(-1, 3)


def icosphere(level: int, order: int) -> Surface:
    uv, w = node_rule(order)
    V, F = icosphere_faces(level)
    X, Xu, Xv = _sphere_chart(V[F[:, 0]], V[F[:, 1]], V[F[:, 2]], uv)
    return Surface(f"icosphere{level}", order, len(F), uv, w, X, Xu, Xv)


def ellipsoid(abc, level: int, order: int) -> Surface:
    s = icosphere(level, order)
    D = np.asarray(abc, dtype=np.float64)[None, :]
    return Surface(f"ellipsoid{tuple(abc)}-{level}", order, s.npatch, s.uv, s.wref,
                   s.X * D, s.Xu * D, s.Xv * D)


def torus(R: float, r: float, n_theta: int, n_phi: int, order: int) -> Surface:
    uv, w = node_rule(order)
    dth = 2 * np.pi / n_theta
    dph = 2 * np.pi / n_phi
    Xs, Xus, Xvs = [], [], []
    u = uv[:, 0]
    v = uv[:, 1]
    for i in range(n_theta):
        for j in range(n_phi):
            for lower in (True, False):
                if lower:
                    th = i * dth + u * dth
                    ph = j * dph + v * dph
                    su, sv = dth, dph
                else:
                    th = (i + 1) * dth - u * dth
                    ph = (j + 1) * dph - v * dph
                    su, sv = -dth, -dph
                rr = R + r * np.cos(ph)
                X = np.stack([rr * np.cos(th), rr * np.sin(th), r * np.sin(ph)], axis=1)
                Xth = np.stack([-rr * np.sin(th), rr * np.cos(th), 0 * th], axis=1)
                Xph = np.stack([-r * np.sin(ph) * np.cos(th), -r * np.sin(ph) * np.sin(th),
                                r * np.cos(ph)], axis=1)
                Xs.append(X)
                Xus.append(su * Xth)
                Xvs.append(sv * Xph)
    return Surface(f"torus({R},{r})", order, 2 * n_theta * n_phi, uv, w,
                   np.concatenate(Xs), np.concatenate(Xus), np.concatenate(Xvs))


# nonzero coefficients delta_{i,j} of the twisted torus (Section 6.3)
TWISTED_DELTA = {(-1, -1): 0.17, (-1, 0): 0.11, (0, 0): 1.0, (1, 0): 4.5,
                 (2, 0): -0.25, (0, 1): 0.01, (2, 1): -0.45}


def _twisted(s, t):
    """X(s, t) and its two partial derivatives for the twisted torus."""
    X = np.zeros(s.shape + (3,))
    Xs = np.zeros_like(X)
    Xt = np.zeros_like(X)
    for (i, j), d in TWISTED_DELTA.items():
        a = (1 - i) * s + j * t
        ca, sa = np.cos(a), np.sin(a)
        ct, st = np.cos(t), np.sin(t)
        X += d * np.stack([ct * ca, st * ca, sa], axis=-1)
        # d/ds: only a depends on s, da/ds = 1 - i
        Xs += d * (1 - i) * np.stack([-ct * sa, -st * sa, ca], axis=-1)
        # d/dt: da/dt = j, plus the explicit cos t / sin t
        Xt += d * np.stack([-st * ca - j * ct * sa, ct * ca - j * st * sa, j * ca], axis=-1)
    return X, Xs, Xt


def twisted_torus(n_u: int, n_v: int, order: int) -> Surface:
    uv, w = node_rule(order)
    du = 2 * np.pi / n_u
    dv = 2 * np.pi / n_v

    def build(swap: bool):
        a = uv[:, 1] if swap else uv[:, 0]
        b = uv[:, 0] if swap else uv[:, 1]
        Xs, Xus, Xvs = [], [], []
        for i in range(n_u):
            for j in range(n_v):
                for sgn, s0, t0 in ((1.0, i * du, j * dv), (-1.0, (i + 1) * du, (j + 1) * dv)):
                    s = s0 + sgn * a * du
                    t = t0 + sgn * b * dv
                    X, Xs_, Xt_ = _twisted(s, t)
                    # d(s,t)/d(u,v): s depends on a, t on b
                    ds = sgn * du * Xs_
                    dt = sgn * dv * Xt_
                    Xs.append(X)
                    Xus.append(dt if swap else ds)
                    Xvs.append(ds if swap else dt)
        return np.concatenate(Xs), np.concatenate(Xus), np.concatenate(Xvs)

    X, Xu, Xv = build(False)
    # orient outward: the signed volume (1/3) sum w x.n must be positive
    wq = np.tile(w, 2 * n_u * n_v)
    if np.sum(wq * np.einsum("ij,ij->i", X, np.cross(Xu, Xv))) < 0:
        X, Xu, Xv = build(True)
    return Surface("twisted_torus", order, 2 * n_u * n_v, uv, w, X, Xu, Xv)
