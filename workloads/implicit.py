"""Closed implicit surfaces of genus 2 and 5, meshed into triangular patches
with smooth charts sampled at the node rule.

Each surface is the zero set of a smooth F with F < 0 inside, so the outward
unit normal is grad F / |grad F|.  The patches come from three steps:

1. Surface nets (Gibson 1998): sample F on a uniform grid, put one vertex
   in every grid cell whose corners change sign (the mean of the edge
   crossings), and one quad across every grid edge whose ends change sign,
   joining the four cells around that edge.  Each quad is split along its
   shorter diagonal.
2. The vertices are moved onto F = 0 by Newton steps along grad F, then
   smoothed tangentially a few times (each step re-projected).
3. Each flat triangle ABC gets the chart
       X(u, v) = P(u, v) + s(u, v) m(u, v),
   with P = A + u (B - A) + v (C - A), m the normalised blend
   (1 - u - v) n_A + u n_B + v n_C of the vertex normals, and s the root of
   F(P + s m) = 0 nearest 0.  Along an edge P and m depend only on that
   edge's two vertices, so neighbouring charts agree there and the patches
   tile the surface.  Differentiating F(X(u, v)) = 0 gives
       s_u = -grad F . (P_u + s m_u) / (grad F . m),
   and X_u = P_u + s_u m + s m_u (likewise for v).

Curvatures of an implicit surface, for the checks (Goldman 2005):
  H = (1/2) div(grad F / |grad F|)
    = (1/2) [tr Hess F / |grad F| - grad F^T Hess F grad F / |grad F|^3],
  K = -det [[Hess F, grad F], [grad F^T, 0]] / |grad F|^4,
with H = +1 and K = +1 on the unit sphere.

Surfaces:
  * ToriChain: a smooth minimum -rho log sum_k exp(-T_k / rho) of tori
    T_k = (|(x - c_k, y)| - R)^2 + z^2 - r^2 set in a row, each touching
    only its neighbours: genus = the number of tori.  The genus-2 and
    genus-5 workloads use it.
  * Genus2Lemniscate: F = (x^2 (1 - x^2) - y^2)^2 + z^2 - eps^2, a thickened
    figure-eight (lemniscate of Gerono), optionally plus a small seeded
    polynomial of degree <= 2.  At eps = 0.1 its cross-section near x = +-1
    is an ellipse of half-width 0.05 and half-height 0.1, with ridges of
    curvature radius 0.025: patches of about 0.05 do not resolve them, so it
    serves only the meshing checks.
"""
from __future__ import annotations

import itertools

import numpy as np

from .nodes import node_rule
from .surfaces import Surface


# ---------------------------------------------------------------------------
# implicit functions: F [M], grad [M, 3], hess [M, 3, 3] at points X [M, 3]

class Genus2Lemniscate:
    genus = 2

    def __init__(self, eps: float = 0.1, pert: float = 0.0, seed: int | None = None):
        self.eps = eps
        # small polynomial of degree <= 2: sum c_a x^a0 y^a1 z^a2
        self.mono = [a for a in itertools.product(range(3), repeat=3) if sum(a) <= 2]
        rng = np.random.default_rng(seed)
        self.coef = pert * rng.standard_normal(len(self.mono)) if pert else np.zeros(len(self.mono))
        self.lo = np.array([-1.2, -0.75, -0.25])
        self.hi = np.array([1.2, 0.75, 0.25])

    def _poly(self, X):
        """The perturbation's value, gradient and Hessian."""
        M = X.shape[0]
        p = np.zeros(M)
        g = np.zeros((M, 3))
        h = np.zeros((M, 3, 3))
        for c, a in zip(self.coef, self.mono):
            if c == 0.0:
                continue
            pw = [[np.ones(M), X[:, k], X[:, k] ** 2] for k in range(3)]

            def term(d):  # d: derivative order per axis
                out = np.full(M, c)
                for k in range(3):
                    e = a[k] - d[k]
                    if e < 0:
                        return np.zeros(M)
                    fac = 1.0
                    for t in range(d[k]):
                        fac *= a[k] - t
                    out = out * fac * pw[k][e]
                return out

            p += term((0, 0, 0))
            for k in range(3):
                d = [0, 0, 0]
                d[k] = 1
                g[:, k] += term(tuple(d))
                for l in range(3):
                    d2 = [0, 0, 0]
                    d2[k] += 1
                    d2[l] += 1
                    h[:, k, l] += term(tuple(d2))
        return p, g, h

    def F(self, X):
        x, y, z = X[:, 0], X[:, 1], X[:, 2]
        g = x * x * (1 - x * x) - y * y
        return g * g + z * z - self.eps ** 2 + self._poly(X)[0]

    def grad(self, X):
        x, y, z = X[:, 0], X[:, 1], X[:, 2]
        g = x * x * (1 - x * x) - y * y
        gx, gy = 2 * x - 4 * x ** 3, -2 * y
        G = np.stack([2 * g * gx, 2 * g * gy, 2 * z], axis=1)
        return G + self._poly(X)[1]

    def hess(self, X):
        x, y = X[:, 0], X[:, 1]
        g = x * x * (1 - x * x) - y * y
        gx, gy = 2 * x - 4 * x ** 3, -2 * y
        gxx, gyy = 2 - 12 * x * x, -2.0
        Hs = np.zeros((X.shape[0], 3, 3))
        Hs[:, 0, 0] = 2 * (gx * gx + g * gxx)
        Hs[:, 1, 1] = 2 * (gy * gy + g * gyy)
        Hs[:, 0, 1] = Hs[:, 1, 0] = 2 * gx * gy
        Hs[:, 2, 2] = 2.0
        return Hs + self._poly(X)[2]


class ToriChain:
    def __init__(self, n: int = 5, R: float = 1.0, r: float = 0.35, spacing: float = 2.3, rho: float = 0.15):
        self.genus = n
        self.R, self.r, self.rho = R, r, rho
        self.c = spacing * np.arange(n)
        pad = R + r + 0.3
        self.lo = np.array([self.c[0] - pad, -pad, -r - 0.3])
        self.hi = np.array([self.c[-1] + pad, pad, r + 0.3])

    def _tori(self, X, order: int = 2):
        """T_k, grad T_k, Hess T_k for every torus: [n, M], [n, M, 3], [n, M, 3, 3]
        (derivatives up to `order`)."""
        n, M = len(self.c), X.shape[0]
        T = np.empty((n, M))
        G = np.empty((n, M, 3)) if order >= 1 else None
        Hs = np.zeros((n, M, 3, 3)) if order >= 2 else None
        for k, ck in enumerate(self.c):
            x, y, z = X[:, 0] - ck, X[:, 1], X[:, 2]
            q = np.maximum(np.sqrt(x * x + y * y), 1e-300)
            a = q - self.R
            T[k] = a * a + z * z - self.r ** 2
            if order < 1:
                continue
            ex, ey = x / q, y / q
            G[k] = np.stack([2 * a * ex, 2 * a * ey, 2 * z], axis=1)
            if order < 2:
                continue
            # d(e_x)/dx = y^2 / q^3, d(e_x)/dy = -x y / q^3, d(e_y)/dy = x^2 / q^3
            q3 = q ** 3
            Hs[k, :, 0, 0] = 2 * ex * ex + 2 * a * y * y / q3
            Hs[k, :, 1, 1] = 2 * ey * ey + 2 * a * x * x / q3
            Hs[k, :, 0, 1] = Hs[k, :, 1, 0] = 2 * ex * ey - 2 * a * x * y / q3
            Hs[k, :, 2, 2] = 2.0
        return T, G, Hs

    def _weights(self, T):
        e = -T / self.rho
        e -= e.max(axis=0, keepdims=True)
        p = np.exp(e)
        return p / p.sum(axis=0, keepdims=True), e

    def F(self, X):
        T = self._tori(X, 0)[0]
        m = (-T / self.rho).max(axis=0)
        return -self.rho * (m + np.log(np.exp(-T / self.rho - m).sum(axis=0)))

    def grad(self, X):
        T, G, _ = self._tori(X, 1)
        p, _ = self._weights(T)
        return np.einsum("km,kmi->mi", p, G)

    def hess(self, X):
        T, G, Hs = self._tori(X)
        p, _ = self._weights(T)
        g = np.einsum("km,kmi->mi", p, G)
        outer = np.einsum("km,kmi,kmj->mij", p, G, G)
        return np.einsum("km,kmij->mij", p, Hs) - (outer - np.einsum("mi,mj->mij", g, g)) / self.rho


def mean_curvature(surf, X):
    g, Hs = surf.grad(X), surf.hess(X)
    gn = np.linalg.norm(g, axis=1)
    tr = np.einsum("mii->m", Hs)
    return 0.5 * (tr / gn - np.einsum("mi,mij,mj->m", g, Hs, g) / gn ** 3)


def gauss_curvature(surf, X):
    g, Hs = surf.grad(X), surf.hess(X)
    M = X.shape[0]
    B = np.zeros((M, 4, 4))
    B[:, :3, :3] = Hs
    B[:, :3, 3] = g
    B[:, 3, :3] = g
    return -np.linalg.det(B) / np.linalg.norm(g, axis=1) ** 4


# ---------------------------------------------------------------------------
# meshing

def project(surf, X, iters: int = 60, tol: float = 1e-15):
    """Newton steps x <- x - F grad F / |grad F|^2 until |F| / |grad F| < tol."""
    X = X.copy()
    for _ in range(iters):
        F, g = surf.F(X), surf.grad(X)
        g2 = np.einsum("ij,ij->i", g, g)
        step = (F / g2)[:, None] * g
        X -= step
        if np.max(np.abs(F) / np.sqrt(g2)) < tol:
            break
    return X


def surface_nets(surf, h: float, offset: float = 0.0):
    """Vertices [V, 3] and outward quads [Q, 4] of {F = 0} on a grid of
    spacing h whose points sit at lo - offset h + h Z^3."""
    lo, hi = surf.lo - offset * h, surf.hi
    n = np.ceil((hi - lo) / h).astype(int) + 1
    axes = [lo[k] + h * np.arange(n[k]) for k in range(3)]
    G = np.stack(np.meshgrid(*axes, indexing="ij"), axis=-1)
    Fg = surf.F(G.reshape(-1, 3)).reshape(tuple(n))
    Fg[Fg == 0.0] = 1e-300  # no corner exactly on the surface
    inside = Fg < 0
    if inside[0].any() or inside[-1].any() or inside[:, 0].any() or inside[:, -1].any() \
            or inside[:, :, 0].any() or inside[:, :, -1].any():
        raise ValueError("the grid box does not enclose the surface")
    # cell vertices: mean of the crossings on the cell's sign-changing edges
    nc = n - 1
    acc = np.zeros(tuple(nc) + (3,))
    cnt = np.zeros(tuple(nc))
    corners = list(itertools.product((0, 1), repeat=3))
    cell_edges = [(a, b) for a in corners for b in corners
                  if sum(abs(a[k] - b[k]) for k in range(3)) == 1 and a < b]
    sl = lambda o: tuple(slice(o[k], o[k] + nc[k]) for k in range(3))
    for a, b in cell_edges:
        Fa, Fb = Fg[sl(a)], Fg[sl(b)]
        ch = (Fa < 0) != (Fb < 0)
        t = np.where(ch, Fa / np.where(ch, Fa - Fb, 1.0), 0.0)
        pa = G[sl(a)]
        pb = G[sl(b)]
        acc += ch[..., None] * (pa + t[..., None] * (pb - pa))
        cnt += ch
    active = cnt > 0
    vid = -np.ones(tuple(nc), dtype=np.int64)
    vid[active] = np.arange(active.sum())
    V = (acc[active] / cnt[active][:, None])
    quads = []
    for ax in range(3):
        # edges along ax from grid point p to p + e_ax; the four cells around
        # it, ordered counterclockwise about +e_ax
        b1, b2 = (ax + 1) % 3, (ax + 2) % 3
        lo_idx = [slice(0, n[k]) for k in range(3)]
        lo_idx[ax] = slice(0, n[ax] - 1)
        hi_idx = list(lo_idx)
        hi_idx[ax] = slice(1, n[ax])
        Fa, Fb = Fg[tuple(lo_idx)], Fg[tuple(hi_idx)]
        ch = (Fa < 0) != (Fb < 0)
        idx = np.argwhere(ch)
        inward = (Fa < 0)[ch]  # inside at p: outward normal along +e_ax
        ring = []
        for d1, d2 in ((-1, -1), (0, -1), (0, 0), (-1, 0)):
            c = idx.copy()
            c[:, b1] += d1
            c[:, b2] += d2
            ring.append(c)
        ok = np.ones(len(idx), bool)
        for c in ring:
            ok &= np.all((c >= 0) & (c < nc[None, :]), axis=1)
        if not ok.all():
            raise ValueError("a sign change on the grid boundary")
        q = np.stack([vid[c[:, 0], c[:, 1], c[:, 2]] for c in ring], axis=1)
        q[~inward] = q[~inward][:, ::-1]
        quads.append(q)
    Q = np.concatenate(quads)
    if (Q < 0).any():
        raise ValueError("a quad references an inactive cell")
    return V, Q


def is_closed_manifold(nv, T):
    """Every directed edge once and its reverse once: a closed, consistently
    oriented 2-manifold (T may be triangles or quads)."""
    k = T.shape[1]
    e = np.concatenate([T[:, [i, (i + 1) % k]] for i in range(k)])
    key = e[:, 0] * nv + e[:, 1]
    rkey = e[:, 1] * nv + e[:, 0]
    return len(np.unique(key)) == len(key) and bool(np.isin(rkey, key).all())


def _neighbours(T, nv):
    e = np.concatenate([T[:, [0, 1]], T[:, [1, 2]], T[:, [2, 0]]])
    e = np.unique(np.sort(e, axis=1), axis=0)
    nbr = [[] for _ in range(nv)]
    for a, b in e:
        nbr[a].append(b)
        nbr[b].append(a)
    return nbr


def mesh(surf, h: float, smooth: int = 8, relax: float = 0.5):
    """Projected, smoothed vertices [V, 3] and outward triangles [T, 3].

    Surface nets can leave a non-manifold edge where the surface crosses one
    grid cell twice; the grid is then shifted by a fraction of h (a fixed
    sequence) until the quads form a closed manifold of the surface's genus."""
    for offset in (0.0, 0.37, 0.21, 0.63, 0.11, 0.83, 0.49, 0.29):
        V, Q = surface_nets(surf, h, offset)
        if is_closed_manifold(len(V), Q) and euler_characteristic(V, Q) == 2 - 2 * surf.genus:
            break
    else:
        raise ValueError(f"no manifold surface-nets mesh of spacing {h}")
    V = project(surf, V)
    # split each quad along its shorter diagonal.  Quads of surface nets are
    # often symmetric, so the two lengths can agree to the last bit, and the
    # last bits of the vertices depend on the host's exp; a near tie therefore
    # takes the 0-2 diagonal (the 1-3 one only when shorter by a relative
    # 1e-9, far above rounding), and quad q gives triangles 2 q and 2 q + 1,
    # so that the mesh, its order included, is the same on every machine.
    d02 = np.linalg.norm(V[Q[:, 0]] - V[Q[:, 2]], axis=1)
    d13 = np.linalg.norm(V[Q[:, 1]] - V[Q[:, 3]], axis=1)
    use13 = (d13 < (1.0 - 1e-9) * d02)[:, None]
    T = np.empty((2 * len(Q), 3), dtype=Q.dtype)
    T[0::2] = np.where(use13, Q[:, [0, 1, 3]], Q[:, [0, 1, 2]])
    T[1::2] = np.where(use13, Q[:, [1, 2, 3]], Q[:, [0, 2, 3]])
    nbr = _neighbours(T, len(V))
    deg = np.array([len(x) for x in nbr])
    rows = np.repeat(np.arange(len(V)), deg)
    cols = np.concatenate([np.asarray(x, dtype=np.int64) for x in nbr])
    for _ in range(smooth):
        mean = np.zeros_like(V)
        np.add.at(mean, rows, V[cols])
        mean /= deg[:, None]
        nrm = surf.grad(V)
        nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
        dv = mean - V
        dv -= np.einsum("ij,ij->i", dv, nrm)[:, None] * nrm
        V = project(surf, V + relax * dv)
    # the quads' orientation is outward by construction; a triangle folded by
    # the smoothing would show here
    A, B, C = V[T[:, 0]], V[T[:, 1]], V[T[:, 2]]
    cen = project(surf, (A + B + C) / 3.0)
    if (np.einsum("ij,ij->i", np.cross(B - A, C - A), surf.grad(cen)) <= 0).any():
        raise ValueError("a triangle is folded against the surface normal")
    return V, T


def euler_characteristic(V, T):
    k = T.shape[1]
    e = np.concatenate([T[:, [i, (i + 1) % k]] for i in range(k)])
    e = np.unique(np.sort(e, axis=1), axis=0)
    return len(V) - len(e) + len(T)


# ---------------------------------------------------------------------------
# charts

def chart(surf, A, B, C, nA, nB, nC, uv, iters: int = 60):
    """X, X_u, X_v [npatch, n_p, 3] of the normal-blend charts at the nodes uv."""
    u = uv[:, 0][None, :, None]
    v = uv[:, 1][None, :, None]
    Pu, Pv = (B - A)[:, None, :], (C - A)[:, None, :]
    P = A[:, None, :] + u * Pu + v * Pv
    mt = (1 - u - v) * nA[:, None, :] + u * nB[:, None, :] + v * nC[:, None, :]
    mn = np.linalg.norm(mt, axis=-1, keepdims=True)
    m = mt / mn
    du, dv = (nB - nA)[:, None, :], (nC - nA)[:, None, :]
    mu = (du - m * np.sum(m * du, axis=-1, keepdims=True)) / mn
    mv = (dv - m * np.sum(m * dv, axis=-1, keepdims=True)) / mn
    shp = P.shape
    P2, m2 = P.reshape(-1, 3), m.reshape(-1, 3)
    s = np.zeros(P2.shape[0])
    scale = np.max(np.abs(P2))
    for _ in range(iters):
        X2 = P2 + s[:, None] * m2
        F, g = surf.F(X2), surf.grad(X2)
        gm = np.einsum("ij,ij->i", g, m2)
        ds = F / gm
        s -= ds
        if np.max(np.abs(ds)) < 1e-15 * scale:
            break
    X2 = P2 + s[:, None] * m2
    g = surf.grad(X2)
    gm = np.einsum("ij,ij->i", g, m2)
    s = s.reshape(shp[:2])[..., None]
    X = X2.reshape(shp)
    g = g.reshape(shp)
    gm = gm.reshape(shp[:2])[..., None]
    su = -np.sum(g * (Pu + s * mu), axis=-1, keepdims=True) / gm
    sv = -np.sum(g * (Pv + s * mv), axis=-1, keepdims=True) / gm
    Xu = Pu + su * m + s * mu
    Xv = Pv + sv * m + s * mv
    return X, Xu, Xv


def implicit_surface(surf, h: float, order: int, name: str, smooth: int = 8) -> Surface:
    """A Surface of normal-blend charts over the surface-nets mesh of spacing h."""
    uv, w = node_rule(order)
    V, T = mesh(surf, h, smooth=smooth)
    nv = surf.grad(V)
    nv /= np.linalg.norm(nv, axis=1, keepdims=True)
    X, Xu, Xv = chart(surf, V[T[:, 0]], V[T[:, 1]], V[T[:, 2]], nv[T[:, 0]], nv[T[:, 1]], nv[T[:, 2]], uv)
    s = Surface(name, order, len(T), uv, w, X.reshape(-1, 3), Xu.reshape(-1, 3), Xv.reshape(-1, 3))
    s.mesh = (V, T, nv)
    s.implicit = surf
    return s


def tori_chain(n: int, h: float, order: int) -> Surface:
    """n blended tori in a row (genus n), surface-nets spacing h."""
    s = implicit_surface(ToriChain(n), h, order, f"tori{n}-h{h:g}-k{order}")
    return s
