"""Genus-2 and genus-5 surfaces: meshing, charts and curvature (CPU only).

The meshes are pinned by topology (closed, consistently oriented
2-manifolds whose Euler characteristic is 2 - 2g), the charts by the implicit
equation, by finite differences and by agreement along shared edges, and the
oracle's geometry on them by the Gauss-Bonnet theorem (the integral of K is
2 pi (2 - 2g)) and by the closed-form mean curvature of a level set.  The
curvature formulas themselves are pinned on a plain torus, whose curvatures
are known in closed form, and against finite differences of the unit normal.
The oracle's layer potentials on the genus-2 surface meet the Gauss and
Green identities at sampled targets.
"""
import numpy as np
import pytest

from workloads import implicit as I
from workloads import surfaces as S


@pytest.fixture(scope="module")
def chain2():
    return I.tori_chain(2, 0.2, 6)


def test_euler_characteristic_of_known_meshes():
    V, F = S.icosphere_faces(1)
    assert I.is_closed_manifold(len(V), F) and I.euler_characteristic(V, F) == 2
    # an m x n torus grid, two triangles per cell
    m, n = 5, 7
    idx = lambda i, j: (i % m) * n + (j % n)
    T = []
    for i in range(m):
        for j in range(n):
            T += [[idx(i, j), idx(i + 1, j), idx(i + 1, j + 1)], [idx(i, j), idx(i + 1, j + 1), idx(i, j + 1)]]
    T = np.array(T)
    assert I.is_closed_manifold(m * n, T) and I.euler_characteristic(np.zeros((m * n, 3)), T) == 0
    # a flipped triangle breaks the orientation check
    T[0] = T[0][[0, 2, 1]]
    assert not I.is_closed_manifold(m * n, T)


@pytest.mark.parametrize("surf,h", [(I.ToriChain(2), 0.2), (I.ToriChain(5), 0.15),
                                    (I.Genus2Lemniscate(0.1, 1e-3, 1004), 0.04)])
def test_mesh_is_a_closed_manifold_of_the_surface_genus(surf, h):
    V, T = I.mesh(surf, h)
    assert I.is_closed_manifold(len(V), T)
    assert I.euler_characteristic(V, T) == 2 - 2 * surf.genus
    assert np.abs(surf.F(V) / np.linalg.norm(surf.grad(V), axis=1)).max() < 1e-13


def test_curvature_formulas_on_a_torus():
    """A single torus of the chain (no blending): K = cos p / (r (R + r cos p)),
    H = (R + 2 r cos p) / (2 r (R + r cos p)); also H against finite
    differences of the unit normal of the blended chain."""
    R, r = 1.0, 0.35
    surf = I.ToriChain(1, R=R, r=r)
    rng = np.random.default_rng(0)
    th, ph = rng.uniform(0, 2 * np.pi, 50), rng.uniform(0, 2 * np.pi, 50)
    X = np.stack([(R + r * np.cos(ph)) * np.cos(th), (R + r * np.cos(ph)) * np.sin(th), r * np.sin(ph)], axis=1)
    K = np.cos(ph) / (r * (R + r * np.cos(ph)))
    H = (R + 2 * r * np.cos(ph)) / (2 * r * (R + r * np.cos(ph)))
    assert np.abs(I.gauss_curvature(surf, X) - K).max() < 1e-12
    assert np.abs(I.mean_curvature(surf, X) - H).max() < 1e-12
    chain = I.ToriChain(2)
    P = I.mesh(chain, 0.2)[0][::7]
    nrm = lambda Y: chain.grad(Y) / np.linalg.norm(chain.grad(Y), axis=1, keepdims=True)
    e = 1e-6
    div = sum((nrm(P + e * np.eye(3)[k])[:, k] - nrm(P - e * np.eye(3)[k])[:, k]) / (2 * e) for k in range(3))
    assert np.abs(0.5 * div - I.mean_curvature(chain, P)).max() < 1e-6


def test_charts_lie_on_the_surface_and_point_outward(chain2):
    s, surf = chain2, chain2.implicit
    g = surf.grad(s.X)
    assert np.abs(surf.F(s.X) / np.linalg.norm(g, axis=1)).max() < 1e-13
    n = np.cross(s.Xu, s.Xv)
    assert (np.einsum("ij,ij->i", n, g) > 0).all()
    # X_u and X_v are tangent: grad F . X_u = 0
    gn = g / np.linalg.norm(g, axis=1, keepdims=True)
    for D in (s.Xu, s.Xv):
        assert np.abs(np.einsum("ij,ij->i", gn, D)).max() < 1e-12 * np.abs(D).max()


def test_chart_derivatives_match_finite_differences(chain2):
    s, surf = chain2, chain2.implicit
    V, T, nv = s.mesh
    sel = np.arange(0, s.npatch, 37)
    args = [V[T[sel, 0]], V[T[sel, 1]], V[T[sel, 2]], nv[T[sel, 0]], nv[T[sel, 1]], nv[T[sel, 2]]]
    e = 1e-6
    X0, Xu, Xv = I.chart(surf, *args, s.uv)
    for k, D in ((0, Xu), (1, Xv)):
        du = np.zeros(2)
        du[k] = e
        Xp = I.chart(surf, *args, s.uv + du)[0]
        Xm = I.chart(surf, *args, s.uv - du)[0]
        assert np.abs((Xp - Xm) / (2 * e) - D).max() < 1e-6 * np.abs(D).max()
    assert np.abs(X0.reshape(-1, 3) - s.X.reshape(s.npatch, -1, 3)[sel].reshape(-1, 3)).max() == 0.0


def test_neighbouring_charts_agree_on_shared_edges(chain2):
    """Points at t = 0.2, 0.5, 0.8 along each mesh edge, from both triangles."""
    s, surf = chain2, chain2.implicit
    V, T, nv = s.mesh
    ts = np.array([0.2, 0.5, 0.8])
    pts = {}
    for a in range(3):   # local edge a -> a + 1
        b = (a + 1) % 3
        bary = np.zeros((3, 3))
        bary[:, a] = 1 - ts
        bary[:, b] = ts
        uv = bary[:, 1:]   # (u, v) = weights of vertices 1, 2
        X = I.chart(surf, V[T[:, 0]], V[T[:, 1]], V[T[:, 2]], nv[T[:, 0]], nv[T[:, 1]], nv[T[:, 2]], uv)[0]
        for p in range(len(T)):
            va, vb = T[p, a], T[p, b]
            key = (min(va, vb), max(va, vb))
            Y = X[p] if va < vb else X[p][::-1]   # ordered from the smaller vertex id
            pts.setdefault(key, []).append(Y)
    assert all(len(v) == 2 for v in pts.values())
    gap = max(np.abs(v[0] - v[1]).max() for v in pts.values())
    assert gap < 1e-13


@pytest.mark.parametrize("n,h", [(2, 0.2), (5, 0.15)])
def test_gauss_bonnet_with_oracle_weights(n, h):
    from oracle.geometry import build_geometry
    s = I.tori_chain(n, h, 6)
    g = build_geometry(s.order, s.uv, s.wref, s.X, s.Xu, s.Xv)
    total = np.sum(g.w * I.gauss_curvature(s.implicit, s.X))
    chi = 2 - 2 * n
    assert abs(total - 2 * np.pi * chi) < 1e-5 * 2 * np.pi * abs(chi)


def test_oracle_mean_curvature_converges_to_the_level_set_formula():
    from oracle.geometry import build_geometry
    errs = []
    for h in (0.2, 0.12):
        s = I.tori_chain(2, h, 6)
        g = build_geometry(s.order, s.uv, s.wref, s.X, s.Xu, s.Xv)
        errs.append(np.abs(g.H - I.mean_curvature(s.implicit, s.X)).max())
    assert errs[0] < 2e-2
    assert errs[1] < errs[0] / 5


def test_genus2_and_genus5_workloads():
    from workloads.configs import config
    w = config(4)
    s = w.surface
    V, T, _ = s.mesh
    assert 3800 <= s.npatch <= 4400 and s.N == 28 * s.npatch
    assert I.euler_characteristic(V, T) == -2
    assert w.f.shape == (1, s.N) and w.extra["u_target"].shape == (s.N,)
    assert np.isfinite(w.f).all()
    # the genus-5 workload's mesh (its charts and data take about 20 s more)
    V, T = I.mesh(I.ToriChain(5), 0.07)
    assert 34000 <= len(T) <= 38000
    assert I.is_closed_manifold(len(V), T) and I.euler_characteristic(V, T) == -8


def test_green_and_gauss_identities_on_genus2_sampled_rows():
    """Oracle layer potentials on the genus-2 surface at 12 sampled targets:
    Gauss D[1] = -1/2 and Green S[dU/dn] - D[U] = U/2 for U = 1/|x - x0|,
    x0 at the centre of a hole (outside the solid, so U is harmonic inside).
    Both converge with the order (discretisation error, not parity)."""
    from oracle import farsum
    from oracle.geometry import build_geometry, near_lists
    from oracle.quadrature import build_corrections
    errs = []
    for order in (4, 6):
        s = I.tori_chain(2, 0.2, order)
        g = build_geometry(s.order, s.uv, s.wref, s.X, s.Xu, s.Xv)
        ptr, pl = near_lists(g, 2.0)
        rows = np.sort(np.random.default_rng(7).choice(g.N, 12, replace=False))
        vals, _ = build_corrections(g, ptr, pl, eps_q=1e-12, rows=rows)
        d = g.X - np.array([0.0, 0.0, 0.0])[None, :]
        r = np.linalg.norm(d, axis=1)
        U, dU, one = 1 / r, -np.einsum("ij,ij->i", d, g.n) / r ** 3, np.ones(g.N)
        far = farsum.far_sums(g, ptr, pl, np.stack([dU, U, one]), targets=rows)

        def near(K, sig):
            out = []
            for i in rows:
                out.append(sum(vals[b, K] @ sig[pl[b] * g.np_:(pl[b] + 1) * g.np_] for b in range(ptr[i], ptr[i + 1])))
            return np.array(out)

        green = far[0, 0] + near(0, dU) - far[1, 1] - near(1, U) - 0.5 * U[rows]
        gauss = far[2, 1] + near(1, one) + 0.5
        errs.append(max(np.abs(green).max(), np.abs(gauss).max()))
    assert errs[1] < 1e-5 and errs[1] < errs[0] / 5
