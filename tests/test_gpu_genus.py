"""Solves and harmonic fields on the genus-2 surface (two blended tori),
with corrections built on the GPU.

* Manufactured solution: the coordinate x_1 satisfies
  Delta_Gamma x_1 = -2 H n_1 on any closed surface, so with f = -2 H n_1
  (H and n from the level-set formulas) the mean-zero solution is
  x_1 - mean(x_1).
* Harmonic fields: on a closed surface of genus g they form a space of
  dimension 2g (Section 5), so the fields H_k and n x H_k of six random
  tangential F span four dimensions, up to discretisation error.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lb():
    import __graft_entry__ as g
    g.build()
    import paper_2111_10743_gb300 as lb
    return lb


@pytest.fixture(scope="module")
def genus2(lb):
    from oracle.geometry import build_geometry
    from workloads import implicit as I
    s = I.tori_chain(2, 0.2, 6)
    g = build_geometry(s.order, s.uv, s.wref, s.X, s.Xu, s.Xv)
    ctx = lb.Context(0, lb.default_params(precision=lb.LB_FP32_REFINED, tol=1e-10, eps_quad=1e-12,
                                          near_factor=2.0))
    ctx.upload_surface(s)
    ctx.build_corrections()
    return ctx, s, g


def test_genus2_manufactured_solution(genus2):
    from workloads import implicit as I
    ctx, s, g = genus2
    surf = s.implicit
    n = surf.grad(s.X)
    n /= np.linalg.norm(n, axis=1, keepdims=True)
    f = -2.0 * I.mean_curvature(surf, s.X) * n[:, 0]
    u, info = ctx.solve_lb(f[None])
    assert info["converged"]
    ue = s.X[:, 0] - np.sum(g.w * s.X[:, 0]) / np.sum(g.w)
    assert np.abs(u[0] - ue).max() < 1e-3 * np.abs(ue).max()


def test_genus2_harmonic_fields_span_four_dimensions(genus2):
    from workloads import rhs as R
    ctx, s, g = genus2
    rng = np.random.default_rng(44)
    Xc = s.X - 0.5 * (s.X.min(0) + s.X.max(0))
    F = []
    for _ in range(6):
        V = R.legendre_field(Xc, rng, 3, 2.5, ncomp=3)
        F.append(-np.cross(g.n, np.cross(g.n, V)))
    H, info = ctx.harmonic_fields(np.stack(F))
    assert H.shape == (12, g.N, 3)
    M = (H * np.sqrt(g.w)[None, :, None]).reshape(12, -1)
    sv = np.linalg.svd(M, compute_uv=False)
    assert sv[3] > 0.05 * sv[0]
    assert sv[4] < 1e-2 * sv[0]
    # and each field is tangential and (discretely) divergence free
    div = ctx.surface_div(H)
    for k in range(12):
        assert np.abs(np.sum(H[k] * g.n, axis=1)).max() < 1e-10 * np.abs(H[k]).max()
        assert np.sqrt(np.sum(g.w * div[k] ** 2)) < 0.05 * np.sqrt(np.sum(g.w * np.sum(H[k] ** 2, 1)))
