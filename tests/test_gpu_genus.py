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


def test_genus2_gradients_against_central_differences(lb):
    """The autograd configuration: genus 2, 4,032 order-6 patches
    (N = 112,896), loss L = |u - u_t|^2 / 2 of the A3 solve.  The density
    gradient (adjoint solve) and the geometry gradient (X, X_u, X_v; the
    corrections and near lists built once and held fixed) against central
    differences along four seeded directions each; the losses come from
    double-float solves to 1e-13."""
    torch = pytest.importorskip("torch")
    from workloads.configs import config
    w = config(4)
    s = w.surface
    dev = "cuda"
    p = lb.default_params(precision=lb.LB_FP64, tol=1e-13, eps_quad=1e-12, near_factor=2.0)
    ctx = lb.Context(0, p)
    ctx.upload_surface(s)
    ctx.build_corrections()
    rp, pa, vals = ctx.get_corrections()
    corr = (torch.tensor(rp, device=dev), torch.tensor(pa, device=dev), torch.tensor(vals, device=dev))
    del vals
    N = s.N
    f = w.f[:1]
    ut = w.extra["u_target"][None]
    pdf = lb.default_params(precision=lb.LB_DF64, tol=1e-13, eps_quad=1e-12, near_factor=2.0)
    ev = lb.Context(0, pdf)

    def loss(ff, X, Xu, Xv):
        ev.upload_geometry(s.npatch, s.order, s.uv, s.wref, X, Xu, Xv)
        ev.load_corrections(*corr)
        u, info = ev.solve_lb(ff)
        assert info["converged"]
        return 0.5 * float(np.sum((u - ut) ** 2))

    u, _ = ctx.solve_lb(f)
    gu = u - ut
    gf, _ = ctx.solve_lb_adjoint(gu)
    gX, gXu, gXv, info = ctx.geometry_gradient(f, gu)
    assert info["converged"]
    rng = np.random.default_rng(1004)
    scale = np.abs(s.X).max()
    for k in range(4):
        v = rng.standard_normal((1, N))
        h = 1e-2 * np.abs(f).max() / np.abs(v).max()   # L is quadratic in f: no truncation error
        fd = (loss(f + h * v, s.X, s.Xu, s.Xv) - loss(f - h * v, s.X, s.Xu, s.Xv)) / (2 * h)
        an = float(np.sum(gf * v))
        assert abs(fd - an) < 1e-6 * abs(an), ("density", k, fd, an)
    for k in range(4):
        dX, dU, dV = (rng.standard_normal((N, 3)) for _ in range(3))
        h = 1e-6 * scale
        Lp = loss(f, s.X + h * dX, s.Xu + h * dU, s.Xv + h * dV)
        Lm = loss(f, s.X - h * dX, s.Xu - h * dU, s.Xv - h * dV)
        fd = (Lp - Lm) / (2 * h)
        an = float(np.sum(gX[0] * dX) + np.sum(gXu[0] * dU) + np.sum(gXv[0] * dV))
        print(f"geometry direction {k}: central difference {fd:.10e}, gradient {an:.10e}")
        assert abs(fd - an) < 1e-5 * abs(an), ("geometry", k, fd, an)
    ctx.close()
    ev.close()
