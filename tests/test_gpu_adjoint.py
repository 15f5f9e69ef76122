"""Density adjoint: transposed applies, the adjoint solve and autograd.

The transposes are checked against the transposes of the oracle's dense
matrices (assembled column by column from its FP64 operators), the adjoint
solve against the dense gradient P^T A3^-T S^T S^T g_u and against the
adjoint identity <g_u, L f> = <L^T g_u, f>, and the torch.autograd wrapper
against central finite differences of a quadratic loss in float64.
"""
import numpy as np
import pytest

from test_gpu_parity import _rel, _rel2, ctx_for, oracle_disc

pytestmark = pytest.mark.gpu

_DENSE = {}


@pytest.fixture(scope="module")
def lb():
    import __graft_entry__ as g
    g.build()
    import paper_2111_10743_gb300 as lb
    return lb


def dense(name, form="A3"):
    """Dense S and A3 (or A2) of the oracle's discretisation."""
    if (name, form) not in _DENSE:
        from oracle.gmres import dense_matrix
        s, d = oracle_disc(name)
        N = d.geo.N
        _DENSE[(name, form)] = (dense_matrix(lambda x: d.S(x), N), dense_matrix(lambda x: d.apply(form, x), N))
    return _DENSE[(name, form)]


@pytest.mark.parametrize("name", ["sphere300", "ellipsoid1200"])
@pytest.mark.parametrize("form", ["A3", "A2"])
def test_transposed_operators(lb, name, form):
    ctx, s, d = ctx_for(lb, name, formulation=lb.LB_A3 if form == "A3" else lb.LB_A2, precision=lb.LB_FP64)
    Smat, Amat = dense(name, form)
    y = np.random.default_rng(40).standard_normal((2, d.geo.N))
    assert _rel(ctx.apply_St(y), y @ Smat) < 1e-12
    assert _rel(ctx.apply_At(y), y @ Amat) < 1e-12


@pytest.mark.parametrize("name", ["sphere300", "ellipsoid1200"])
@pytest.mark.parametrize("form", ["A3", "A2"])
def test_adjoint_solve_matches_dense_gradient(lb, name, form):
    ctx, s, d = ctx_for(lb, name, formulation=lb.LB_A3 if form == "A3" else lb.LB_A2, precision=lb.LB_FP64,
                        tol=1e-14)
    Smat, Amat = dense(name, form)
    g = d.geo
    N = g.N
    rng = np.random.default_rng(41)
    f = rng.standard_normal((1, N))
    gu = rng.standard_normal((1, N))
    u, _ = ctx.solve_lb(f)
    gf, info = ctx.solve_lb_adjoint(gu)
    assert info["converged"] and info["iterations"] > 0
    # adjoint identity of the linear map f -> u
    lhs, rhs = float(np.sum(gu * u)), float(np.sum(gf * f))
    assert abs(lhs - rhs) < 1e-10 * np.linalg.norm(gu) * np.linalg.norm(u) * 10
    # dense gradient: u = S S A3^-1 P f or S A2^-1 S P f, P = I - 1 w^T / |Gamma|
    P = np.eye(N) - np.outer(np.ones(N), g.w) / g.w.sum()
    L = Smat @ Smat @ np.linalg.solve(Amat, P) if form == "A3" else Smat @ np.linalg.solve(Amat, Smat @ P)
    assert _rel2(gf[0], L.T @ gu[0]) < 1e-9
    assert _rel2(u[0], L @ f[0]) < 1e-9


def test_autograd_solve_and_apply(lb):
    torch = pytest.importorskip("torch")
    name = "ellipsoid1200"
    ctx, s, d = ctx_for(lb, name, formulation=lb.LB_A3, precision=lb.LB_FP64, tol=1e-14)
    N = d.geo.N
    rng = np.random.default_rng(42)
    dev = "cuda"
    f0 = torch.tensor(rng.standard_normal((1, N)), device=dev)
    ut = torch.tensor(rng.standard_normal((1, N)), device=dev)
    v = torch.tensor(rng.standard_normal((1, N)), device=dev)

    def loss(f):
        u = lb.solve_lb_autograd(f, ctx)
        return ((u - ut) ** 2).sum()

    f = f0.clone().requires_grad_(True)
    L = loss(f)
    L.backward()
    g = float((f.grad * v).sum())
    h = 1e-3   # the loss is quadratic in f: central differences are exact up to rounding
    with torch.no_grad():
        fd = (float(loss(f0 + h * v)) - float(loss(f0 - h * v))) / (2 * h)
    assert abs(fd - g) < 1e-8 * max(abs(g), 1.0)
    # the apply's gradient is A3^T
    tau = torch.tensor(rng.standard_normal((2, N)), device=dev, requires_grad=True)
    gy = torch.tensor(rng.standard_normal((2, N)), device=dev)
    (lb.apply_A_autograd(tau, ctx) * gy).sum().backward()
    Smat, Amat = dense(name)
    assert _rel(tau.grad.cpu().numpy(), gy.cpu().numpy() @ Amat) < 1e-12


def test_adjoint_refuses_A1(lb):
    ctx, s, d = ctx_for(lb, "sphere300", formulation=lb.LB_A1, precision=lb.LB_FP64)
    with pytest.raises(lb.LBError) as e:
        ctx.apply_At(np.zeros((1, d.geo.N)))
    assert e.value.code == lb.LB_EINVAL


@pytest.mark.parametrize("name", ["sphere300", "ellipsoid1200"])
def test_shape_gradient_matches_oracle(lb, name):
    """Node-position gradient of an A3-solve loss (corrections held fixed)
    against the oracle's dense gradient, which its own pin checks against
    central differences."""
    from oracle.shape import shape_gradient_A3
    ctx, s, d = ctx_for(lb, name, formulation=lb.LB_A3, precision=lb.LB_FP64, tol=1e-14)
    N = d.geo.N
    rng = np.random.default_rng(43)
    f = rng.standard_normal((2, N))
    gu = rng.standard_normal((2, N))
    grad, info = ctx.shape_gradient(f, gu)
    assert grad.shape == (2, N, 3)
    assert info["converged"] and info["iterations"] > 0
    for r in range(2):
        ref = shape_gradient_A3(d, f[r], gu[r])
        assert _rel(grad[r], ref) < 1e-9
    if name == "sphere300":
        ctx2, _, _ = ctx_for(lb, name, formulation=lb.LB_A2, precision=lb.LB_FP64)
        with pytest.raises(lb.LBError) as e:
            ctx2.shape_gradient(f[:1], gu[:1])
        assert e.value.code == lb.LB_EINVAL


@pytest.mark.parametrize("name", ["sphere300", "ellipsoid1200"])
def test_geometry_gradient_matches_oracle(lb, name):
    """Gradients of an A3-solve loss with respect to X, X_u and X_v
    (corrections and near lists held fixed) against the oracle's dense
    gradients, whose own pins check them against central differences."""
    from oracle.shape import shape_gradient_A3, tangent_gradient_A3
    ctx, s, d = ctx_for(lb, name, formulation=lb.LB_A3, precision=lb.LB_FP64, tol=1e-14)
    N = d.geo.N
    rng = np.random.default_rng(47)
    f = rng.standard_normal((2, N))
    gu = rng.standard_normal((2, N))
    gX, gXu, gXv, info = ctx.geometry_gradient(f, gu)
    assert info["converged"] and gXu.shape == (2, N, 3)
    for r in range(1 if name == "ellipsoid1200" else 2):
        ru, rv = tangent_gradient_A3(d, f[r], gu[r])
        assert _rel(gXu[r], ru) < 1e-9 and _rel(gXv[r], rv) < 1e-9
        assert _rel(gX[r], shape_gradient_A3(d, f[r], gu[r])) < 1e-9
    # tangents only: the same numbers
    _, gXu2, gXv2, _ = ctx.geometry_gradient(f, gu, want_x=False)
    assert np.array_equal(gXu2, gXu) and np.array_equal(gXv2, gXv)


def test_autograd_geometry_path(lb):
    """solve_lb_autograd with device tensors X, X_u, X_v: their gradients
    against the oracle's, and an X that differs from the upload is refused."""
    torch = pytest.importorskip("torch")
    from oracle.shape import shape_gradient_A3, tangent_gradient_A3
    ctx, s, d = ctx_for(lb, "sphere300", formulation=lb.LB_A3, precision=lb.LB_FP64, tol=1e-14)
    g = d.geo
    N = g.N
    dev = "cuda"
    rng = np.random.default_rng(48)
    f = torch.tensor(rng.standard_normal((1, N)), device=dev, requires_grad=True)
    ut = torch.tensor(rng.standard_normal((1, N)), device=dev)
    X = torch.tensor(s.X, device=dev, requires_grad=True)
    Xu = torch.tensor(s.Xu, device=dev, requires_grad=True)
    Xv = torch.tensor(s.Xv, device=dev, requires_grad=True)
    u = lb.solve_lb_autograd(f, ctx, X=X, Xu=Xu, Xv=Xv)
    (0.5 * ((u - ut) ** 2).sum()).backward()
    gu = (u.detach() - ut).cpu().numpy()[0]
    fn = f.detach().cpu().numpy()[0]
    assert _rel(X.grad.cpu().numpy(), shape_gradient_A3(d, fn, gu)) < 1e-9
    ru, rv = tangent_gradient_A3(d, fn, gu)
    assert _rel(Xu.grad.cpu().numpy(), ru) < 1e-9 and _rel(Xv.grad.cpu().numpy(), rv) < 1e-9
    assert f.grad is not None
    with pytest.raises(ValueError, match="differs"):
        lb.solve_lb_autograd(f, ctx, X=X.detach() * (1.0 + 1e-12))
