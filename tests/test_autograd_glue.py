"""The torch.autograd wrappers' plumbing, on the CPU.

A stand-in context answers solve_lb, solve_lb_adjoint and geometry_gradient
from the oracle's dense FP64 matrices, so these tests check only what the
wrappers add: which calls the backward pass makes, the sums of the geometry
gradients over right-hand sides, the shapes and the refusal of a surface that
differs from the uploaded one.  The library
calls themselves are checked against the oracle on the GPU.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")


class OracleContext:
    def __init__(self, disc):
        from oracle.gmres import dense_matrix
        self.d = disc
        N = disc.geo.N
        self.S = dense_matrix(lambda x: disc.S(x), N)
        self.A = dense_matrix(lambda x: disc.apply("A3", x), N)
        w = disc.geo.w
        self.P = np.eye(N) - np.outer(np.ones(N), w) / w.sum()
        self.L = self.S @ self.S @ np.linalg.solve(self.A, self.P)   # u = L f
        self.calls = []
        self.cache = {}

    def solve_lb(self, f, out):
        self.calls.append("solve")
        out.copy_(torch.from_numpy(f.numpy() @ self.L.T))

    def solve_lb_adjoint(self, gu, out):
        self.calls.append("adjoint")
        out.copy_(torch.from_numpy(gu.numpy() @ self.L))

    def grad(self, f, gu):
        """The oracle's node-position gradient, cached per input pair."""
        from oracle.shape import shape_gradient_A3
        key = (f.tobytes(), gu.tobytes())
        if key not in self.cache:
            self.cache[key] = shape_gradient_A3(self.d, f, gu)
        return self.cache[key]

    def tgrad(self, f, gu):
        """The oracle's tangent gradient (dL/dX_u, dL/dX_v), cached."""
        from oracle.shape import tangent_gradient_A3
        key = ("t", f.tobytes(), gu.tobytes())
        if key not in self.cache:
            self.cache[key] = tangent_gradient_A3(self.d, f, gu)
        return self.cache[key]

    def check_geometry(self, **arrays):
        g = self.d.geo
        for k, a in arrays.items():
            if a is not None and not np.array_equal(a.detach().numpy(), getattr(g, k)):
                raise ValueError(f"{k} differs from the uploaded surface")

    def geometry_gradient(self, f, gu, want_x, want_t, out):
        self.calls.append("geometry")
        for r in range(f.shape[0]):
            fr, gr = f[r].numpy(), gu[r].numpy()
            if want_x:
                out[0][r] = torch.from_numpy(self.grad(fr, gr))
            if want_t:
                gxu, gxv = self.tgrad(fr, gr)
                out[1][r] = torch.from_numpy(gxu)
                out[2][r] = torch.from_numpy(gxv)


@pytest.fixture(scope="module")
def octx():
    from workloads import surfaces as S
    from oracle.layers import discretise
    s = S.icosphere(0, 3)   # 20 patches of order 3, N = 200
    return OracleContext(discretise(s.order, s.uv, s.wref, s.X, s.Xu, s.Xv, eta=2.0, eps_q=1e-10))


def test_solve_autograd_density_and_positions(octx):
    import paper_2111_10743_gb300 as lb
    N = octx.d.geo.N
    rng = np.random.default_rng(45)
    f = torch.tensor(rng.standard_normal((2, N)), requires_grad=True)
    X = torch.tensor(octx.d.geo.X.copy(), requires_grad=True)
    ut = torch.tensor(rng.standard_normal((2, N)))
    octx.calls.clear()
    u = lb.solve_lb_autograd(f, octx, X=X)
    loss = ((u - ut) ** 2).sum()
    loss.backward()
    assert octx.calls == ["solve", "adjoint", "geometry"]
    gu = 2.0 * (u.detach() - ut).numpy()
    assert np.allclose(f.grad.numpy(), gu @ octx.L, rtol=0, atol=1e-12)
    ref = sum(octx.grad(f.detach()[r].numpy(), gu[r]) for r in range(2))
    assert X.grad.shape == (N, 3)
    assert np.abs(X.grad.numpy() - ref).max() < 1e-12 * np.abs(ref).max()
    # positions only: no adjoint solve for f
    octx.calls.clear()
    f2 = f.detach()[:1]
    (lb.solve_lb_autograd(f2, octx, X=X) ** 2).sum().backward()
    assert octx.calls == ["solve", "geometry"]
    # without X the wrapper is the density-only one
    octx.calls.clear()
    g = torch.tensor(rng.standard_normal((1, N)), requires_grad=True)
    (lb.solve_lb_autograd(g, octx) ** 2).sum().backward()
    assert octx.calls == ["solve", "adjoint"]


def test_solve_autograd_tangents_and_refusal(octx):
    """Gradients with respect to the chart tangents come from the geometry
    gradient, summed over right-hand sides; an X that differs from the
    uploaded surface is refused before anything is solved."""
    import paper_2111_10743_gb300 as lb
    g = octx.d.geo
    N = g.N
    rng = np.random.default_rng(46)
    f = torch.tensor(rng.standard_normal((2, N)))
    Xu = torch.tensor(g.Xu.copy(), requires_grad=True)
    Xv = torch.tensor(g.Xv.copy(), requires_grad=True)
    ut = torch.tensor(rng.standard_normal((2, N)))
    octx.calls.clear()
    u = lb.solve_lb_autograd(f, octx, Xu=Xu, Xv=Xv)
    ((u - ut) ** 2).sum().backward()
    assert octx.calls == ["solve", "geometry"]
    gu = 2.0 * (u.detach() - ut).numpy()
    refs = [octx.tgrad(f[r].numpy(), gu[r]) for r in range(2)]
    ru, rv = refs[0][0] + refs[1][0], refs[0][1] + refs[1][1]
    assert np.abs(Xu.grad.numpy() - ru).max() < 1e-12 * np.abs(ru).max()
    assert np.abs(Xv.grad.numpy() - rv).max() < 1e-12 * np.abs(rv).max()
    X = torch.tensor(g.X + 1e-9, requires_grad=True)
    octx.calls.clear()
    with pytest.raises(ValueError, match="differs"):
        lb.solve_lb_autograd(f, octx, X=X)
    assert octx.calls == []
