"""Failure paths of the C ABI, driven from the host (no GPU fault involved).

* GMRES that reaches max_iter before tol returns LB_ENOTCONVERGED with the
  best iterate written and the residual history filled (Section 6 caps GMRES
  at 100 iterations; here the cap is 2): the iterate equals the oracle's
  GMRES after the same two iterations.
* A device allocation made to fail (lb_debug_fail_alloc, the library's
  failure-injection hook) returns LB_ENOMEM, and the same context then solves
  again with results identical to an undisturbed context.
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
def sphere():
    from oracle.layers import discretise
    from workloads.configs import config
    w = config(1)
    s = w.surface
    d = discretise(s.order, s.uv, s.wref, s.X, s.Xu, s.Xv, eta=2.0, eps_q=1e-12)
    return w, d


def _ctx(lb, w, d, **kw):
    ctx = lb.Context(0, lb.default_params(eps_quad=1e-12, **kw))
    ctx.upload_surface(w.surface)
    ctx.load_corrections(d.near_ptr, d.near_patch, d.vals)
    return ctx


def test_not_converged_returns_best_iterate(lb, sphere):
    from oracle.gmres import gmres
    w, d = sphere
    ctx = _ctx(lb, w, d, precision=lb.LB_FP64, tol=1e-14, max_iter=2)
    with pytest.raises(lb.LBError) as e:
        ctx.solve_lb(w.f)
    assert e.value.code == lb.LB_ENOTCONVERGED
    u, info = ctx.solve_lb(w.f, allow_unconverged=True)
    assert not info["converged"] and info["iterations"] == 2
    b = d.rhs("A3", w.f)[0]
    sig, it, hist = gmres(lambda x: d.apply("A3", x)[0], b, tol=1e-14, max_iter=2)
    assert it == 2
    u_ref = d.solution("A3", sig)[0]
    assert np.linalg.norm(u[0] - u_ref) / np.linalg.norm(u_ref) < 1e-10
    assert len(info["history"]) == 3
    assert np.allclose(info["history"], hist, rtol=1e-8, atol=0)
    assert info["history"][-1] > 1e-14
    # the lockstep solver (several right-hand sides) reports the same status
    ctx2 = _ctx(lb, w, d, precision=lb.LB_DF64, tol=1e-14, max_iter=2)
    f2 = np.stack([w.f[0], np.roll(w.f[0], 7)])
    with pytest.raises(lb.LBError) as e:
        ctx2.solve_lb(f2)
    assert e.value.code == lb.LB_ENOTCONVERGED
    u2, info2 = ctx2.solve_lb(f2, allow_unconverged=True)
    assert not info2["converged"] and np.all(np.isfinite(u2))
    assert np.linalg.norm(u2[0] - u_ref) / np.linalg.norm(u_ref) < 1e-9
    ctx.close()
    ctx2.close()


def test_simulated_out_of_memory_keeps_context_usable(lb, sphere):
    w, d = sphere
    ref_ctx = _ctx(lb, w, d, precision=lb.LB_FP64, tol=1e-12)
    u0, _ = ref_ctx.solve_lb(w.f)
    ref_ctx.close()
    # the next workspace allocation of a solve fails
    ctx = _ctx(lb, w, d, precision=lb.LB_FP64, tol=1e-12)
    ctx.debug_fail_alloc(0)
    with pytest.raises(lb.LBError) as e:
        ctx.solve_lb(w.f)
    assert e.value.code == lb.LB_ENOMEM
    assert "simulated" in str(e.value)
    u1, info = ctx.solve_lb(w.f)
    assert info["converged"] and np.array_equal(u1, u0)
    # an allocation in the middle of the geometry upload fails: no geometry is
    # kept, and a second upload restores the context
    ctx.debug_fail_alloc(3)
    with pytest.raises(lb.LBError) as e:
        ctx.upload_surface(w.surface)
    assert e.value.code == lb.LB_ENOMEM
    with pytest.raises(lb.LBError) as e:
        ctx.solve_lb(w.f)
    assert e.value.code == lb.LB_ESTATE
    ctx.upload_surface(w.surface)
    ctx.load_corrections(d.near_ptr, d.near_patch, d.vals)
    u2, _ = ctx.solve_lb(w.f)
    assert np.array_equal(u2, u0)
    # disarmed: nothing fails
    ctx.debug_fail_alloc(5)
    ctx.debug_fail_alloc(-1)
    u3, _ = ctx.solve_lb(w.f)
    assert np.array_equal(u3, u0)
    ctx.close()


def test_load_corrections_refuses_bad_lists(lb, sphere):
    """Out-of-range patch ids and unsorted rows never reach a kernel: the
    binding refuses host arrays, and the library's own device check refuses
    device arrays (LB_EINVAL, no corrections kept)."""
    torch = pytest.importorskip("torch")
    w, d = sphere
    ctx = lb.Context(0, lb.default_params(eps_quad=1e-12))
    ctx.upload_surface(w.surface)
    bad = d.near_patch.copy()
    bad[10] = w.surface.npatch
    with pytest.raises(lb.LBError) as e:
        ctx.load_corrections(d.near_ptr, bad, d.vals)
    assert e.value.code == lb.LB_EINVAL
    for arr, msg in ((bad, "outside"), (np.ascontiguousarray(d.near_patch[::-1]), "ascending")):
        with pytest.raises(lb.LBError) as e:
            ctx.load_corrections(torch.tensor(d.near_ptr, device="cuda"), torch.tensor(arr, device="cuda"),
                                 torch.tensor(d.vals, device="cuda"))
        assert e.value.code == lb.LB_EINVAL and msg in str(e.value)
        assert ctx.info()["corrections"] == 0
    rp = d.near_ptr.copy()
    rp[5] = rp[6] + 1
    with pytest.raises(lb.LBError) as e:
        ctx.load_corrections(torch.tensor(rp, device="cuda"), torch.tensor(d.near_patch, device="cuda"),
                             torch.tensor(d.vals, device="cuda"))
    assert e.value.code == lb.LB_EINVAL
    ctx.load_corrections(d.near_ptr, d.near_patch, d.vals)
    assert ctx.info()["corrections"] == 1
    ctx.close()
