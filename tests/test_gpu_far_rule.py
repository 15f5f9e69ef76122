"""The oversampled far-field rule on the GPU against the oracle (Section 4).

The paper evaluates its far field on an oversampled smooth rule: the chart
and the density are interpolated from the node rule to a finer rule on every
patch.  lb_set_far_rule does this on the device; the oracle's FarRule
(oracle/geometry.py oversample) does it on the host.  Far sums, potentials,
the A3 and A2 applies and the solves must match in float64 to 1e-12 (1e-10
for solves) and float32 to 2e-5, with the oracle's
near lists and correction blocks loaded on both sides (double-float far sums
to 5e-12: the S''+D' sums cancel).
"""
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

WORKERS = min(16, os.cpu_count() or 1)


def _rel(a, b):
    return np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(np.asarray(b)).max(), 1e-300)


@pytest.fixture(scope="module")
def lb():
    import __graft_entry__ as g
    g.build()
    import paper_2111_10743_gb300 as lb
    return lb


_CACHE = {}


def _setup(name):
    if name not in _CACHE:
        from oracle.geometry import oversample
        from oracle.layers import Discretisation, discretise
        from workloads import surfaces as S
        from workloads.configs import config
        from workloads.nodes import node_rule
        s = config(1).surface if name == "sphere300" else S.ellipsoid((1.0, 1.5, 2.0), 1, 4)
        d = discretise(s.order, s.uv, s.wref, s.X, s.Xu, s.Xv, eta=2.0, eps_q=1e-12, workers=WORKERS)
        uv8, w8 = node_rule(8)
        df = Discretisation(d.geo, d.near_ptr, d.near_patch, d.vals, d.eta, d.eps_q, far=oversample(d.geo, uv8, w8))
        _CACHE[name] = (s, d, df, uv8, w8)
    return _CACHE[name]


def _ctx(lb, name, **kw):
    s, d, df, uv8, w8 = _setup(name)
    ctx = lb.Context(0, lb.default_params(eps_quad=1e-12, **kw))
    ctx.upload_surface(s)
    ctx.load_corrections(d.near_ptr, d.near_patch, d.vals)
    ctx.set_far_rule(8, uv8, w8)
    return ctx, s, d, df


@pytest.mark.parametrize("name", ["sphere300", "ellipsoid1200"])
def test_far_sums_and_potentials(lb, name):
    from oracle import farsum
    ctx, s, d, df = _ctx(lb, name)
    rng = np.random.default_rng(51)
    sig = rng.standard_normal((2, d.geo.N))
    ref = farsum.far_sums(d.geo, d.near_ptr, d.near_patch, sig, far=df.far)
    # double-float: the S''+D' sums cancel to about 1e-12 of the largest term
    for prec, tol in ((lb.LB_FP64, 1e-12), (lb.LB_DF64, 5e-12), (lb.LB_FP32, 2e-5)):
        got = ctx.far_sums(sig, precision=prec)
        for r in range(2):
            for k in range(4):
                assert _rel(got[r, k], ref[r, k]) < tol, (prec, r, k, _rel(got[r, k], ref[r, k]))
    pot = df.potentials(sig)
    for fn, k in ((ctx.apply_S, 0), (ctx.apply_D, 1), (ctx.apply_Sp, 2), (ctx.apply_SppDp, 3)):
        assert _rel(fn(sig), pot[:, k]) < 1e-12, k
    # the oversampled sums differ from the node-rule sums: the rule is in use
    base = farsum.far_sums(d.geo, d.near_ptr, d.near_patch, sig)
    assert _rel(ref[0, 0], base[0, 0]) > 1e-9
    # order 0 restores the node rule exactly
    ctx.set_far_rule(0)
    fresh = lb.Context(0, lb.default_params(eps_quad=1e-12))
    fresh.upload_surface(s)
    fresh.load_corrections(d.near_ptr, d.near_patch, d.vals)
    assert np.array_equal(ctx.far_sums(sig, precision=lb.LB_FP64), fresh.far_sums(sig, precision=lb.LB_FP64))
    ctx.close()
    fresh.close()


@pytest.mark.parametrize("form", ["A3", "A2"])
def test_operators_and_solves(lb, form):
    name = "ellipsoid1200"
    formulation = lb.LB_A3 if form == "A3" else lb.LB_A2
    ctx, s, d, df = _ctx(lb, name, formulation=formulation, tol=1e-12, precision=lb.LB_FP64)
    tau = np.random.default_rng(52).standard_normal((3, d.geo.N))
    assert _rel(ctx.apply_A(tau), df.apply(form, tau)) < 1e-12
    from oracle.gmres import solve_lb
    f = np.sin(2.0 * d.geo.X[:, 0]) * d.geo.X[:, 2]
    u_ref, _, _, _ = solve_lb(df, f, form, tol=1e-12)
    u, info = ctx.solve_lb(f[None])
    assert info["converged"]
    assert np.linalg.norm(u[0] - u_ref) / np.linalg.norm(u_ref) < 1e-10
    # float32 applies (several densities: single-density passes under the far rule)
    p = ctx.get_params()
    p.precision = lb.LB_FP32
    ctx.set_params(p)
    assert _rel(ctx.apply_A(tau), df.apply(form, tau)) < 2e-5
    # the refined solve and a batch of right-hand sides
    p.precision, p.tol = lb.LB_FP32_REFINED, 1e-10
    ctx.set_params(p)
    f2 = np.stack([f, np.cos(d.geo.X[:, 1])])
    u2, info2 = ctx.solve_lb(f2)
    assert info2["converged"]
    assert np.linalg.norm(u2[0] - u_ref) / np.linalg.norm(u_ref) < 1e-9
    ctx.close()


def test_far_rule_refusals(lb):
    from workloads.nodes import node_rule
    ctx, s, d, df = _ctx(lb, "sphere300")
    y = np.ones((1, d.geo.N))
    for fn in (ctx.apply_St, ctx.apply_At):
        with pytest.raises(lb.LBError) as e:
            fn(y)
        assert e.value.code == lb.LB_EINVAL
    with pytest.raises(lb.LBError) as e:
        ctx.solve_lb_adjoint(y)
    assert e.value.code == lb.LB_EINVAL
    uv, w = node_rule(6)
    with pytest.raises(lb.LBError) as e:
        ctx.set_far_rule(6, uv, 2.0 * w)            # weights must sum to 1/2
    assert e.value.code == lb.LB_EINVAL
    ctx.set_far_rule(0)
    ctx.apply_St(y)                                  # the node rule again: allowed
    ctx.close()
