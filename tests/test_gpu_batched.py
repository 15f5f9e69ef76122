"""Batched applies and lockstep solves (several right-hand sides at once).

The batched A3 apply evaluates each (target, source) pair once for up to 8
densities; the lockstep solver advances several GMRES systems with one such
apply per iteration.  Both are checked against the FP64 oracle per density /
right-hand side, and against properties that hold exactly: a zero density
gives an exactly zero result, two equal densities in one batch give
bit-identical results, and the chunking (8 per pass, then 4) and grouping
(64 systems per lockstep group) leave each result unchanged.
"""
import numpy as np
import pytest

from test_gpu_parity import _rel, _rel2, ctx_for, oracle_disc

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lb():
    import __graft_entry__ as g
    g.build()
    import paper_2111_10743_gb300 as lb
    return lb


@pytest.mark.parametrize("name", ["ellipsoid1200", "torus1920"])
@pytest.mark.parametrize("prec", ["fp32", "df64"])
@pytest.mark.parametrize("R", [5, 11])
def test_batched_a3_apply(lb, name, prec, R):
    ctx, s, d = ctx_for(lb, name, formulation=lb.LB_A3,
                        precision=lb.LB_FP32 if prec == "fp32" else lb.LB_DF64)
    rng = np.random.default_rng(31 + R)
    tau = rng.standard_normal((R, d.geo.N))
    tau[1] = 0.0
    tau[3] = tau[2]
    got = ctx.apply_A(tau)
    ref = d.apply("A3", tau)
    tol = 2e-5 if prec == "fp32" else 1e-12
    for r in range(R):
        if r == 1:
            assert np.all(got[r] == 0.0)
            continue
        assert _rel(got[r], ref[r]) < tol, r
    assert np.array_equal(got[2], got[3])
    # one density at a time goes through the single-density kernels
    single = np.stack([ctx.apply_A(tau[r:r + 1])[0] for r in (0, R - 1)])
    assert _rel(got[[0, R - 1]], single) < tol


@pytest.mark.parametrize("prec", ["df64", "fp32_refined"])
def test_lockstep_solve_matches_oracle(lb, prec):
    from oracle.gmres import solve_lb
    from workloads.rhs import legendre_field
    name = "torus1920"
    s, d = oracle_disc(name)
    rng = np.random.default_rng(33)
    f = np.stack([legendre_field(d.geo.X, rng, 4, 2.75) for _ in range(3)])
    f = np.concatenate([f, np.zeros((1, d.geo.N)), f[:1]])  # a zero and a repeated right-hand side
    tol = 1e-12 if prec == "df64" else 1e-11
    ctx, _, _ = ctx_for(lb, name, formulation=lb.LB_A3, tol=tol,
                        precision=lb.LB_DF64 if prec == "df64" else lb.LB_FP32_REFINED)
    u, info = ctx.solve_lb(f)
    assert info["converged"] and info["nrhs"] == 5
    assert info["rel_residual"] < tol
    assert np.all(u[3] == 0.0)
    assert np.array_equal(u[0], u[4])
    its = []
    for r in range(3):
        u_ref, _, it_ref, _ = solve_lb(d, f[r], "A3", tol=1e-12)
        its.append(it_ref)
        assert _rel2(u[r], u_ref) < (1e-10 if prec == "df64" else 1e-9), r
    if prec == "df64":
        # each system stops at its own tolerance, as it would alone (the zero
        # right-hand side takes no iteration, the repeated one as many as the first)
        assert abs(info["iterations"] - (sum(its) + its[0])) <= 4
        u1, info1 = ctx.solve_lb(f[:1])
        assert _rel2(u[0], u1[0]) < 1e-11
    else:
        assert info["refinements"] >= 4 and info["applies_fp32"] > info["applies_fp64"]


def test_lockstep_groups(lb):
    """66 right-hand sides: two lockstep groups (64 + 2) and all chunk shapes."""
    from oracle.gmres import solve_lb
    name = "sphere300"
    s, d = oracle_disc(name)
    rng = np.random.default_rng(34)
    f = rng.standard_normal((66, d.geo.N))
    ctx, _, _ = ctx_for(lb, name, formulation=lb.LB_A3, tol=1e-12, precision=lb.LB_DF64)
    u, info = ctx.solve_lb(f)
    assert info["converged"] and info["nrhs"] == 66
    for r in (0, 63, 64, 65):
        u_ref, _, _, _ = solve_lb(d, f[r], "A3", tol=1e-12)
        assert _rel2(u[r], u_ref) < 1e-10, r


@pytest.mark.parametrize("prec", ["df64", "fp32_refined"])
def test_lockstep_graphs_match_direct_launches(lb, prec):
    """Replaying each GMRES iteration as a captured CUDA graph runs the same
    kernels on the same data as launching them directly: identical results,
    and with profiling on every replayed far-field launch is still timed."""
    from workloads.rhs import legendre_field
    name = "torus1920"
    s, d = oracle_disc(name)
    rng = np.random.default_rng(35)
    f = np.stack([legendre_field(d.geo.X, rng, 4, 2.75) for _ in range(5)])
    kw = dict(formulation=lb.LB_A3, tol=1e-11,
              precision=lb.LB_DF64 if prec == "df64" else lb.LB_FP32_REFINED)
    out = {}
    for graphs in (0, 1):
        ctx, _, _ = ctx_for(lb, name, graphs=graphs, **kw)
        out[graphs] = ctx.solve_lb(f)
    (u0, i0), (u1, i1) = out[0], out[1]
    assert i0["graph_iterations"] == 0 and i1["graph_iterations"] > 0
    assert i0["iterations"] == i1["iterations"] and i0["pairs"] == i1["pairs"]
    assert np.array_equal(u0, u1)
    ctx.set_profiling(True)
    u2, i2 = ctx.solve_lb(f)
    prof = ctx.get_profile()
    ctx.set_profiling(False)
    assert i2["graph_iterations"] > 0 and np.array_equal(u2, u1)
    far = sum(v["pairs"] for k, v in prof.items() if isinstance(v, dict) and k.startswith("far"))
    assert far == i2["pairs"]


@pytest.mark.parametrize("shape", [0, 1, 2])
def test_batched_launch_shapes(lb, shape, monkeypatch):
    """Every launch shape the tuner chooses between (threads per block x
    sources per tile: 128 x 64, 128 x 128, 256 x 64) gives the oracle's A3."""
    monkeypatch.setenv("GBLB_BATCH_SHAPE", str(shape))
    name = "torus1920"
    for prec, tol in (("fp32", 2e-5), ("df64", 1e-12)):
        ctx, s, d = ctx_for(lb, name, formulation=lb.LB_A3,
                            precision=lb.LB_FP32 if prec == "fp32" else lb.LB_DF64)
        tau = np.random.default_rng(36).standard_normal((6, d.geo.N))
        got = ctx.apply_A(tau)
        ref = d.apply("A3", tau)
        for r in range(6):
            assert _rel(got[r], ref[r]) < tol, (prec, r)


def test_tuning_recorded(lb):
    """After batched passes have run, the tuner reports a shape for each
    (precision, pass, density count) it has seen."""
    ctx, s, d = ctx_for(lb, "ellipsoid1200", formulation=lb.LB_A3, precision=lb.LB_FP32)
    ctx.apply_A(np.random.default_rng(37).standard_normal((11, d.geo.N)))   # 8 + 3 densities
    t = ctx.get_tuning()
    for k in ("far32_k1_rc8", "far32_k2_rc8", "far32_k1_rc4", "far32_k2_rc4"):
        assert t[k] in ("128x64", "128x128", "256x64"), (k, t)
