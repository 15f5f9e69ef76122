"""Parity at the benchmark's own size, in the benchmark's launch shapes.

Surface: the ellipsoid (1, 1.5, 2) from the icosahedron subdivided three
times, 1,280 order-8 patches, N = 57,600 nodes, near-field corrections built
on the GPU (the set-up the benchmark times).  The oracle cannot form the
whole operator at this size (its quadrature would take hours on the host), so
the checks are on outputs it can compute one by one, and on properties that
hold at any size:
  * far sums and correction blocks of sampled rows (Section 4);
  * the A3 apply (Section 4.3) of a density supported on two patches: its
    first pass S tau, S' tau at every node (the oracle builds the correction
    blocks of the two patches for all rows), its second pass at 64 sampled
    rows; A3 tau is compared up to the constant W S mu2, the one term that
    needs every row of the correction matrix;
  * the mixed-precision solve the benchmark times (float32 inner GMRES,
    double-float residual) against the plain float64 solve of the same
    right-hand side.
"""
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

WORKERS = min(16, os.cpu_count() or 1)


def _rel(a, b):
    return np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(np.asarray(b)).max(), 1e-300)


@pytest.fixture(scope="module")
def full():
    import __graft_entry__ as g
    g.build()
    import paper_2111_10743_gb300 as lb
    from oracle.geometry import build_geometry, near_lists
    from workloads.configs import config
    w = config(2)
    s = w.surface
    ctx = lb.Context(0, lb.default_params(eps_quad=1e-12, tol=1e-12, precision=lb.LB_FP64))
    ctx.upload_surface(s)
    ctx.build_corrections()
    geo = build_geometry(s.order, s.uv, s.wref, s.X, s.Xu, s.Xv)
    ptr, pl = near_lists(geo, 2.0)
    yield lb, w, ctx, geo, ptr, pl
    ctx.close()


def test_full_size_sampled_rows(full):
    """Near lists bit-exact; GPU-built correction blocks of 24 sampled rows
    against the oracle's; far sums of those rows in every pair precision."""
    from oracle import farsum
    from oracle.layers import Discretisation
    from oracle.quadrature import build_corrections
    lb, w, ctx, g, ptr, pl = full
    rp, pa, vals = ctx.get_corrections()
    assert np.array_equal(rp, ptr) and np.array_equal(pa, pl)
    rows = np.random.default_rng(29).choice(g.N, 24, replace=False)
    ov, hits = build_corrections(g, ptr, pl, eps_q=1e-12, rows=rows, workers=WORKERS)
    assert hits == 0
    sel = np.isin(np.repeat(np.arange(g.N), np.diff(ptr)), rows)
    assert np.abs(vals[sel] - ov[sel]).max() < 1e-10 * np.abs(ov[sel]).max()
    sig = np.random.default_rng(30).standard_normal(g.N)
    ref = farsum.far_sums(g, ptr, pl, sig, targets=rows)[0]
    # the FP64 oracle sums 57,600 terms of random sign in plain order: its own
    # rounding is about 1e-11 of the largest sum here, which bounds the DF64 check
    for prec, tol in ((lb.LB_FP64, 1e-12), (lb.LB_DF64, 2e-11), (lb.LB_FP32, 2e-5)):
        got = ctx.far_sums(sig, precision=prec)[0][:, rows]
        for k in range(4):
            assert _rel(got[k], ref[k]) < tol, (prec, k)
    disc = Discretisation(g, ptr, pl, np.where(sel[:, None, None], ov, 0.0), 2.0, 1e-12)
    pot = ctx.apply_S(sig)[0][rows]
    assert _rel(pot, disc.potentials(sig, targets=rows)[0, 0]) < 1e-10


def test_a3_apply_of_local_density(full):
    """A3 tau for tau supported on two patches far apart: S tau and S' tau at
    all 57,600 nodes, and A3 tau at 64 sampled rows up to the constant W S mu2
    (float64, double-float and float32 pair sums)."""
    from oracle.layers import Discretisation, K_S, K_SD, K_SP
    from oracle.quadrature import build_corrections
    lb, w, ctx, g, ptr, pl = full
    rng = np.random.default_rng(31)
    npn = g.np_
    d0 = np.linalg.norm(g.centroid - g.centroid[0], axis=1)
    T = [0, int(np.argmax(d0))]
    tau = np.zeros(g.N)
    for P in T:
        tau[P * npn:(P + 1) * npn] = rng.standard_normal(npn)
    rows = np.sort(rng.choice(g.N, 64, replace=False))
    # the oracle's blocks: every block on the two patches (first pass, all
    # rows) and every block of the sampled rows (second pass)
    ov, hits = build_corrections(g, ptr, pl, eps_q=1e-12, rows=rows, blocks=np.isin(pl, T), workers=WORKERS)
    assert hits == 0
    disc = Discretisation(g, ptr, pl, ov, 2.0, 1e-12)
    p1 = disc.potentials(tau)[0]
    mu1, mu2 = p1[K_SP], p1[K_S]
    q = disc.potentials(np.stack([mu1, mu2]), targets=rows)
    H = g.H[rows]
    a3_no_eta = -0.25 * tau[rows] + q[0, K_SP] - q[1, K_SD] - 2.0 * H * q[1, K_SP]
    tol = {lb.LB_FP64: 1e-10, lb.LB_DF64: 1e-10, lb.LB_FP32: 2e-5}
    tol_a3 = {lb.LB_FP64: 1e-9, lb.LB_DF64: 1e-9, lb.LB_FP32: 2e-5}
    p = ctx.get_params()
    try:
        for prec in (lb.LB_FP64, lb.LB_DF64, lb.LB_FP32):
            p.precision = prec
            ctx.set_params(p)
            e_s = _rel(ctx.apply_S(tau)[0], mu2)
            e_sp = _rel(ctx.apply_Sp(tau)[0], mu1)
            a3 = ctx.apply_A(tau)[0][rows]
            diff = a3 - a3_no_eta
            # the same constant eta = W S mu2 on every row
            e_a3 = (diff.max() - diff.min()) / np.abs(a3_no_eta).max()
            print(f"precision {prec}: S {e_s:.2e}, S' {e_sp:.2e}, A3 up to eta {e_a3:.2e}")
            assert e_s < tol[prec] and e_sp < tol[prec] and e_a3 < tol_a3[prec], (prec, e_s, e_sp, e_a3)
    finally:
        p.precision = lb.LB_FP64
        ctx.set_params(p)


def test_refined_solve_matches_fp64_solve(full):
    """The benchmark's solve (LB_FP32_REFINED to 1e-10) against the plain
    float64 solve to 1e-12 of the same right-hand side: relative L2 and
    largest elementwise difference of u below 1e-9."""
    lb, w, ctx, g, ptr, pl = full
    p = ctx.get_params()
    try:
        p.precision, p.tol = lb.LB_FP32_REFINED, 1e-10
        ctx.set_params(p)
        ur, ir = ctx.solve_lb(w.f)
        assert ir["converged"] and ir["rel_residual"] < 1e-10 and ir["applies_fp64"] >= 1
        p.precision, p.tol = lb.LB_FP64, 1e-12
        ctx.set_params(p)
        u64, i64 = ctx.solve_lb(w.f)
        assert i64["converged"] and i64["rel_residual"] < 1e-12
        err2 = np.linalg.norm(ur - u64) / np.linalg.norm(u64)
        errinf = _rel(ur, u64)
        assert err2 < 1e-9 and errinf < 1e-9, (err2, errinf)
        print(f"refined vs float64 solve: rel L2 {err2:.2e}, max {errinf:.2e}")
    finally:
        p.precision, p.tol = lb.LB_FP64, 1e-12
        ctx.set_params(p)
