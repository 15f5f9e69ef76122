"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Small surfaces span several target blocks and source tiles with ragged tails
(N = 300, 1200, 1920 against blocks of 256/512 targets and tiles of 64/128
sources).  Float64 results must match the oracle to 1e-12 relative for
single applies and 1e-10 relative L2 for solves when both use the same near
lists and correction blocks; float32 pair sums to 1e-5; GPU-built correction
blocks match the oracle's within the quadrature tolerance.
"""
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

WORKERS = min(16, os.cpu_count() or 1)


def _rel(a, b):
    return np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(np.asarray(b)).max(), 1e-300)


def _rel2(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b))


@pytest.fixture(scope="module")
def lb():
    import __graft_entry__ as g
    g.build()
    import paper_2111_10743_gb300 as lb
    return lb


def _case(name):
    from workloads import surfaces as S
    from workloads.configs import config
    if name == "sphere300":
        return config(1).surface, 1e-12
    if name == "ellipsoid1200":
        return S.ellipsoid((1.0, 1.5, 2.0), 1, 4), 1e-11
    if name == "torus1920":
        return S.torus(2.0, 0.75, 8, 8, 4), 1e-11
    raise KeyError(name)


_CACHE = {}


def oracle_disc(name):
    if name not in _CACHE:
        from oracle.layers import discretise
        s, eps = _case(name)
        _CACHE[name] = (s, discretise(s.order, s.uv, s.wref, s.X, s.Xu, s.Xv, eta=2.0, eps_q=eps,
                                      workers=WORKERS))
    return _CACHE[name]


def ctx_for(lb, name, load=True, **kw):
    s, d = oracle_disc(name)
    p = lb.default_params(eps_quad=d.eps_q, near_factor=2.0, **kw)
    ctx = lb.Context(0, p)
    ctx.upload_surface(s)
    if load:
        ctx.load_corrections(d.near_ptr, d.near_patch, d.vals)
    return ctx, s, d


CASES = ["sphere300", "ellipsoid1200", "torus1920"]


@pytest.mark.parametrize("name", CASES)
def test_geometry_and_near_lists(lb, name):
    ctx, s, d = ctx_for(lb, name, load=False)
    n, w, H = ctx.get_geometry()
    g = d.geo
    assert np.abs(n - g.n).max() < 1e-14
    assert _rel(w, g.w) < 1e-14
    assert np.abs(H - g.H).max() < 1e-11 * max(1.0, np.abs(g.H).max())
    ctx.build_near()
    rp, pa, _ = ctx.get_corrections(with_vals=False)
    assert np.array_equal(rp, d.near_ptr) and np.array_equal(pa, d.near_patch)


@pytest.mark.parametrize("name", CASES)
def test_far_sums_fp64_fp32(lb, name):
    from oracle import farsum
    ctx, s, d = ctx_for(lb, name)
    rng = np.random.default_rng(21)
    sig = rng.standard_normal((2, d.geo.N))
    ref = farsum.far_sums(d.geo, d.near_ptr, d.near_patch, sig)
    got64 = ctx.far_sums(sig, precision=lb.LB_FP64)
    got32 = ctx.far_sums(sig, precision=lb.LB_FP32)
    gotdf = ctx.far_sums(sig, precision=lb.LB_DF64)
    for k in range(4):
        assert _rel(got64[:, k], ref[:, k]) < 1e-12, k
        assert _rel(got32[:, k], ref[:, k]) < 2e-5, k
        # double-float sums: ~1e-14 per pair; S''+D' cancels partly (measured 2.2e-12)
        assert _rel(gotdf[:, k], ref[:, k]) < 5e-12, k


def test_far_sums_df64_coarse_grid(lb):
    """Double-float far sums when the position grid is coarse next to the
    pair distances: two spheres of radius 0.05 twelve units apart (2 x 80
    order-6 patches, N = 4,480).  The recentred coordinates reach 6, so the
    grid step of the hi parts is 2^-20, and close far pairs are about 0.02
    apart: the lo parts of the differences are up to 5e-5 of the hi parts.
    Unless the differences are renormalised before they are squared, the
    dropped lo * lo products alone put about 1e-9 into the closest terms;
    with it the error is that of the 48-bit positions (2^-44 absolute)."""
    from oracle import farsum
    from oracle.geometry import build_geometry, near_lists
    from workloads import surfaces as S
    from workloads.surfaces import Surface
    a = S.icosphere(1, 6)
    parts = []
    for c in ((-6.0, 0.3, 0.0), (6.0, 0.0, -0.2)):
        parts.append((np.asarray(c) + 0.05 * a.X, 0.05 * a.Xu, 0.05 * a.Xv))
    s = Surface("two_spheres", a.order, 2 * a.npatch, a.uv, a.wref, *(np.concatenate(z) for z in zip(*parts)))
    g = build_geometry(s.order, s.uv, s.wref, s.X, s.Xu, s.Xv)
    ptr, pl = near_lists(g, 2.0)
    ctx = lb.Context(0, lb.default_params(eps_quad=1e-10, near_factor=2.0))
    ctx.upload_surface(s)
    ctx.build_near()
    rp, pa, _ = ctx.get_corrections(with_vals=False)
    assert np.array_equal(rp, ptr) and np.array_equal(pa, pl)
    rng = np.random.default_rng(23)
    sig = rng.standard_normal((2, s.N))
    ref = farsum.far_sums(g, ptr, pl, sig)
    gotdf = ctx.far_sums(sig, precision=lb.LB_DF64)
    got64 = ctx.far_sums(sig, precision=lb.LB_FP64)
    for k in range(4):
        assert _rel(got64[:, k], ref[:, k]) < 1e-12, k
        e = _rel(gotdf[:, k], ref[:, k])
        print(f"kernel {k}: double-float {e:.2e}")
        assert e < 2e-11, (k, e)
    ctx.close()


@pytest.mark.parametrize("name", CASES)
def test_potentials_with_oracle_corrections(lb, name):
    ctx, s, d = ctx_for(lb, name)
    rng = np.random.default_rng(22)
    sig = rng.standard_normal((3, d.geo.N))
    ref = d.potentials(sig)
    for k, fn in enumerate((ctx.apply_S, ctx.apply_D, ctx.apply_Sp, ctx.apply_SppDp)):
        assert _rel(fn(sig), ref[:, k]) < 1e-12, k


@pytest.mark.parametrize("name", CASES)
@pytest.mark.parametrize("form", ["A3", "A2"])
@pytest.mark.parametrize("prec", ["fp64", "df64"])
def test_operators(lb, name, form, prec):
    ctx, s, d = ctx_for(lb, name, formulation=lb.LB_A3 if form == "A3" else lb.LB_A2,
                        precision=lb.LB_FP64 if prec == "fp64" else lb.LB_DF64)
    rng = np.random.default_rng(23)
    tau = rng.standard_normal((2, d.geo.N))
    assert _rel(ctx.apply_A(tau), d.apply(form, tau)) < 1e-12


@pytest.mark.parametrize("name", CASES)
def test_operators_fp32_every_variant(lb, name):
    """Every float32 launch variant against the oracle: A3 through K1 and K2
    (variants 0-6, 3 to 6 the symmetric kernels), A2 through all-four and
    K4 (0-2).  Float32 pairs: 2e-5 relative, as for the far sums."""
    rng = np.random.default_rng(25)
    tau = None
    for form, kinds, nvar in (("A3", (0, 2), 7), ("A2", (1, 3), 3)):
        ctx, s, d = ctx_for(lb, name, formulation=lb.LB_A3 if form == "A3" else lb.LB_A2,
                            precision=lb.LB_FP32)
        tau = rng.standard_normal((1, d.geo.N))
        ref = d.apply(form, tau)
        for v in range(nvar):
            for k in kinds:
                ctx.debug_set_variant(k, v)
            got = ctx.apply_A(tau)
            assert _rel(got, ref) < 2e-5, (form, v, _rel(got, ref))
        with pytest.raises(lb.LBError):
            ctx.debug_set_variant(kinds[1], nvar)
        ctx.close()


@pytest.mark.parametrize("name", CASES)
def test_operator_df64_every_variant(lb, name):
    """Both launch variants of the symmetric double-float A3 passes (one or
    two targets per thread) against the oracle at 1e-12."""
    ctx, s, d = ctx_for(lb, name, formulation=lb.LB_A3, precision=lb.LB_DF64)
    tau = np.random.default_rng(26).standard_normal((1, d.geo.N))
    ref = d.apply("A3", tau)
    for v in range(2):
        ctx.debug_set_variant(4, v)
        ctx.debug_set_variant(5, v)
        assert _rel(ctx.apply_A(tau), ref) < 1e-12, v
    with pytest.raises(lb.LBError):
        ctx.debug_set_variant(5, 2)
    ctx.close()


@pytest.mark.parametrize("name", ["sphere300", "torus1920"])
@pytest.mark.parametrize("form", ["A3", "A2"])
@pytest.mark.parametrize("prec", ["fp64", "df64"])
def test_solve_fp64_matches_oracle(lb, name, form, prec):
    from oracle.gmres import solve_lb
    from workloads.rhs import legendre_field
    ctx, s, d = ctx_for(lb, name, formulation=lb.LB_A3 if form == "A3" else lb.LB_A2, tol=1e-12,
                        precision=lb.LB_FP64 if prec == "fp64" else lb.LB_DF64)
    f = legendre_field(d.geo.X, np.random.default_rng(24), 4, 2.75)
    u_ref, _, it_ref, _ = solve_lb(d, f, form, tol=1e-12)
    u, info = ctx.solve_lb(f[None, :])
    assert info["converged"] and abs(info["iterations"] - it_ref) <= 1
    assert _rel2(u[0], u_ref) < 1e-10
    # the discrete A3/A2 solution is mean zero only to discretisation accuracy:
    # compare its mean with the oracle's
    assert abs(np.sum(d.geo.w * (u[0] - u_ref))) < 1e-10 * np.abs(u_ref).max() * d.geo.w.sum()


def test_solve_refined_and_fp32(lb):
    from oracle.gmres import solve_lb
    from workloads.rhs import legendre_field
    name = "ellipsoid1200"
    s, d = oracle_disc(name)
    f = legendre_field(d.geo.X, np.random.default_rng(25), 4, 2.75)
    u_ref, _, _, _ = solve_lb(d, f, "A3", tol=1e-12)
    ctx, _, _ = ctx_for(lb, name, precision=lb.LB_FP32_REFINED, tol=1e-11)
    u, info = ctx.solve_lb(f[None, :])
    assert info["converged"] and info["refinements"] >= 1 and info["applies_fp32"] > info["applies_fp64"]
    assert info["rel_residual"] < 1e-11
    assert _rel2(u[0], u_ref) < 1e-9
    ctx32, _, _ = ctx_for(lb, name, precision=lb.LB_FP32, tol=1e-6)
    u32, info32 = ctx32.solve_lb(f[None, :])
    assert _rel2(u32[0], u_ref) < 1e-4


@pytest.mark.parametrize("name", CASES)
def test_built_corrections_match_oracle(lb, name):
    ctx, s, d = ctx_for(lb, name, load=False)
    ctx.build_corrections()
    rp, pa, vals = ctx.get_corrections()
    assert np.array_equal(rp, d.near_ptr) and np.array_equal(pa, d.near_patch)
    # two independent adaptive quadratures converged to eps_quad
    scale = np.abs(d.vals).max()
    err = np.abs(vals - d.vals).max()
    assert err < 1e-10 * scale, err / scale
    # potentials with the library's own corrections
    rng = np.random.default_rng(26)
    sig = rng.standard_normal(d.geo.N)
    assert _rel(ctx.apply_S(sig), d.potentials(sig)[:, 0]) < 1e-9


def test_gradS_and_surface_div(lb):
    from oracle.hodge import grad_S
    from oracle.geometry import surface_divergence
    ctx, s, d = ctx_for(lb, "ellipsoid1200")
    rng = np.random.default_rng(27)
    sig = rng.standard_normal(d.geo.N)
    assert _rel(ctx.apply_gradS(sig)[0], grad_S(d, sig)) < 1e-11
    F = np.cross(d.geo.n, rng.standard_normal((d.geo.N, 3)))
    assert _rel(ctx.surface_div(F)[0], surface_divergence(d.geo, F)) < 1e-11


def test_harmonic_fields_torus(lb):
    from oracle.hodge import harmonic_field
    from oracle.geometry import surface_divergence
    from workloads.rhs import current_source_field
    ctx, s, d = ctx_for(lb, "torus1920", tol=1e-11)
    g = d.geo
    V = current_source_field(g.X)
    F = -np.cross(g.n, np.cross(g.n, V))
    H, info = ctx.harmonic_fields(F[None])
    Href, nHref, _ = harmonic_field(d, F, tol=1e-11)
    assert _rel2(H[0], Href) < 1e-8 and _rel2(H[1], nHref) < 1e-8
    # both fields are (discretely) divergence free to discretisation accuracy
    # (this 128-patch order-4 torus resolves div H to about 7 %)
    for k in range(2):
        assert np.sqrt(np.sum(g.w * surface_divergence(g, H[k]) ** 2)) < 0.1 * np.sqrt(
            np.sum(g.w * np.sum(H[k] ** 2, 1)))


def test_device_pointers_batches_and_errors(lb):
    torch = pytest.importorskip("torch")
    ctx, s, d = ctx_for(lb, "sphere300")
    rng = np.random.default_rng(28)
    sig = rng.standard_normal((4, d.geo.N))
    ref = d.potentials(sig)[:, 0]
    dev = torch.tensor(sig, device="cuda")
    out = torch.empty_like(dev)
    ctx.set_stream(torch.cuda.current_stream())
    ctx.apply_S(dev, out=out)
    torch.cuda.synchronize()
    assert _rel(out.cpu().numpy(), ref) < 1e-12
    with pytest.raises(lb.LBError) as e:
        ctx.solve_lb(np.full((1, d.geo.N), np.nan))
    assert e.value.code == lb.LB_EINVAL
    fresh = lb.Context(0)
    fresh.upload_surface(s)
    with pytest.raises(lb.LBError) as e:
        fresh.apply_S(sig[0])
    assert e.value.code == lb.LB_ESTATE
    # a zero right-hand side solves to zero
    u, info = ctx.solve_lb(np.zeros((1, d.geo.N)))
    assert np.all(u == 0.0)


def test_twisted_torus_against_paper_table(lb):
    """Harmonic fields on the twisted torus with the settings of Section 6.3
    (order-9 patches, N = 27,000, eps 5e-8, GMRES 5e-10, A3, float64) against
    the values the paper prints (tests/golden/twisted_torus_table5.txt): the
    iteration counts of the two Laplace-Beltrami solves, the divergence norms
    of H and n x H, and |H|."""
    import os
    from workloads import surfaces as S
    from workloads.rhs import current_source_field
    gold = [l.split() for l in open(os.path.join(os.path.dirname(__file__), "golden", "twisted_torus_table5.txt"))
            if l.strip() and not l.startswith("#")]
    row = [float(x) for x in gold[0]]
    h_norm = float([g for g in gold if g[0] == "H_norm"][0][1])
    s = S.twisted_torus(10, 30, 8)
    assert s.N == int(row[0])
    ctx = lb.Context(0, lb.default_params(eps_quad=5e-8, tol=5e-10, formulation=lb.LB_A3, precision=lb.LB_FP64))
    ctx.upload_surface(s)
    ctx.build_corrections()
    n, w, _ = ctx.get_geometry()
    F = -np.cross(n, np.cross(n, current_source_field(s.X)))
    its = [ctx.solve_lb(f)[1]["iterations"]
           for f in (ctx.surface_div(F[None]), -ctx.surface_div(np.cross(n, F)[None]))]
    H, info = ctx.harmonic_fields(F[None])
    l2 = lambda f: np.sqrt(np.sum(w * f * f))
    # the GMRES details (norm, orthogonalisation) and the far rule are not fixed
    # by the paper: the counts agree within a few iterations
    assert abs(its[0] - row[1]) <= 3 and abs(its[1] - row[2]) <= 3, its
    assert abs(l2(np.linalg.norm(H[0], axis=1)) - h_norm) < 0.01 * h_norm
    # discretisation errors: same order of magnitude as the paper's
    assert row[3] / 2 < l2(ctx.surface_div(H[0][None])[0]) < 2 * row[3]
    assert l2(ctx.surface_div(H[1][None])[0]) < 2 * row[4]


@pytest.mark.parametrize("name", ["sphere300", "ellipsoid1200"])
@pytest.mark.parametrize("prec", ["fp64", "df64"])
def test_operator_A1(lb, name, prec):
    """A1 = div S grad_Gamma S + S W S (Section 4.1) against the oracle."""
    ctx, s, d = ctx_for(lb, name, formulation=lb.LB_A1,
                        precision=lb.LB_FP64 if prec == "fp64" else lb.LB_DF64)
    tau = np.random.default_rng(38).standard_normal((2, d.geo.N))
    # two nodal differentiations amplify the pair sums' rounding (~1e-15 in
    # float64, ~1e-14 in double-float) by about 1e3
    assert _rel(ctx.apply_A(tau), d.apply("A1", tau)) < (1e-11 if prec == "fp64" else 1e-10)
