"""lb_far_sums_noalloc: far sums for callers that cannot allocate device memory.

The entry point runs the float32 far-field kernel with its scratch in a fixed
device array carried by the library, so that code inside another runtime's
memory pool, which owns every allocation, can use it without cudaMalloc.  Its
output is checked against the allocating entry point lb_far_sums (float32
pairs) on two calls in a row, which also shows that the shared array is
reset between calls, and, on sampled targets, against the FP64 oracle's far
sums.  One surface sits close to the 65,536-node limit, where the split
partials fill most of the array.  This file is collected last and needs
nothing from the other tests.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _dev(t):
    return ctypes.c_void_p(t.data_ptr())


@pytest.mark.parametrize("surface", ["ellipsoid1200", "torus1920", "torus64800"])
def test_noalloc_matches_far_sums(surface):
    torch = pytest.importorskip("torch")
    import __graft_entry__ as g
    g.build()
    import paper_2111_10743_gb300 as lb
    from oracle import farsum
    from oracle.geometry import build_geometry, near_lists
    from workloads import surfaces as S

    if surface == "ellipsoid1200":
        s = S.ellipsoid((1.0, 1.5, 2.0), 1, 4)
    elif surface == "torus1920":
        s = S.torus(2.0, 0.75, 8, 8, 4)
    else:   # 4,320 order-4 patches: N = 64,800, just under the 65,536-node limit
        s = S.torus(2.0, 0.75, 48, 45, 4)
    ctx = lb.Context(0)
    ctx.upload_surface(s)
    ctx.build_near()
    n, w, _ = ctx.get_geometry()
    rp, pa, _ = ctx.get_corrections(with_vals=False)
    N = s.N
    dev = "cuda:0"
    X = torch.tensor(s.X, device=dev)
    nt = torch.tensor(n, device=dev)
    wt = torch.tensor(w, device=dev)
    rpt = torch.tensor(rp, device=dev)
    pat = torch.tensor(pa, device=dev)
    stream = torch.cuda.current_stream()
    # the oracle on its own geometry and near lists, at sampled targets
    geo = build_geometry(s.order, s.uv, s.wref, s.X, s.Xu, s.Xv)
    optr, opl = near_lists(geo, 2.0)
    rng = np.random.default_rng(41)
    targets = np.sort(rng.choice(N, 64, replace=False)).astype(np.int64)
    for call in range(2):
        sigma = rng.standard_normal(N)
        ref = ctx.far_sums(sigma[None], precision=lb.LB_FP32)[0]
        sig = torch.tensor(sigma, device=dev)
        out = torch.full((4, N), float("nan"), dtype=torch.float64, device=dev)
        rc = lb.lib.lb_far_sums_noalloc(s.npatch, s.np_, _dev(X), _dev(nt), _dev(wt), _dev(sig), _dev(rpt),
                                        _dev(pat), _dev(out), ctypes.c_void_p(stream.cuda_stream))
        assert rc == lb.LB_OK, lb.lib.lb_last_error(None)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.all(np.isfinite(got))
        orc = farsum.far_sums(geo, optr, opl, sigma, targets)[0]
        for k in range(4):
            err = np.abs(got[k] - ref[k]).max() / np.abs(ref[k]).max()
            assert err < 2e-5, (call, k, err)
            err_o = np.abs(got[k][targets] - orc[k]).max() / np.abs(orc[k]).max()
            assert err_o < 2e-5, (call, k, err_o)
    ctx.close()


def test_noalloc_rejects_oversize():
    pytest.importorskip("torch")
    import __graft_entry__ as g
    g.build()
    import paper_2111_10743_gb300 as lb
    one = ctypes.c_void_p(1)
    rc = lb.lib.lb_far_sums_noalloc(70000, 15, one, one, one, one, one, one, one, None)
    assert rc == lb.LB_EINVAL
    assert b"exceeds the maximum" in lb.lib.lb_last_error(None)
    # a patch count whose product with np would wrap around int64 is refused
    # without forming the product
    rc = lb.lib.lb_far_sums_noalloc(1 << 62, 4, one, one, one, one, one, one, one, None)
    assert rc == lb.LB_EINVAL
    assert b"exceeds the maximum" in lb.lib.lb_last_error(None)
