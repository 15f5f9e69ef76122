"""Correction checkpoints: digest, round trip and refusals (host only)."""
import numpy as np
import pytest

from paper_2111_10743_gb300 import checkpoint as ck


def _geom(seed=0):
    from workloads.configs import config
    s = config(1).surface
    return (s.npatch, s.order, s.uv, s.wref, s.X.copy(), s.Xu, s.Xv)


def _csr(rng, N=300, npatch=20, np_=15):
    counts = rng.integers(1, 5, N)
    rp = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    pa = np.concatenate([np.sort(rng.choice(npatch, k, replace=False)) for k in counts]).astype(np.int32)
    vals = rng.standard_normal((rp[-1], 4, np_))
    return rp, pa, vals


def test_digest_is_stable_and_sensitive():
    g = _geom()
    d0 = ck.geometry_digest(*g)
    assert d0 == ck.geometry_digest(*_geom())
    X = g[4].copy()
    X[17, 1] = np.nextafter(X[17, 1], 2.0)   # one ulp of one coordinate
    assert ck.geometry_digest(*g[:4], X, *g[5:]) != d0
    assert ck.geometry_digest(g[0], g[1] + 1, *g[2:]) != d0


def test_round_trip_and_refusals(tmp_path):
    rng = np.random.default_rng(1)
    rp, pa, vals = _csr(rng)
    d = ck.geometry_digest(*_geom())
    path = tmp_path / "corr.npz"
    ck.save(path, d, 2.0, 1e-12, rp, pa, vals)
    a, b, c = ck.load(path, d, 2.0, 1e-12)
    assert np.array_equal(a, rp) and np.array_equal(b, pa) and np.array_equal(c, vals)
    with pytest.raises(ck.CheckpointError, match="another geometry"):
        ck.load(path, "0" * 64, 2.0, 1e-12)
    with pytest.raises(ck.CheckpointError, match="parameters"):
        ck.load(path, d, 3.0, 1e-12)
    with pytest.raises(ck.CheckpointError, match="parameters"):
        ck.load(path, d, 2.0, 1e-10)
    # malformed CSR is refused on save
    bad = rp.copy()
    bad[-1] += 1
    with pytest.raises(ck.CheckpointError):
        ck.save(tmp_path / "bad.npz", d, 2.0, 1e-12, bad, pa, vals)
    v2 = vals.copy()
    v2[3, 1, 2] = np.nan
    with pytest.raises(ck.CheckpointError):
        ck.save(tmp_path / "bad2.npz", d, 2.0, 1e-12, rp, pa, v2)


def test_csr_structure_refusals():
    """Patch indices outside [0, npatch), rows that are not strictly
    ascending, a decreasing row pointer and a wrong vals shape are refused
    before anything reaches the library."""
    rng = np.random.default_rng(2)
    rp, pa, vals = _csr(rng)
    ck._check_csr(rp, pa, vals, N=300, npatch=20, np_=15)
    p2 = pa.copy()
    p2[5] = 20
    with pytest.raises(ck.CheckpointError, match="outside"):
        ck._check_csr(rp, p2, vals, N=300, npatch=20, np_=15)
    p2[5] = -1
    with pytest.raises(ck.CheckpointError, match="outside"):
        ck._check_csr(rp, p2, vals, N=300, npatch=20, np_=15)
    # swap two patches inside a row of at least two blocks
    i = int(np.nonzero(np.diff(rp) >= 2)[0][0])
    p3 = pa.copy()
    p3[rp[i]], p3[rp[i] + 1] = p3[rp[i] + 1], p3[rp[i]]
    with pytest.raises(ck.CheckpointError, match="ascending"):
        ck._check_csr(rp, p3, vals, N=300, npatch=20, np_=15)
    r2 = rp.copy()
    r2[10] = r2[11] + 1
    with pytest.raises(ck.CheckpointError, match="row pointer"):
        ck._check_csr(r2, pa, vals)
    with pytest.raises(ck.CheckpointError, match="n_p"):
        ck._check_csr(rp, pa, vals[:, :3])
    with pytest.raises(ck.CheckpointError, match="N \\+ 1"):
        ck._check_csr(rp, pa, vals, N=299)
