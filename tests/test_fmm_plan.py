"""Octree plan for a fast-multipole far field (host only, no GPU).

Checked by brute force on small node sets: the Morton order and the leaf
ranges partition the nodes, each node lies in its leaf's cell (decoded here
from the key bits), U lists are exactly the adjacent leaves, V lists are
non-adjacent children of the parent's neighbours, and every pair of leaves
is covered exactly once (by U, or by V at exactly one level).  With the
leaf side set from the near criterion every near (node, patch) pair lies in
adjacent leaves.
"""
import numpy as np
import pytest


@pytest.fixture(scope="module")
def lb():
    import __graft_entry__ as g
    g.build()
    import paper_2111_10743_gb300 as lb
    return lb


def _decode(key):
    """Integer cell coordinates from an interleaved key (x bit 0, y bit 1, z bit 2)."""
    c = np.zeros((len(key), 3), np.int64)
    for bit in range(21):
        for k in range(3):
            c[:, k] |= ((key >> (3 * bit + k)) & 1) << bit
    return c


def _check(p, X):
    n = X.shape[0]
    d = p["depth"]
    lp = p["level_ptr"]
    assert np.array_equal(np.sort(p["perm"]), np.arange(n))
    L0, nb = lp[d], lp[d + 1]
    nleaf = nb - L0
    npt = p["node_ptr"]
    assert npt[0] == 0 and npt[-1] == n and np.all(np.diff(npt) > 0)
    keys = p["box_key"]
    for l in range(d + 1):
        assert np.all(np.diff(keys[lp[l]:lp[l + 1]]) > 0)
    for b in range(lp[1], nb):
        assert keys[p["box_parent"][b]] == keys[b] >> 3
    # every node inside its leaf's cell
    cells = _decode(keys[L0:])
    h = p["side"] / 2 ** d
    leaf_of = np.repeat(np.arange(nleaf), np.diff(npt))
    Y = X[p["perm"]]
    lo = p["lo"][None, :] + cells[leaf_of] * h
    assert np.all(Y >= lo - 1e-12 * p["side"]) and np.all(Y <= lo + h + 1e-12 * p["side"])
    # U lists: exactly the adjacent leaves
    adj = np.all(np.abs(cells[:, None, :] - cells[None, :, :]) <= 1, axis=2)
    U = np.zeros((nleaf, nleaf), bool)
    for b in range(nleaf):
        U[b, p["u_idx"][p["u_ptr"][b]:p["u_ptr"][b + 1]]] = True
    assert np.array_equal(U, adj)
    # V lists: same level, not adjacent, parents adjacent; coverage exactly once
    level = np.searchsorted(lp, np.arange(nb), side="right") - 1
    allc = np.concatenate([_decode(keys[lp[l]:lp[l + 1]]) for l in range(d + 1)])
    anc = np.zeros((d + 1, nleaf), np.int64)   # ancestor box of each leaf per level
    anc[d] = np.arange(L0, nb)
    for l in range(d - 1, -1, -1):
        anc[l] = p["box_parent"][anc[l + 1]]
    cover = U.astype(np.int64)
    for b in range(nb):
        vs = p["v_idx"][p["v_ptr"][b]:p["v_ptr"][b + 1]]
        if len(vs) == 0:
            continue
        assert level[b] >= 2 and np.all(level[vs] == level[b])
        assert np.all(np.abs(allc[vs] - allc[b]).max(axis=1) >= 2)
        pb, pv = p["box_parent"][b], p["box_parent"][vs]
        assert np.all(np.abs(allc[pv] - allc[pb]).max(axis=1) <= 1)
        l = level[b]
        rows = np.nonzero(anc[l] == b)[0]
        cols = np.nonzero(np.isin(anc[l], vs))[0]
        cover[np.ix_(rows, cols)] += 1
    assert np.all(cover == 1)
    return leaf_of


@pytest.mark.parametrize("min_side,n", [(0.5, 400), (0.2, 1500), (0.1, 3000)])
def test_plan_on_sphere_nodes(lb, min_side, n):
    X = np.random.default_rng(n).standard_normal((n, 3))
    X /= np.linalg.norm(X, axis=1, keepdims=True)
    p = lb.fmm_plan(X, min_side)
    assert p["side"] / 2 ** p["depth"] >= min_side
    assert p["depth"] == 20 or p["side"] / 2 ** (p["depth"] + 1) < min_side
    _check(p, X)


def test_near_pairs_lie_in_adjacent_leaves(lb):
    from oracle.geometry import build_geometry, near_lists
    from workloads import surfaces as S
    s = S.ellipsoid((1.0, 1.5, 2.0), 3, 3)
    g = build_geometry(s.order, s.uv, s.wref, s.X, s.Xu, s.Xv)
    ptr, pl = near_lists(g, 2.0)
    p = lb.fmm_plan(g.X, (2.0 + 1.0) * g.radius.max())
    assert p["depth"] >= 3
    leaf_of = np.empty(g.N, np.int64)
    leaf_of[p["perm"]] = np.repeat(np.arange(len(p["node_ptr"]) - 1), np.diff(p["node_ptr"]))
    for i in range(g.N):
        nbr = set(p["u_idx"][p["u_ptr"][leaf_of[i]]:p["u_ptr"][leaf_of[i] + 1]])
        for P in pl[ptr[i]:ptr[i + 1]]:
            assert set(leaf_of[P * g.np_:(P + 1) * g.np_]) <= nbr


def test_plan_errors(lb):
    with pytest.raises(lb.LBError) as e:
        lb.fmm_plan(np.zeros((0, 3)), 0.1)
    assert e.value.code == lb.LB_EINVAL
    X = np.zeros((4, 3))
    X[2, 1] = np.nan
    with pytest.raises(lb.LBError) as e:
        lb.fmm_plan(X, 0.1)
    assert e.value.code == lb.LB_EINVAL
    # one node: a single box at depth 0 ... max_depth, covered by U alone
    p = lb.fmm_plan(np.ones((1, 3)), 0.5, max_depth=3)
    assert p["node_ptr"].tolist() == [0, 1] and p["u_idx"].tolist() == [0]
