"""Pins for the oracle octree and Barnes-Hut walk (CPU only)."""
import numpy as np
import pytest

import ics


def _set(name, scale):
    w = ics.make(name, scale)
    return w


def _h(w):
    return 2.8 * w.eps


@pytest.mark.parametrize("name,scale", [("uniform4096", 700), ("nfw256", 12), ("zoom8m", 800)])
def test_node_moments(orc, name, scale):
    w = _set(name, scale)
    T = orc.Tree(w.pos, w.mass, _h(w), leaf_size=8)
    nd = T.nodes()
    M = T.nnodes
    assert nd["count"][0] == w.n
    # children: mass, count and member sets add up; leaves partition the set
    seen = np.zeros(w.n, np.int64)
    for k in range(M):
        mem = T.members(k)
        assert nd["mass"][k] == pytest.approx(w.mass[mem].sum(), rel=1e-14)
        com = (w.mass[mem, None] * w.pos[mem]).sum(0) / w.mass[mem].sum()
        # both sums run over positive terms: each is within (count - 1) ulp of exact
        assert np.allclose(nd["com"][k], com, rtol=2.3e-16 * len(mem), atol=0)
        assert nd["hmax"][k] == _h(w)[mem].max()
        if nd["leaf"][k]:
            seen[mem] += 1
            assert nd["count"][k] <= 8 or nd["level"][k] == 21
        else:
            c0, nc = nd["child0"][k], nd["nchild"][k]
            assert nd["count"][k] > 8
            assert nd["count"][c0:c0 + nc].sum() == nd["count"][k]
            assert nd["mass"][c0:c0 + nc].sum() == pytest.approx(nd["mass"][k], rel=1e-14)
            assert np.all(nd["level"][c0:c0 + nc] == nd["level"][k] + 1)
            # each child's cell sits inside the parent's
            assert np.all((nd["cell"][c0:c0 + nc] >> 1) == nd["cell"][k])
    assert np.all(seen == 1)


def test_tree_equals_key_prefix_runs(orc):
    """The octree's nodes are exactly the maximal runs of sorted Hilbert keys
    that share a 3*level-bit prefix, inside parents with more than B members
    (the key-sorted construction relies on this)."""
    w = _set("nfw256", 16)
    B = 8
    T = orc.Tree(w.pos, w.mass, _h(w), leaf_size=B)
    nd = T.nodes()
    keys, _, _ = orc.keys(w.pos)
    ks, _ = orc.sort(keys)
    tree_nodes = set()
    for k in range(T.nnodes):
        lev = int(nd["level"][k])
        pref = int(orc.hilbert_grid([nd["cell"][k]], lev)[0]) if lev > 0 else 0
        tree_nodes.add((lev, pref, int(nd["count"][k])))
    runs = set()
    frontier = [(0, 0, len(ks))]
    while frontier:
        lev, a, b = frontier.pop()
        pref = int(ks[a]) >> (63 - 3 * lev) if lev > 0 else 0
        runs.add((lev, pref, b - a))
        if b - a > B and lev < 21:
            sub = (ks[a:b] >> np.uint64(63 - 3 * (lev + 1))).astype(np.int64)
            cuts = np.flatnonzero(np.diff(sub)) + 1
            edges = [0] + cuts.tolist() + [b - a]
            for s, e in zip(edges[:-1], edges[1:]):
                frontier.append((lev + 1, a + s, a + e))
    assert tree_nodes == runs


@pytest.mark.parametrize("name,scale", [("uniform4096", 512), ("nfw256", 10), ("zoom8m", 600)])
def test_theta_zero_equals_direct(orc, name, scale):
    w = _set(name, scale)
    T = orc.Tree(w.pos, w.mass, _h(w))
    at, ct = T.walk(w.r_s, w.rcut, 0.0)
    ad, cd = orc.direct(w.pos, w.mass, _h(w), 1.0, w.r_s, w.rcut)
    assert np.array_equal(ct, cd)
    rel = np.linalg.norm(at - ad, axis=1) / np.maximum(np.linalg.norm(ad, axis=1), 1e-300)
    assert rel.max() < 1e-13


@pytest.mark.parametrize("theta", [0.0, 0.3, 0.5, 0.9])
def test_walk_covers_every_particle_once(orc, theta):
    w = _set("nfw256", 12)
    T = orc.Tree(w.pos, w.mass, _h(w))
    tg = np.arange(0, w.n, 7)
    assert T.cover_errors(w.rcut, theta, tg) == 0


def test_theta_half_accuracy_is_recorded(orc):
    """Monopole Barnes-Hut at theta = 0.5 against the direct sum: the error is
    measured (not a tolerance of the method); sanity bounds only."""
    w = _set("uniform4096", None)
    T = orc.Tree(w.pos, w.mass, _h(w))
    at, ct = T.walk(w.r_s, w.rcut, 0.5)
    ad, cd = orc.direct(w.pos, w.mass, _h(w), 1.0, w.r_s, w.rcut)
    rel = np.linalg.norm(at - ad, axis=1) / np.linalg.norm(ad, axis=1)
    assert np.sqrt(np.mean(rel ** 2)) < 0.05
    assert ct.sum() < cd.sum()
    # a smaller opening angle is more accurate
    a2, _ = T.walk(w.r_s, w.rcut, 0.2)
    rel2 = np.linalg.norm(a2 - ad, axis=1) / np.linalg.norm(ad, axis=1)
    assert np.percentile(rel2, 99) < 5e-3 < np.percentile(rel, 99)
