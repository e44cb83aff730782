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


# ---------------------------------------------------------------- acceptance branch at theta > 0
# Hand-built trees whose outcome follows from the opening rule alone.  With
# leaf_size 12, a clump of 12 particles inside the level-4 cube
# C = [0.5, 0.5625)^3 (side s = 1/16, centre c = 0.53125 (1, 1, 1)) is one
# leaf node once every enclosing cube holds more than 12 particles.  For a
# lone target the walk either accepts that node (one monopole term at the
# clump's centre of mass, the value computed here from its definition) or
# opens it (the 12 particle pairs, inside the cut: the oracle's direct sum,
# itself pinned by closed forms).

def _short_range_F(r, r_s):
    """K(r) f(r) for r beyond the softening: f(u) / r^3 with u = r / (2 r_s),
    f(u) = erfc(u) + (2u / sqrt(pi)) exp(-u^2)."""
    from scipy.special import erfc
    u = r / (2.0 * r_s)
    return (erfc(u) + 2.0 * u / np.sqrt(np.pi) * np.exp(-u * u)) / r ** 3


def _clump(rng, lo, hi):
    return lo + (hi - lo) * rng.random((12, 3))


def _monopole(pos, mass, clump_idx, t, r_s):
    M = mass[clump_idx].sum()
    X = (mass[clump_idx, None] * pos[clump_idx]).sum(0) / M
    d = pos[t] - X
    return -M * _short_range_F(np.linalg.norm(d), r_s) * d


def _far_clump_set():
    rng = np.random.default_rng(2024)
    clump = _clump(rng, 0.5005, 0.562)            # spread over C
    # one extra particle in each enclosing cube (levels 1-3) but outside the
    # next one, all beyond any cut used below from the target
    extra = np.array([[0.9, 0.9, 0.9], [0.7, 0.7, 0.7], [0.6, 0.6, 0.6]])
    target = np.array([[0.45, 0.45, 0.45]])
    pos = np.concatenate([clump, extra, target])
    mass = np.concatenate([rng.uniform(0.5, 2.0, 12), np.ones(3), [1.0]])
    return pos, mass


def test_accepted_node_is_one_monopole_at_com(orc):
    """(i) theta = 0.5, rcut = 0.225: the clump's cube is inside the cut,
    outside the 1.2x enlargement around the target and s^2 < theta^2 d^2, so
    the target gets one term: -M F(|x - X|) (x - X), X the clump's COM."""
    pos, mass = _far_clump_set()
    r_s = 0.05
    t = len(pos) - 1
    T = orc.Tree(pos, mass, np.full(len(pos), 1e-4), leaf_size=12)
    a, c = T.walk(r_s, 4.5 * r_s, 0.5, [t])
    assert c[0] == 1
    ref = _monopole(pos, mass, np.arange(12), t, r_s)
    assert np.allclose(a[0], ref, rtol=1e-12, atol=0)


def test_node_straddling_the_cut_is_opened(orc):
    """(iii) the same clump with rcut = 0.15: its COM is inside the cut but
    its far corner is not, so the node is opened and each pair takes the cut
    on its own distance: the result is the direct pair sum."""
    pos, mass = _far_clump_set()
    r_s = 0.15 / 4.5
    t = len(pos) - 1
    h = np.full(len(pos), 1e-4)
    T = orc.Tree(pos, mass, h, leaf_size=12)
    a, c = T.walk(r_s, 0.15, 0.5, [t])
    ad, cd = orc.direct(pos, mass, h, 1.0, r_s, 0.15, [t])
    assert 0 < cd[0] < 12                       # the cut splits the clump
    assert c[0] == cd[0]
    assert np.allclose(a[0], ad[0], rtol=1e-12, atol=0)
    # a monopole of the whole clump would differ
    ref = _monopole(pos, mass, np.arange(12), t, r_s)
    assert np.linalg.norm(ref - ad[0]) > 1e-3 * np.linalg.norm(ad[0])


@pytest.mark.parametrize("offset,opened", [(0.59, True), (0.61, False)])
def test_containment_of_the_enlarged_cube(orc, offset, opened):
    """(ii) theta = 0.9, the clump packed in the corner of C away from the
    target, the target at c + offset s x (outside C, in the sibling cube).
    |x - COM| is large enough for s^2 < theta^2 d^2 but |x - c| is not, so a
    distance taken to the geometric centre would open both cases.  At
    offset 0.59 the target is inside the cube enlarged 1.2x (0.6 s) and the
    node is opened (the 12 pairs); at 0.61 it is accepted (one monopole)."""
    rng = np.random.default_rng(7)
    s = 0.0625
    clump = _clump(rng, 0.5005, 0.51)
    c = np.full(3, 0.53125)
    target = (c + np.array([offset * s, 0.0, 0.0]))[None, :]
    pos = np.concatenate([clump, target])
    mass = np.concatenate([rng.uniform(0.5, 2.0, 12), [1.0]])
    r_s = 0.05
    t = 12
    h = np.full(13, 1e-4)
    T = orc.Tree(pos, mass, h, leaf_size=12)
    a, cnt = T.walk(r_s, 4.5 * r_s, 0.9, [t])
    X = (mass[:12, None] * clump).sum(0) / mass[:12].sum()
    assert s * s < 0.81 * np.sum((pos[t] - X) ** 2)       # the angle test alone would accept
    assert s * s > 0.81 * np.sum((pos[t] - c) ** 2)       # ... measured from the centre it would not
    if opened:
        ad, cd = orc.direct(pos, mass, h, 1.0, r_s, 4.5 * r_s, [t])
        assert cnt[0] == cd[0] == 12
        assert np.allclose(a[0], ad[0], rtol=1e-12, atol=0)
    else:
        assert cnt[0] == 1
        assert np.allclose(a[0], _monopole(pos, mass, np.arange(12), t, r_s), rtol=1e-12, atol=0)
