"""K6/K6d parity: the GPU walks against the oracle.

Tolerances (from the stated precision pattern):
* FP32-Kahan vs the oracle tree at the same theta: rms relative <= 1e-5;
* FP32-Kahan at theta = 0 vs the oracle direct sum: rms relative <= 1e-6;
* FP64 walk vs the oracle tree: max relative <= 1e-11 (rounding order only);
* interaction counts: equal per particle (decisions are re-taken in FP64 when
  FP32 cannot settle them, so the sets of terms are the oracle's).
"""
import numpy as np
import pytest

import ics
from gpu_util import GRAD_TOL, device, err_stats, forward, grad_scaled_err, og, torch

pytestmark = pytest.mark.gpu


def _oracle_tree(orc, w):
    return orc.Tree(w.pos, w.mass, 2.8 * w.eps)


def test_uniform4096_theta0_vs_direct(orc):
    dev = device()
    w = ics.make("uniform4096")
    a, tot, cnt, _ = forward(w, dev, 0.0)
    ad, cd = orc.direct(w.pos, w.mass, 2.8 * w.eps, 1.0, w.r_s, w.rcut)
    assert np.array_equal(cnt, cd)
    assert tot == cd.sum()
    st = err_stats(a, ad)
    print("theta=0 vs direct", st)
    assert st["rms"] <= 1e-6


def test_uniform4096_theta_half_vs_tree(orc):
    dev = device()
    w = ics.make("uniform4096")
    a, tot, cnt, _ = forward(w, dev, 0.5)
    ao, co = _oracle_tree(orc, w).walk(w.r_s, w.rcut, 0.5)
    assert np.array_equal(cnt, co)
    st = err_stats(a, ao)
    print("theta=0.5 vs tree", st)
    assert st["rms"] <= 1e-5


@pytest.mark.parametrize("name,scale,theta", [("zeldovich128", 32, 0.5), ("nfw256", 32, 0.5),
                                              ("zoom8m", 20000, 0.5), ("nfw256", 24, 0.0),
                                              ("nfw256", 24, 0.9), ("uniform4096", 1000, 0.3)])
def test_small_sets_vs_tree(orc, name, scale, theta):
    dev = device()
    w = ics.make(name, scale)
    a, tot, cnt, _ = forward(w, dev, theta)
    ao, co = _oracle_tree(orc, w).walk(w.r_s, w.rcut, theta)
    assert np.array_equal(cnt, co)
    st = err_stats(a, ao)
    print(name, theta, st)
    assert st["rms"] <= 1e-5


@pytest.mark.parametrize("theta", [0.0, 0.5])
def test_fp64_walk_vs_tree(orc, theta):
    dev = device()
    w = ics.make("nfw256", 24)
    a, tot, cnt, _ = forward(w, dev, theta, prec="fp64")
    ao, co = _oracle_tree(orc, w).walk(w.r_s, w.rcut, theta)
    assert np.array_equal(cnt, co)
    st = err_stats(a, ao)
    assert st["max"] <= 1e-11


@pytest.mark.parametrize("n", [1, 2, 9, 33, 1000])
def test_ragged_and_tiny(orc, n):
    dev = device()
    w = ics.make("uniform4096", n)
    w.r_s = 0.05
    a, tot, cnt, _ = forward(w, dev, 0.5)
    ao, co = _oracle_tree(orc, w).walk(w.r_s, w.rcut, 0.5)
    assert np.array_equal(cnt, co)
    if n > 1:
        assert err_stats(a, ao)["rms"] <= 1e-5


def test_non_unit_box_and_leaf_sizes(orc):
    dev = device()
    w = ics.make("nfw256", 16)
    w.pos = w.pos * 64.0
    w.box = 64.0
    w.r_s = w.r_s * 64.0
    w.eps = w.eps * 64.0
    for B in (1, 8, 32):
        a, tot, cnt, _ = forward(w, dev, 0.5, leaf_size=B)
        ao, co = orc.Tree(w.pos, w.mass, 2.8 * w.eps, box=64.0, leaf_size=B).walk(w.r_s, w.rcut, 0.5)
        assert np.array_equal(cnt, co)
        assert err_stats(a, ao)["rms"] <= 1e-5


@pytest.mark.slow
@pytest.mark.parametrize("name", ["zeldovich128", "nfw256", "zoom8m"])
def test_full_size_sampled(orc, name):
    """Full-size sets in the benchmark's launch configuration; the oracle
    walks a seeded sample of targets."""
    dev = device()
    w = ics.make(name)
    a, tot, cnt, _ = forward(w, dev, 0.5)
    s = np.random.default_rng(123).choice(w.n, 512, replace=False)
    T = _oracle_tree(orc, w)
    ao, co = T.walk(w.r_s, w.rcut, 0.5, s)
    assert np.array_equal(cnt[s], co)
    st = err_stats(a[s], ao)
    print(name, st, "interactions", tot)
    assert st["rms"] <= 1e-5
    assert np.all(np.isfinite(a))
    # momentum-like sanity at any size: total interactions match the counts
    assert tot == int(cnt.astype(np.int64).sum())


def test_deterministic_repeat():
    dev = device()
    w = ics.make("nfw256", 20)
    a1, t1, c1, _ = forward(w, dev, 0.5)
    a2, t2, c2, _ = forward(w, dev, 0.5)
    assert np.array_equal(a1, a2) and t1 == t2


def test_walk_iteration_cap_reports_error():
    """A walk that exceeds its node-visit cap stops and reports OG_EWALK
    through the workspace status (no trap, the context stays usable)."""
    dev = device()
    m = og()
    w = ics.make("uniform4096", 2000)
    from gpu_util import build_tree
    tree, _, _ = build_tree(w, dev, max_walk_iters=5)
    with pytest.raises(m.OGError) as e:
        m.shortrange_accel(tree, w.r_s, 0.5)
    assert e.value.code == 4
    # the device is still usable afterwards
    tree2, _, _ = build_tree(w, dev)
    acc, tot, _ = m.shortrange_accel(tree2, w.r_s, 0.5)
    assert tot.item() > 0


def test_walk_refuses_a_failed_tree():
    """A tree whose build ran out of node capacity is flagged; the walk
    refuses it with OG_ETREE instead of reading it."""
    dev = device()
    m = og()
    w = ics.make("uniform4096", 3000)
    pos = torch.tensor(w.pos, device=dev)
    mass = torch.tensor(w.mass, device=dev)
    keys, order = m.keys_sort(pos, 1.0)
    tree = m.tree_build(keys, order, pos, mass, 1.0 / 480, 1.0, p=m.params(node_capacity=40), check=False)
    with pytest.raises(m.OGError) as e:
        m.shortrange_accel(tree, w.r_s, 0.5)
    assert e.value.code == 5


def _dense_clump(seed=77, n_clump=3000, n_bg=1000):
    """A compact clump much smaller than r_cut in a uniform background: every
    batch of the clump's groups has all 32 x 32 (target, source) pairs inside
    the cut, more than the pair list holds at once."""
    rng = np.random.default_rng(seed)
    clump = 0.5 + rng.normal(scale=0.002, size=(n_clump, 3))
    pos = np.concatenate([clump, rng.random((n_bg, 3))])
    n = pos.shape[0]
    return ics.Workload("dense_clump", pos, np.full(n, 1.0 / n), np.full(n, 1e-4), 1.0, 0.004, (0.0, 0.5, 0.9))


@pytest.mark.parametrize("theta", [0.0, 0.5, 0.9])
def test_dense_clump_vs_tree(orc, theta):
    dev = device()
    w = _dense_clump()
    a, tot, cnt, _ = forward(w, dev, theta)
    ao, co = _oracle_tree(orc, w).walk(w.r_s, w.rcut, theta)
    assert np.array_equal(cnt, co)
    st = err_stats(a, ao)
    print("dense clump", theta, st, "interactions", tot)
    assert st["rms"] <= 1e-5


def test_dense_clump_adjoint(orc):
    dev = device()
    m = og()
    w = _dense_clump(seed=78)
    wt = ics.loss_weights(w.n, 9).astype(np.float32).astype(np.float64)
    from gpu_util import build_tree
    tree, _, _ = build_tree(w, dev)
    dpos, dmass = m.shortrange_adjoint(tree, w.r_s, 0.5, torch.tensor(wt, dtype=torch.float32, device=dev))
    gp, gm = dpos.cpu().numpy(), dmass.cpu().numpy()
    s = np.arange(0, w.n, 13)
    op, om, pa, ma = _oracle_tree(orc, w).adjoint(w.r_s, w.rcut, 0.5, wt, s, with_scale=True)
    ep = np.abs(gp[s] - op).max() / np.abs(op).max()
    em = np.abs(gm[s] - om).max() / np.abs(om).max()
    print("dense clump adjoint", ep, em, grad_scaled_err(gp[s], op, pa), grad_scaled_err(gm[s], om, ma))
    assert ep < 2e-5 and em < 2e-5
    assert grad_scaled_err(gp[s], op, pa) < GRAD_TOL and grad_scaled_err(gm[s], om, ma) < GRAD_TOL


@pytest.mark.parametrize("name,scale,deep", [("nfw256", 24, 1), ("zoom8m", 20000, 3), ("uniform4096", None, 2)])
def test_single_range_pops_vs_tree(orc, name, scale, deep):
    """With the deep-stack threshold lowered, most traversal steps pop a
    single child range; the terms must stay exactly the per-target walk's."""
    dev = device()
    w = ics.make(name, scale) if scale else ics.make(name)
    a, tot, cnt, _ = forward(w, dev, 0.5, deep_stack=deep)
    ao, co = _oracle_tree(orc, w).walk(w.r_s, w.rcut, 0.5)
    assert np.array_equal(cnt, co)
    assert err_stats(a, ao)["rms"] <= 1e-5


def test_single_range_pops_adjoint(orc):
    dev = device()
    m = og()
    w = _dense_clump(seed=79, n_clump=1500, n_bg=1500)
    wt = ics.loss_weights(w.n, 10).astype(np.float32).astype(np.float64)
    from gpu_util import build_tree
    tree, _, _ = build_tree(w, dev, deep_stack=1)
    dpos, dmass = m.shortrange_adjoint(tree, w.r_s, 0.5, torch.tensor(wt, dtype=torch.float32, device=dev))
    gp, gm = dpos.cpu().numpy(), dmass.cpu().numpy()
    s = np.arange(0, w.n, 11)
    op, om, pa, ma = _oracle_tree(orc, w).adjoint(w.r_s, w.rcut, 0.5, wt, s, with_scale=True)
    assert np.abs(gp[s] - op).max() / np.abs(op).max() < 2e-5
    assert np.abs(gm[s] - om).max() / np.abs(om).max() < 2e-5
    assert grad_scaled_err(gp[s], op, pa) < GRAD_TOL and grad_scaled_err(gm[s], om, ma) < GRAD_TOL


def _scaled(w, L):
    w.pos = w.pos * L
    w.box = L
    w.r_s = w.r_s * L
    w.eps = w.eps * L
    return w


def test_non_power_of_two_box_vs_tree(orc):
    """Box side 3 (not a power of two): the tree build divides by L."""
    dev = device()
    w = _scaled(ics.make("nfw256", 20), 3.0)
    a, tot, cnt, _ = forward(w, dev, 0.5)
    ao, co = orc.Tree(w.pos, w.mass, 2.8 * w.eps, box=3.0).walk(w.r_s, w.rcut, 0.5)
    assert np.array_equal(cnt, co)
    assert err_stats(a, ao)["rms"] <= 1e-5


def test_non_power_of_two_box_adjoint(orc):
    dev = device()
    m = og()
    w = _scaled(ics.make("nfw256", 16), 3.0)
    wt = ics.loss_weights(w.n, 12).astype(np.float32).astype(np.float64)
    from gpu_util import build_tree
    tree, _, _ = build_tree(w, dev)
    dpos, dmass = m.shortrange_adjoint(tree, w.r_s, 0.5, torch.tensor(wt, dtype=torch.float32, device=dev))
    gp, gm = dpos.cpu().numpy(), dmass.cpu().numpy()
    s = np.arange(0, w.n, 7)
    op, om, pa, ma = orc.Tree(w.pos, w.mass, 2.8 * w.eps, box=3.0).adjoint(w.r_s, w.rcut, 0.5, wt, s,
                                                                          with_scale=True)
    assert np.abs(gp[s] - op).max() / np.abs(op).max() < 2e-5
    assert np.abs(gm[s] - om).max() / np.abs(om).max() < 2e-5
    assert grad_scaled_err(gp[s], op, pa) < GRAD_TOL and grad_scaled_err(gm[s], om, ma) < GRAD_TOL


def test_momentum_at_theta_zero():
    """At theta = 0 every term is a particle pair, and pair forces are
    antisymmetric: sum_i m_i a_i vanishes up to FP32 rounding of the terms."""
    dev = device()
    w = ics.make("zeldovich128", 27)   # 19,683 particles
    a, tot, cnt, _ = forward(w, dev, 0.0)
    ma = w.mass[:, None] * a
    assert np.abs(ma.sum(axis=0)).max() <= 1e-5 * np.abs(ma).sum(axis=0).max()


def test_large_opening_angle_vs_tree(orc):
    """theta = 1.2: far more accepted nodes and mixed decisions."""
    dev = device()
    w = ics.make("nfw256", 24)
    a, tot, cnt, _ = forward(w, dev, 1.2)
    ao, co = _oracle_tree(orc, w).walk(w.r_s, w.rcut, 1.2)
    assert np.array_equal(cnt, co)
    assert err_stats(a, ao)["rms"] <= 1e-5


def test_coincident_particles(orc):
    """100 particles at one point (a level-21 leaf that cannot split) in a
    background: their mutual pairs count and give zero force, nothing is NaN."""
    dev = device()
    rng = np.random.default_rng(93)
    pos = np.concatenate([np.full((100, 3), 0.3141592653589793), rng.random((1900, 3))])
    n = pos.shape[0]
    w = ics.Workload("coincident", pos, np.full(n, 1.0 / n), np.full(n, 1e-3), 1.0, 0.02, (0.5,))
    a, tot, cnt, _ = forward(w, dev, 0.5)
    ao, co = _oracle_tree(orc, w).walk(w.r_s, w.rcut, 0.5)
    assert np.all(np.isfinite(a))
    assert np.array_equal(cnt, co)
    assert cnt[:100].min() >= 99
    assert err_stats(a[100:], ao[100:])["rms"] <= 1e-5
    # the coincident ones feel only the background
    assert np.abs(a[:100] - ao[:100]).max() <= 1e-5 * np.abs(ao[:100]).max() + 1e-12

