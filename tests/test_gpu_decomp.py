"""Group-range walks (og_shortrange_accel_range / og_shortrange_adjoint_range),
the per-rank part of the key-range decomposition, on one GPU: the ranges of a
partition reproduce the full walk bit for bit and their partial-loss
gradients add up to the full gradient; the decomposition driver with one
rank gives the full results."""
import numpy as np
import pytest

import ics
from gpu_util import build_tree, device, og, to_dev, torch

pytestmark = pytest.mark.gpu


def _set():
    return ics.make("nfw256", 24)   # 13,824 clustered particles, 432 groups


def test_range_walks_reproduce_the_full_walk():
    from paper_2606_17145_gb300.decomp import partition
    dev = device()
    m = og()
    w = _set()
    tree, _, _ = build_tree(w, dev)
    a_full, t_full, c_full = m.shortrange_accel(tree, w.r_s, 0.5, counts=True)
    ng = int(tree.header.n_groups)
    rng = np.random.default_rng(3)
    for nranks in (2, 3, 5):
        acc = torch.zeros_like(a_full)
        tot = 0
        for g0, g1 in partition(rng.random(ng), nranks):
            _, t, _ = m.shortrange_accel(tree, w.r_s, 0.5, out=acc, groups=(g0, g1))
            tot += int(t.item())
        assert torch.equal(acc, a_full)
        assert tot == int(t_full.item())


def test_range_counts_and_untouched_rows():
    dev = device()
    m = og()
    w = _set()
    tree, keys, order = build_tree(w, dev)
    a_full, _, c_full = m.shortrange_accel(tree, w.r_s, 0.5, counts=True)
    g0, g1 = 100, 200
    sentinel = torch.full((w.n, 3), 7.0, dtype=torch.float32, device=dev)
    acc, t, _ = m.shortrange_accel(tree, w.r_s, 0.5, out=sentinel, groups=(g0, g1))
    rows = order[32 * g0: 32 * g1].long()
    mine = torch.zeros(w.n, dtype=torch.bool, device=dev)
    mine[rows] = True
    assert torch.equal(acc[mine], a_full[mine])
    assert bool((acc[~mine] == 7.0).all())
    assert int(t.item()) == int(c_full[rows].sum().item())


def test_range_adjoints_add_up_to_the_full_adjoint():
    from paper_2606_17145_gb300.decomp import partition
    dev = device()
    m = og()
    w = _set()
    tree, _, _ = build_tree(w, dev)
    wt = torch.tensor(ics.loss_weights(w.n, 12), dtype=torch.float32, device=dev)
    dp, dm = m.shortrange_adjoint(tree, w.r_s, 0.5, wt)
    ng = int(tree.header.n_groups)
    sp = torch.zeros_like(dp)
    sm = torch.zeros_like(dm)
    for g0, g1 in partition(np.ones(ng), 4):
        p, q = m.shortrange_adjoint(tree, w.r_s, 0.5, wt, groups=(g0, g1))
        sp += p
        sm += q
    assert float((sp - dp).abs().max()) <= 1e-12 * float(dp.abs().max())
    assert float((sm - dm).abs().max()) <= 1e-12 * float(dm.abs().max())


def test_empty_and_invalid_ranges():
    dev = device()
    m = og()
    w = _set()
    tree, _, _ = build_tree(w, dev)
    ng = int(tree.header.n_groups)
    sentinel = torch.full((w.n, 3), 3.0, dtype=torch.float32, device=dev)
    acc, t, _ = m.shortrange_accel(tree, w.r_s, 0.5, out=sentinel, groups=(5, 5))
    assert int(t.item()) == 0 and bool((acc == 3.0).all())
    wt = torch.ones((w.n, 3), dtype=torch.float32, device=dev)
    dp, dm = m.shortrange_adjoint(tree, w.r_s, 0.5, wt, groups=(ng, ng))
    assert float(dp.abs().max()) == 0.0 and float(dm.abs().max()) == 0.0
    for bad in ((-1, 3), (4, 2), (0, ng + 1)):
        with pytest.raises(m.OGError) as e:
            m.shortrange_accel(tree, w.r_s, 0.5, groups=bad)
        assert e.value.code == 1


def test_decomposition_driver_on_one_gpu():
    from paper_2606_17145_gb300.decomp import CudaCompute, KeyRangeDecomposition
    dev = device()
    m = og()
    w = _set()
    pos, mass, eps = to_dev(w, dev)
    tree, _, _ = build_tree(w, dev)
    a_full, _, c_full = m.shortrange_accel(tree, w.r_s, 0.5, counts=True)
    wt = torch.tensor(ics.loss_weights(w.n, 13), dtype=torch.float32, device=dev)
    dp, dm = m.shortrange_adjoint(tree, w.r_s, 0.5, wt)
    D = KeyRangeDecomposition(0, 1, CudaCompute(w.n, mass, eps, w.box, w.r_s, 0.5)).build(pos)
    acc, cnt = D.accel()
    assert torch.equal(acc, a_full) and torch.equal(cnt, c_full)
    gp, gm = D.adjoint(wt)
    assert float((gp - dp).abs().max()) <= 1e-12 * float(dp.abs().max())
    assert float((gm - dm).abs().max()) <= 1e-12 * float(dm.abs().max())
    assert D.rebalance(cnt) == [(0, int(tree.header.n_groups))]
