"""Key-range decomposition (the multi-GPU layout of the walk): its host
logic and collectives on 2 and 4 gloo ranks on CPU, with the FP64 oracle as
every rank's compute.  Each rank walks a contiguous range of walk groups of
the same tree; the assembled accelerations must equal the single-process
walk exactly and the summed partial-loss gradients the full gradient, and
the rebalanced ranges must split the interaction counts evenly."""
import socket

import numpy as np
import pytest

import ics
from paper_2606_17145_gb300.decomp import GROUP, group_work, partition


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


@pytest.mark.parametrize("nranks", [1, 2, 3, 4, 7])
def test_partition_is_contiguous_and_balanced(nranks):
    rng = np.random.default_rng(nranks)
    work = rng.pareto(1.5, 500) + 0.01
    r = partition(work, nranks)
    assert len(r) == nranks and r[0][0] == 0 and r[-1][1] == 500
    assert all(a[1] == b[0] for a, b in zip(r, r[1:]))          # contiguous, disjoint, covering
    sums = [work[g0:g1].sum() for g0, g1 in r]
    assert max(sums) <= work.sum() / nranks + work.max() + 1e-9


def test_partition_edge_cases():
    assert partition([], 3) == [(0, 0)] * 3
    assert partition([1.0, 1.0], 4)[-1][1] == 2
    assert partition(np.zeros(8), 2) == [(0, 4), (4, 8)]        # no work: split by groups
    c = np.arange(70)
    gw = group_work(c, 3)
    assert gw.tolist() == [c[:32].sum(), c[32:64].sum(), c[64:].sum()] and GROUP == 32


@pytest.mark.parametrize("nranks", [2, 4])
def test_ranks_reproduce_the_single_process_walk(orc, nranks):
    pytest.importorskip("torch")
    import multiprocessing as mp

    import decomp_workers
    name, scale = "nfw256", 12
    w = ics.make(name, scale)
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=decomp_workers.decomp_rank, args=(r, nranks, port, q, name, scale))
             for r in range(nranks)]
    for p in procs:
        p.start()
    out = sorted((q.get(timeout=180) for _ in procs), key=lambda t: t[0])
    errs = [o[2] for o in out if len(o) == 3 and o[1] == "error"]
    assert not errs, errs[0]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    T = orc.Tree(w.pos, w.mass, 2.8 * w.eps)
    a_ref, c_ref = T.walk(w.r_s, w.rcut, 0.5)
    wt = ics.loss_weights(w.n, 41)
    dp_ref, dm_ref = T.adjoint(w.r_s, w.rcut, 0.5, wt)
    rows_all = np.concatenate([o[2] for o in out])
    assert np.array_equal(np.sort(rows_all), np.arange(w.n))     # each particle owned by one rank
    moved = w.pos + 1e-4 * np.random.default_rng(7).standard_normal((w.n, 3))
    for rank, gathered, rows, acc, cnt, dpos, dmass, r1, r2, acc2 in out:
        assert np.array_equal(gathered, moved)                  # the all-gather by rows
        assert np.array_equal(acc, a_ref) and np.array_equal(cnt, c_ref)
        assert np.array_equal(acc2, a_ref)                      # after rebalancing too
        assert np.abs(dpos - dp_ref).max() <= 1e-12 * np.abs(dp_ref).max()
        assert np.abs(dmass - dm_ref).max() <= 1e-12 * np.abs(dm_ref).max()
        assert r2 == out[0][8]                                   # every rank takes the same ranges
    order = orc.sort(orc.keys(w.pos)[0])[1]
    gw = group_work(c_ref[order], (w.n + 31) // 32)
    sums = [gw[g0:g1].sum() for g0, g1 in out[0][8]]
    assert max(sums) <= gw.sum() / nranks + gw.max()
