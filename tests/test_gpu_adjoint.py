"""K7/K8 parity: GPU adjoint (frozen decisions) against the oracle's analytic
gradient, the oracle's finite differences, and the autograd wrapper."""
import numpy as np
import pytest

import ics
from gpu_util import build_tree, device, og, to_dev, torch

pytestmark = pytest.mark.gpu

# FP32 interactions with FP64 accumulators: per-term rounding ~1e-7 relative;
# tolerance on max |error| / max |gradient| over the checked particles.
TOL = 2e-5


def _gpu_adjoint(w, dev, theta, wt):
    m = og()
    tree, _, _ = build_tree(w, dev)
    wt_d = torch.tensor(wt, dtype=torch.float32, device=dev)
    dpos, dmass = m.shortrange_adjoint(tree, w.r_s, theta, wt_d)
    return dpos.cpu().numpy(), dmass.cpu().numpy()


@pytest.mark.parametrize("name,scale,theta", [("uniform4096", 1500, 0.5), ("nfw256", 20, 0.5),
                                              ("nfw256", 16, 0.0), ("zoom8m", 8000, 0.5)])
def test_adjoint_vs_oracle(orc, name, scale, theta):
    dev = device()
    w = ics.make(name, scale)
    wt = ics.loss_weights(w.n, 31).astype(np.float32).astype(np.float64)
    gp, gm = _gpu_adjoint(w, dev, theta, wt)
    T = orc.Tree(w.pos, w.mass, 2.8 * w.eps)
    s = np.arange(0, w.n, max(1, w.n // 400))
    op, om = T.adjoint(w.r_s, w.rcut, theta, wt, s)
    ep = np.abs(gp[s] - op).max() / np.abs(op).max()
    em = np.abs(gm[s] - om).max() / np.abs(om).max()
    print(name, theta, "pos", ep, "mass", em)
    assert ep < TOL and em < TOL


def test_autograd_function(orc):
    dev = device()
    m = og()
    w = ics.make("nfw256", 16)
    pos, mass, eps = to_dev(w, dev)
    pos.requires_grad_(True)
    mass.requires_grad_(True)
    acc = m.ShortRangeAccel.apply(pos, mass, eps, w.box, w.r_s, 0.5)
    wt = torch.tensor(ics.loss_weights(w.n, 5), dtype=torch.float32, device=dev)
    loss = (acc * wt).sum()
    gp, gm = torch.autograd.grad(loss, (pos, mass))
    dp, dm = _gpu_adjoint(w, dev, 0.5, wt.double().cpu().numpy())
    # The source-side sums are FP64 atomics whose order is not fixed, so two
    # runs agree up to FP64 summation-order rounding, not bit for bit.
    gp, gm = gp.cpu().numpy(), gm.cpu().numpy()
    assert np.abs(gp - dp).max() <= 1e-12 * np.abs(dp).max()
    assert np.abs(gm - dm).max() <= 1e-12 * np.abs(dm).max()


@pytest.mark.slow
def test_adjoint_fd_full_size(orc):
    """nfw128 adjoint set (2.1M clustered, seeded weights w ~ N(0, I)): GPU
    gradient vs central finite differences of the FP64 oracle's frozen-list
    loss (h = 1e-6 for positions, 1e-6 m for masses) on 64 seeded particles.
    The finite differences run in a spawn process pool (oracle only)."""
    import concurrent.futures as cf
    import multiprocessing as mp
    import os

    import oracle_workers
    w = ics.make("nfw128_adjoint")
    s = np.random.default_rng(64).choice(w.n, 64, replace=False)
    workers = max(1, min(16, os.cpu_count() or 1))
    chunks = [s[i::workers] for i in range(workers)]
    with cf.ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
        futs = [ex.submit(oracle_workers.fd_chunk, ("nfw128_adjoint", c, 0.5)) for c in chunks]
        dev = device()
        wt = w.w.astype(np.float32).astype(np.float64)
        gp, gm = _gpu_adjoint(w, dev, 0.5, wt)
        res = [f.result() for f in futs]
    fp = np.zeros((64, 3))
    fm = np.zeros(64)
    for i, (p, m) in enumerate(res):
        fp[i::workers] = p
        fm[i::workers] = m
    ep = np.abs(gp[s] - fp).max() / np.abs(fp).max()
    em = np.abs(gm[s] - fm).max() / np.abs(fm).max()
    print("fd: gpu pos", ep, "gpu mass", em)
    assert ep < TOL and em < TOL
