"""K7/K8 parity: GPU adjoint (frozen decisions) against the oracle's analytic
gradient, the oracle's finite differences, and the autograd wrapper against
the oracle.

Per-particle criterion: every component of dL/dx_k and dL/dm_k is within
GRAD_TOL of the oracle's sum of the absolute values of that component's terms
(the scale of its rounding error; tests/gpu_util.py gives the error budget).
A global check, max |error| / max |gradient| < TOL, is kept beside it."""
import numpy as np
import pytest

import ics
from gpu_util import GRAD_TOL, build_tree, device, grad_scaled_err, og, to_dev, torch

pytestmark = pytest.mark.gpu

# FP32 interactions with FP64 accumulators: per-term rounding ~1e-7 relative;
# tolerance on max |error| / max |gradient| over the checked particles.
TOL = 2e-5


def _gpu_adjoint(w, dev, theta, wt, **pkw):
    m = og()
    tree, _, _ = build_tree(w, dev, **pkw)
    wt_d = torch.tensor(wt, dtype=torch.float32, device=dev)
    dpos, dmass = m.shortrange_adjoint(tree, w.r_s, theta, wt_d)
    return dpos.cpu().numpy(), dmass.cpu().numpy()


def _check(gp, gm, orc_tree, w, theta, wt, s, what):
    op, om, pa, ma = orc_tree.adjoint(w.r_s, w.rcut, theta, wt, s, with_scale=True)
    ep, em = grad_scaled_err(gp, op, pa), grad_scaled_err(gm, om, ma)
    gep = np.abs(gp - op).max() / np.abs(op).max()
    gem = np.abs(gm - om).max() / np.abs(om).max()
    print(what, "per-particle pos", ep, "mass", em, "| global pos", gep, "mass", gem)
    assert ep < GRAD_TOL and em < GRAD_TOL
    assert gep < TOL and gem < TOL


@pytest.mark.parametrize("name,scale,theta", [("uniform4096", 1500, 0.5), ("nfw256", 20, 0.5),
                                              ("nfw256", 16, 0.0), ("zoom8m", 8000, 0.5)])
def test_adjoint_vs_oracle(orc, name, scale, theta):
    dev = device()
    w = ics.make(name, scale)
    wt = ics.loss_weights(w.n, 31).astype(np.float32).astype(np.float64)
    gp, gm = _gpu_adjoint(w, dev, theta, wt)
    T = orc.Tree(w.pos, w.mass, 2.8 * w.eps)
    s = np.arange(0, w.n, max(1, w.n // 400))
    _check(gp[s], gm[s], T, w, theta, wt, s, f"{name} theta={theta}")


def test_autograd_function(orc):
    """ShortRangeAccel (torch.autograd.Function): the gradients autograd
    returns for pos and mass against the oracle's analytic gradient, per
    particle, and against the direct adjoint call."""
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
    gp, gm = gp.cpu().numpy(), gm.cpu().numpy()
    wd = wt.double().cpu().numpy()
    T = orc.Tree(w.pos, w.mass, 2.8 * w.eps)
    s = np.arange(0, w.n, 9)
    _check(gp[s], gm[s], T, w, 0.5, wd, s, "autograd")
    # the direct adjoint call: the source-side sums are FP64 atomics whose
    # order is not fixed, so two runs agree up to FP64 summation order
    dp, dm = _gpu_adjoint(w, dev, 0.5, wd)
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
    for i, (p, m, *_rest) in enumerate(res):
        fp[i::workers] = p
        fm[i::workers] = m
    fl = np.zeros(64, np.int32)
    ap, am, sp_, sm_ = np.zeros((64, 3)), np.zeros(64), np.zeros((64, 3)), np.zeros(64)
    for i, (p, m, f, a1, a2, a3, a4) in enumerate(res):
        fl[i::workers] = f
        ap[i::workers], am[i::workers], sp_[i::workers], sm_[i::workers] = a1, a2, a3, a4
    ok = fl == 0
    print("fd: samples whose steps cross h or rcut (excluded):", int((~ok).sum()), "of 64",
          "(h:", int(((fl & 1) != 0).sum()), "rcut:", int(((fl & 2) != 0).sum()), ")")
    assert ok.sum() >= 48
    ep = np.abs(gp[s][ok] - fp[ok]).max() / np.abs(fp[ok]).max()
    em = np.abs(gm[s][ok] - fm[ok]).max() / np.abs(fm[ok]).max()
    print("fd: gpu pos", ep, "gpu mass", em)
    assert ep < TOL and em < TOL
    # the same 64 particles against the oracle's analytic gradient, per particle
    ep2, em2 = grad_scaled_err(gp[s], ap, sp_), grad_scaled_err(gm[s], am, sm_)
    print("analytic per-particle: pos", ep2, "mass", em2)
    assert ep2 < GRAD_TOL and em2 < GRAD_TOL

