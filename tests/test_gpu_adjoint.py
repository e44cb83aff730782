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
    assert np.array_equal(gp.cpu().numpy(), dp)
    assert np.array_equal(gm.cpu().numpy(), dm)


@pytest.mark.slow
def test_adjoint_fd_full_size(orc):
    """nfw128 adjoint set (2.1M clustered): GPU gradient vs the oracle's
    central finite differences (h = 1e-6) on 64 seeded particles."""
    dev = device()
    w = ics.make("nfw128_adjoint")
    wt = w.w.astype(np.float32).astype(np.float64)
    gp, gm = _gpu_adjoint(w, dev, 0.5, wt)
    T = orc.Tree(w.pos, w.mass, 2.8 * w.eps)
    s = np.random.default_rng(64).choice(w.n, 64, replace=False)
    fp, fm = T.fd(w.r_s, w.rcut, 0.5, wt, s, hx=1e-6, hm_rel=1e-6)
    op, om = T.adjoint(w.r_s, w.rcut, 0.5, wt, s)
    ep = np.abs(gp[s] - fp).max() / np.abs(fp).max()
    em = np.abs(gm[s] - fm).max() / np.abs(fm).max()
    eo = np.abs(op - fp).max() / np.abs(fp).max()
    print("fd: gpu pos", ep, "gpu mass", em, "oracle analytic vs fd", eo)
    assert eo < 1e-6
    assert ep < TOL and em < TOL
