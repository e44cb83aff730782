"""Parity of the fused forward + adjoint walk (og_shortrange_accel_adjoint).

The fused walk takes the same decisions, batches and summation order as the
separate walks, so:
* acc, the interaction total and the per-particle counts equal
  og_shortrange_accel's bit for bit;
* dpos, dmass equal og_shortrange_adjoint's up to the order of the FP64
  atomic additions of the node sums (well below 1e-12 of each component's
  term-magnitude scale);
* both sides also meet the oracle's criteria directly: counts equal to the
  oracle tree's, acc within rms 1e-5 of it, gradients within GRAD_TOL of the
  oracle's term-magnitude scale per component.
"""
import numpy as np
import pytest

import ics
from gpu_util import GRAD_TOL, build_tree, device, err_stats, grad_scaled_err, og, torch

pytestmark = pytest.mark.gpu


def _run(w, dev, theta, wt):
    m = og()
    tree, _, _ = build_tree(w, dev)
    wt_d = torch.tensor(wt, dtype=torch.float32, device=dev)
    af, tf, cf = m.shortrange_accel(tree, w.r_s, theta, counts=True)
    dps, dms = m.shortrange_adjoint(tree, w.r_s, theta, wt_d)
    au, tu, cu, dpu, dmu = m.shortrange_accel_adjoint(tree, w.r_s, theta, wt_d, counts=True)
    torch.cuda.synchronize()
    cpu = lambda t: t.cpu().numpy()
    return dict(af=cpu(af), tf=int(tf.item()), cf=cpu(cf), dps=cpu(dps), dms=cpu(dms),
                au=cpu(au), tu=int(tu.item()), cu=cpu(cu), dpu=cpu(dpu), dmu=cpu(dmu))


@pytest.mark.parametrize("name,scale,theta", [("uniform4096", 1500, 0.5), ("nfw256", 20, 0.5),
                                              ("nfw256", 16, 0.0), ("zoom8m", 8000, 0.5),
                                              ("zeldovich128", 32, 0.9)])
def test_fused_equals_separate_and_oracle(orc, name, scale, theta):
    dev = device()
    w = ics.make(name, scale)
    wt = ics.loss_weights(w.n, 31).astype(np.float32).astype(np.float64)
    r = _run(w, dev, theta, wt)
    # forward outputs: bit for bit
    assert np.array_equal(r["au"].view(np.uint32), r["af"].view(np.uint32))
    assert np.array_equal(r["cu"], r["cf"])
    assert r["tu"] == r["tf"]
    # against the oracle tree
    T = orc.Tree(w.pos, w.mass, 2.8 * w.eps)
    ao, co = T.walk(w.r_s, w.rcut, theta)
    assert np.array_equal(r["cu"], co)
    st = err_stats(r["au"].astype(np.float64), ao)
    assert st["rms"] <= 1e-5
    # gradients: against the separate adjoint (atomic order only) and the oracle
    s = np.arange(0, w.n, max(1, w.n // 300))
    op, om, pa, ma = T.adjoint(w.r_s, w.rcut, theta, wt, s, with_scale=True)
    e_sep = max(grad_scaled_err(r["dpu"][s], r["dps"][s], pa), grad_scaled_err(r["dmu"][s], r["dms"][s], ma))
    e_orc = max(grad_scaled_err(r["dpu"][s], op, pa), grad_scaled_err(r["dmu"][s], om, ma))
    print(name, theta, "fused vs separate", e_sep, "vs oracle", e_orc, st)
    assert e_sep < 1e-12
    assert e_orc < GRAD_TOL


@pytest.mark.parametrize("n", [1, 2, 33, 1000])
def test_fused_ragged_and_tiny(orc, n):
    """Tiny sets and a ragged last group: fused outputs against the separate
    calls and the oracle."""
    dev = device()
    w = ics.make("uniform4096", n)
    w.r_s = 0.05
    wt = ics.loss_weights(w.n, 7).astype(np.float32).astype(np.float64)
    r = _run(w, dev, 0.5, wt)
    assert np.array_equal(r["au"].view(np.uint32), r["af"].view(np.uint32))
    assert np.array_equal(r["cu"], r["cf"])
    assert r["tu"] == r["tf"]
    s = np.arange(w.n)
    op, om, pa, ma = orc.Tree(w.pos, w.mass, 2.8 * w.eps).adjoint(w.r_s, w.rcut, 0.5, wt, s, with_scale=True)
    assert max(grad_scaled_err(r["dpu"], r["dps"], pa), grad_scaled_err(r["dmu"], r["dms"], ma)) < 1e-12
    assert max(grad_scaled_err(r["dpu"], op, pa), grad_scaled_err(r["dmu"], om, ma)) < GRAD_TOL


def test_fused_argument_errors():
    dev = device()
    m = og()
    w = ics.make("uniform4096", 1000)
    tree, _, _ = build_tree(w, dev)
    wt = torch.zeros((w.n, 3), dtype=torch.float32, device=dev)
    with pytest.raises(ValueError):
        m.shortrange_accel_adjoint(tree, w.r_s, 0.5, wt.double())
    # a workspace one byte short
    import ctypes as C
    L = m.lib()
    need = L.og_adjoint_ws_bytes(C.byref(tree.header), 1)
    ws = torch.empty(need - 1 + 256, dtype=torch.uint8, device=dev)
    ws = ws[(-ws.data_ptr()) % 256:][: need - 1]
    with pytest.raises(m.OGError):
        m.shortrange_accel_adjoint(tree, w.r_s, 0.5, wt, ws=ws)


def test_linear_loss_autograd(orc):
    """ShortRangeLinearLoss: L = sum w . a and, through autograd, dL/dx, dL/dm
    and dL/dw from the fused walk, against the two-walk autograd path, the
    oracle's gradient per particle and the oracle's accelerations."""
    dev = device()
    m = og()
    w = ics.make("nfw256", 16)
    wt = torch.tensor(ics.loss_weights(w.n, 5), dtype=torch.float32, device=dev)
    pos = torch.tensor(w.pos, dtype=torch.float64, device=dev, requires_grad=True)
    mass = torch.tensor(w.mass, dtype=torch.float64, device=dev, requires_grad=True)
    eps = torch.tensor(w.eps, dtype=torch.float64, device=dev)
    wr = wt.clone().requires_grad_(True)
    L = m.ShortRangeLinearLoss.apply(pos, mass, eps, wr, w.box, w.r_s, 0.5)
    # a factor 2 (exact in FP32): the two-walk path receives 2 w as its weights
    gp, gm, gw = torch.autograd.grad(2.0 * L, (pos, mass, wr))
    # the two-walk path
    pos2 = pos.detach().clone().requires_grad_(True)
    mass2 = mass.detach().clone().requires_grad_(True)
    acc = m.ShortRangeAccel.apply(pos2, mass2, eps, w.box, w.r_s, 0.5)
    L2 = (acc.double() * wt.double()).sum()
    gp2, gm2 = torch.autograd.grad(2.0 * L2, (pos2, mass2))
    assert abs(L.item() - L2.item()) <= 1e-12 * abs(L2.item())
    assert torch.equal(gw, 2.0 * acc.detach())
    assert (gp - gp2).abs().max().item() <= 1e-12 * gp2.abs().max().item()
    assert (gm - gm2).abs().max().item() <= 1e-12 * gm2.abs().max().item()
    # against the oracle
    wd = wt.double().cpu().numpy()
    T = orc.Tree(w.pos, w.mass, 2.8 * w.eps)
    s = np.arange(0, w.n, 9)
    op, om, pa, ma = T.adjoint(w.r_s, w.rcut, 0.5, wd, s, with_scale=True)
    assert grad_scaled_err(gp.cpu().numpy()[s] / 2.0, op, pa) < GRAD_TOL
    assert grad_scaled_err(gm.cpu().numpy()[s] / 2.0, om, ma) < GRAD_TOL
    ao, _ = T.walk(w.r_s, w.rcut, 0.5)
    assert err_stats(gw.double().cpu().numpy() / 2.0, ao)["rms"] <= 1e-5
