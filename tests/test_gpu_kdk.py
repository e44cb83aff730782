"""Device-resident kick-drift-kick steps against the FP64 oracle step
(oracle/og_kdk.py).

Tolerance.  The GPU forces are FP32: the theta = 0 walk is within 1e-6 rms
of the direct sum, and the mesh within 5e-6 of rms |a|.  Five oracle steps
of the 512-particle set with a 1e-5 relative error put into every force
component moved positions by 2.8e-8 rms (4.8e-7 max) and velocities by
2.5e-6 rms (3.6e-5 max).  The bounds below are ten times those.
"""
import numpy as np
import pytest

from gpu_util import device, og, torch
from oracle import og_kdk as K

pytestmark = pytest.mark.gpu

BOX = 1.0
N = 16
R_S = 1.25 / N
RCUT = 4.5 * R_S


def _t(a, dev, dtype=torch.float64):
    return torch.tensor(np.ascontiguousarray(a), dtype=dtype, device=dev)


def test_kick_and_drift():
    dev = device()
    m = og()
    rng = np.random.default_rng(3)
    v = rng.normal(size=(100, 3))
    x = rng.normal(size=(100, 3))
    a = rng.normal(size=(100, 3)).astype(np.float32)
    b = rng.normal(size=(100, 3)).astype(np.float32)
    vt, xt = _t(v, dev), _t(x, dev)
    m.kick(vt, _t(a, dev, torch.float32), _t(b, dev, torch.float32), 0.25)
    m.drift(xt, vt, 0.5)
    v1 = v + 0.25 * (a.astype(np.float64) + b.astype(np.float64))
    np.testing.assert_allclose(vt.cpu().numpy(), v1, rtol=1e-15, atol=1e-15)
    np.testing.assert_allclose(xt.cpu().numpy(), x + 0.5 * v1, rtol=1e-15, atol=1e-15)
    m.kick(vt, _t(a, dev, torch.float32), None, -0.25)  # acc_b may be absent
    np.testing.assert_allclose(vt.cpu().numpy(), v1 - 0.25 * a.astype(np.float64), rtol=1e-14, atol=1e-14)


def test_steps_against_the_oracle():
    dev = device()
    m = og()
    rng = np.random.default_rng(12)
    n = 512
    pos = rng.random((n, 3))
    vel = rng.normal(size=(n, 3)) * 0.05
    mass = np.full(n, 1.0 / n)
    eps = 1.0 / 400.0
    acc = K.accel(pos, mass, 2.8 * eps, BOX, R_S, RCUT, N)
    p1, v1, _ = K.kdk(pos, vel, acc, mass, 2.8 * eps, BOX, R_S, RCUT, N, 0.01, 5)

    S = m.TreePMStepper(_t(pos, dev), _t(vel, dev), _t(mass, dev), eps, BOX, R_S, 0.0, N)
    for _ in range(5):
        S.step(0.01)
    torch.cuda.synchronize()
    pg, vg = S.pos.cpu().numpy(), S.vel.cpu().numpy()
    S.close()
    dx = np.linalg.norm(pg - p1, axis=1)
    dv = np.linalg.norm(vg - v1, axis=1)
    assert np.sqrt(np.mean(dx ** 2)) < 3e-7 and dx.max() < 5e-6, (np.sqrt(np.mean(dx ** 2)), dx.max())
    assert np.sqrt(np.mean(dv ** 2)) < 3e-5 and dv.max() < 4e-4, (np.sqrt(np.mean(dv ** 2)), dv.max())
    # momentum: pairwise walk forces and the mesh conserve it up to FP32 rounding
    dp = np.abs((mass[:, None] * (vg - vel)).sum(0)).max()
    assert dp < 1e-4 * (mass * np.linalg.norm(vg - vel, axis=1)).sum(), dp


def test_binary_returns_after_one_kepler_period():
    """The oracle's pin on the device: 200 steps per period bring a tight
    binary back within 1.0e-3 of its separation (oracle: 1.03e-3)."""
    dev = device()
    m = og()
    r0, M = 1e-3, 1.0
    x0 = np.array([0.3, 0.4, 0.5])
    pos = np.array([x0 - [r0 / 2, 0.0, 0.0], x0 + [r0 / 2, 0.0, 0.0]])
    v = np.sqrt(M / r0) / 2.0
    vel = np.array([[0.0, -v, 0.0], [0.0, v, 0.0]])
    T = 2.0 * np.pi * np.sqrt(r0 ** 3 / M)
    S = m.TreePMStepper(_t(pos, dev), _t(vel, dev), _t(np.array([0.5, 0.5]), dev), 1e-5 / 2.8, BOX, R_S, 0.5, N)
    for _ in range(200):
        S.step(T / 200)
    torch.cuda.synchronize()
    err = np.linalg.norm(S.pos.cpu().numpy() - pos, axis=1).max() / r0
    S.close()
    assert err < 1.5e-3, err


def test_stepper_reports_a_failed_tree():
    """A step whose tree build runs out of node capacity raises (the status
    words are polled once per step), and an unchecked step leaves NaN
    short-range forces rather than the previous step's."""
    import numpy as np
    from gpu_util import device, og, to_dev
    import ics
    dev = device()
    m = og()
    w = ics.make("uniform4096", 2000)
    pos, mass, eps = to_dev(w, dev)
    S = m.TreePMStepper(pos.clone(), torch.zeros_like(pos), mass, eps, w.box, w.r_s, 0.5, 16)
    S.step(1e-4)                         # a clean step polls without error
    S.p = m.params(node_capacity=40)     # the same buffer, too few nodes allowed
    with pytest.raises(m.OGError) as e:
        S.step(1e-4)
    assert e.value.code == 2             # OG_ENOSPACE from the tree build
    S.step(1e-4, check=False)
    assert torch.isnan(S.acc_s).all()
    S.close()
