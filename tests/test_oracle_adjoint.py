"""Pins for the oracle's adjoint (CPU only): the analytic gradient of
L = sum_i w_i . a_i with frozen opening / cut decisions is compared with
central finite differences of the forward sum over the same frozen lists."""
import numpy as np
import pytest

import ics


def _rel(a, b):
    return np.abs(a - b) / np.maximum(np.abs(b), 1e-300)


@pytest.mark.parametrize("theta", [0.0, 0.5])
def test_adjoint_matches_finite_differences(orc, theta):
    w = ics.make("nfw256", 10)
    h = 2.8 * w.eps
    wt = ics.loss_weights(w.n, 99)
    T = orc.Tree(w.pos, w.mass, h)
    samples = np.random.default_rng(1).choice(w.n, 24, replace=False)
    dp, dm = T.adjoint(w.r_s, w.rcut, theta, wt, samples)
    fp, fm = T.fd(w.r_s, w.rcut, theta, wt, samples, hx=1e-6, hm_rel=1e-6)
    scale_p = np.abs(dp).max()
    assert np.abs(dp - fp).max() < 1e-6 * scale_p
    assert np.abs(dm - fm).max() < 1e-6 * np.abs(dm).max()


def test_adjoint_fd_multimass(orc):
    w = ics.make("zoom8m", 900)
    h = 2.8 * w.eps
    T = orc.Tree(w.pos, w.mass, h)
    samples = np.random.default_rng(2).choice(w.n, 16, replace=False)
    dp, dm = T.adjoint(w.r_s, w.rcut, 0.5, w.w, samples)
    fp, fm = T.fd(w.r_s, w.rcut, 0.5, w.w, samples)
    assert np.abs(dp - fp).max() < 1e-6 * np.abs(dp).max()
    assert np.abs(dm - fm).max() < 1e-6 * np.abs(dm).max()


def test_sampled_adjoint_equals_full(orc):
    w = ics.make("uniform4096", 600)
    h = 2.8 * w.eps
    wt = ics.loss_weights(w.n, 5)
    T = orc.Tree(w.pos, w.mass, h)
    fp, fm = T.adjoint(w.r_s, w.rcut, 0.5, wt)
    s = np.arange(0, w.n, 13)
    sp, sm = T.adjoint(w.r_s, w.rcut, 0.5, wt, s)
    assert np.allclose(sp, fp[s], rtol=1e-12, atol=1e-12 * np.abs(fp).max())
    assert np.allclose(sm, fm[s], rtol=1e-12, atol=1e-12 * np.abs(fm).max())


def test_adjoint_is_gradient_of_full_loss(orc):
    # global check: moving one particle changes the whole tree-walk loss by the
    # predicted amount as long as no decision flips (tiny step)
    w = ics.make("uniform4096", 400)
    h = 2.8 * w.eps
    wt = ics.loss_weights(w.n, 8)
    T = orc.Tree(w.pos, w.mass, h)
    dp, dm = T.adjoint(w.r_s, w.rcut, 0.0, wt)
    k, step = 17, 1e-7
    for c in range(3):
        pp = w.pos.copy(); pp[k, c] += step
        pn = w.pos.copy(); pn[k, c] -= step
        Lp = orc.Tree(pp, w.mass, h).loss(w.r_s, w.rcut, 0.0, wt)
        Ln = orc.Tree(pn, w.mass, h).loss(w.r_s, w.rcut, 0.0, wt)
        assert (Lp - Ln) / (2 * step) == pytest.approx(dp[k, c], rel=1e-5)


def test_two_body_gradient(orc):
    # L = w . a_0 for two bodies: dL/dx_1 = -dL/dx_0 and dL/dm_1 = w . a_0 / m_1
    pos = np.array([[0.5, 0.5, 0.5], [0.52, 0.51, 0.49]])
    mass = np.array([1.0, 2.0])
    h = np.full(2, 0.003)
    wt = np.array([[0.3, -1.0, 2.0], [0.0, 0.0, 0.0]])
    T = orc.Tree(pos, mass, h, leaf_size=1)
    r_s = 0.02
    dp, dm = T.adjoint(r_s, 4.5 * r_s, 0.0, wt)
    a, _ = T.walk(r_s, 4.5 * r_s, 0.0)
    assert np.allclose(dp[1], -dp[0], rtol=1e-13)
    assert dm[1] == pytest.approx(float(wt[0] @ a[0]) / mass[1], rel=1e-13)
    assert dm[0] == pytest.approx(0.0, abs=1e-12)
