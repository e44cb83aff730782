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


def test_adjoint_term_scale(orc):
    """The term-magnitude sums bound the gradients (triangle inequality) and
    equal them where one term of one sign makes up a component: two bodies
    with the loss on body 0 only, so dL/dx_0 is a single target-side term and
    dL/dm_1 the single source-side term w . g."""
    w = ics.make("nfw256", 10)
    T = orc.Tree(w.pos, w.mass, 2.8 * w.eps)
    wt = ics.loss_weights(w.n, 98)
    s = np.arange(0, w.n, 37)
    dp, dm, pa, ma = T.adjoint(w.r_s, w.rcut, 0.5, wt, s, with_scale=True)
    dp2, dm2 = T.adjoint(w.r_s, w.rcut, 0.5, wt, s)
    assert np.array_equal(dp, dp2) and np.array_equal(dm, dm2)
    assert np.all(np.abs(dp) <= pa * (1 + 1e-12)) and np.all(np.abs(dm) <= ma * (1 + 1e-12))
    # many terms of both signs: the scale is well above the sum for most particles
    assert np.median(ma / np.maximum(np.abs(dm), 1e-300)) > 2.0
    pos = np.array([[0.5, 0.5, 0.5], [0.52, 0.51, 0.49]])
    mass = np.array([1.0, 2.0])
    T2 = orc.Tree(pos, mass, np.full(2, 0.003), leaf_size=1)
    w2 = np.array([[0.3, -1.0, 2.0], [0.0, 0.0, 0.0]])
    dp, dm, pa, ma = T2.adjoint(0.02, 0.09, 0.0, w2, with_scale=True)
    assert np.allclose(pa[0], np.abs(dp[0]), rtol=1e-14)
    assert ma[1] == pytest.approx(abs(dm[1]), rel=1e-14)


def test_fd_crossing_flags(orc):
    """A position step that moves a term across its softening length h sets
    bit 0, across rcut bit 1; a pair well inside both sets neither."""
    h, r_s = 0.004, 0.02
    rcut = 4.5 * r_s
    mass = np.array([1.0, 1.0])
    cases = [(0.02, 0), (h - 2e-7, 1), (h + 2e-7, 1), (rcut - 2e-7, 2)]
    for dx, want in cases:
        pos = np.array([[0.5, 0.5, 0.5], [0.5 + dx, 0.5, 0.5]])
        T = orc.Tree(pos, mass, np.full(2, h), leaf_size=1)
        wt = np.array([[1.0, 0.5, 0.25], [0.0, 0.0, 0.0]])
        _, _, fl = T.fd(r_s, rcut, 0.0, wt, np.array([0]), hx=1e-6, with_flags=True)
        assert int(fl[0]) == want, (dx, int(fl[0]))
