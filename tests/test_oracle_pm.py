"""Pins of the PM long-range oracle (oracle/og_pm.py) against facts fixed
outside it: mass conservation, the node-exact CIC deposit, zero self-force and
momentum conservation (the deposit and interpolation kernels are the same and
the difference operator is antisymmetric), the exact long-range Fourier series
of a point mass, and short + long against an Ewald sum whose splitting
parameter is unrelated to r_s (the total periodic force does not depend on it).

The long-range bounds are the CIC mesh's own discretisation error at
r_s = 1.25 mesh cells, measured on these seeds (max 2.3 % of |F| at 2-4 cells,
rms 1.8 % of |F_long| at 3 cells).  The same checks with the CIC
deconvolution dropped give 4.1 % and 8.8 %, and with the split scale off by
sqrt(2) give 18-32 %.
"""
import numpy as np
import pytest

import oracle
from oracle import og_pm as P
from pm_ref import ewald, long_series

L = 1.0
N = 32
D = L / N
R_S = 1.25 * D


def _pair(rng, r):
    x0 = rng.random(3) * L
    u = rng.normal(size=3)
    u /= np.linalg.norm(u)
    d = r * D * u
    # a massless probe at x0 + d feels the long-range force of the unit mass at x0
    return np.array([x0, x0 + d]), np.array([1.0, 1e-12]), d


def test_deposit_conserves_mass():
    rng = np.random.default_rng(1)
    pos = rng.random((500, 3)) * 3.0 - 1.0  # also outside [0, L): wrapped
    m = rng.random(500)
    rho = P.deposit(pos, m, L, N)
    assert abs(rho.sum() * D ** 3 - m.sum()) <= 1e-12 * m.sum()


def test_deposit_on_a_node_and_between_nodes():
    rho = P.deposit(np.array([[3 * D, 5 * D, 7 * D]]), np.array([2.0]), L, N)
    assert rho[3, 5, 7] == pytest.approx(2.0 / D ** 3, rel=1e-14)
    assert np.count_nonzero(rho) == 1
    # a quarter cell along x, on nodes in y and z: 3/4 and 1/4 of the mass
    rho = P.deposit(np.array([[3.25 * D, 5 * D, 7 * D]]), np.array([1.0]), L, N)
    assert rho[3, 5, 7] == pytest.approx(0.75 / D ** 3, rel=1e-12)
    assert rho[4, 5, 7] == pytest.approx(0.25 / D ** 3, rel=1e-12)
    # periodic: the upper neighbour of the last node is node 0
    rho = P.deposit(np.array([[(N - 0.5) * D, 0.0, 0.0]]), np.array([1.0]), L, N)
    assert rho[N - 1, 0, 0] == pytest.approx(0.5 / D ** 3, rel=1e-12)
    assert rho[0, 0, 0] == pytest.approx(0.5 / D ** 3, rel=1e-12)


def test_lone_particle_feels_no_force():
    rng = np.random.default_rng(2)
    scale = 1.0 / D ** 2  # the force of a unit mass one cell away
    for _ in range(5):
        a = P.pm_accel(rng.random((1, 3)) * L, np.array([1.0]), L, N, R_S)
        assert np.abs(a).max() <= 1e-12 * scale


def test_momentum_is_conserved():
    rng = np.random.default_rng(3)
    pos = rng.random((64, 3)) * L
    m = 0.5 + rng.random(64)
    a = P.pm_accel(pos, m, L, N, R_S)
    tot = (m[:, None] * a).sum(0)
    assert np.abs(tot).max() <= 1e-12 * (m * np.linalg.norm(a, axis=1)).sum()


def test_ewald_reference_is_split_independent_and_newtonian_up_close():
    d = np.array([0.11, -0.23, 0.05])
    np.testing.assert_allclose(ewald(d, 6.0), ewald(d, 9.0), rtol=1e-10)
    # a close pair: the periodic images change the force by far less than 1e-6
    d = np.array([1e-3, 0.0, 0.0])
    assert ewald(d, 6.0)[0] == pytest.approx(-1.0 / d[0] ** 2, rel=1e-6)
    # the middle of the box between a mass and its image: no net force
    assert np.abs(ewald(np.array([0.5, 0.0, 0.0]), 6.0)).max() < 1e-9


def test_long_range_matches_the_exact_series():
    rng = np.random.default_rng(4)
    for r in (2.0, 3.0, 4.0):
        errs = []
        for _ in range(40):
            pos, m, d = _pair(rng, r)
            a = P.pm_accel(pos, m, L, N, R_S)[1]
            ex = long_series(d, R_S)
            errs.append(np.linalg.norm(a - ex) / np.linalg.norm(ex))
        rms = float(np.sqrt(np.mean(np.square(errs))))
        assert rms < 0.04 if r == 3.0 else rms < 0.06, (r, rms)


def test_short_plus_long_is_the_periodic_newtonian_force():
    rng = np.random.default_rng(5)
    for r in (0.5, 1.0, 2.0, 3.0, 4.0, 6.0, 12.0):
        worst = 0.0
        for _ in range(20):
            pos, m, d = _pair(rng, r)
            a = P.pm_accel(pos, m, L, N, R_S)[1]
            # short-range part from the pinned direct sum, cut far out (f(10 r_s) ~ 1e-10)
            s, _ = oracle.direct(pos, m, 1e-9, L, R_S, 10.0 * R_S)
            ew = ewald(d, 6.0)
            worst = max(worst, float(np.linalg.norm(a + s[1] - ew) / np.linalg.norm(ew)))
        assert worst < 0.03, (r, worst)
