"""Pins of the kick-drift-kick oracle (oracle/og_kdk.py) against facts fixed
outside it:
- time reversibility of the leapfrog (forces depend on positions only);
- momentum conservation (pairwise short-range forces; a momentum-conserving
  mesh);
- Kepler's law: a tight binary (separation 1/80 of r_s, where the split
  factor is 1 to 1e-7) returns to its start after one period
  2 pi sqrt(r^3 / M).  The return error falls as dt^2: 4.1e-3, 1.0e-3 and
  2.6e-4 of the separation for 100, 200 and 400 steps per period.
"""
import numpy as np

import oracle
from oracle import og_kdk as K

BOX = 1.0
N = 16
R_S = 1.25 / N
RCUT = 4.5 * R_S


def _random_set(seed, n=48):
    rng = np.random.default_rng(seed)
    pos = rng.random((n, 3)) * BOX
    vel = rng.normal(size=(n, 3)) * 0.05
    mass = np.full(n, 1.0 / n)
    return pos, vel, mass


def test_reversible():
    pos, vel, mass = _random_set(1)
    h = 2.8 / 400.0
    acc = K.accel(pos, mass, h, BOX, R_S, RCUT, N)
    p, v, a = K.kdk(pos, vel, acc, mass, h, BOX, R_S, RCUT, N, 0.01, 6)
    assert np.abs(p - pos).max() > 1e-3  # the particles did move
    p2, v2, _ = K.kdk(p, -v, a, mass, h, BOX, R_S, RCUT, N, 0.01, 6)
    assert np.abs(p2 - pos).max() < 1e-12
    assert np.abs(v2 + vel).max() < 1e-12


def test_momentum_is_conserved():
    pos, vel, mass = _random_set(2)
    h = 2.8 / 400.0
    acc = K.accel(pos, mass, h, BOX, R_S, RCUT, N)
    p0 = (mass[:, None] * vel).sum(0)
    _, v, _ = K.kdk(pos, vel, acc, mass, h, BOX, R_S, RCUT, N, 0.01, 6)
    p1 = (mass[:, None] * v).sum(0)
    assert np.abs(p1 - p0).max() < 1e-13 * (mass * np.linalg.norm(v, axis=1)).sum() + 1e-16


def _binary():
    r0, M = 1e-3, 1.0
    x0 = np.array([0.3, 0.4, 0.5])
    pos = np.array([x0 - [r0 / 2, 0.0, 0.0], x0 + [r0 / 2, 0.0, 0.0]])
    v = np.sqrt(M / r0) / 2.0  # each body on the circular orbit about the centre
    vel = np.array([[0.0, -v, 0.0], [0.0, v, 0.0]])
    return pos, vel, np.array([0.5, 0.5]), r0, 2.0 * np.pi * np.sqrt(r0 ** 3 / M)


def test_binary_returns_after_one_kepler_period_at_second_order():
    pos, vel, mass, r0, T = _binary()
    h = 1e-5
    acc = K.accel(pos, mass, h, BOX, R_S, RCUT, N)
    err = []
    for nst in (100, 200):
        p, _, _ = K.kdk(pos, vel, acc, mass, h, BOX, R_S, RCUT, N, T / nst, nst)
        err.append(np.linalg.norm(p - pos, axis=1).max() / r0)
    assert err[1] < 2e-3, err
    assert 3.5 < err[0] / err[1] < 4.5, err  # second order in dt
