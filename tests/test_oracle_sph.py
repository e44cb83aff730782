"""Pins of the SPH density oracle (oracle/og_sph.py) against facts fixed
outside it:
- the cubic spline's unit integral (scipy quadrature);
- the density of a uniform lattice, m / a^3, with h -> a (3 N_ngb / 4 pi)^(1/3)
  (measured within 0.4 % for 32-100 neighbours on a 12^3 lattice);
- neighbour counts against scipy's periodic k-d tree;
- the scaling of h and rho with the box;
- the root condition N_eff(h) = N_ngb.
"""
import numpy as np
import pytest
from scipy.integrate import quad
from scipy.spatial import cKDTree

from oracle import og_sph as S


@pytest.mark.parametrize("h", [1.0, 0.37])
def test_kernel_has_unit_integral(h):
    val, _ = quad(lambda r: 4.0 * np.pi * r * r * float(S.kernel(np.array([r]), h)[0]), 0.0, h,
                  points=[0.5 * h], epsabs=1e-13, epsrel=1e-13)
    assert abs(val - 1.0) < 1e-10


def _lattice(n, box=1.0):
    a = box / n
    g = (np.arange(n) + 0.5) * a
    return np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3), a


@pytest.mark.parametrize("n_ngb", [32, 64, 100])
def test_uniform_lattice_density(n_ngb):
    pos, a = _lattice(12)
    m = np.full(len(pos), 1.0 / len(pos))
    tg = np.array([0, 100, 777])
    h = S.smoothing_length(pos, 1.0, n_ngb, targets=tg)
    rho = S.density(pos, m, h, 1.0, targets=tg)
    np.testing.assert_allclose(rho * a ** 3 / m[0], 1.0, atol=5e-3)
    np.testing.assert_allclose(h / a, (3.0 * n_ngb / (4.0 * np.pi)) ** (1.0 / 3.0), rtol=5e-3)


def _random(n=400, seed=3):
    return np.random.default_rng(seed).random((n, 3))


def test_neighbour_counts_match_a_periodic_kd_tree():
    pos = _random()
    h = S.smoothing_length(pos, 1.0, 40, targets=np.arange(50))
    cnt = S.neighbour_count(pos, np.concatenate([h, np.full(len(pos) - 50, 0.1)]), 1.0)[:50]
    T = cKDTree(pos, boxsize=1.0)
    ref = np.array([len(T.query_ball_point(pos[i], h[i] * (1 - 1e-12))) - 1 for i in range(50)])
    np.testing.assert_array_equal(cnt, ref)


def test_root_condition_and_scaling():
    pos = _random()
    tg = np.arange(20)
    h = S.smoothing_length(pos, 1.0, 50, targets=tg)
    for k, i in enumerate(tg):
        r = S.distances(pos, int(i), 1.0)
        assert S.n_eff(r, h[k]) == pytest.approx(50.0, rel=1e-9)
        assert S.n_eff(r, h[k] * (1 - 1e-6)) < 50.0
    s = 7.5
    h2 = S.smoothing_length(pos * s, s, 50, targets=tg)
    np.testing.assert_allclose(h2, s * h, rtol=1e-10)
    m = np.full(len(pos), 2.0)
    np.testing.assert_allclose(S.density(pos * s, m, h2, s, targets=tg) * s ** 3,
                               S.density(pos, m, h, 1.0, targets=tg), rtol=1e-10)
