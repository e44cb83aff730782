"""Pins for the oracle's force law (CPU only).

* K_h, the softened kernel, is pinned to its definition as the force of the
  cubic-spline mass distribution: K_h(r) = M(<r) / r^3 with M the enclosed
  mass of W(r, h) = 8/(pi h^3) [1 - 6v^2 + 6v^3] (v < 1/2), 16/(pi h^3)(1-v)^3
  (1/2 <= v < 1), integrated numerically here.
* f, the short-range factor, is pinned to its closed-form derivative
  f'(r) = -(r^2 / (2 sqrt(pi) r_s^3)) exp(-r^2 / 4 r_s^2) (a wrong coefficient
  on either term breaks it), to f(0) = 1, to the series 1 - (4/(3 sqrt(pi))) u^3
  and to f -> 1 as r_s -> infinity.
"""
import math

import numpy as np
import pytest

quad = pytest.importorskip("scipy.integrate").quad


def _spline_density(r, h):
    v = r / h
    if v < 0.5:
        return 8.0 / (math.pi * h ** 3) * (1.0 - 6.0 * v * v + 6.0 * v ** 3)
    if v < 1.0:
        return 16.0 / (math.pi * h ** 3) * (1.0 - v) ** 3
    return 0.0


def _enclosed(r, h):
    rr = min(r, h)
    pts = [0.5 * h] if rr > 0.5 * h else None
    val, _ = quad(lambda s: 4.0 * math.pi * s * s * _spline_density(s, h), 0.0, rr, points=pts,
                  epsabs=0.0, epsrel=1e-13, limit=200)
    return val


@pytest.mark.parametrize("v", [0.01, 0.1, 0.3, 0.49, 0.5, 0.51, 0.7, 0.9, 0.999, 1.0, 1.5, 3.0])
def test_spline_kernel_is_enclosed_mass_force(orc, v):
    h = 0.37
    r = v * h
    assert _enclosed(10 * h, h) == pytest.approx(1.0, rel=1e-12)
    expect = _enclosed(r, h) / r ** 3
    assert orc.kernel_K(r, h) == pytest.approx(expect, rel=1e-11)


def test_spline_continuity_and_limit(orc):
    h = 0.5
    for v in (0.5, 1.0):
        lo, hi = orc.kernel_K(v * h * (1 - 1e-12), h), orc.kernel_K(v * h * (1 + 1e-12), h)
        assert lo == pytest.approx(hi, rel=1e-9)
        dl = (orc.kernel_K(v * h, h) - orc.kernel_K(v * h - 1e-6, h)) / 1e-6
        dr = (orc.kernel_K(v * h + 1e-6, h) - orc.kernel_K(v * h, h)) / 1e-6
        assert dl == pytest.approx(dr, rel=1e-4)
    # the acceleration r K_h(r) goes to zero linearly at the centre
    assert orc.kernel_K(0.0, h) == pytest.approx(32.0 / 3.0 / h ** 3, rel=1e-15)


def test_short_range_factor_derivative(orc):
    r_s = 0.013
    for r in np.linspace(0.002, 4.5 * r_s, 17):
        step = 1e-7 * r_s
        fd = (orc.kernel_f(r + step, r_s) - orc.kernel_f(r - step, r_s)) / (2 * step)
        closed = -(r * r / (2.0 * math.sqrt(math.pi) * r_s ** 3)) * math.exp(-(r / (2 * r_s)) ** 2)
        assert fd == pytest.approx(closed, rel=2e-6, abs=1e-9 / r_s)


def test_short_range_factor_limits(orc):
    r_s = 0.05
    assert orc.kernel_f(0.0, r_s) == 1.0
    for u in (1e-3, 1e-2, 3e-2):
        r = 2 * r_s * u
        series = 1.0 - 4.0 / (3.0 * math.sqrt(math.pi)) * u ** 3
        assert orc.kernel_f(r, r_s) == pytest.approx(series, abs=2 * u ** 5)
    assert orc.kernel_f(0.3, 1e9) == pytest.approx(1.0, abs=1e-20)
    # decreasing on the whole cut range, small but non-zero at the cut
    f = [orc.kernel_f(r, r_s) for r in np.linspace(0, 4.5 * r_s, 50)]
    assert all(a > b for a, b in zip(f, f[1:]))
    assert 0.017 < orc.kernel_f(4.5 * r_s, r_s) < 0.018
