"""Pins for the oracle's direct periodic short-range sum (CPU only)."""
import math

import numpy as np
import pytest

from ics import uniform


def test_two_body_closed_form(orc):
    # two particles across the periodic boundary: minimum image separation 0.04
    pos = np.array([[0.98, 0.5, 0.5], [0.02, 0.5, 0.5]])
    mass = np.array([2.0, 3.0])
    h = np.array([0.001, 0.001])
    r_s = 0.02
    acc, cnt = orc.direct(pos, mass, h, 1.0, r_s, 4.5 * r_s)
    r = 0.04
    u = r / (2 * r_s)
    f = math.erfc(u) + 2 * u / math.sqrt(math.pi) * math.exp(-u * u)
    # particle 0 is pulled toward +x (through the boundary), particle 1 toward -x
    assert acc[0, 0] == pytest.approx(3.0 * f / r ** 2, rel=1e-14)
    assert acc[1, 0] == pytest.approx(-2.0 * f / r ** 2, rel=1e-14)
    assert np.all(acc[:, 1:] == 0.0)
    assert list(cnt) == [1, 1]
    assert mass[0] * acc[0, 0] + mass[1] * acc[1, 0] == pytest.approx(0.0, abs=1e-12)


def test_cut_is_strict(orc):
    r_s = 0.01
    rcut = 4.5 * r_s
    pos = np.array([[0.5, 0.5, 0.5], [0.5 + rcut, 0.5, 0.5], [0.5, 0.5 + 0.999 * rcut, 0.5]])
    acc, cnt = orc.direct(pos, np.ones(3), np.full(3, 1e-4), 1.0, r_s, rcut, targets=[0])
    assert cnt[0] <= 2 and cnt[0] >= 1
    assert acc[0, 1] > 0.0


def test_newtonian_limit(orc):
    # compact cluster (size 1) in a huge box (1000) with r_s = 100: the short-range
    # factor differs from 1 by at most (4/(3 sqrt(pi))) (D / 2 r_s)^3 ~ 1e-7
    rng = np.random.default_rng(5)
    n = 300
    pos = 500.0 + rng.random((n, 3))
    mass = rng.random(n) + 0.5
    h = np.full(n, 0.05)
    acc, cnt = orc.direct(pos, mass, h, 1000.0, 100.0, 450.0)
    assert np.all(cnt == n - 1)
    ref = np.zeros((n, 3))
    for i in range(n):
        d = pos[i] - pos
        r = np.sqrt((d * d).sum(1))
        for j in range(n):
            if j != i:
                ref[i] -= mass[j] * orc.kernel_K(r[j], 0.05) * d[j]
    rel = np.linalg.norm(acc - ref, axis=1) / np.linalg.norm(ref, axis=1)
    bound = 4.0 / (3.0 * math.sqrt(math.pi)) * (math.sqrt(3.0) / 200.0) ** 3
    assert rel.max() < 1.5 * bound
    assert rel.max() > 0.0


def test_momentum_conservation(orc):
    pos = uniform(2000, 41)
    rng = np.random.default_rng(41)
    mass = rng.random(2000)
    h = 0.01 + 0.01 * rng.random(2000)          # unequal softenings: pairing is max(h_i, h_j)
    acc, _ = orc.direct(pos, mass, h, 1.0, 0.03, 0.135)
    p = (mass[:, None] * acc).sum(0)
    scale = (mass[:, None] * np.abs(acc)).sum(0)
    assert np.all(np.abs(p) < 1e-13 * scale)


def test_pair_count_against_kdtree(orc):
    ckd = pytest.importorskip("scipy.spatial").cKDTree
    pos = uniform(3000, 42)
    rcut = 0.09
    _, cnt = orc.direct(pos, np.ones(3000), np.full(3000, 1e-3), 1.0, rcut / 4.5, rcut)
    pairs = ckd(pos, boxsize=1.0).query_pairs(rcut * (1 - 1e-12))
    assert int(cnt.sum()) == 2 * len(pairs)


def test_cell_list_equals_all_pairs(orc):
    # rcut > box/3 forces the all-pairs branch; a slightly smaller box-relative
    # rcut uses cells.  Compare both against per-target brute force on a subset.
    pos = uniform(1500, 43)
    m = np.full(1500, 1.0 / 1500)
    h = np.full(1500, 0.002)
    for rcut in (0.2, 0.34):
        a, c = orc.direct(pos, m, h, 1.0, rcut / 4.5, rcut)
        sub = np.arange(0, 1500, 37)
        a2, c2 = orc.direct(pos, m, h, 1.0, rcut / 4.5, rcut, targets=sub)
        assert np.array_equal(c[sub], c2)
        assert np.allclose(a[sub], a2, rtol=1e-13, atol=0)
