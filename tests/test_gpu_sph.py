"""SPH density on the device against the FP64 oracle (oracle/og_sph.py).

The oracle solves N_eff(h) = N_ngb by FP64 bisection to 1e-12 of h.  The
device's grouped walk converges in FP32 (to ~1e-7) and finishes with one
Newton step whose sums come from float-float minimum-image distances on the
split-float positions (~1e-11 relative in q), with the density carried to
the new h to first order (~1e-11).  So h and rho agree to 1e-9 relative,
and neighbour counts exactly (ties at r = h have measure zero).
"""
import numpy as np
import pytest

import ics
from gpu_util import device, og, torch
from oracle import og_sph as S

pytestmark = pytest.mark.gpu


def _run(pos, mass, box, n_ngb, dev, eps=1e-3):
    m = og()
    pt = torch.tensor(pos, dtype=torch.float64, device=dev)
    mt = torch.tensor(mass, dtype=torch.float64, device=dev)
    keys, order = m.keys_sort(pt, box)
    tree = m.tree_build(keys, order, pt, mt, eps, box)
    h, rho, ngb = m.sph_density(tree, n_ngb)
    torch.cuda.synchronize()
    return h.cpu().numpy(), rho.cpu().numpy(), ngb.cpu().numpy()


def _compare(pos, mass, box, n_ngb, dev, nsamp=120, seed=0):
    h, rho, ngb = _run(pos, mass, box, n_ngb, dev)
    tg = np.random.default_rng(seed).choice(len(pos), size=min(nsamp, len(pos)), replace=False)
    ho = S.smoothing_length(pos, box, n_ngb, targets=tg)
    ro = S.density(pos, mass, ho, box, targets=tg)
    co = np.array([int((S.distances(pos, int(i), box) < ho[k]).sum()) - 1 for k, i in enumerate(tg)])
    np.testing.assert_allclose(h[tg], ho, rtol=1e-9)
    np.testing.assert_allclose(rho[tg], ro, rtol=1e-9)
    np.testing.assert_array_equal(ngb[tg], co)
    assert np.isfinite(h).all() and np.isfinite(rho).all()


def test_uniform_random():
    dev = device()
    rng = np.random.default_rng(1)
    pos = rng.random((3000, 3))
    _compare(pos, np.full(3000, 1.0 / 3000), 1.0, 32, dev)


def test_clustered_set_and_unequal_masses():
    dev = device()
    w = ics.make("nfw256", 16)
    m = w.mass * (0.5 + np.random.default_rng(2).random(w.n))
    _compare(w.pos, m, w.box, 48, dev)


def test_non_unit_box():
    dev = device()
    rng = np.random.default_rng(3)
    pos = rng.random((2000, 3)) * 3.0
    _compare(pos, np.full(2000, 2.0), 3.0, 40, dev)


def test_uniform_lattice_density():
    dev = device()
    n = 12
    a = 1.0 / n
    g = (np.arange(n) + 0.5) * a
    pos = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    m = np.full(len(pos), 1.0 / len(pos))
    h, rho, _ = _run(pos, m, 1.0, 64, dev)
    np.testing.assert_allclose(rho * a ** 3 / m[0], 1.0, atol=5e-3)


def test_too_many_neighbours_is_flagged():
    dev = device()
    m = og()
    rng = np.random.default_rng(4)
    pos = torch.tensor(rng.random((50, 3)), device=dev)
    mass = torch.full((50,), 0.02, dtype=torch.float64, device=dev)
    keys, order = m.keys_sort(pos, 1.0)
    tree = m.tree_build(keys, order, pos, mass, 1e-3, 1.0)
    with pytest.raises(m.OGError):
        m.sph_density(tree, 500.0)  # more than a half-box sphere can hold


def test_clustered_set_full_tree_depth():
    """A clustered set large enough for haloes much denser than the mean
    (the start radius comes from the tree, and Newton steps span decades)."""
    dev = device()
    w = ics.make("nfw256", 48)   # 110,592 particles
    _compare(w.pos, w.mass, w.box, 32, dev, nsamp=60, seed=5)


def test_small_and_ragged():
    """Fewer particles than a group, and a ragged last group."""
    dev = device()
    rng = np.random.default_rng(6)
    for n in (40, 1000 + 17):
        pos = rng.random((n, 3))
        _compare(pos, np.full(n, 1.0 / n), 1.0, 16, dev, nsamp=40, seed=n)
