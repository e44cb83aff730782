"""K1/K2 parity: GPU Hilbert keys and sort order are bit-exact against the
oracle (integer work: exact equality required)."""
import numpy as np
import pytest

import ics
from gpu_util import device, og, torch

pytestmark = pytest.mark.gpu


def _gpu_keys(pos, box=1.0):
    dev = device()
    m = og()
    p = torch.tensor(pos, dtype=torch.float64, device=dev)
    keys, order = m.keys_sort(p, box)
    return keys.cpu().numpy().view(np.uint64), order.cpu().numpy()


def _check(pos, orc, box=1.0):
    ks, order = _gpu_keys(pos, box)
    k_ref, bad, _ = orc.keys(pos, box)
    assert bad == 0
    ks_ref, order_ref = orc.sort(k_ref)
    assert np.array_equal(ks, ks_ref)
    assert np.array_equal(order, order_ref)


@pytest.mark.parametrize("n", [1, 2, 31, 33, 2047, 2048, 2049, 4096, 100003])
def test_uniform_sizes(orc, n):
    _check(ics.uniform(n, 500 + n), orc)


def test_exhaustive_grid_centres(orc):
    # every cell centre of a 2^7-per-axis grid (bijection and order of the curve)
    b = 7
    ax = (np.arange(1 << b) + 0.5) / (1 << b)
    g = np.stack(np.meshgrid(ax, ax, ax, indexing="ij"), axis=-1).reshape(-1, 3)
    perm = np.random.default_rng(0).permutation(g.shape[0])
    _check(g[perm], orc)


def test_full_depth_random_points(orc):
    _check(ics.uniform(2_000_000, 77), orc)


def test_ties_are_stable(orc):
    rng = np.random.default_rng(9)
    base = rng.random((300, 3))
    pos = base[rng.integers(0, 300, 50000)]          # many exact duplicates
    _check(pos, orc)


def test_periodic_wrap_and_edges(orc):
    rng = np.random.default_rng(4)
    pos = rng.random((20000, 3)) * 6.0 - 3.0          # far outside the box
    edge = np.array([[0.0, 1.0, -1e-300], [1.0 - 2 ** -53, 0.5, 0.25], [-0.0, 2.0, -3.0],
                     [2 ** -21, 1 - 2 ** -21, 0.5]])
    _check(np.concatenate([pos, edge]), orc)


def test_non_unit_box(orc):
    pos = ics.uniform(30000, 8) * 250.0
    _check(pos, orc, box=250.0)


def test_clustered_full_size_keys(orc):
    w = ics.make("nfw256", 128)                       # 2.1M clustered: long runs of near-equal keys
    _check(w.pos, orc)


def test_nonfinite_positions_flagged():
    dev = device()
    m = og()
    pos = torch.rand((1000, 3), dtype=torch.float64, device=dev)
    pos[17, 1] = float("nan")
    with pytest.raises(m.OGError) as e:
        m.keys_sort(pos, 1.0)
    assert e.value.code == 1


def test_non_power_of_two_box_with_wrap(orc):
    """A box side that is not a power of two takes the IEEE division in the
    wrap and the quantisation; positions span several periods."""
    rng = np.random.default_rng(91)
    L = 3.0
    pos = rng.random((50000, 3)) * 5.0 * L - 2.0 * L
    # and points just around quantisation boundaries of that box
    q = rng.integers(0, 1 << 21, size=(5000, 3)).astype(np.float64)
    edge = np.concatenate([q * (L / (1 << 21)), np.nextafter(q * (L / (1 << 21)), -np.inf)])
    _check(np.concatenate([pos, edge]), orc, box=L)
