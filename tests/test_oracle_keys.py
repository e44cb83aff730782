"""Pins for the oracle's Peano-Hilbert keys and key sort (CPU only).

The keys are pinned against facts about Hilbert curves that do not depend on
how the oracle computes them: the first-order curve is the reflected Gray code
(golden fixture), every order is a bijection onto [0, 8^b), consecutive cells
share a face, and the index of a cell's parent is the index's top bits.
"""
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "hilbert_order1.txt")


def _grid(b):
    n = 1 << b
    ax = np.arange(n, dtype=np.uint32)
    g = np.stack(np.meshgrid(ax, ax, ax, indexing="ij"), axis=-1).reshape(-1, 3)
    return g


def test_order1_is_reflected_gray_code(orc):
    rows = np.loadtxt(GOLDEN, dtype=np.int64)
    for idx, x0, x1, x2 in rows:
        assert int(orc.hilbert_grid([[x0, x1, x2]], 1)[0]) == idx


@pytest.mark.parametrize("b", [1, 2, 3, 4, 5])
def test_bijection_and_face_adjacency(orc, b):
    g = _grid(b)
    k = orc.hilbert_grid(g, b)
    assert np.array_equal(np.sort(k), np.arange(8 ** b, dtype=np.uint64))
    walk = g[np.argsort(k)].astype(np.int64)
    step = np.abs(np.diff(walk, axis=0)).sum(axis=1)
    assert np.all(step == 1), "consecutive Hilbert cells must share a face"


def test_nested_prefixes_small_grid(orc):
    b = 5
    g = _grid(b)
    k = orc.hilbert_grid(g, b)
    parent = orc.hilbert_grid(g >> 1, b - 1)
    assert np.array_equal(k >> np.uint64(3), parent)


def test_nested_prefixes_full_depth(orc):
    rng = np.random.default_rng(7)
    q = rng.integers(0, 1 << 21, size=(300, 3), dtype=np.uint32)
    L = orc.lib()
    for a, b, c in q:
        full = L.orc_hilbert_cell(int(a), int(b), int(c))
        for lev in (1, 2, 5, 9, 14, 20):
            sh = 21 - lev
            coarse = L.orc_hilbert_grid(int(a) >> sh, int(b) >> sh, int(c) >> sh, lev)
            assert full >> (3 * sh) == coarse


def test_keys_are_63_bit_and_match_cells(orc):
    rng = np.random.default_rng(3)
    pos = rng.random((2000, 3))
    k, bad, cells = orc.keys(pos)
    assert bad == 0
    assert int(k.max()) < (1 << 63)
    # the integer cell is floor(x * 2^21) for x in [0, 1)
    assert np.array_equal(cells, np.floor(pos * 2.0 ** 21).astype(np.uint32))
    L = orc.lib()
    for i in range(0, 2000, 97):
        assert int(k[i]) == L.orc_hilbert_cell(int(cells[i, 0]), int(cells[i, 1]), int(cells[i, 2]))


def test_quantisation_edge_cases(orc):
    # rows: input x (all three axes) -> expected integer cell
    cases = [
        (0.0, 0),
        (1.0, 0),                      # x = box wraps to 0
        (1.5, 1 << 20),                # periodic wrap: 1.5 -> 0.5
        (-0.25, 3 << 19),              # -0.25 -> 0.75
        (0.5, 1 << 20),
        (1.0 - 2.0 ** -30, (1 << 21) - 1),
        (-1e-300, (1 << 21) - 1),      # wraps to 1.0 after rounding: clamped to the last cell
        (2.0 ** -21, 1),
        (2.0 ** -21 * (1 - 2.0 ** -40), 0),
    ]
    pos = np.array([[x, x, x] for x, _ in cases])
    _, bad, cells = orc.keys(pos)
    assert bad == 0
    for (x, q), c in zip(cases, cells):
        assert int(c[0]) == q, (x, int(c[0]), q)


def test_non_finite_positions_flagged(orc):
    pos = np.array([[0.1, 0.2, 0.3], [np.nan, 0.1, 0.1], [0.2, np.inf, 0.2]])
    _, bad, _ = orc.keys(pos)
    assert bad == 2


def test_sort_stable_against_numpy(orc):
    rng = np.random.default_rng(11)
    k = rng.integers(0, 1 << 10, size=5000).astype(np.uint64) << np.uint64(53)  # many ties
    ks, order = orc.sort(k)
    ref = np.argsort(k, kind="stable")
    assert np.array_equal(order, ref.astype(np.int32))
    assert np.array_equal(ks, k[ref])
