"""FP64 CPU oracle for the SPH density / smoothing-length iteration.

TEST INFRASTRUCTURE ONLY: the slow, obviously-correct reference that the
device's grouped density walk (og_sph_density) is compared with.  Only the
tests and the benchmark's CPU legs use it.

The paper's SPH density module iterates the smoothing length of each
particle until its sphere holds a fixed number of neighbours, and its
neighbour walks first gather all neighbours inside a sphere and then
evaluate them (Sec. 2.1).  It prints no formula.  The reading here is the
GADGET-2 one, with periodic minimum-image distances:

  kernel   W(r, h) = 8 / (pi h^3) w(q), q = r / h, with
           w = 1 - 6 q^2 + 6 q^3 for q <= 1/2, 2 (1 - q)^3 for 1/2 < q <= 1,
           and 0 beyond (support h, unit integral);
  density  rho_i = sum_j m_j W(|x_i - x_j|, h_i), the particle itself included;
  h_i      the root of N_eff(h) = (4 pi / 3) h^3 sum_j W(|x_i - x_j|, h) = N_ngb,
           the kernel-weighted neighbour count (for equal masses
           (4 pi / 3) h^3 rho / m).  It is increasing in h, and bisection
           finds it.

Parity status (pins in tests/test_oracle_sph.py): pinned by the kernel's unit
integral, the density of a uniform lattice (m / a^3), neighbour counts
against scipy's periodic k-d tree, the scaling of h and rho with the box,
and the root condition.
"""
from __future__ import annotations

import numpy as np


def w_spline(q: np.ndarray) -> np.ndarray:
    """The dimensionless cubic spline w(q) (support q <= 1)."""
    q = np.asarray(q, dtype=np.float64)
    out = np.zeros_like(q)
    a = q <= 0.5
    b = (q > 0.5) & (q <= 1.0)
    out[a] = 1.0 - 6.0 * q[a] ** 2 + 6.0 * q[a] ** 3
    out[b] = 2.0 * (1.0 - q[b]) ** 3
    return out


def kernel(r, h):
    """W(r, h) = 8 / (pi h^3) w(r / h)."""
    h = np.asarray(h, dtype=np.float64)
    return 8.0 / (np.pi * h ** 3) * w_spline(np.asarray(r, dtype=np.float64) / h)


def distances(pos: np.ndarray, i: int, box: float) -> np.ndarray:
    """Minimum-image distances from particle i to every particle (itself: 0)."""
    d = pos - pos[i]
    d -= box * np.round(d / box)
    return np.sqrt((d ** 2).sum(axis=1))


def n_eff(r: np.ndarray, h: float) -> float:
    """(4 pi / 3) h^3 sum_j W(r_j, h) = (32 / 3) sum_j w(r_j / h)."""
    return (4.0 * np.pi / 3.0) * h ** 3 * float(kernel(r, h).sum())


def smoothing_length(pos, box: float, n_ngb: float, targets=None, rel_tol: float = 1e-12):
    """h_i with N_eff(h_i) = n_ngb for the targets (default: every particle),
    by bisection; neighbours are all particles."""
    pos = np.asarray(pos, dtype=np.float64)
    tg = np.arange(pos.shape[0]) if targets is None else np.asarray(targets)
    h = np.empty(tg.shape[0])
    for k, i in enumerate(tg):
        r = distances(pos, int(i), box)
        lo, hi = 0.0, 0.5 * box  # minimum image holds below half the box
        if n_eff(r, hi) < n_ngb:
            raise ValueError("n_ngb needs h >= box / 2")
        while hi - lo > rel_tol * hi:
            mid = 0.5 * (lo + hi)
            if n_eff(r, mid) < n_ngb:
                lo = mid
            else:
                hi = mid
        h[k] = hi
    return h


def density(pos, mass, h, box: float, targets=None) -> np.ndarray:
    """rho_i = sum_j m_j W(r_ij, h_i) for the targets (default: every particle)."""
    pos = np.asarray(pos, dtype=np.float64)
    m = np.asarray(mass, dtype=np.float64)
    tg = np.arange(pos.shape[0]) if targets is None else np.asarray(targets)
    h = np.broadcast_to(np.asarray(h, dtype=np.float64), (tg.shape[0],))
    return np.array([float((m * kernel(distances(pos, int(i), box), h[k])).sum()) for k, i in enumerate(tg)])


def neighbour_count(pos, h, box: float) -> np.ndarray:
    """Number of particles j != i with r_ij < h_i."""
    pos = np.asarray(pos, dtype=np.float64)
    h = np.broadcast_to(np.asarray(h, dtype=np.float64), (pos.shape[0],))
    return np.array([int((distances(pos, i, box) < h[i]).sum()) - 1 for i in range(pos.shape[0])])
