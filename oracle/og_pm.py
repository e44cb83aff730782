"""FP64 CPU oracle for the PM long-range complement of the TreePM split.

TEST INFRASTRUCTURE ONLY: the slow, obviously-correct reference that the
CUDA PM path is compared against.  Only the tests, ``__graft_entry__.smoke()``
and the benchmark's CPU-baseline / reference leg use it; the product path
never calls it and has no CPU fallback.  It shares no code with the CUDA
library.

The paper (Sec. 3.1) computes the long-range gravity on a particle mesh with
FFTW on the host and prints no formula for it.  The steps below are the
standard GADGET-2 TreePM long-range scheme, written out plainly, with G = 1.
They are the exact complement of the short-range factor
f(r) = erfc(r / 2 r_s) + (r / (sqrt(pi) r_s)) exp(-r^2 / 4 r_s^2): the
long-range potential of a point mass is the Fourier series of
-4 pi m exp(-k^2 r_s^2) / k^2.

  1. CIC deposit.  Mesh of N^3 nodes at x = i D (D = L / N, periodic).  A
     particle at u = x N / L (x wrapped into [0, L]) gives, along each axis,
     weight 1 - f to node floor(u) and f to node floor(u) + 1 (mod N), with
     f = u - floor(u); rho_node = sum m W / D^3.
  2. Forward DFT: rho_hat(kappa) = sum_node rho exp(-2 pi i kappa . node / N).
  3. Potential: phi_hat = -4 pi rho_hat exp(-k^2 r_s^2) / (k^2 S), with
     k = 2 pi kappa / L and S = prod_a sinc^4(kappa_a / N), sinc(t) =
     sin(pi t) / (pi t): the CIC window, once for the deposit and once for
     the interpolation.  phi_hat(0) = 0 (the mean density does not pull).
  4. Inverse DFT with the 1 / N^3 normalisation.
  5. Mesh force by the four-point central difference per axis:
     F = -[(2/3)(phi(+1) - phi(-1)) - (1/12)(phi(+2) - phi(-2))] / D.
  6. CIC interpolation of the mesh force to the particles, with the
     weights of step 1.

Parity status (pins in tests/test_oracle_pm.py): pinned by mass
conservation, the node-exact deposit, zero self-force, momentum
conservation, the exact long-range Fourier series of a point mass, and the
total short + long force against an Ewald sum with an unrelated splitting
parameter.
"""
from __future__ import annotations

import numpy as np


def wrap(x: np.ndarray, L: float) -> np.ndarray:
    """x folded into [0, L]: x - L floor(x / L)."""
    return x - L * np.floor(x / L)


def cic_weights(pos: np.ndarray, L: float, N: int):
    """Step 1: lower node index i0 (int64, in [0, N)) and fraction f per axis."""
    u = wrap(np.asarray(pos, dtype=np.float64), L) * N / L
    fl = np.floor(u)
    f = u - fl
    i0 = fl.astype(np.int64) % N
    return i0, f


def _corners():
    for dx in (0, 1):
        for dy in (0, 1):
            for dz in (0, 1):
                yield dx, dy, dz


def _corner_weight(f: np.ndarray, dx: int, dy: int, dz: int) -> np.ndarray:
    wx = f[:, 0] if dx else 1.0 - f[:, 0]
    wy = f[:, 1] if dy else 1.0 - f[:, 1]
    wz = f[:, 2] if dz else 1.0 - f[:, 2]
    return wx * wy * wz


def deposit(pos: np.ndarray, mass: np.ndarray, L: float, N: int) -> np.ndarray:
    """Step 1: the CIC density rho on the N^3 mesh (index [ix, iy, iz])."""
    i0, f = cic_weights(pos, L, N)
    m = np.asarray(mass, dtype=np.float64)
    rho = np.zeros((N, N, N))
    for dx, dy, dz in _corners():
        ix = (i0[:, 0] + dx) % N
        iy = (i0[:, 1] + dy) % N
        iz = (i0[:, 2] + dz) % N
        np.add.at(rho, (ix, iy, iz), m * _corner_weight(f, dx, dy, dz))
    D = L / N
    return rho / D ** 3


def green(N: int, L: float, r_s: float) -> np.ndarray:
    """Step 3: the factor phi_hat / rho_hat on the rfftn layout [N, N, N/2 + 1]."""
    kx = np.fft.fftfreq(N) * N
    kz = np.fft.rfftfreq(N) * N
    KX, KY, KZ = np.meshgrid(kx, kx, kz, indexing="ij")
    k2 = (2.0 * np.pi / L) ** 2 * (KX ** 2 + KY ** 2 + KZ ** 2)
    S = (np.sinc(KX / N) * np.sinc(KY / N) * np.sinc(KZ / N)) ** 4
    g = np.zeros_like(k2)
    nz = k2 > 0
    g[nz] = -4.0 * np.pi * np.exp(-k2[nz] * r_s ** 2) / (k2[nz] * S[nz])
    return g


def potential(rho: np.ndarray, L: float, r_s: float) -> np.ndarray:
    """Steps 2-4: the long-range potential on the mesh."""
    N = rho.shape[0]
    rho_hat = np.fft.rfftn(rho)
    return np.fft.irfftn(rho_hat * green(N, L, r_s), s=rho.shape, axes=(0, 1, 2))


def mesh_force(phi: np.ndarray, L: float) -> np.ndarray:
    """Step 5: F[a] on the mesh, a = 0, 1, 2 (shape [3, N, N, N])."""
    D = L / phi.shape[0]
    F = np.empty((3,) + phi.shape)
    for a in range(3):
        p1 = np.roll(phi, -1, axis=a)   # phi at node + 1
        m1 = np.roll(phi, 1, axis=a)    # phi at node - 1
        p2 = np.roll(phi, -2, axis=a)
        m2 = np.roll(phi, 2, axis=a)
        F[a] = -((2.0 / 3.0) * (p1 - m1) - (1.0 / 12.0) * (p2 - m2)) / D
    return F


def interpolate(F: np.ndarray, pos: np.ndarray, L: float) -> np.ndarray:
    """Step 6: CIC interpolation of the mesh force to the particles."""
    N = F.shape[1]
    i0, f = cic_weights(pos, L, N)
    acc = np.zeros((i0.shape[0], 3))
    for dx, dy, dz in _corners():
        ix = (i0[:, 0] + dx) % N
        iy = (i0[:, 1] + dy) % N
        iz = (i0[:, 2] + dz) % N
        w = _corner_weight(f, dx, dy, dz)
        for a in range(3):
            acc[:, a] += w * F[a][ix, iy, iz]
    return acc


def pm_accel(pos: np.ndarray, mass: np.ndarray, L: float, N: int, r_s: float) -> np.ndarray:
    """Long-range accelerations [n, 3] of every particle (steps 1-6)."""
    rho = deposit(pos, mass, L, N)
    phi = potential(rho, L, r_s)
    return interpolate(mesh_force(phi, L), pos, L)
