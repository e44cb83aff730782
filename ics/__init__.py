"""Seeded synthetic particle sets for the short-range gravity workloads.

This module is shared by the oracle-side tests and the CUDA-side tests and
benchmark.  It only draws particle positions, masses, softenings and loss
weights; it holds none of the force, key, tree or walk arithmetic.

The paper's own initial conditions (the Magneticum Box1a/mr dark-matter box of
Sec. 3.1 and the Dianoga zoom clusters of Secs. 3.3-3.4) are not available, so
these generators stand in for them with the same kind of structure:

* ``uniform``      -- uniform random points (homogeneous, like the early,
                      near-homogeneous start of the scaling runs in Sec. 4.1);
* ``zeldovich``    -- a lattice displaced by a Gaussian random field with
                      P(k) ~ k^-2 (a cosmological-box start, Sec. 3.1);
* ``nfw_clustered``-- NFW haloes plus a uniform background (an evolved,
                      clustered box);
* ``zoom``         -- a high-resolution NFW region inside a low-resolution
                      uniform background with heavier particles and larger
                      softening (the multi-mass zoom-in set-up of Secs. 3.3-3.4).

All randomness comes from numpy's PCG64 with an explicit seed; positions are
float64 in the periodic unit box [0, 1).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

BOX = 1.0


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def _wrap(x: np.ndarray) -> np.ndarray:
    x = np.mod(x, BOX)
    # np.mod can return BOX for tiny negative inputs; fold those to 0.
    x[x >= BOX] = 0.0
    return x


def uniform(n: int, seed: int) -> np.ndarray:
    """n points uniform in [0, 1)^3."""
    return _rng(seed).random((n, 3), dtype=np.float64)


def zeldovich(ngrid: int, seed: int, rms_disp_cells: float = 0.5) -> np.ndarray:
    """ngrid^3 lattice displaced by a Zel'dovich field.

    delta(k) is Gaussian with power P(k) ~ k^-2 on the grid's modes (modes on
    the Nyquist planes are dropped so the displacement is real), the
    displacement is psi(k) = i k delta(k) / k^2, and psi is rescaled so that
    its rms length is ``rms_disp_cells`` grid spacings.
    """
    rng = _rng(seed)
    n = ngrid
    white = rng.standard_normal((n, n, n))
    wk = np.fft.rfftn(white)
    kx = np.fft.fftfreq(n) * n
    kz = np.fft.rfftfreq(n) * n
    KX, KY, KZ = np.meshgrid(kx, kx, kz, indexing="ij")
    k2 = KX * KX + KY * KY + KZ * KZ
    nyq = n // 2
    keep = (np.abs(KX) < nyq) & (np.abs(KY) < nyq) & (np.abs(KZ) < nyq) & (k2 > 0)
    amp = np.zeros_like(k2)
    amp[keep] = 1.0 / np.sqrt(k2[keep])          # sqrt(P) with P ~ k^-2
    dk = wk * amp
    inv_k2 = np.zeros_like(k2)
    inv_k2[keep] = 1.0 / k2[keep]
    psi = np.empty((3, n, n, n))
    for a, K in enumerate((KX, KY, KZ)):
        psi[a] = np.fft.irfftn(1j * K * dk * inv_k2, s=(n, n, n))
    rms = math.sqrt(float(np.mean(np.sum(psi * psi, axis=0))))
    psi *= (rms_disp_cells / n) / rms
    g = (np.arange(n, dtype=np.float64) + 0.5) / n
    QX, QY, QZ = np.meshgrid(g, g, g, indexing="ij")
    pos = np.stack([QX + psi[0], QY + psi[1], QZ + psi[2]], axis=-1).reshape(-1, 3)
    return _wrap(pos)


def _nfw_radii(rng: np.random.Generator, count: int, r200: float, conc: float) -> np.ndarray:
    """Radii drawn from an NFW profile truncated at r200 (inverse CDF by Newton)."""
    if count == 0:
        return np.zeros(0)
    mu = lambda x: np.log1p(x) - x / (1.0 + x)
    target = rng.random(count) * mu(conc)
    # Newton on mu(x) = target; mu'(x) = x / (1 + x)^2.  Start from a safe guess.
    x = np.clip(target * 2.0, 1e-8, conc)
    for _ in range(60):
        fx = mu(x) - target
        dfx = x / (1.0 + x) ** 2
        step = fx / np.maximum(dfx, 1e-300)
        x_new = np.clip(x - step, x * 0.1, np.minimum(x * 10.0 + 1e-12, conc))
        if np.max(np.abs(x_new - x) / np.maximum(x, 1e-300)) < 1e-14:
            x = x_new
            break
        x = x_new
    return x * (r200 / conc)


def _isotropic(rng: np.random.Generator, count: int) -> np.ndarray:
    v = rng.standard_normal((count, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    return v


def nfw_clustered(n: int, seed: int, n_halos: int = 2000, halo_frac: float = 0.6,
                  m_lo: float = 1e-5, m_hi: float = 1e-2, slope: float = -1.9,
                  c_lo: float = 5.0, c_hi: float = 15.0) -> np.ndarray:
    """n equal-mass points: ``halo_frac`` of them in NFW haloes, the rest uniform.

    Halo masses follow dN/dM ~ M^slope on [m_lo, m_hi] (fractions of the total
    mass) and are rescaled so they sum to ``halo_frac``; particles are assigned
    by largest-remainder rounding; concentrations are uniform in [c_lo, c_hi];
    r200 encloses 200 times the mean density (mean density 1 in the unit box);
    centres are uniform; positions wrap periodically.
    """
    rng = _rng(seed)
    a = slope + 1.0
    u = rng.random(n_halos)
    mh = (m_lo ** a + u * (m_hi ** a - m_lo ** a)) ** (1.0 / a)
    mh *= halo_frac / mh.sum()
    n_halo_total = int(round(halo_frac * n))
    raw = mh / mh.sum() * n_halo_total
    cnt = np.floor(raw).astype(np.int64)
    rem = n_halo_total - int(cnt.sum())
    if rem > 0:
        order = np.argsort(-(raw - cnt), kind="stable")
        cnt[order[:rem]] += 1
    conc = rng.uniform(c_lo, c_hi, n_halos)
    centres = rng.random((n_halos, 3))
    parts = []
    for h in range(n_halos):
        r200 = (3.0 * mh[h] / (800.0 * math.pi)) ** (1.0 / 3.0)
        r = _nfw_radii(rng, int(cnt[h]), r200, conc[h])
        parts.append(centres[h] + r[:, None] * _isotropic(rng, int(cnt[h])))
    bg = rng.random((n - n_halo_total, 3))
    pos = np.concatenate(parts + [bg], axis=0)
    pos = pos[rng.permutation(n)]
    return _wrap(pos)


def zoom(n_hr: int, n_lr: int, seed: int, r_trunc: float = 0.1, conc: float = 10.0):
    """High-resolution NFW sphere at the box centre plus a uniform low-res background.

    Returns (pos, mass, species) with species 0 = high-res (mass m), 1 = low-res
    (mass 64 m); m is chosen so the total mass is 1.
    """
    rng = _rng(seed)
    r = _nfw_radii(rng, n_hr, r_trunc, conc)
    hr = 0.5 + r[:, None] * _isotropic(rng, n_hr)
    lr = rng.random((n_lr, 3))
    m = 1.0 / (n_hr + 64.0 * n_lr)
    pos = _wrap(np.concatenate([hr, lr], axis=0))
    mass = np.concatenate([np.full(n_hr, m), np.full(n_lr, 64.0 * m)])
    species = np.concatenate([np.zeros(n_hr, np.int8), np.ones(n_lr, np.int8)])
    perm = rng.permutation(n_hr + n_lr)
    return pos[perm], mass[perm], species[perm]


def loss_weights(n: int, seed: int) -> np.ndarray:
    """w_i ~ N(0, I_3) weights of the loss L = sum_i w_i . a_i."""
    return _rng(seed).standard_normal((n, 3))


@dataclass
class Workload:
    """One seeded particle set plus the short-range parameters it is run with."""
    name: str
    pos: np.ndarray                 # float64 [n, 3], in [0, box)
    mass: np.ndarray                # float64 [n]
    eps: np.ndarray                 # float64 [n] softening lengths (Plummer-equivalent)
    box: float
    r_s: float
    thetas: tuple
    w: np.ndarray | None = None     # float64 [n, 3] loss weights (adjoint workloads)
    notes: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.pos.shape[0])

    @property
    def rcut(self) -> float:
        return 4.5 * self.r_s


def make(name: str, scale: int | None = None) -> Workload:
    """Build a named workload.

    ``scale`` shrinks the set for fast tests: for the lattice / clustered sets
    it is the number of particles per side, for ``uniform4096`` the particle
    count, for ``zoom`` the high-res count (low-res = scale / 4).
    Seeds are 1000 + workload index.
    """
    if name == "uniform4096":
        n = scale or 4096
        pos = uniform(n, 1000)
        return Workload(name, pos, np.full(n, 1.0 / n), np.full(n, 1.0 / 480.0),
                        BOX, 1.25 / 16.0, (0.5, 0.0))
    if name == "zeldovich128":
        side = scale or 128
        pos = zeldovich(side, 1001)
        n = side ** 3
        return Workload(name, pos, np.full(n, 1.0 / n), np.full(n, 1.0 / (30.0 * side)),
                        BOX, 1.25 / (2.0 * side), (0.5,))
    if name == "nfw256":
        side = scale or 256
        n = side ** 3
        pos = nfw_clustered(n, 1002)
        return Workload(name, pos, np.full(n, 1.0 / n), np.full(n, 1.0 / (30.0 * side)),
                        BOX, 1.25 / (2.0 * side), (0.5,))
    if name == "nfw128_adjoint":
        side = scale or 128
        n = side ** 3
        pos = nfw_clustered(n, 1003)
        return Workload(name, pos, np.full(n, 1.0 / n), np.full(n, 1.0 / (30.0 * side)),
                        BOX, 1.25 / (2.0 * side), (0.5,), w=loss_weights(n, 2003))
    if name == "zoom8m":
        n_hr = scale or (1 << 23)
        n_lr = max(n_hr // 4, 1)
        pos, mass, species = zoom(n_hr, n_lr, 1004)
        eps_hr = 1.0 / 20000.0
        eps = np.where(species == 0, eps_hr, 4.0 * eps_hr)
        # r_s follows the 512-per-side resolution of the full-size set.
        return Workload(name, pos, mass, eps, BOX, 1.25 / 512.0, (0.5,),
                        w=loss_weights(n_hr + n_lr, 2004))
    raise KeyError(name)


NAMES = ("uniform4096", "zeldovich128", "nfw256", "nfw128_adjoint", "zoom8m")
