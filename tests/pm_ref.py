"""Closed-form references for the PM long-range tests: the exact long-range
Fourier series of a point mass and the Ewald sum of the periodic Newtonian
force (unit mass, G = 1, unit box by default).  They share nothing with the
oracle or the CUDA path."""
import numpy as np
from scipy.special import erfc

L = 1.0


def _kvectors(kmax, L=L):
    k1 = np.arange(-kmax, kmax + 1)
    KX, KY, KZ = np.meshgrid(k1, k1, k1, indexing="ij")
    kv = np.stack([KX.ravel(), KY.ravel(), KZ.ravel()], 1) * 2.0 * np.pi / L
    k2 = (kv ** 2).sum(1)
    keep = k2 > 0
    return kv[keep], k2[keep]


def long_series(d, r_s, L=L):
    """Exact periodic long-range force of a unit mass at separation d:
    -(4 pi / L^3) sum_k k exp(-k^2 r_s^2) / k^2 sin(k . d)."""
    kmax = int(np.ceil(np.sqrt(45.0) / (2.0 * np.pi * r_s / L))) + 1
    kv, k2 = _kvectors(kmax, L)
    w = np.exp(-k2 * r_s ** 2) / k2 * np.sin(kv @ d)
    return -(4.0 * np.pi / L ** 3) * (w[:, None] * kv).sum(0)


def ewald(d, alpha, L=L):
    """Periodic Newtonian force of a unit mass at separation d (Ewald sum with
    splitting parameter alpha, neutralising background)."""
    F = np.zeros(3)
    for a in range(-2, 3):
        for b in range(-2, 3):
            for c in range(-2, 3):
                s = d + L * np.array([a, b, c])
                r = np.linalg.norm(s)
                F -= (erfc(alpha * r) + 2.0 * alpha * r / np.sqrt(np.pi) * np.exp(-(alpha * r) ** 2)) * s / r ** 3
    kv, k2 = _kvectors(int(np.ceil(7.0 * alpha * L / np.pi)) + 1, L)
    w = np.exp(-k2 / (4.0 * alpha ** 2)) / k2 * np.sin(kv @ d)
    F -= (4.0 * np.pi / L ** 3) * (w[:, None] * kv).sum(0)
    return F
