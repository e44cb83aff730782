"""Writes short_range_poly.inc: the polynomial used by the FP32 walk for the
short-range force factor.

f(u) = erfc(u) + (2u/sqrt(pi)) exp(-u^2) = exp(-u^2) g(u),
g(u) = erfcx(u) + 2u/sqrt(pi),   u = r / (2 r_s) in [0, 2.25] (r < 4.5 r_s).

g is fitted by relative-weighted least squares on Chebyshev nodes as a
degree-11 polynomial in t = u / 1.125 - 1 in [-1, 1] (centring keeps the
coefficients decaying, so FP32 Horner evaluation stays within ~2e-7 of g).
exp(-u^2) is evaluated separately with the hardware base-2 exponential.
Run: python fit_short_range_poly.py  (needs numpy and scipy).
"""
import os

import numpy as np
from scipy.special import erfcx

DEG = 11
HALF = 1.125


def fit():
    g = lambda u: erfcx(u) + 2.0 * u / np.sqrt(np.pi)
    m = 6 * DEG
    t = np.cos(np.pi * (np.arange(m) + 0.5) / m)
    u = (t + 1.0) * HALF
    c = np.polyfit(t, g(u), DEG, w=1.0 / g(u))[::-1]  # c[0] + c[1] t + ...
    uu = np.linspace(0.0, 2.0 * HALF, 400001)
    tt = (uu.astype(np.float32) * np.float32(1.0 / HALF) - np.float32(1.0)).astype(np.float32)
    cf = c.astype(np.float32)
    acc = np.full_like(tt, cf[-1])
    for k in range(DEG - 1, -1, -1):
        acc = (acc * tt + cf[k]).astype(np.float32)
    err = float(np.abs(acc.astype(np.float64) / g(uu) - 1.0).max())
    return c, err


def main():
    c, err = fit()
    here = os.path.dirname(os.path.abspath(__file__))
    lines = ["// Generated by fit_short_range_poly.py -- do not edit.",
             f"// g(u) = erfcx(u) + 2u/sqrt(pi) ~ sum_k c_k t^k, t = u / {HALF} - 1, u in [0, {2 * HALF}]",
             f"// max relative error of FP32 Horner evaluation on the interval: {err:.2e}",
             f"#define OG_SR_POLY_DEG {DEG}",
             f"#define OG_SR_POLY_INV_HALF {1.0 / HALF!r}",
             "__constant__ float og_sr_poly[OG_SR_POLY_DEG + 1] = {"]
    lines += [f"    {float(np.float32(v))!r}f," for v in c]
    lines += ["};", ""]
    with open(os.path.join(here, "short_range_poly.inc"), "w") as f:
        f.write("\n".join(lines))
    print("max rel err", err)


if __name__ == "__main__":
    main()
