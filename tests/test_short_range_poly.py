"""The FP32 polynomial of the walk's short-range factor.

f(u) = erfc(u) + (2u/sqrt(pi)) exp(-u^2) = exp(-u^2) g(u) with
g(u) = erfcx(u) + 2u/sqrt(pi) on u in [0, 2.25] (r < 4.5 r_s).  The kernel
evaluates g as a degree-11 polynomial in t = u / 1.125 - 1 by FP32 Horner
with fused multiply-adds; this checks the committed table against scipy's
erfcx (independent of the oracle and of the kernels).
"""
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
INC = os.path.join(ROOT, "paper_2606_17145_gb300", "csrc", "short_range_poly.inc")


def _coefficients():
    text = open(INC).read()
    deg = int(re.search(r"#define OG_SR_POLY_DEG (\d+)", text).group(1))
    body = text[text.index("{") + 1:text.index("}")]
    c = np.array([float(x) for x in re.findall(r"(-?\d[\d.]*(?:e-?\d+)?)f", body)], dtype=np.float32)
    assert c.shape[0] == deg + 1
    return c


def _fma32(a, b, c):
    # product of two FP32 values is exact in FP64; one rounding to FP32
    return (a.astype(np.float64) * b.astype(np.float64) + c.astype(np.float64)).astype(np.float32)


def _horner32(c, t):
    acc = np.full_like(t, c[-1])
    for k in range(c.shape[0] - 2, -1, -1):
        acc = _fma32(acc, t, np.full_like(t, c[k]))
    return acc


def test_polynomial_accuracy_on_the_cut_interval():
    special = pytest.importorskip("scipy.special")
    c = _coefficients()
    u = np.linspace(0.0, 2.25, 200001)
    t = (u.astype(np.float32) * np.float32(1.0 / 1.125) - np.float32(1.0)).astype(np.float32)
    g = special.erfcx(u) + 2.0 * u / np.sqrt(np.pi)
    rel = np.abs(_horner32(c, t).astype(np.float64) / g - 1.0)
    assert rel.max() <= 2.0e-7
    # the factor itself (with the exact exponential): f(0) = 1, f(2.25) ~ 0.0175
    f = _horner32(c, t).astype(np.float64) * np.exp(-u * u)
    ref = special.erfc(u) + 2.0 * u / np.sqrt(np.pi) * np.exp(-u * u)
    assert np.abs(f / ref - 1.0).max() <= 2.0e-7
    assert abs(f[0] - 1.0) <= 2.5e-7


def test_table_is_what_the_generator_writes():
    pytest.importorskip("scipy")
    import importlib.util
    spec = importlib.util.spec_from_file_location(
        "fit_short_range_poly", os.path.join(ROOT, "paper_2606_17145_gb300", "csrc", "fit_short_range_poly.py"))
    mod = importlib.util.module_from_spec(spec)
    import sys
    keep = sys.dont_write_bytecode
    sys.dont_write_bytecode = True  # no cache files next to the CUDA sources
    try:
        spec.loader.exec_module(mod)
    finally:
        sys.dont_write_bytecode = keep
    coeffs, err = mod.fit()
    assert np.array_equal(np.asarray(coeffs, dtype=np.float64).astype(np.float32), _coefficients())
    assert err <= 2.5e-7
