"""Integer-pipe roundings of the tree build (csrc/split_coord.cuh) on the CPU.

The kernels store positions as split floats (hi = rint(xi 2^23) 2^-23,
lo = xi - hi rounded to FP32), masses and softenings as FP32 copies of FP64
products with 2^-2e, and cube centres (q + 1/2) 2^(e - l) in FP64.
split_coord.cuh computes these from bit patterns on the integer pipe; this
test compiles that header with g++ and holds it, bit for bit, against the
FP64 expressions written out in numpy, over random values and the rounding
edges (ties, powers of two, range ends).
"""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2606_17145_gb300", "csrc")

HARNESS = r"""
#include "split_coord.cuh"
#include <cstring>
extern "C" void t_split(const double* x, long n, int s, float* hi, float* lo, int* ok) {
  for (long i = 0; i < n; ++i) {
    uint64_t b;
    std::memcpy(&b, &x[i], 8);
    ok[i] = og::split_bits(b, s, hi[i], lo[i]) ? 1 : 0;
  }
}
extern "C" void t_cic(const double* x, long n, int s, int* i0, float* f, int* ok) {
  for (long i = 0; i < n; ++i) {
    uint64_t b;
    std::memcpy(&b, &x[i], 8);
    ok[i] = og::cic_bits(b, s, i0[i], f[i]) ? 1 : 0;
  }
}
extern "C" void t_odd(const unsigned* v, const int* x, long n, double* out, int* ok) {
  for (long i = 0; i < n; ++i) ok[i] = og::double_odd_scaled(v[i], x[i], out[i]) ? 1 : 0;
}
extern "C" void t_d2f(const double* x, long n, int s, float* out, int* ok) {
  for (long i = 0; i < n; ++i) {
    uint64_t b;
    std::memcpy(&b, &x[i], 8);
    ok[i] = og::d2f_scaled(b, s, out[i]) ? 1 : 0;
  }
}
"""


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    d = tmp_path_factory.mktemp("split")
    src = d / "h.cpp"
    src.write_text(HARNESS)
    so = d / "libh.so"
    subprocess.run([gxx, "-O2", "-std=c++17", "-shared", "-fPIC", "-I", CSRC, str(src), "-o", str(so)], check=True)
    L = ctypes.CDLL(str(so))
    P = ctypes.c_void_p
    L.t_split.argtypes = [P, ctypes.c_long, ctypes.c_int, P, P, P]
    L.t_d2f.argtypes = [P, ctypes.c_long, ctypes.c_int, P, P]
    L.t_odd.argtypes = [P, P, ctypes.c_long, P, P]
    L.t_cic.argtypes = [P, ctypes.c_long, ctypes.c_int, P, P, P]
    return L


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _split(lib, x, s):
    x = np.ascontiguousarray(x, dtype=np.float64)
    hi = np.zeros(x.shape, np.float32)
    lo = np.zeros(x.shape, np.float32)
    ok = np.zeros(x.shape, np.int32)
    lib.t_split(_ptr(x), x.size, s, _ptr(hi), _ptr(lo), _ptr(ok))
    return hi, lo, ok.astype(bool)


def _d2f(lib, x, s):
    x = np.ascontiguousarray(x, dtype=np.float64)
    out = np.zeros(x.shape, np.float32)
    ok = np.zeros(x.shape, np.int32)
    lib.t_d2f(_ptr(x), x.size, s, _ptr(out), _ptr(ok))
    return out, ok.astype(bool)


def _split_f64(xi):
    """The FP64 definition of the split-float format."""
    k = np.rint(xi * 8388608.0)
    h = k * (1.0 / 8388608.0)
    return h.astype(np.float32), (xi - h).astype(np.float32)


def _bits(a):
    return a.view(np.uint32)


def _coordinates(rng):
    u = rng.random(200000)
    k = rng.integers(0, 1 << 23, 100000).astype(np.float64)
    ties = (k + 0.5) / 2.0 ** 23
    near = np.concatenate([ties, np.nextafter(ties, 0), np.nextafter(ties, 2), k / 2.0 ** 23,
                           np.nextafter(k / 2.0 ** 23, 2)])
    scales = 2.0 ** rng.integers(-26, 1, 100000) * (1.0 + rng.random(100000))
    edges = np.array([2.0 ** -24, np.nextafter(2.0 ** -24, 1), np.nextafter(2.0 ** -24, 0), 1.5 * 2.0 ** -24,
                      2.0 ** -23, 3 * 2.0 ** -24, 0.5, 1.0, np.nextafter(1.0, 0), np.nextafter(1.0, 2),
                      1.5, np.nextafter(2.0, 0), 2.0, 0.0, 5e-324, 1e-310, np.inf, np.nan, -0.5, -0.0])
    return np.concatenate([u, near, scales, edges])


@pytest.mark.parametrize("s", [0, 1, -1, 3, -6])
def test_split_matches_fp64_definition(lib, s):
    rng = np.random.default_rng(11 + s)
    xi = _coordinates(rng)
    x = np.ldexp(xi, s)  # xi = x 2^-s exactly for these (normal) values
    hi, lo, ok = _split(lib, x, s)
    with np.errstate(invalid="ignore"):
        in_range = np.isfinite(xi) & (xi >= 2.0 ** -24) & (xi < 2.0)
    # applies exactly on [2^-24, 2), declines everything else
    np.testing.assert_array_equal(ok, in_range)
    eh, el = _split_f64(xi[ok])
    np.testing.assert_array_equal(_bits(hi[ok]), _bits(eh))
    np.testing.assert_array_equal(_bits(lo[ok]), _bits(el))
    # the format's own invariants: hi on the 2^-23 grid, hi + lo within FP32 of xi
    assert np.all(np.rint(hi[ok].astype(np.float64) * 2.0 ** 23) == hi[ok].astype(np.float64) * 2.0 ** 23)
    assert np.all(np.abs(lo[ok]) <= 2.0 ** -24)


def test_split_ties_round_to_even(lib):
    # xi = (k + 1/2) 2^-23 exactly: hi takes the even neighbour, lo = +-2^-24
    k = np.arange(0, 4096, dtype=np.float64)
    xi = (k + 0.5) / 2.0 ** 23
    hi, lo, ok = _split(lib, xi, 0)
    assert ok[1:].all()
    kk = k[1:]
    even = np.where(kk % 2 == 0, kk, kk + 1)
    np.testing.assert_array_equal(hi[1:].astype(np.float64), even / 2.0 ** 23)
    np.testing.assert_array_equal(lo[1:].astype(np.float64), np.where(kk % 2 == 0, 2.0 ** -24, -(2.0 ** -24)))


@pytest.mark.parametrize("s", [0, 2, -4, 20, -30])
def test_d2f_matches_fp64_conversion(lib, s):
    rng = np.random.default_rng(5 + abs(s))
    e = rng.integers(-170, 170, 200000)
    x = np.ldexp(1.0 + rng.random(200000), e + s)
    fmax = np.float64(np.finfo(np.float32).max)
    fmin = np.float64(np.finfo(np.float32).tiny)
    ulp_top = 2.0 ** (127 - 23)
    edges = np.array([fmax, fmax + ulp_top / 2, np.nextafter(fmax + ulp_top / 2, 0), fmin, np.nextafter(fmin, 0),
                      1.0, 1.0 + 2.0 ** -24, 1.0 + 3 * 2.0 ** -24, 1.0 + 2.0 ** -24 + 2.0 ** -40,
                      0.0, 5e-324, np.inf, np.nan, -1.0])
    m = rng.integers(1 << 23, 1 << 24, 50000).astype(np.float64)
    ties = np.ldexp(m + 0.5, rng.integers(-100, 100, 50000) - 23)
    xs = np.concatenate([x, np.ldexp(edges, s), np.ldexp(ties, s), np.ldexp(np.nextafter(ties, 0), s)])
    out, ok = _d2f(lib, xs, s)
    with np.errstate(invalid="ignore", over="ignore"):
        v = np.ldexp(xs, -s)
        expect = v.astype(np.float32)
        applies = np.isfinite(xs) & (xs > 0) & (v >= fmin) & (v < 2.0 ** 128) & (xs >= 2.0 ** -1022)
    # declines only outside the normal FP32 range (or for non-positive input)
    assert not np.any(ok & ~applies)
    assert np.all(ok[applies & (v <= fmax)])
    np.testing.assert_array_equal(_bits(out[ok]), _bits(expect[ok]))


def test_odd_scaled_is_the_exact_cell_centre(lib):
    rng = np.random.default_rng(17)
    lev = rng.integers(0, 22, 100000)
    q = (rng.random(100000) * (2.0 ** lev)).astype(np.int64)
    e = rng.integers(-40, 40, 100000)
    v = (2 * q + 1).astype(np.uint32)
    x = (e - lev - 1).astype(np.int32)
    # range ends: largest and smallest normal results, and just beyond them
    v = np.concatenate([v, np.array([1, 1, 1, 1, (1 << 22) - 1, (1 << 22) - 1, 3, 2], np.uint32)])
    x = np.concatenate([x, np.array([-1022, -1023, 1023, 1024, 1023 - 21, 1024 - 21, -1050, 0], np.int32)])
    out = np.zeros(v.shape, np.float64)
    ok = np.zeros(v.shape, np.int32)
    lib.t_odd(_ptr(v), _ptr(x), v.size, _ptr(out), _ptr(ok))
    ok = ok.astype(bool)
    with np.errstate(over="ignore"):
        expect = np.ldexp(v.astype(np.float64), x)  # exact where normal
    normal = np.isfinite(expect) & (expect >= np.finfo(np.float64).tiny) & (v % 2 == 1)
    np.testing.assert_array_equal(ok, normal)
    np.testing.assert_array_equal(out[ok].view(np.uint64), expect[ok].view(np.uint64))
    # the centre form used by the tree: (q + 1/2) 2^(e - lev)
    m = ok[:100000]
    centre = (q[m] + 0.5) * np.ldexp(1.0, e[m] - lev[m])
    np.testing.assert_array_equal(out[:100000][m], centre)


@pytest.mark.parametrize("s", [0, -8, -10, 3])
def test_cic_matches_fp64_floor_and_fraction(lib, s):
    """Mesh coordinate u = x 2^-s (e.g. x N / L for L = 1, N = 2^8: s = -8):
    i0 = floor(u) and f = (float)(u - floor(u)) as FP64 gives them."""
    rng = np.random.default_rng(23 + abs(s))
    u = np.concatenate([rng.random(200000) * 1024.0, rng.random(50000),
                        np.arange(0, 1025, dtype=np.float64),                      # nodes: f = 0
                        np.nextafter(np.arange(1, 1025, dtype=np.float64), 0),     # just below a node
                        np.arange(0, 1024) + 0.5, rng.integers(0, 1024, 50000) + 2.0 ** -30,
                        np.array([0.0, 2.0 ** -126, 2.0 ** -127, 5e-324, 2.0 ** 31, 2.0 ** 30 + 0.5,
                                  np.inf, np.nan, -0.25, -0.0])])
    x = np.ldexp(u, s)
    x = np.ascontiguousarray(x)
    i0 = np.zeros(x.shape, np.int32)
    f = np.zeros(x.shape, np.float32)
    ok = np.zeros(x.shape, np.int32)
    lib.t_cic(_ptr(x), x.size, s, _ptr(i0), _ptr(f), _ptr(ok))
    ok = ok.astype(bool)
    with np.errstate(invalid="ignore"):
        uu = np.ldexp(x, -s)
        applies = (x == 0) & ~np.signbit(x) | (np.isfinite(uu) & (uu >= 2.0 ** -126) & (uu < 2.0 ** 31)
                                              & (x >= 2.0 ** -1022))
    np.testing.assert_array_equal(ok, applies)
    fl = np.floor(uu[ok])
    np.testing.assert_array_equal(i0[ok], fl.astype(np.int64))
    np.testing.assert_array_equal(f[ok].view(np.uint32), (uu[ok] - fl).astype(np.float32).view(np.uint32))
