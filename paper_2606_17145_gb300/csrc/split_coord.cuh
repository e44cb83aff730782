// split_coord.cuh -- integer-pipe forms of two FP64 roundings used when the
// tree stores FP32 copies of positions and masses (the FP64 pipe runs at a
// small fraction of the integer rate on this GPU).  Each works on the bit
// pattern of a positive double x and a power-of-two scale 2^-s, gives the
// same bits as the FP64 expression it replaces, and returns false (writing
// nothing) where it does not apply, so the caller then evaluates that FP64
// expression.  Host-compilable, so that a CPU test can hold it against the
// FP64 definitions.
#pragma once

#include <cstdint>
#include <cstring>

#if defined(__CUDACC__)
#define OG_HD __host__ __device__ __forceinline__
#else
#define OG_HD inline
#endif

namespace og {

OG_HD int clz64(uint64_t u) {  // u != 0
#if defined(__CUDA_ARCH__)
  return __clzll((long long)u);
#else
  return __builtin_clzll(u);
#endif
}

OG_HD float float_from_bits(uint32_t b) {
#if defined(__CUDA_ARCH__)
  return __uint_as_float(b);
#else
  float f;
  std::memcpy(&f, &b, sizeof f);
  return f;
#endif
}

// Round-to-nearest-even of the significand bits below bit c (0 < c < 64):
// 1 when the discarded part r of v exceeds half an ulp, or equals it and the
// kept part q is odd.
OG_HD uint32_t round_up(uint64_t q, uint64_t r, int c) {
  const uint64_t half = 1ull << (c - 1);
  return (r > half || (r == half && (q & 1ull))) ? 1u : 0u;
}

// Split of xi = x 2^-s, with b the bits of x:
//   hi = rint(xi 2^23) 2^-23 (ties to even) and lo = (float)(xi - hi),
// the FP64 expressions of the split-float position format.  Applies when
// 2^-24 <= xi < 2.
//
// With xi = S 2^(ex - 52) (S the 53-bit significand), rint(xi 2^23) is S
// shifted right by c = 29 - ex and rounded to even, R = q + up; hi = R 2^-23
// is exact in FP32 since R <= 2^24.  xi - hi = D 2^(ex - 52) with
// D = (S mod 2^c) - up 2^c, |D| <= 2^52, which FP64 holds exactly; lo rounds
// D to 24 significant bits and places the exponent.
OG_HD bool split_bits(uint64_t b, int s, float& hi, float& lo) {
  const int E = (int)(b >> 52);  // a set sign bit gives E >= 2048
  if (E == 0 || E >= 2047) return false;
  const int ex = E - 1023 - s;
  if (ex < -24 || ex > 0) return false;
  const uint64_t S = (b & 0x000fffffffffffffull) | 0x0010000000000000ull;
  const int c = 29 - ex;  // 29 .. 53
  const uint64_t q = S >> c;
  const uint64_t rem = S & ((1ull << c) - 1ull);
  const uint32_t up = round_up(q, rem, c);
  hi = (float)((uint32_t)q + up) * 0x1p-23f;
  const int64_t D = (int64_t)rem - (up ? (int64_t)(1ull << c) : 0);
  if (D == 0) {
    lo = 0.0f;
    return true;
  }
  const uint64_t u = D < 0 ? (uint64_t)(-D) : (uint64_t)D;
  const int lz = clz64(u);            // >= 11
  const uint64_t v = u << lz;         // leading one at bit 63
  const uint32_t m = (uint32_t)(v >> 40);
  const uint32_t r = round_up(m, v & 0xffffffffffull, 40);
  // |lo| = m 2^(11 - lz + ex - 23): biased exponent 138 - lz + ex (51 .. 127)
  const uint32_t fb = ((uint32_t)(138 - lz + ex) << 23) + (m - 0x800000u) + r;
  lo = float_from_bits(fb | (D < 0 ? 0x80000000u : 0u));
  return true;
}

// out = (float)(x 2^-s) for x > 0 whose scaled value is a normal FP32
// number, from the bits b of x.  The scaling by 2^-s is exact in FP64 there,
// so this equals (float)(x * 2^-s).  A carry out of the largest exponent
// gives infinity, as the FP64 -> FP32 conversion does.
OG_HD bool d2f_scaled(uint64_t b, int s, float& out) {
  const int E = (int)(b >> 52);
  if (E == 0 || E >= 2047) return false;
  const int ef = E - 1023 - s + 127;
  if (ef < 1 || ef > 254) return false;
  const uint64_t man = b & 0x000fffffffffffffull;
  const uint32_t m23 = (uint32_t)(man >> 29);
  const uint32_t fb = ((uint32_t)ef << 23) + m23 + round_up(m23, man & 0x1fffffffull, 29);
  out = float_from_bits(fb);
  return true;
}

// CIC node and fraction of u = x 2^-s, from the bits b of x >= 0:
//   i0 = floor(u) and f = (float)(u - floor(u)),
// the FP64 expressions of a mesh coordinate.  u - floor(u) is exact in FP64
// (the low bits of the significand); f rounds it to 24 bits.  Applies for
// x = 0 and for 2^-126 <= u < 2^31; returns false, writing nothing, otherwise
// (negative, subnormal or non-finite x, or u out of that range).
OG_HD bool cic_bits(uint64_t b, int s, int& i0, float& f) {
  if (b == 0) {
    i0 = 0;
    f = 0.0f;
    return true;
  }
  const int E = (int)(b >> 52);
  if (E == 0 || E >= 2047) return false;
  const int eu = E - 1023 - s;  // u = S 2^(eu - 52)
  if (eu > 30) return false;
  if (eu < 0) {  // u < 1
    if (!d2f_scaled(b, s, f)) return false;
    i0 = 0;
    return true;
  }
  const uint64_t S = (b & 0x000fffffffffffffull) | 0x0010000000000000ull;
  const int sh = 52 - eu;  // 22 .. 52
  const uint64_t frac = S & ((1ull << sh) - 1ull);
  i0 = (int)(S >> sh);
  if (frac == 0) {
    f = 0.0f;
    return true;
  }
  const int lz = clz64(frac);  // >= 64 - sh
  const uint64_t v = frac << lz;
  const uint32_t m = (uint32_t)(v >> 40);
  const uint32_t r = round_up(m, v & 0xffffffffffull, 40);
  // frac 2^-sh lies in [2^(63 - lz - sh), 1): biased exponent 190 - lz - sh
  f = float_from_bits(((uint32_t)(190 - lz - sh) << 23) + (m - 0x800000u) + r);
  return true;
}

}  // namespace og

namespace og {

// The double v 2^x for an odd integer 1 <= v < 2^31, built from its bits:
// exact, like the FP64 product (v / 2) 2^(x + 1) it replaces (the centre of
// cell q at level l of a box 2^e is (q + 1/2) 2^(e - l) = (2q + 1) 2^(e - l - 1)).
// Returns false, writing nothing, where the result would not be a normal
// double.
OG_HD bool double_odd_scaled(uint32_t v, int x, double& out) {
  if ((v & 1u) == 0u) return false;
#if defined(__CUDA_ARCH__)
  const int nb = 31 - __clz((int)v);  // floor(log2 v)
#else
  const int nb = 31 - __builtin_clz(v);
#endif
  const int E = nb + x + 1023;
  if (E < 1 || E > 2046) return false;
  const uint64_t man = ((uint64_t)v << (52 - nb)) & 0x000fffffffffffffull;
  const uint64_t b = ((uint64_t)E << 52) | man;
#if defined(__CUDA_ARCH__)
  out = __longlong_as_double((long long)b);
#else
  std::memcpy(&out, &b, sizeof out);
#endif
  return true;
}

}  // namespace og
