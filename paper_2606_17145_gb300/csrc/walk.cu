// walk.cu -- K6 FP32+Kahan walk, K6d FP64 walk, K7 adjoint walk.
//
// One warp walks the tree for one group of 32 Hilbert-consecutive targets
// (lane = target).  The warp keeps a stack of (first node, node count, lane
// mask) ranges in shared memory: a node is visited once per warp, every
// active lane takes its own decision (discard / accept / open), and the
// children of a node are pushed with the mask of the lanes that opened it.
// Each target therefore receives exactly the terms of its own per-particle
// walk (the rules are listed in og.h), while node data is read once per warp
// and broadcast.
//
// FP32 path.  Positions are split floats in box units (hi a multiple of 2^-23,
// lo the rest), so hi_i - hi_j is exact and every displacement
// (hi_i - hi_j) + (lo_i - lo_j) is the FP64 difference rounded to FP32.  A
// decision whose FP32 test falls within a small relative band of its
// threshold is re-taken in FP64 with the same operation order as the CPU
// reference, so decisions agree with an FP64 walk.  Interactions use the
// special-function unit (rsqrt, ex2) and a polynomial for
// erfcx(u) + 2u/sqrt(pi); per-target sums are Kahan-compensated after every
// node visit.
#include "og_internal.cuh"
#include "short_range_poly.inc"

namespace og {

constexpr int kWarpsPerBlock = 4;
constexpr int kStack = 24;

enum : int { DEC_DISCARD = 0, DEC_OPEN = 1, DEC_ACCEPT = 2, DEC_ACCEPT_OUT = 3, DEC_UNSURE = 4 };


// ------------------------------------------------------------------ helpers

__device__ __forceinline__ float rsqrt_approx(float x) {
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float mi1(float t) { return t > 0.5f ? t - 1.0f : (t < -0.5f ? t + 1.0f : t); }

__device__ __forceinline__ float sr_poly(float t) {
  float p = og_sr_poly[OG_SR_POLY_DEG];
#pragma unroll
  for (int k = OG_SR_POLY_DEG - 1; k >= 0; --k) p = fmaf(p, t, og_sr_poly[k]);
  return p;
}

// FP64 forms with the reference's operation order (no contraction).
__device__ __forceinline__ double mi64(double t, double L) {
  const double h = __dmul_rn(0.5, L);
  if (t > h) return __dsub_rn(t, L);
  if (t < -h) return __dadd_rn(t, L);
  return t;
}
__device__ __forceinline__ double norm2_64(double a, double b, double c) {
  return __dadd_rn(__dadd_rn(__dmul_rn(a, a), __dmul_rn(b, b)), __dmul_rn(c, c));
}

// Exact (FP64) node decision for sorted target k.
__device__ int decide_exact(const WalkArgs& A, int64_t k, int node, int level) {
  const TreeDev& T = A.T;
  const double L = A.box;
  const double side = ldexp(L, -level);
  const double half = __dmul_rn(0.5, side);
  double dc[3], cmax = 0.0, e[3], f[3], d[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    dc[c] = fabs(mi64(__dsub_rn(T.x64[3 * k + c], T.cen64[3 * (int64_t)node + c]), L));
    if (dc[c] > cmax) cmax = dc[c];
    e[c] = __dsub_rn(dc[c], half);
    if (e[c] < 0.0) e[c] = 0.0;
  }
  const double e2 = norm2_64(e[0], e[1], e[2]);
  if (e2 > A.rc2_64) return DEC_DISCARD;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    f[c] = __dadd_rn(dc[c], half);
    d[c] = mi64(__dsub_rn(T.x64[3 * k + c], T.com64[3 * (int64_t)node + c]), L);
  }
  const double far2 = norm2_64(f[0], f[1], f[2]);
  const double d2 = norm2_64(d[0], d[1], d[2]);
  const bool inside = cmax <= __dmul_rn(0.6, side);
  if (__dmul_rn(side, side) < __dmul_rn(A.th2_64, d2) && !inside && far2 < A.rc2_64)
    return d2 < A.rc2_64 ? DEC_ACCEPT : DEC_ACCEPT_OUT;
  return DEC_OPEN;
}

__device__ __forceinline__ bool pair_inside_exact(const WalkArgs& A, int64_t k, int64_t j) {
  const double* x = A.T.x64;
  const double L = A.box;
  const double a = mi64(__dsub_rn(x[3 * k], x[3 * j]), L);
  const double b = mi64(__dsub_rn(x[3 * k + 1], x[3 * j + 1]), L);
  const double c = mi64(__dsub_rn(x[3 * k + 2], x[3 * j + 2]), L);
  return norm2_64(a, b, c) < A.rc2_64;
}

// Softened kernel K_h(r) inside r < h (v = r / h), FP32.
__device__ __forceinline__ void spline_f32(float r, float h2, float& K, float& Kp_r) {
  const float h = sqrtf(h2);
  const float hinv = 1.0f / h;
  const float v = r * hinv;
  const float h3 = hinv * hinv * hinv;
  if (v < 0.5f) {
    K = h3 * (10.6666666667f + v * v * (32.0f * v - 38.4f));
    Kp_r = h3 * hinv * hinv * (96.0f * v - 76.8f);
  } else {
    const float v3 = v * v * v;
    K = h3 * (21.3333333333f - 48.0f * v + 38.4f * v * v - 10.6666666667f * v3 - 0.0666666667f / v3);
    Kp_r = h3 * hinv * hinv * (-48.0f / v + 76.8f - 32.0f * v + 0.2f / (v3 * v * v));
  }
}

// Force factor F = K_h(r) f(r) (and its radial derivative over r if wanted).
template <bool DERIV>
__device__ __forceinline__ void force_f32(const WalkArgs& A, float r2, float h2, float& F, float& Fr) {
  float K, Kp_r, r;
  if (r2 >= h2) {
    const float ri = rsqrt_approx(r2);
    r = r2 * ri;
    K = ri * ri * ri;
    Kp_r = -3.0f * K * ri * ri;
  } else {
    r = sqrtf(r2);
    spline_f32(r, h2, K, Kp_r);
  }
  const float e = ex2_approx(r2 * A.ex2c);
  const float g = sr_poly(fmaf(r, A.t_scale, -1.0f));
  const float f = g * e;
  F = K * f;
  if (DERIV) Fr = fmaf(Kp_r, f, K * (A.fp_c * e * r));  // f'(r)/r = fp_c r exp(-u^2)
  else Fr = 0.0f;
}

__device__ __forceinline__ void kahan_add(float& T, float& C, float x) {
  const float y = x - C;
  const float t = T + y;
  C = (t - T) - y;
  T = t;
}

__device__ __forceinline__ float warp_sum(float v, uint32_t m = 0xffffffffu) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(m, v, o);
  return v;
}

struct GroupInfo {
  float cx, cy, cz;  // group box centre
  float ex, ey, ez;  // group box half extents
};

// ------------------------------------------------------------------ lanes

// FP32 lane: forward (ADJ = false) or adjoint (ADJ = true).
template <bool ADJ>
struct LaneF32 {
  int64_t k;          // sorted index of this lane's target
  float xh[3], xl[3]; // split position
  float h2;           // own softening support squared (box units)
  float d[3], d2;     // displacement to the last decided node's COM
  float P[3];         // partial sum since the last fold
  float S[3], C[3];   // Kahan total and compensation
  float w[3];         // adjoint weight
  int nint;

  __device__ void init(const WalkArgs& A, int64_t kk, bool valid) {
    k = kk;
    const float4 a = valid ? A.T.pA[kk] : make_float4(0.f, 0.f, 0.f, 0.f);
    const float4 b = valid ? A.T.pB[kk] : make_float4(0.f, 0.f, 0.f, 0.f);
    xh[0] = a.x; xh[1] = a.y; xh[2] = a.z;
    xl[0] = b.x; xl[1] = b.y; xl[2] = b.z;
    h2 = b.w;
#pragma unroll
    for (int c = 0; c < 3; ++c) { P[c] = 0.f; S[c] = 0.f; C[c] = 0.f; w[c] = 0.f; }
    if (ADJ && valid) {
      const int32_t i = A.T.order[kk];
#pragma unroll
      for (int c = 0; c < 3; ++c) w[c] = A.w[3 * (int64_t)i + c];
    }
    nint = 0;
  }

  __device__ int decide(const WalkArgs& A, int node, const int4& ND, const float4& NC) {
    const float s = NC.w, hs = 0.5f * s;
    // the hi differences are exact, so the minimum image is applied before
    // the lo parts are added (no loss of relative precision across the box edge)
    const float ax = fabsf(mi1(NC.x - xh[0]) - xl[0]);
    const float ay = fabsf(mi1(NC.y - xh[1]) - xl[1]);
    const float az = fabsf(mi1(NC.z - xh[2]) - xl[2]);
    const float ex = fmaxf(ax - hs, 0.f), ey = fmaxf(ay - hs, 0.f), ez = fmaxf(az - hs, 0.f);
    const float e2 = fmaf(ex, ex, fmaf(ey, ey, ez * ez));
    if (e2 > A.rc2_hi) return DEC_DISCARD;
    const float4 NA = A.T.nA[node];
    const float4 NB = A.T.nB[node];
    d[0] = mi1(xh[0] - NA.x) + (xl[0] - NB.x);
    d[1] = mi1(xh[1] - NA.y) + (xl[1] - NB.y);
    d[2] = mi1(xh[2] - NA.z) + (xl[2] - NB.z);
    d2 = fmaf(d[0], d[0], fmaf(d[1], d[1], d[2] * d[2]));
    int dec;
    if (e2 >= A.rc2_lo) {
      dec = DEC_UNSURE;
    } else {
      const float fx = ax + hs, fy = ay + hs, fz = az + hs;
      const float far2 = fmaf(fx, fx, fmaf(fy, fy, fz * fz));
      const float lhs = s * s;
      const float cmax = fmaxf(ax, fmaxf(ay, az));
      const int a1 = lhs < A.th2_lo * d2 ? 1 : (lhs > A.th2_hi * d2 ? 0 : 2);
      const int a2 = cmax > A.lim_hi * s ? 1 : (cmax < A.lim_lo * s ? 0 : 2);
      const int a3 = far2 < A.rc2_lo ? 1 : (far2 > A.rc2_hi ? 0 : 2);
      if (a1 == 0 || a2 == 0 || a3 == 0) dec = DEC_OPEN;
      else if (a1 == 2 || a2 == 2 || a3 == 2) dec = DEC_UNSURE;
      else dec = d2 < A.rc2_lo ? DEC_ACCEPT : (d2 > A.rc2_hi ? DEC_ACCEPT_OUT : DEC_UNSURE);
    }
    if (dec == DEC_UNSURE) dec = decide_exact(A, k, node, meta_level(ND.w));
    return dec;
  }

  // One interaction with source mass m (box units) at displacement dv.
  __device__ __forceinline__ void term(const WalkArgs& A, const float* dv, float r2, float m, float hh2, float* jw,
                                       float& wg) {
    float F, Fr;
    force_f32<ADJ>(A, r2, fmaxf(h2, hh2), F, Fr);
    if (!ADJ) {
      const float sc = -m * F;
#pragma unroll
      for (int c = 0; c < 3; ++c) P[c] = fmaf(sc, dv[c], P[c]);
    } else {
      const float dw = fmaf(dv[0], w[0], fmaf(dv[1], w[1], dv[2] * w[2]));
      const float q = Fr * dw;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        jw[c] = -fmaf(F, w[c], q * dv[c]);
        P[c] = fmaf(m, jw[c], P[c]);
      }
      wg = -F * dw;
    }
    ++nint;
  }

  __device__ __forceinline__ void fold() {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      kahan_add(S[c], C[c], P[c]);
      P[c] = 0.f;
    }
  }

  __device__ void node_term(const WalkArgs& A, int node, bool mine, uint32_t amask) {
    float jw[3] = {0.f, 0.f, 0.f}, wg = 0.f;
    if (mine) {
      const float4 NA = A.T.nA[node];
      const float4 NB = A.T.nB[node];
      term(A, d, d2, NA.w, NB.w, jw, wg);
    }
    if (ADJ) {
      const float g0 = warp_sum(jw[0]), g1 = warp_sum(jw[1]), g2 = warp_sum(jw[2]), sg = warp_sum(wg);
      if ((threadIdx.x & 31) == (__ffs(amask) - 1)) {
        atomicAdd(&A.Gn[3 * (int64_t)node], (double)g0);
        atomicAdd(&A.Gn[3 * (int64_t)node + 1], (double)g1);
        atomicAdd(&A.Gn[3 * (int64_t)node + 2], (double)g2);
        atomicAdd(&A.Sn[node], (double)sg);
      }
    }
    fold();
  }

  template <bool UNIFORM>
  __device__ void leaf_loop(const WalkArgs& A, int j0, int jn, bool open, const float* sh) {
    const float xs0 = xh[0] + sh[0], xs1 = xh[1] + sh[1], xs2 = xh[2] + sh[2];
    for (int j = j0; j < j0 + jn; ++j) {
      const float4 SA = A.T.pA[j];
      const float4 SB = A.T.pB[j];
      float jw[3] = {0.f, 0.f, 0.f}, wg = 0.f;
      bool hit = false;
      if (open && j != k) {
        float dv[3];
        if (UNIFORM) {
          dv[0] = (xs0 - SA.x) + (xl[0] - SB.x);
          dv[1] = (xs1 - SA.y) + (xl[1] - SB.y);
          dv[2] = (xs2 - SA.z) + (xl[2] - SB.z);
        } else {
          dv[0] = mi1(xh[0] - SA.x) + (xl[0] - SB.x);
          dv[1] = mi1(xh[1] - SA.y) + (xl[1] - SB.y);
          dv[2] = mi1(xh[2] - SA.z) + (xl[2] - SB.z);
        }
        const float r2 = fmaf(dv[0], dv[0], fmaf(dv[1], dv[1], dv[2] * dv[2]));
        if (r2 < A.pp_lo) hit = true;
        else if (r2 <= A.pp_hi) hit = pair_inside_exact(A, k, j);
        if (hit) term(A, dv, r2, SA.w, SB.w, jw, wg);
      }
      if (ADJ) {
        const uint32_t hm = __ballot_sync(0xffffffffu, hit);
        if (hm) {
          const float g0 = warp_sum(jw[0]), g1 = warp_sum(jw[1]), g2 = warp_sum(jw[2]), sg = warp_sum(wg);
          if ((threadIdx.x & 31) == (__ffs(hm) - 1)) {
            atomicAdd(&A.Gp[3 * (int64_t)j], (double)g0);
            atomicAdd(&A.Gp[3 * (int64_t)j + 1], (double)g1);
            atomicAdd(&A.Gp[3 * (int64_t)j + 2], (double)g2);
            atomicAdd(&A.Sp[j], (double)sg);
          }
        }
      }
    }
    fold();
  }

  __device__ void leaf(const WalkArgs& A, const int4& ND, const float4& NC, bool open, const GroupInfo& G) {
    // A warp-uniform periodic image for the whole leaf exists when every
    // (target, source) pair that can lie inside rcut is certainly put at its
    // minimum image by one shift of the leaf.
    const float hs = 0.5f * NC.w;
    const float dx = NC.x - G.cx, dy = NC.y - G.cy, dz = NC.z - G.cz;
    const float nx = rintf(dx), ny = rintf(dy), nz = rintf(dz);
    const bool uni = fabsf(dx - nx) + G.ex + hs < A.uni_lim && fabsf(dy - ny) + G.ey + hs < A.uni_lim &&
                     fabsf(dz - nz) + G.ez + hs < A.uni_lim;
    const float sh[3] = {nx, ny, nz};
    if (uni) leaf_loop<true>(A, ND.x, ND.y, open, sh);
    else leaf_loop<false>(A, ND.x, ND.y, open, sh);
  }

  __device__ void finish(const WalkArgs& A, bool valid) {
    if (!valid) return;
    const int32_t i = A.T.order[k];
    if (!ADJ) {
#pragma unroll
      for (int c = 0; c < 3; ++c) A.accf[3 * (int64_t)i + c] = S[c] - C[c];
      if (A.counts) A.counts[i] = nint;
    } else {
#pragma unroll
      for (int c = 0; c < 3; ++c) A.tgt[3 * k + c] = (double)S[c] - (double)C[c];
    }
  }
};

// FP64 lane (forward only): the same walk in double precision.
struct LaneF64 {
  int64_t k;
  double x[3];
  double h;
  double a[3];
  int nint;

  __device__ void init(const WalkArgs& A, int64_t kk, bool valid) {
    k = kk;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      x[c] = valid ? A.T.x64[3 * kk + c] : 0.0;
      a[c] = 0.0;
    }
    h = valid ? A.T.h64[kk] : 0.0;
    nint = 0;
  }

  __device__ int decide(const WalkArgs& A, int node, const int4& ND, const float4&) {
    return decide_exact(A, k, node, meta_level(ND.w));
  }

  __device__ void term(const WalkArgs& A, const double* dv, double m, double hs) {
    const double r2 = norm2_64(dv[0], dv[1], dv[2]);
    const double r = sqrt(r2);
    const double hh = fmax(h, hs);
    double K;
    if (r >= hh) {
      K = 1.0 / (r * r * r);
    } else {
      const double v = r / hh;
      const double h3 = 1.0 / (hh * hh * hh);
      if (v < 0.5) K = h3 * (32.0 / 3.0 + v * v * (32.0 * v - 38.4));
      else K = h3 * (64.0 / 3.0 - 48.0 * v + 38.4 * v * v - (32.0 / 3.0) * v * v * v - (1.0 / 15.0) / (v * v * v));
    }
    const double u = r * A.inv2rs64;
    const double f = erfc(u) + 1.1283791670955126 * u * exp(-u * u);
    const double sc = -m * K * f;
#pragma unroll
    for (int c = 0; c < 3; ++c) a[c] += sc * dv[c];
    ++nint;
  }

  __device__ void node_term(const WalkArgs& A, int node, bool mine, uint32_t) {
    if (!mine) return;
    double dv[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) dv[c] = mi64(__dsub_rn(x[c], A.T.com64[3 * (int64_t)node + c]), A.box);
    term(A, dv, A.T.mass64[node], A.T.hmax64[node]);
  }

  __device__ void leaf(const WalkArgs& A, const int4& ND, const float4&, bool open, const GroupInfo&) {
    if (!open) return;
    for (int j = ND.x; j < ND.x + ND.y; ++j) {
      if (j == k) continue;
      double dv[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) dv[c] = mi64(__dsub_rn(x[c], A.T.x64[3 * (int64_t)j + c]), A.box);
      if (norm2_64(dv[0], dv[1], dv[2]) < A.rc2_64) term(A, dv, A.T.m64[j], A.T.h64[j]);
    }
  }

  __device__ void finish(const WalkArgs& A, bool valid) {
    if (!valid) return;
    const int32_t i = A.T.order[k];
#pragma unroll
    for (int c = 0; c < 3; ++c) A.accd[3 * (int64_t)i + c] = a[c];
    if (A.counts) A.counts[i] = nint;
  }
};

// ------------------------------------------------------------------ traversal

template <class Lane>
__global__ void __launch_bounds__(kWarpsPerBlock * 32) k_walk(WalkArgs A) {
  __shared__ int s_first[kWarpsPerBlock][kStack];
  __shared__ int s_cnt[kWarpsPerBlock][kStack];
  __shared__ uint32_t s_mask[kWarpsPerBlock][kStack];
  const TreeDev& T = A.T;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int64_t g = (int64_t)blockIdx.x * kWarpsPerBlock + wib;
  if (g >= T.ngroups) return;
  if (T.sb->status != 0 || T.sb->magic != kMagicTree) {
    if (lane == 0) set_status(A.wsb, ST_NOTREE);
    return;
  }
  int nodes_total = 0;
  for (int l = 0; l < kLevels; ++l) nodes_total += T.sb->level_cnt[l];
  if (nodes_total > T.cap) nodes_total = (int)T.cap;

  const int64_t k = g * kGroup + lane;
  const bool valid = k < T.n;
  const uint32_t vmask = __ballot_sync(0xffffffffu, valid);

  GroupInfo G;
  {
    const float4 lo = T.gbox[2 * g], hi = T.gbox[2 * g + 1];
    G.cx = 0.5f * (lo.x + hi.x); G.cy = 0.5f * (lo.y + hi.y); G.cz = 0.5f * (lo.z + hi.z);
    G.ex = 0.5f * (hi.x - lo.x) * 1.0001f + 1e-7f;
    G.ey = 0.5f * (hi.y - lo.y) * 1.0001f + 1e-7f;
    G.ez = 0.5f * (hi.z - lo.z) * 1.0001f + 1e-7f;
  }

  Lane L;
  L.init(A, k, valid);

  int* sf = s_first[wib];
  int* sc = s_cnt[wib];
  uint32_t* sm = s_mask[wib];
  if (lane == 0) { sf[0] = 0; sc[0] = 1; sm[0] = vmask; }
  int sp = 1;
  long long iters = 0;
  __syncwarp();
  while (sp > 0) {
    if (++iters > A.max_iters) {
      if (lane == 0) set_status(A.wsb, ST_WALKCAP);
      break;
    }
    const int top = sp - 1;
    const int node = sf[top];
    const int cnt = sc[top];
    const uint32_t mask = sm[top];
    __syncwarp();
    if (cnt > 1) {
      if (lane == 0) { sf[top] = node + 1; sc[top] = cnt - 1; }
    } else {
      sp = top;
    }
    __syncwarp();
    if (node < 0 || node >= nodes_total) {
      if (lane == 0) set_status(A.wsb, ST_TREELINK);
      break;
    }
    const float4 NC = T.nC[node];
    {
      // all lanes certainly discard: the node cube is beyond rcut of the group box
      const float hs = 0.5f * NC.w;
      const float gx = fmaxf(fabsf(mi1(NC.x - G.cx)) - hs - G.ex, 0.f);
      const float gy = fmaxf(fabsf(mi1(NC.y - G.cy)) - hs - G.ey, 0.f);
      const float gz = fmaxf(fabsf(mi1(NC.z - G.cz)) - hs - G.ez, 0.f);
      if (fmaf(gx, gx, fmaf(gy, gy, gz * gz)) > A.grp_rc2) continue;
    }
    const int4 ND = T.nD[node];
    const bool active = (mask >> lane) & 1u;
    const int dec = active ? L.decide(A, node, ND, NC) : DEC_DISCARD;
    const uint32_t amask = __ballot_sync(0xffffffffu, dec == DEC_ACCEPT);
    const uint32_t omask = __ballot_sync(0xffffffffu, dec == DEC_OPEN);
    if (amask) L.node_term(A, node, dec == DEC_ACCEPT, amask);
    if (omask) {
      if (meta_leaf(ND.w)) {
        if (ND.x < 0 || ND.y < 0 || (int64_t)ND.x + ND.y > T.n) {
          if (lane == 0) set_status(A.wsb, ST_TREELINK);
          break;
        }
        L.leaf(A, ND, NC, dec == DEC_OPEN, G);
      } else {
        const int nch = meta_nchild(ND.w);
        if (nch <= 0 || ND.z <= node || ND.z + nch > nodes_total) {
          if (lane == 0) set_status(A.wsb, ST_TREELINK);
          break;
        }
        if (sp >= kStack) {
          if (lane == 0) set_status(A.wsb, ST_STACK);
          break;
        }
        if (lane == 0) { sf[sp] = ND.z; sc[sp] = nch; sm[sp] = omask; }
        ++sp;
        __syncwarp();
      }
    }
  }
  L.finish(A, valid);
  if (A.total) {
    const unsigned cnt = __reduce_add_sync(0xffffffffu, (unsigned)(valid ? L.nint : 0));
    if (lane == 0 && cnt) atomicAdd(A.total, (unsigned long long)cnt);
  }
}

cudaError_t launch_walk(const WalkArgs& A, int prec, bool adjoint, cudaStream_t s) {
  const int64_t blocks = (A.T.ngroups + kWarpsPerBlock - 1) / kWarpsPerBlock;
  if (blocks <= 0) return cudaSuccess;
  if (adjoint) k_walk<LaneF32<true>><<<(unsigned)blocks, kWarpsPerBlock * 32, 0, s>>>(A);
  else if (prec == OG_FP64) k_walk<LaneF64><<<(unsigned)blocks, kWarpsPerBlock * 32, 0, s>>>(A);
  else k_walk<LaneF32<false>><<<(unsigned)blocks, kWarpsPerBlock * 32, 0, s>>>(A);
  return cudaGetLastError();
}

}  // namespace og
