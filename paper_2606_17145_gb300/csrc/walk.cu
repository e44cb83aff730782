// walk.cu -- K6 FP32+Kahan walk, K6d FP64 walk, K7 adjoint walk.
//
// One warp walks the tree for one group of 32 Hilbert-consecutive targets
// (lane = target).  The warp keeps a stack of (first node, node count, lane
// mask) ranges in shared memory and pops up to 32 nodes per step, one per
// lane.  Each node is first classified against the bounding box of the whole
// group (drop / open / accept / mixed); a mixed node is classified again
// against the boxes of the four 8-target sub-groups, and only the sub-groups
// left undecided take per-lane decisions.  Opened internal nodes push their
// children as one range with the mask of the lanes that opened them; opened
// leaves and accepted nodes are queued.  Each target therefore receives
// exactly the terms of its own per-particle walk (the rules are listed in
// og.h), while node data is read once per warp.
//
// Evaluation.  Queued entries are expanded into source slots; a source
// beyond r_cut of the group box is dropped and the others are staged in a
// ring of two 32-slot batches.  For a batch, a cheap conservative test
// (|x_i|^2 + |x_j|^2 - 2 x_i.x_j against r_cut^2, with a per-slot rounding
// margin) marks the (target, source) pairs that can lie inside the cut; the
// marked pairs are compacted into a target-major list by a warp prefix sum,
// and each warp iteration evaluates 32 listed pairs.  A segmented scan over
// the lanes sums each target's run in a fixed order, so the result does not
// depend on scheduling.  In the adjoint, the lane that owns a slot sums that
// source's terms over the iteration's lanes in lane order (their lanes are
// found through a shared-memory bit mask per slot).  The FP64 variant shares
// all of this with FP64 decisions and pair arithmetic.
//
// FP32 path.  Positions are split floats in box units (hi a multiple of 2^-23,
// lo the rest), so hi_i - hi_j is exact and every displacement
// (hi_i - hi_j) + (lo_i - lo_j) is the FP64 difference rounded to FP32.  A
// decision whose FP32 test falls within a small relative band of its
// threshold is re-taken in FP64 with the same operation order as the CPU
// reference, so decisions agree with an FP64 walk.  Interactions use the
// special-function unit (rsqrt, ex2) and a polynomial for
// erfcx(u) + 2u/sqrt(pi); per-target sums are Kahan-compensated after every
// batch of 32 staged sources (at most 32 terms per target).
#include <type_traits>

#include "og_internal.cuh"
#include "short_range_poly.inc"

namespace og {

constexpr int kWarpsPerBlock = 2;

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
// Minimum image of a box-unit difference t (|t| < 1.5): t - rint(t), with
// rint by the 1.5 * 2^23 rounding constant (round to nearest even, so
// +-0.5 stay), equal bit for bit to t - 1 / t + 1 / t on t > 0.5 / t < -0.5 /
// otherwise.
__device__ __forceinline__ float mi1(float t) {
  const float r = __fadd_rn(__fadd_rn(t, 12582912.0f), -12582912.0f);
  return __fadd_rn(t, -r);
}

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
__device__ __noinline__ int decide_exact(const WalkArgs& A, int64_t k, int node, int level) {
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

__device__ __noinline__ bool pair_inside_exact(const WalkArgs& A, int64_t k, int64_t j) {
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

// Exact float -> double by bit manipulation on the integer pipe (the FP64
// pipe is a small fraction of the FP32 rate on this GPU).  Subnormal inputs
// flush to zero, like the FP32 arithmetic that produced them.
__device__ __forceinline__ double f2d_exact(float x) {
  const uint32_t u = __float_as_uint(x);
  const uint32_t e = (u >> 23) & 0xffu;
  const uint64_t sign = (uint64_t)(u >> 31) << 63;
  const uint64_t exp = e == 0xffu ? 0x7ffull : (uint64_t)(e + (1023u - 127u));
  const uint64_t man = (uint64_t)(u & 0x7fffffu) << 29;
  const uint64_t bits = e == 0u ? sign : (sign | (exp << 52) | man);
  return __longlong_as_double((long long)bits);
}

struct GroupInfo {
  float cx, cy, cz;  // group box centre
  float ex, ey, ez;  // group box half extents (padded outward)
};

// ------------------------------------------------------------------ per-warp shared buffers

// Traversal stack of child ranges.  A step pops ranges holding up to 32
// nodes and pushes at most one range per popped node (net growth <= 31).
// Above kDeep entries a step pops a single range (<= 8 nodes, growth <= 7
// per level), so the depth stays below kDeep + 31 + 7 x 20 + 8 for any tree.
constexpr int kStack = 276;
constexpr int kStackNeed = 32;   // pushes of one step
constexpr int kDeep = 64;
static_assert(kDeep + 31 + 7 * 20 + 8 <= kStack - kStackNeed, "stack bound");
constexpr int kQueue = 128;      // queued leaves / accepted nodes per warp
constexpr int kQueueNeed = 64;   // a step queues at most 2 entries per node
constexpr int kSlots = 32;       // sources per evaluation batch
constexpr int kRing = 2 * kSlots; // staged sources: two batches
constexpr int kList = 512;       // (node or slot, target) list entries

// Stack entry: (first node | node count << 28, lane mask); node indices stay
// below 2^28 (checked on the host).  Queue entry: (first particle or node,
// particle count or -1 for an accepted node, lane mask, image flags).
// Image flags bit 0: one shift puts the whole entry at the minimum image of
// every target of the group (bits 1-6: the shift per axis, 0 / +1 / -1).
struct WarpBufs {
  int2* stack;
  int4* queue;
  int* qoff;
  unsigned short* list;  // per-lane decision list (traversal) or pair list (evaluation)
};

// Nodes of one traversal step that need per-lane decisions.
struct MixedScratch {
  int4 D[kGroup];
  float4 C[kGroup], A[kGroup], B[kGroup];  // C, A image-shifted when the node has a common image
  int node[kGroup], fl[kGroup];
  uint32_t mask[kGroup], acc[kGroup], open[kGroup];
  uint32_t dmask[kGroup];  // lanes whose sub-group box leaves the node undecided
};

constexpr int kSub = 4;  // sub-groups of 8 Hilbert-consecutive targets

enum : int { CL_NONE = -1, CL_DROP = 0, CL_OPEN = 1, CL_ACCEPT = 2, CL_MIXED = 3 };

// Group-level classification of a node against the whole group box (box
// units, FP32, conservative margins): DROP if the cube is beyond rcut of
// every point of the box; OPEN if no point of the box can accept it; ACCEPT
// if every point of the box accepts it (cube inside rcut, outside the 1.2x
// cube, side < theta d); MIXED otherwise (exact per-lane decisions follow).
__device__ __forceinline__ int classify(const WalkArgs& A, const GroupInfo& G, const float4& NC, const float4& NA,
                                        const float4& NB) {
  const float s = NC.w, hs = 0.5f * s;
  const float tcx = fabsf(mi1(NC.x - G.cx)), tcy = fabsf(mi1(NC.y - G.cy)), tcz = fabsf(mi1(NC.z - G.cz));
  const float gx = fmaxf(tcx - G.ex - hs, 0.f), gy = fmaxf(tcy - G.ey - hs, 0.f), gz = fmaxf(tcz - G.ez - hs, 0.f);
  if (fmaf(gx, gx, fmaf(gy, gy, gz * gz)) > A.grp_rc2) return CL_DROP;
  if (s > 0.25f || G.ex > 0.125f || G.ey > 0.125f || G.ez > 0.125f) return CL_MIXED;
  if (A.th2_hi == 0.0f) return CL_OPEN;  // theta = 0: nothing is ever accepted
  const float txx = fabsf(mi1((NA.x - G.cx) + NB.x));
  const float txy = fabsf(mi1((NA.y - G.cy) + NB.y));
  const float txz = fabsf(mi1((NA.z - G.cz) + NB.z));
  const float m_lo = 0.999f, m_hi = 1.001f;
  const float ax = txx + G.ex, ay = txy + G.ey, az = txz + G.ez;
  const float dmax2 = fmaf(ax, ax, fmaf(ay, ay, az * az));
  const float bx = fmaxf(txx - G.ex, 0.f), by = fmaxf(txy - G.ey, 0.f), bz = fmaxf(txz - G.ez, 0.f);
  const float dmin2 = fmaf(bx, bx, fmaf(by, by, bz * bz));
  const float fx0 = fmaxf(tcx - G.ex, 0.f) + hs, fy0 = fmaxf(tcy - G.ey, 0.f) + hs, fz0 = fmaxf(tcz - G.ez, 0.f) + hs;
  const float minfar2 = fmaf(fx0, fx0, fmaf(fy0, fy0, fz0 * fz0));
  const float fx1 = tcx + G.ex + hs, fy1 = tcy + G.ey + hs, fz1 = tcz + G.ez + hs;
  const float maxfar2 = fmaf(fx1, fx1, fmaf(fy1, fy1, fz1 * fz1));
  const float lim = 0.6f * s;
  const bool all_inside = tcx + G.ex < lim * m_lo && tcy + G.ey < lim * m_lo && tcz + G.ez < lim * m_lo;
  const bool all_outside = tcx - G.ex > lim * m_hi || tcy - G.ey > lim * m_hi || tcz - G.ez > lim * m_hi;
  const float s2 = s * s;
  if (s2 > A.th2_hi * dmax2 * m_hi || all_inside || minfar2 > A.rc2 * m_hi) return CL_OPEN;
  if (s2 < A.th2_lo * dmin2 * m_lo && all_outside && maxfar2 < A.rc2 * m_lo) return CL_ACCEPT;
  return CL_MIXED;
}

// Image shift that puts every (target, source) pair of an entry that can lie
// inside rcut at its minimum image, if one exists for the whole cube.
__device__ __forceinline__ int image_flags(const WalkArgs& A, const GroupInfo& G, const float4& NC) {
  const float hs = 0.5f * NC.w;
  const float dx = NC.x - G.cx, dy = NC.y - G.cy, dz = NC.z - G.cz;
  const float nx = rintf(dx), ny = rintf(dy), nz = rintf(dz);
  const bool uni = fabsf(dx - nx) + G.ex + hs < A.uni_lim && fabsf(dy - ny) + G.ey + hs < A.uni_lim &&
                   fabsf(dz - nz) + G.ez + hs < A.uni_lim;
  if (!uni) return 0;
  const int cx = nx > 0.5f ? 1 : (nx < -0.5f ? 2 : 0);
  const int cy = ny > 0.5f ? 1 : (ny < -0.5f ? 2 : 0);
  const int cz = nz > 0.5f ? 1 : (nz < -0.5f ? 2 : 0);
  return 1 | (cx << 1) | (cy << 3) | (cz << 5);
}

__device__ __forceinline__ float shift_of(int flags, int axis) {
  const int c = (flags >> (1 + 2 * axis)) & 3;
  return c == 1 ? 1.0f : (c == 2 ? -1.0f : 0.0f);
}

// Validates the queue and writes the slot offsets; returns the slot count or
// -1 if an entry is malformed (then nothing may be evaluated).
__device__ __forceinline__ int queue_offsets(const WalkArgs& A, const WarpBufs& W, int nq, int lane) {
  int run = 0;
  bool badq = false;
  for (int b0 = 0; b0 < nq; b0 += 32) {
    const int e = b0 + lane;
    int c = 0;
    if (e < nq) {
      const int4 Q = W.queue[e];
      if (Q.y == -1) {
        c = 1;
        badq = badq || Q.x < 0 || Q.x >= A.T.cap;
      } else {
        c = Q.y;
        badq = badq || Q.y < 1 || Q.x < 0 || (int64_t)Q.x + Q.y > A.T.n;
      }
    }
    int incl = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    if (e < nq) W.qoff[e] = run + incl - c;
    run += __shfl_sync(0xffffffffu, incl, 31);
  }
  __syncwarp();
  if (__any_sync(0xffffffffu, badq)) return -1;
  return run;
}


// 32 x 32 bit-matrix transpose across the warp: lane r holds row r (bit c =
// column c) and receives column r.  Five stages swap the off-diagonal blocks
// of side 16, 8, 4, 2, 1 between partner lanes.
__device__ __forceinline__ uint32_t transpose32(uint32_t x, int lane) {
  const uint32_t keep[5] = {0x0000ffffu, 0x00ff00ffu, 0x0f0f0f0fu, 0x33333333u, 0x55555555u};
  int j = 16;
#pragma unroll
  for (int st = 0; st < 5; ++st, j >>= 1) {
    const uint32_t y = __shfl_xor_sync(0xffffffffu, x, j);
    x = (lane & j) == 0 ? ((x & keep[st]) | ((y & keep[st]) << j)) : ((x & ~keep[st]) | ((y & ~keep[st]) >> j));
  }
  return x;
}

// ------------------------------------------------------------------ lanes

__device__ __forceinline__ unsigned long long pack2(float lo, float hi) {
  return ((unsigned long long)__float_as_uint(hi) << 32) | __float_as_uint(lo);
}
__device__ __forceinline__ unsigned long long add2(unsigned long long a, unsigned long long b) {
  unsigned long long d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ unsigned long long fma2(unsigned long long a, unsigned long long b, unsigned long long c) {
  unsigned long long d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}

// Exact per-target decision for a node (FP32 with an FP64 re-check in the
// band), target given by its split position.  With uni, NC and NA are
// already shifted to the image that is the minimum image for every target
// of the group, so no per-target minimum image is taken.
__device__ __forceinline__ float mi1_if(bool per_target, float t) { return per_target ? mi1(t) : t; }

__device__ __forceinline__ int decide_f32(const WalkArgs& A, int64_t k, const float4& th, const float4& tl, int node,
                                          const int4& ND, const float4& NC, const float4& NA, const float4& NB,
                                          bool uni) {
  const float s = NC.w, hs = 0.5f * s;
  // hi differences are exact: the minimum image is taken before the lo parts are added
  const float ax = fabsf(mi1_if(!uni, NC.x - th.x) - tl.x);
  const float ay = fabsf(mi1_if(!uni, NC.y - th.y) - tl.y);
  const float az = fabsf(mi1_if(!uni, NC.z - th.z) - tl.z);
  const float ex = fmaxf(ax - hs, 0.f), ey = fmaxf(ay - hs, 0.f), ez = fmaxf(az - hs, 0.f);
  const float e2 = fmaf(ex, ex, fmaf(ey, ey, ez * ez));
  if (e2 > A.rc2_hi) return DEC_DISCARD;
  const float d0 = mi1_if(!uni, th.x - NA.x) + (tl.x - NB.x);
  const float d1 = mi1_if(!uni, th.y - NA.y) + (tl.y - NB.y);
  const float dz = mi1_if(!uni, th.z - NA.z) + (tl.z - NB.z);
  const float d2 = fmaf(d0, d0, fmaf(d1, d1, dz * dz));
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

// One pair's result on the target side: FP32 (with the hit flag in w) or
// FP64 (hit flag separate).
template <bool F64> struct Term { float x, y, z, w; };
template <> struct Term<true> { double x, y, z; float w; };

// Lane of the walk: FP32 + Kahan forward (ADJ = false) or adjoint
// (ADJ = true), or the all-FP64 forward comparison variant (F64 = true:
// FP64 decisions, FP64 pair arithmetic with CUDA's erfc / exp, plain double
// sums).  All share the traversal, the box test, the FP32 cut filter (a
// conservative superset of the pairs inside the cut) and the compaction.
// FUSED (with ADJ): the adjoint walk that also writes the forward
// accelerations, each pair's force factor serving both (one traversal for a
// loss whose weights are known before the walk).
template <bool ADJ, bool F64, bool FUSED = false>
struct LaneFP {
  static_assert(!FUSED || (ADJ && !F64), "the fused walk is the FP32 adjoint plus the forward sums");
  // per-warp data that lives through the whole walk
  struct Smem {
    float4 tA[kGroup];    // targets: hi part, h^2
    float4 tB[kGroup];    // targets: lo part
    float4 tW[ADJ ? kGroup : 1];   // adjoint: dL/da of each target
    float4 SG[ADJ ? kGroup : 1];     // adjoint: source-side term (G, S) of each lane's listed pair
    uint32_t smask[ADJ ? kSlots : 1];  // adjoint: the lanes whose listed pair has this slot
    int self[kGroup];     // staged slot holding the target itself, or -1
    typename std::conditional<F64, double3, float4>::type Ps[kGroup];  // each target's sum over the batch
    float4 Pf[FUSED ? kGroup : 1];  // fused: each target's forward sum over the batch
    int fneg[kGroup];     // listed pairs of the batch found outside the exact cut
  };
  // per-batch staging (dead between evaluations; shares memory with the
  // traversal's scratch)
  // Staged sources live in a ring of two batches: survivors of the box test
  // are appended at the tail, and a batch is evaluated once 32 are pending.
  struct Stage {
    float4 sa[kRing];     // staged source: hi part (image-shifted), mass
    float4 sb[kRing];     // lo part, h^2
    int2 sc[kRing];       // id (particle, or -2 - node), per-pair image flag
    uint32_t sq[kRing];   // lane mask of the source's queue entry
    float fX[kRing], fY[kRing], fZ[kRing], fW[kRing];  // filter form (see put)
  };
  // a slot's source as read from the tree, hi part image-shifted when its
  // entry has a common image (uni)
  struct Fetch {
    float4 a, b;
    int id;
    uint32_t q;
    bool node, uni;
  };

  int64_t k;          // sorted index of this lane's target
  bool valid;
  float xr[3], sr;    // position relative to the group centre and its square (filter)
  float P[3];         // partial sum since the last fold
  float S[3], C[3];   // Kahan total and compensation
  float Pf[3], Sf[3], Cf[3];  // fused: the forward sums likewise
  double a64[3];      // FP64 variant: plain double sums
  int nint;
  float4 gs;          // adjoint: this lane's slot, source-side sums (G, S) over the batch

  __device__ void init(const WalkArgs& A, Smem& M, int64_t kk, bool v, int lane, const GroupInfo& G) {
    k = kk;
    valid = v;
    const int64_t kc = v ? kk : 0;  // never form an out-of-range address
    const float4 a = A.T.pA[kc];
    const float4 b = A.T.pB[kc];
    M.tA[lane] = make_float4(a.x, a.y, a.z, b.w);
    M.tB[lane] = make_float4(b.x, b.y, b.z, 0.f);
    if constexpr (F64) M.Ps[lane] = make_double3(0.0, 0.0, 0.0);
    else M.Ps[lane] = make_float4(0.f, 0.f, 0.f, 0.f);
    a64[0] = a64[1] = a64[2] = 0.0;
    M.fneg[lane] = 0;
    if (ADJ) { gs = make_float4(0.f, 0.f, 0.f, 0.f); M.smask[lane] = 0u; }
    xr[0] = (a.x - G.cx) + b.x;
    xr[1] = (a.y - G.cy) + b.y;
    xr[2] = (a.z - G.cz) + b.z;
    sr = fmaf(xr[0], xr[0], fmaf(xr[1], xr[1], xr[2] * xr[2]));
#pragma unroll
    for (int c = 0; c < 3; ++c) { P[c] = 0.f; S[c] = 0.f; C[c] = 0.f; Pf[c] = 0.f; Sf[c] = 0.f; Cf[c] = 0.f; }
    if constexpr (FUSED) M.Pf[lane] = make_float4(0.f, 0.f, 0.f, 0.f);
    if (ADJ) {
      float4 w = make_float4(0.f, 0.f, 0.f, 0.f);
      if (v) {
        const int32_t i = A.T.order[kk];
        w = make_float4(A.w[3 * (int64_t)i], A.w[3 * (int64_t)i + 1], A.w[3 * (int64_t)i + 2], 0.f);
      }
      M.tW[lane] = w;
    }
    nint = 0;
  }

  __device__ __forceinline__ int decide_for(const WalkArgs& A, const Smem& M, int t, int64_t kt, int node,
                                            const int4& ND, const float4& NC, const float4& NA, const float4& NB,
                                            bool uni) const {
    if constexpr (F64) return decide_exact(A, kt, node, meta_level(ND.w));
    else return decide_f32(A, kt, M.tA[t], M.tB[t], node, ND, NC, NA, NB, uni);
  }

  // FP64 variant: target gbase + i against staged slot s, read from the
  // FP64 tree arrays; the cut is taken on the FP64 distance (accepted nodes
  // are inside by decision).
  __device__ __forceinline__ Term<true> pair_eval64(const WalkArgs& A, const Stage& St, int i, int s,
                                                    int64_t gbase) const {
    const int id = St.sc[s].x;
    const int64_t kt = gbase + i;
    const double* x = A.T.x64;
    double sp[3], m, h;
    if (id >= 0) {
#pragma unroll
      for (int c = 0; c < 3; ++c) sp[c] = x[3 * (int64_t)id + c];
      m = A.T.m64[id];
      h = A.T.h64[id];
    } else {
      const int64_t n = -2 - id;
#pragma unroll
      for (int c = 0; c < 3; ++c) sp[c] = A.T.com64[3 * n + c];
      m = A.T.mass64[n];
      h = A.T.hmax64[n];
    }
    double dv[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) dv[c] = mi64(__dsub_rn(x[3 * kt + c], sp[c]), A.box);
    const double r2 = norm2_64(dv[0], dv[1], dv[2]);
    Term<true> t;
    t.x = t.y = t.z = 0.0;
    t.w = 0.f;
    if (id >= 0 && !(r2 < A.rc2_64)) return t;
    const double r = sqrt(r2);
    const double hh = fmax(A.T.h64[kt], h);
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
    t.x = sc * dv[0];
    t.y = sc * dv[1];
    t.z = sc * dv[2];
    t.w = 1.f;
    return t;
  }

  // Fetch slot s of queue entry e.
  __device__ __forceinline__ Fetch fetch(const WalkArgs& A, const WarpBufs& W, int e, int s) const {
    Fetch f;
    const int4 Q = W.queue[e];
    f.node = Q.y < 0;
    if (f.node) {
      f.a = A.T.nA[Q.x];
      f.b = A.T.nB[Q.x];
      f.id = -2 - Q.x;
    } else {
      const int j = Q.x + (s - W.qoff[e]);
      f.a = A.T.pA[j];
      f.b = A.T.pB[j];
      f.id = j;
    }
    f.uni = (Q.w & 1) != 0;
    if (f.uni) {
      f.a.x -= shift_of(Q.w, 0);
      f.a.y -= shift_of(Q.w, 1);
      f.a.z -= shift_of(Q.w, 2);
    }
    f.q = (uint32_t)Q.z;
    return f;
  }

  // Position of a fetched source relative to the group centre, and whether
  // it can have a pair inside the cut with some target of the group (its
  // distance to the padded group box within the conservative group
  // threshold).  Accepted nodes and entries without a common image are
  // always kept.
  __device__ __forceinline__ bool keep(const WalkArgs& A, const Fetch& f, const GroupInfo& G, float& x0, float& x1,
                                       float& x2) const {
    x0 = (f.a.x - G.cx) + f.b.x;
    x1 = (f.a.y - G.cy) + f.b.y;
    x2 = (f.a.z - G.cz) + f.b.z;
    if (f.node || !f.uni) return true;
    const float g0 = fmaxf(fabsf(x0) - G.ex, 0.f), g1 = fmaxf(fabsf(x1) - G.ey, 0.f), g2 = fmaxf(fabsf(x2) - G.ez, 0.f);
    return fmaf(g0, g0, fmaf(g1, g1, g2 * g2)) <= A.grp_rc2;
  }

  // Stage a fetched source at ring position pos.
  // Filter form: (-2 x, -2 y, -2 z, |x|^2 - r_cut^2 - margin) relative to the
  // group centre, so |x_i - x_j|^2 - r_cut^2 - margin evaluates as
  // fW + |x_i|^2 + fX x_i + fY y_i + fZ z_i.  The FP32 evaluation of that
  // chain is within 18 u (|x_i| + |x_j|)^2 + 18 u r_cut^2 of the exact value
  // (u = 2^-24); the margin is 64 u times that bound's bracket, so every pair
  // inside the cut gives a negative value.
  __device__ __forceinline__ void put(const WalkArgs& A, Stage& S, Smem& M, const Fetch& f, int pos, float x0,
                                      float x1, float x2, int64_t gbase, float Rg) const {
    float fx = 0.f, fy = 0.f, fz = 0.f, fw = -1e30f;  // accepted node or per-pair image: always a candidate
    if (f.uni && !f.node) {
      const float sj = fmaf(x0, x0, fmaf(x1, x1, x2 * x2));
      const float rr = sqrtf(sj) + Rg;
      fx = -2.f * x0;
      fy = -2.f * x1;
      fz = -2.f * x2;
      fw = (sj - A.rc2_hi) - 3.814697265625e-06f * fmaf(rr, rr, A.rc2_hi);
    }
    S.sa[pos] = f.a;
    S.sb[pos] = f.b;
    S.sc[pos] = make_int2(f.id, f.uni ? 0 : 1);
    S.sq[pos] = f.q;
    S.fX[pos] = fx;
    S.fY[pos] = fy;
    S.fZ[pos] = fz;
    S.fW[pos] = fw;
    if (f.id >= gbase && f.id < gbase + kGroup) M.self[f.id - gbase] = pos;
  }

  __device__ __forceinline__ void fold() {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      kahan_add(S[c], C[c], P[c]);
      P[c] = 0.f;
      if constexpr (FUSED) {
        kahan_add(Sf[c], Cf[c], Pf[c]);
        Pf[c] = 0.f;
      }
    }
  }

  // Target i of the group against staged slot s: the exact cut decision, and
  // the interaction (target-side term, hit flag).  In the adjoint the
  // source-side terms go to sg.
  __device__ __forceinline__ float4 pair_eval(const WalkArgs& A, const Stage& St, const Smem& M, int i, int s,
                                              int64_t gbase, float4& sg, float3& fw) const {
    fw = make_float3(0.f, 0.f, 0.f);
    const float4 ta = M.tA[i], tb = M.tB[i];
    const float4 a = St.sa[s], b = St.sb[s];
    const int2 c = St.sc[s];
    float dh0 = ta.x - a.x, dh1 = ta.y - a.y, dh2 = ta.z - a.z;
    if (c.y) {
      dh0 = mi1(dh0);
      dh1 = mi1(dh1);
      dh2 = mi1(dh2);
    }
    float dv[3];
    dv[0] = dh0 + (tb.x - b.x);
    dv[1] = dh1 + (tb.y - b.y);
    dv[2] = dh2 + (tb.z - b.z);
    const float r2 = fmaf(dv[0], dv[0], fmaf(dv[1], dv[1], dv[2] * dv[2]));
    // accepted node (id < 0): inside by decision; particle: cut band, then FP64
    bool in = c.x < 0 || r2 < A.pp_lo;
    if (!in) in = r2 <= A.pp_hi && pair_inside_exact(A, gbase + i, c.x);
    sg = make_float4(0.f, 0.f, 0.f, 0.f);
    if (!in) return make_float4(0.f, 0.f, 0.f, 0.f);
    float F, Fr;
    force_f32<ADJ>(A, r2, fmaxf(ta.w, b.w), F, Fr);
    if (!ADJ) {
      const float sc = -a.w * F;
      return make_float4(sc * dv[0], sc * dv[1], sc * dv[2], 1.f);
    } else {
      const float4 w = M.tW[i];
      const float dw = fmaf(dv[0], w.x, fmaf(dv[1], w.y, dv[2] * w.z));
      const float qq = Fr * dw;
      const float j0 = -fmaf(F, w.x, qq * dv[0]);
      const float j1 = -fmaf(F, w.y, qq * dv[1]);
      const float j2 = -fmaf(F, w.z, qq * dv[2]);
      sg = make_float4(j0, j1, j2, -F * dw);
      if constexpr (FUSED) {
        const float sc = -a.w * F;
        fw = make_float3(sc * dv[0], sc * dv[1], sc * dv[2]);
      }
      return make_float4(a.w * j0, a.w * j1, a.w * j2, 1.f);
    }
  }

  // Evaluate the queued entries (see the header comment).
  __device__ void evaluate(const WalkArgs& A, const WarpBufs& W, Stage& St, Smem& M, int nq, int lane,
                           const GroupInfo& G, int64_t gbase, uint32_t vmask, float Rg) {
    const int total = queue_offsets(A, W, nq, lane);
    if (total < 0) {
      if (lane == 0) set_status(A.wsb, ST_TREELINK);
      return;
    }
    const uint32_t lt = (1u << lane) - 1u;
    M.self[lane] = -1;
    __syncwarp();
    // raw slots are fetched 32 at a time and the survivors of the box test
    // are appended to the ring; pending slots occupy positions
    // [32 half, 32 half + pend) mod 64
    // Each window of 32 slots finds its slots' entries without a search:
    // ecur holds the window's first slot, the entries starting inside the
    // window set bit (start - rb) of one OR-reduced mask (an entry holds at
    // least one slot, so at most 31 start inside it), and slot rb + l lies
    // in entry ecur + (number of starts at or before bit l).
    int pend = 0, tail = 0, half = 0;
    int ecur = 0;
    for (int rb = 0; rb < total; rb += 32) {
      const int ek = ecur + 1 + lane;
      const int sk = ek < nq ? W.qoff[ek] - rb : 32;
      const uint32_t starts = __reduce_or_sync(0xffffffffu, (sk > 0 && sk < 32) ? (1u << sk) : 0u);
      Fetch cur = {};
      bool kp = false;
      float x0 = 0.f, x1 = 0.f, x2 = 0.f;
      if (rb + lane < total) {
        cur = fetch(A, W, ecur + __popc(starts & ((2u << lane) - 1u)), rb + lane);
        kp = keep(A, cur, G, x0, x1, x2);
      }
      const uint32_t km = __ballot_sync(0xffffffffu, kp);
      if (kp) put(A, St, M, cur, (tail + __popc(km & lt)) & (kRing - 1), x0, x1, x2, gbase, Rg);
      tail = (tail + __popc(km)) & (kRing - 1);
      pend += __popc(km);
      __syncwarp();
      const bool last = rb + 32 >= total;
      while (pend >= kSlots || (last && pend > 0)) {
        const int cnt = min(pend, kSlots);
        batch(A, W, St, M, half * kSlots, cnt, lane, gbase, vmask);
        pend -= cnt;
        half ^= 1;
      }
      // the entry holding the next window's first slot
      int en = ecur + __popc(starts);
      if (en + 1 < nq && W.qoff[en + 1] == rb + 32) ++en;
      ecur = en;
    }
  }

  // One batch: the cnt staged sources at ring positions [hb, hb + cnt).
  __device__ void batch(const WalkArgs& A, const WarpBufs& W, Stage& St, Smem& M, int hb, int cnt, int lane,
                        int64_t gbase, uint32_t vmask) {
    const unsigned long long X2 = pack2(xr[0], xr[0]), Y2 = pack2(xr[1], xr[1]), Z2 = pack2(xr[2], xr[2]);
    const unsigned long long S2 = pack2(sr, sr);
    // bit s of msk: slot s is in this lane's part of its entry's lane mask
    const bool has = lane < cnt;
    const uint32_t q = has ? St.sq[hb + lane] : 0u;
    const uint32_t cm = cnt == 32 ? 0xffffffffu : ((1u << cnt) - 1u);
    uint32_t msk;
    if (__any_sync(0xffffffffu, has && q != vmask)) msk = transpose32(q, lane);
    else msk = valid ? cm : 0u;
    // conservative cut test for all 32 slots, two per instruction; the sign
    // bit of each result is shifted into acc (slot 0 ends up at bit 31)
    uint32_t acc = 0;
#pragma unroll
    for (int s = 0; s < kSlots; s += 4) {
      const float4 fx = *reinterpret_cast<const float4*>(St.fX + hb + s);
      const float4 fy = *reinterpret_cast<const float4*>(St.fY + hb + s);
      const float4 fz = *reinterpret_cast<const float4*>(St.fZ + hb + s);
      const float4 fw = *reinterpret_cast<const float4*>(St.fW + hb + s);
      unsigned long long r01 = add2(pack2(fw.x, fw.y), S2);
      unsigned long long r23 = add2(pack2(fw.z, fw.w), S2);
      r01 = fma2(pack2(fz.x, fz.y), Z2, r01);
      r23 = fma2(pack2(fz.z, fz.w), Z2, r23);
      r01 = fma2(pack2(fy.x, fy.y), Y2, r01);
      r23 = fma2(pack2(fy.z, fy.w), Y2, r23);
      r01 = fma2(pack2(fx.x, fx.y), X2, r01);
      r23 = fma2(pack2(fx.z, fx.w), X2, r23);
      acc = __funnelshift_l((uint32_t)r01, acc, 1);
      acc = __funnelshift_l((uint32_t)(r01 >> 32), acc, 1);
      acc = __funnelshift_l((uint32_t)r23, acc, 1);
      acc = __funnelshift_l((uint32_t)(r23 >> 32), acc, 1);
    }
    uint32_t hit = __brev(acc) & msk;
    const int so = M.self[lane];
    const bool self_here = so >= hb && so < hb + cnt;
    if (self_here) hit &= ~(1u << (so - hb));
    const int nhit = (int)__reduce_add_sync(0xffffffffu, (unsigned)__popc(hit));
    // a batch with more pairs than the list holds is processed in two
    // halves of its slots (at most 32 x 16 pairs each)
    const bool split = nhit > kList;
    for (int part = 0; part < (split ? 2 : 1); ++part) {
      const uint32_t hp = split ? (hit & (part == 0 ? 0x0000ffffu : 0xffff0000u)) : hit;
      // compaction: target-major pair list
      const int c = __popc(hp);
      int incl = c;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
      }
      const int T = __shfl_sync(0xffffffffu, incl, 31);
      const int off = incl - c;
      {
        uint32_t m = hp;
        int t = off;
        while (m) {
          const int s = __ffs(m) - 1;
          m &= m - 1;
          W.list[t++] = (unsigned short)((lane << 5) | s);
        }
      }
      nint += c;  // listed pairs; those outside the exact cut are subtracted below
      __syncwarp();
      {
        const int we = T;
        for (int p0 = 0; p0 < we; p0 += 32) {
          const int p = p0 + lane;
          const bool hv = p < we;
          int i = 0, slot = 0;
          Term<F64> r;
          r.x = r.y = r.z = 0;
          r.w = 0.f;
          float4 sg = make_float4(0.f, 0.f, 0.f, 0.f);
          float3 fw = make_float3(0.f, 0.f, 0.f);
          if (hv) {
            const int e = W.list[p];
            i = e >> 5;
            slot = e & 31;
            if constexpr (F64) {
              r = pair_eval64(A, St, i, hb + slot, gbase);
            } else {
              const float4 rr = pair_eval(A, St, M, i, hb + slot, gbase, sg, fw);
              r.x = rr.x;
              r.y = rr.y;
              r.z = rr.z;
              r.w = rr.w;
            }
            if (r.w == 0.f) atomicAdd(&M.fneg[i], 1);
          }
          // segmented inclusive scan over the lanes: the pairs of one target
          // are consecutive, so each target's run is summed in a fixed tree
          // order and its last lane adds the sum to the target's batch total
          const int oi = __shfl_sync(0xffffffffu, off, i);
          const int ci = __shfl_sync(0xffffffffu, c, i);
          const int first = max(oi - p0, 0);
          // the longest run reaching back into this iteration: steps beyond
          // it add nothing (warp-uniform, so skipping them changes no sum)
          const int span = (int)__reduce_max_sync(0xffffffffu, (unsigned)(hv ? lane - first : 0));
#pragma unroll
          for (int d = 1; d < 32; d <<= 1) {
            if (d > 4 && span < d) break;
            const auto y0 = __shfl_up_sync(0xffffffffu, r.x, d);
            const auto y1 = __shfl_up_sync(0xffffffffu, r.y, d);
            const auto y2 = __shfl_up_sync(0xffffffffu, r.z, d);
            if (lane - d >= first) {
              r.x += y0;
              r.y += y1;
              r.z += y2;
            }
            if constexpr (FUSED) {
              const float f0 = __shfl_up_sync(0xffffffffu, fw.x, d);
              const float f1 = __shfl_up_sync(0xffffffffu, fw.y, d);
              const float f2 = __shfl_up_sync(0xffffffffu, fw.z, d);
              if (lane - d >= first) {
                fw.x += f0;
                fw.y += f1;
                fw.z += f2;
              }
            }
          }
          if (hv && p == min(min(oi + ci, we), p0 + 32) - 1) {
            auto a = M.Ps[i];
            a.x += r.x;
            a.y += r.y;
            a.z += r.z;
            M.Ps[i] = a;
            if constexpr (FUSED) {
              float4 b = M.Pf[i];
              b.x += fw.x;
              b.y += fw.y;
              b.z += fw.z;
              M.Pf[i] = b;
            }
          }
          if (ADJ) {
            // source-side terms: each listed pair's term goes to shared
            // memory with its lane bit in its slot's mask; the lane that owns
            // the slot sums them in lane order and adds the sum to its batch
            // total, kept in registers
            M.SG[lane] = sg;
            if (hv) atomicOr(&M.smask[slot], 1u << lane);
            __syncwarp();
            uint32_t mk = M.smask[lane];
            if (mk) {
              M.smask[lane] = 0u;
              float4 acc = M.SG[__ffs(mk) - 1];
              mk &= mk - 1u;
              while (mk) {
                const float4 v = M.SG[__ffs(mk) - 1];
                acc.x += v.x;
                acc.y += v.y;
                acc.z += v.z;
                acc.w += v.w;
                mk &= mk - 1u;
              }
              gs.x += acc.x;
              gs.y += acc.y;
              gs.z += acc.z;
              gs.w += acc.w;
            }
          }
          __syncwarp();
        }
        __syncwarp();
      }
    }
    // this batch's sums (at most 32 terms per target) into the Kahan totals
    // (FP64 variant: into the plain double sums)
    {
      const auto ps = M.Ps[lane];
      if constexpr (F64) {
        a64[0] += ps.x;
        a64[1] += ps.y;
        a64[2] += ps.z;
        M.Ps[lane] = make_double3(0.0, 0.0, 0.0);
      } else {
        P[0] += ps.x;
        P[1] += ps.y;
        P[2] += ps.z;
        M.Ps[lane] = make_float4(0.f, 0.f, 0.f, 0.f);
        if constexpr (FUSED) {
          const float4 pf = M.Pf[lane];
          Pf[0] += pf.x;
          Pf[1] += pf.y;
          Pf[2] += pf.z;
          M.Pf[lane] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
      }
      nint -= M.fneg[lane];
      M.fneg[lane] = 0;
    }
    if constexpr (!F64) fold();
    if (ADJ) {
      const float4 g = gs;
      if (has && (g.x != 0.f || g.y != 0.f || g.z != 0.f || g.w != 0.f)) {
        const int id = St.sc[hb + lane].x;
        double* Gd = id >= 0 ? A.Gp + 3 * (int64_t)id : A.Gn + 3 * (int64_t)(-2 - id);
        double* Sd = id >= 0 ? A.Sp + id : A.Sn + (-2 - id);
        atomicAdd(Gd, f2d_exact(g.x));
        atomicAdd(Gd + 1, f2d_exact(g.y));
        atomicAdd(Gd + 2, f2d_exact(g.z));
        atomicAdd(Sd, f2d_exact(g.w));
      }
      gs = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    // this batch held the target's own slot
    if (self_here) M.self[lane] = -1;
    __syncwarp();
  }

  __device__ void finish(const WalkArgs& A) {
    if (!valid) return;
    const int32_t i = A.T.order[k];
    if (F64) {
#pragma unroll
      for (int c = 0; c < 3; ++c) A.accd[3 * (int64_t)i + c] = a64[c];
      if (A.counts) A.counts[i] = nint;
    } else if (!ADJ) {
#pragma unroll
      for (int c = 0; c < 3; ++c) A.accf[3 * (int64_t)i + c] = S[c] - C[c];
      if (A.counts) A.counts[i] = nint;
    } else {
#pragma unroll
      for (int c = 0; c < 3; ++c) A.tgt[3 * k + c] = (double)S[c] - (double)C[c];
      if constexpr (FUSED) {
#pragma unroll
        for (int c = 0; c < 3; ++c) A.accf[3 * (int64_t)i + c] = Sf[c] - Cf[c];
        if (A.counts) A.counts[i] = nint;
      }
    }
  }
};

template <bool ADJ>
using LaneF32 = LaneFP<ADJ, false>;
using LaneF64 = LaneFP<false, true>;
using LaneFused = LaneFP<true, false, true>;

// ------------------------------------------------------------------ traversal

template <class Lane>
union WarpScratch {
  MixedScratch mix;
  typename Lane::Stage stage;
};

template <class Lane>
__global__ void __launch_bounds__(kWarpsPerBlock * 32) k_walk(WalkArgs A) {
  __shared__ int2 s_stack[kWarpsPerBlock][kStack];
  __shared__ int4 s_queue[kWarpsPerBlock][kQueue];
  __shared__ int s_qoff[kWarpsPerBlock][kQueue + 1];
  __shared__ unsigned short s_list[kWarpsPerBlock][kList];
  __shared__ WarpScratch<Lane> s_scr[kWarpsPerBlock];
  __shared__ typename Lane::Smem s_lane[kWarpsPerBlock];
  __shared__ float4 s_sgb[kWarpsPerBlock][2 * kSub];
  const TreeDev& T = A.T;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int64_t g = A.g_begin + (int64_t)blockIdx.x * kWarpsPerBlock + wib;
  if (g >= A.g_end) return;
  if (T.sb->status != 0 || T.sb->magic != kMagicTree) {
    // a failed or missing tree: flag it and give every output of this
    // group's targets NaN, so that nothing downstream can take stale values
    // for forces.  A tree whose build started wrote its permutation first;
    // for one that was never built the sorted index stands in for it.
    if (lane == 0) set_status(A.wsb, ST_NOTREE);
    const int64_t kk = g * kGroup + lane;
    if (kk < T.n) {
      const float nf = __int_as_float(0x7fc00000);
      const double nd = __longlong_as_double(0x7ff8000000000000ll);
      int64_t io = kk;
      if (T.sb->magic == kMagicTree) {
        const int64_t o = T.order[kk];
        if (o >= 0 && o < T.n) io = o;
      }
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        if (A.accf) A.accf[3 * io + c] = nf;
        if (A.accd) A.accd[3 * io + c] = nd;
        if (A.tgt) A.tgt[3 * kk + c] = nd;
      }
      if (A.counts) A.counts[io] = -1;
    }
    return;
  }
  WarpBufs W;
  W.stack = s_stack[wib];
  W.queue = s_queue[wib];
  W.qoff = s_qoff[wib];
  W.list = s_list[wib];
  MixedScratch& X = s_scr[wib].mix;
  typename Lane::Stage& St = s_scr[wib].stage;
  typename Lane::Smem& M = s_lane[wib];
  int nodes_total = 0;
  for (int l = 0; l < kLevels; ++l) nodes_total += T.sb->level_cnt[l];
  if (nodes_total > T.cap) nodes_total = (int)T.cap;

  const int64_t gbase = g * kGroup;
  const int64_t k = gbase + lane;
  const bool valid = k < T.n;
  const uint32_t vmask = __ballot_sync(0xffffffffu, valid);
  const uint32_t lt = (1u << lane) - 1u;

  GroupInfo G;
  {
    const float4 lo = T.gbox[2 * g], hi = T.gbox[2 * g + 1];
    G.cx = 0.5f * (lo.x + hi.x); G.cy = 0.5f * (lo.y + hi.y); G.cz = 0.5f * (lo.z + hi.z);
    G.ex = 0.5f * (hi.x - lo.x) * 1.0001f + 1e-7f;
    G.ey = 0.5f * (hi.y - lo.y) * 1.0001f + 1e-7f;
    G.ez = 0.5f * (hi.z - lo.z) * 1.0001f + 1e-7f;
  }
  // bound on |x_i - group centre| for the evaluation's cut filter
  const float Rg = sqrtf(fmaf(G.ex, G.ex, fmaf(G.ey, G.ey, G.ez * G.ez))) * 1.0001f + 1e-6f;
  // boxes of the 4 sub-groups of 8 targets (box units, padded outward by
  // more than the FP32 rounding of a position in [0, 1))
  float4* SGB = s_sgb[wib];
  {
    const float4 pa = T.pA[valid ? k : 0], pb = T.pB[valid ? k : 0];
    float lo[3] = {pa.x + pb.x, pa.y + pb.y, pa.z + pb.z};
    float hi[3] = {lo[0], lo[1], lo[2]};
    if (!valid) {
#pragma unroll
      for (int c = 0; c < 3; ++c) { lo[c] = 1e30f; hi[c] = -1e30f; }
    }
#pragma unroll
    for (int o = 4; o > 0; o >>= 1)
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        lo[c] = fminf(lo[c], __shfl_xor_sync(0xffffffffu, lo[c], o));
        hi[c] = fmaxf(hi[c], __shfl_xor_sync(0xffffffffu, hi[c], o));
      }
    if ((lane & 7) == 0) {
      const float pad = 2e-7f;
      SGB[2 * (lane >> 3)] = make_float4(0.5f * (lo[0] + hi[0]), 0.5f * (lo[1] + hi[1]), 0.5f * (lo[2] + hi[2]), 0.f);
      SGB[2 * (lane >> 3) + 1] = make_float4(0.5f * (hi[0] - lo[0]) * 1.0001f + pad,
                                             0.5f * (hi[1] - lo[1]) * 1.0001f + pad,
                                             0.5f * (hi[2] - lo[2]) * 1.0001f + pad, 0.f);
    }
  }

  Lane L;
  L.init(A, M, k, valid, lane, G);

  if (lane == 0) W.stack[0] = make_int2((int)(1u << 28), (int)vmask);  // the root: node 0, one node
  int sp = 1, nq = 0;
  long long visits = 0;
  __syncwarp();
  for (;;) {
    if (sp > 0 && nq <= kQueue - kQueueNeed) {
      if (sp > kStack - kStackNeed) {
        if (lane == 0) set_status(A.wsb, ST_STACK);
        break;
      }
      // Pop whole child ranges from the top until up to 32 nodes are gathered
      // (one range when the stack is deep).  The index is clamped so no lane
      // forms an address outside the stack, and every pop completes before
      // any push.
      const int m = sp > min(A.deep, kDeep) ? 1 : min(sp, 32);
      const int2 E = W.stack[max(sp - 1 - lane, 0)];
      __syncwarp();
      const uint32_t ex = (uint32_t)E.x;
      const int rcnt = lane < m ? (int)(ex >> 28) : 0;
      const int rfirst_l = (int)(ex & 0x0fffffffu);
      if (__any_sync(0xffffffffu, lane < m && (rcnt < 1 || rcnt > 8))) {
        if (lane == 0) set_status(A.wsb, ST_TREELINK);
        break;
      }
      int incl = rcnt;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
      }
      const int take = __popc(__ballot_sync(0xffffffffu, lane < m && incl <= 32));  // >= 4 ranges or all
      const int total = __shfl_sync(0xffffffffu, incl, take - 1);
      sp -= take;
      visits += total;
      if (visits > A.max_iters) {
        if (lane == 0) set_status(A.wsb, ST_WALKCAP);
        break;
      }
      // lane s takes node s of the gathered ranges: r = ranges ending at or before s
      int r = 0;
#pragma unroll
      for (int b = 16; b > 0; b >>= 1) {
        const int cand = r + b;
        const int v = __shfl_sync(0xffffffffu, incl, (cand - 1) & 31);
        if (cand <= take && v <= lane) r = cand;
      }
      // every lane executes the shuffle (a full-mask shuffle reached by only
      // some lanes is undefined); the value is selected afterwards
      const int prev = __shfl_sync(0xffffffffu, incl, (r - 1) & 31);
      const int excl = r > 0 ? prev : 0;
      const int rfirst = __shfl_sync(0xffffffffu, rfirst_l, r & 31);
      const uint32_t mask = (uint32_t)__shfl_sync(0xffffffffu, E.y, r & 31);
      const bool has = lane < total;
      const int node = has ? rfirst + (lane - excl) : 0;
      if (__any_sync(0xffffffffu, has && (node < 0 || node >= nodes_total))) {
        if (lane == 0) set_status(A.wsb, ST_TREELINK);
        break;
      }
      const int nc = has ? node : 0;
      const float4 NC = T.nC[nc];
      const int4 ND = T.nD[nc];
      const float4 NA = T.nA[nc];
      const float4 NB = T.nB[nc];
      const int cls = has ? classify(A, G, NC, NA, NB) : CL_NONE;
      const bool leaf = meta_leaf(ND.w);
      const int nch = meta_nchild(ND.w);
      bool bad = false;
      if (has && cls != CL_DROP) {
        if (leaf) bad = ND.x < 0 || ND.y < 1 || (int64_t)ND.x + ND.y > T.n;
        else bad = nch <= 0 || nch > 8 || ND.z <= node || ND.z + nch > nodes_total;
      }
      if (__any_sync(0xffffffffu, bad)) {
        if (lane == 0) set_status(A.wsb, ST_TREELINK);
        break;
      }
      // OPEN internal nodes: push their child range with the same lanes
      const bool push = cls == CL_OPEN && !leaf;
      const uint32_t pm = __ballot_sync(0xffffffffu, push);
      if (push) W.stack[sp + __popc(pm & lt)] = make_int2((int)((uint32_t)ND.z | ((uint32_t)nch << 28)), (int)mask);
      sp += __popc(pm);
      // OPEN leaves and ACCEPTed nodes: queue them for evaluation
      const bool q = (cls == CL_OPEN && leaf) || cls == CL_ACCEPT;
      const uint32_t qm = __ballot_sync(0xffffffffu, q);
      if (q) {
        const int fl = image_flags(A, G, NC);
        W.queue[nq + __popc(qm & lt)] =
            cls == CL_ACCEPT ? make_int4(node, -1, (int)mask, fl) : make_int4(ND.x, ND.y, (int)mask, fl);
      }
      nq += __popc(qm);
      // MIXED nodes: exact decisions for every (node, target in its mask),
      // 32 at a time from a node-major list; the results are OR-ed into
      // per-node accept / open masks
      const uint32_t mm = __ballot_sync(0xffffffffu, cls == CL_MIXED);
      if (mm) {
        const int nm = __popc(mm);
        if (cls == CL_MIXED) {
          const int ix = __popc(mm & lt);
          const int xfl = image_flags(A, G, NC);
          float4 SC = NC, SA = NA;
          if (xfl & 1) {
            const float sx = shift_of(xfl, 0), sy = shift_of(xfl, 1), sz = shift_of(xfl, 2);
            SC.x -= sx; SC.y -= sy; SC.z -= sz;
            SA.x -= sx; SA.y -= sy; SA.z -= sz;
          }
          X.node[ix] = node;
          X.fl[ix] = xfl;
          X.D[ix] = ND;
          X.C[ix] = SC;
          X.A[ix] = SA;
          X.B[ix] = NB;
          X.mask[ix] = mask & vmask;
          X.acc[ix] = 0u;
          X.open[ix] = 0u;
          X.dmask[ix] = 0u;
        }
        __syncwarp();
        // each (node, sub-group) pair is first classified against the
        // sub-group's box; only undecided sub-groups need per-lane decisions
        for (int j = lane; j < kSub * nm; j += 32) {
          const int ix = j >> 2, g = j & 3;
          const uint32_t gm = X.mask[ix] & (0xffu << (8 * g));
          if (gm) {
            const float4 c4 = SGB[2 * g], e4 = SGB[2 * g + 1];
            GroupInfo Gs;
            Gs.cx = c4.x; Gs.cy = c4.y; Gs.cz = c4.z;
            Gs.ex = e4.x; Gs.ey = e4.y; Gs.ez = e4.z;
            const int cg = classify(A, Gs, X.C[ix], X.A[ix], X.B[ix]);
            if (cg == CL_OPEN) atomicOr(&X.open[ix], gm);
            else if (cg == CL_ACCEPT) atomicOr(&X.acc[ix], gm);
            else if (cg == CL_MIXED) atomicOr(&X.dmask[ix], gm);
          }
        }
        __syncwarp();
        // at most kList / 32 nodes per list
        for (int m0 = 0; m0 < nm; m0 += kList / 32) {
          const int m1 = min(nm, m0 + kList / 32);
          int nd = 0;
          for (int ix = m0; ix < m1; ++ix) {
            const uint32_t mk = X.dmask[ix];
            if ((mk >> lane) & 1u) W.list[nd + __popc(mk & lt)] = (unsigned short)((ix << 5) | lane);
            nd += __popc(mk);
          }
          __syncwarp();
          for (int d = lane; d < nd; d += 32) {
            const int e = W.list[d];
            const int ix = e >> 5, t = e & 31;
            const int dec =
                L.decide_for(A, M, t, gbase + t, X.node[ix], X.D[ix], X.C[ix], X.A[ix], X.B[ix], (X.fl[ix] & 1) != 0);
            if (dec == DEC_ACCEPT) atomicOr(&X.acc[ix], 1u << t);
            else if (dec == DEC_OPEN) atomicOr(&X.open[ix], 1u << t);
          }
          __syncwarp();
        }
        const bool hm = lane < nm;
        const int hx = hm ? lane : 0;
        const uint32_t am = hm ? X.acc[hx] : 0u;
        const uint32_t om = hm ? X.open[hx] : 0u;
        const int4 XD = X.D[hx];
        const int xnode = X.node[hx];
        const bool xleaf = meta_leaf(XD.w);
        const int fl = X.fl[hx];
        const bool qa = am != 0u, qo = om != 0u && xleaf, po = om != 0u && !xleaf;
        const uint32_t ba = __ballot_sync(0xffffffffu, qa);
        const uint32_t bo = __ballot_sync(0xffffffffu, qo);
        const uint32_t bp = __ballot_sync(0xffffffffu, po);
        if (qa) W.queue[nq + __popc(ba & lt)] = make_int4(xnode, -1, (int)am, fl);
        nq += __popc(ba);
        if (qo) W.queue[nq + __popc(bo & lt)] = make_int4(XD.x, XD.y, (int)om, fl);
        nq += __popc(bo);
        if (po)
          W.stack[sp + __popc(bp & lt)] =
              make_int2((int)((uint32_t)XD.z | ((uint32_t)meta_nchild(XD.w) << 28)), (int)om);
        sp += __popc(bp);
      }
      __syncwarp();
    } else if (nq > 0) {
      L.evaluate(A, W, St, M, nq, lane, G, gbase, vmask, Rg);
      nq = 0;
      __syncwarp();
    } else {
      break;
    }
  }
  L.finish(A);
  if (A.total) {
    const unsigned cnt = __reduce_add_sync(0xffffffffu, (unsigned)(valid ? L.nint : 0));
    if (lane == 0 && cnt) atomicAdd(A.total, (unsigned long long)cnt);
  }
}

cudaError_t launch_walk(const WalkArgs& A, int prec, bool adjoint, cudaStream_t s, bool fused) {
  const int64_t blocks = (A.g_end - A.g_begin + kWarpsPerBlock - 1) / kWarpsPerBlock;
  if (blocks <= 0) return cudaSuccess;
  if (fused) k_walk<LaneFused><<<(unsigned)blocks, kWarpsPerBlock * 32, 0, s>>>(A);
  else if (adjoint) k_walk<LaneF32<true>><<<(unsigned)blocks, kWarpsPerBlock * 32, 0, s>>>(A);
  else if (prec == OG_FP64) k_walk<LaneF64><<<(unsigned)blocks, kWarpsPerBlock * 32, 0, s>>>(A);
  else k_walk<LaneF32<false>><<<(unsigned)blocks, kWarpsPerBlock * 32, 0, s>>>(A);
  return cudaGetLastError();
}

}  // namespace og
