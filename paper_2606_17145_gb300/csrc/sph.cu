// sph.cu -- SPH density and smoothing length on the device (declared in
// include/og.h: og_sph_ws_bytes / og_sph_density).
//
// The paper's SPH density module iterates each particle's smoothing length
// until its sphere holds a fixed number of neighbours, gathering the
// neighbours inside a sphere before evaluating them; its walks group nearby
// targets (Sec. 2, 2.1).  The reading is GADGET-2's: W is the cubic spline
// with support h, rho_i = sum_j m_j W(r_ij, h_i) (the particle itself
// included), and h_i is the root of the kernel-weighted count
// N_eff(h) = (4 pi / 3) h^3 sum_j W(r_ij, h) = (32 / 3) sum_j w(r_ij / h) = N_ngb.
//
// Grouped walk.  One warp serves a group of 32 Hilbert-consecutive targets
// (lane = target), as in the gravity walk.  Each pass gathers, from one
// traversal of the tree (a range stack popped 32 nodes at a time), every leaf
// whose cube comes within R of the box of the lanes still iterating (R their
// largest radius).  The leaves' particles are fetched 32 at a time (each
// lane finds its slot's leaf from a start mask and a popcount), a particle
// beyond R of that box is dropped, and every lane evaluates the staged ones
// against its own radius.
//   1. Start: the density of the smallest ancestor of the target's leaf that
//      holds at least N_ngb particles gives h = (3 N_ngb / 4 pi n)^(1/3).
//   2. FP32 passes: Newton steps on ln h, ln N_eff(h) = ln N_ngb, with
//      d ln N_eff / d ln h = -sum q w'(q) / sum w(q), a bracket of the root kept
//      from every evaluation (a step leaving it is replaced by the bracket's
//      geometric mean) and steps clamped to a factor 2, until a step below
//      1e-2 (taken, leaving ~3e-5).
//      Distances come from the split-float positions (FP64 accuracy rounded
//      to FP32).
//   3. Finishing pass: each lane lists its candidates within h (1 + 4e-4)
//      (FP32 test with a margin) and their periodic image in shared memory,
//      and the lists are evaluated lane-parallel in float-float arithmetic
//      on the split-float positions (about 1e-11 relative in q; the FP64
//      pipe, 1/64 of FP32 on this GPU, keeps only the sums): sum w and sum
//      m w in FP64; sum q w' and sum m q w' (compensated FP32) and sum
//      q^2 w'' and sum m q^2 w'' (FP32).  A second-order step in ln h from
//      those sums gives h (error ~20 d^3 for a step d; steps up to 3e-4 are
//      accepted) and the density at it; the neighbour count at the new h is
//      the count at the evaluated one corrected by the neighbours within
//      4e-4 h of it (their distances are kept, up to two; with more, or a
//      larger step, the pass is repeated at the new h).
// Every loop is bounded (node-visit cap, pass caps, the stack bound); a
// particle whose h does not converge below half the box gets NaN / -1 and
// sets a status bit.
#include <cmath>

#include "og_internal.cuh"

namespace og {

constexpr int kSphWarps = 2;          // warps per block
constexpr int kSphStack = 276;        // range stack entries (same bound as the gravity walk)
constexpr int kSphStackNeed = 32;     // pushes of one step
constexpr int kSphDeep = 64;          // above this depth a step pops a single range
static_assert(kSphDeep + 31 + 7 * 20 + 8 <= kSphStack - kSphStackNeed, "stack bound");
constexpr int kSphQueue = 128;        // queued leaves per warp
constexpr int kSphQueueNeed = 32;     // a step queues at most one leaf per popped node
constexpr int kSphList = 32;          // finishing pass: listed candidates per lane before a flush
constexpr int kSphPass32 = 32;        // FP32 Newton passes at most
constexpr int kSphPass64 = 8;         // finishing passes at most
// FP32 passes stop once a Newton step on ln h is below this; the step is
// still taken, and Newton's quadratic convergence leaves an error of about
// (f''/2f') dl^2 ~ 3e-5 (f = ln N_eff(ln h), f' ~ 3), inside the 3e-4 step
// that the finishing pass accepts in one evaluation.
constexpr float kSphConv32 = 1e-2f;
// The finishing pass lists neighbours within (1 + kSphBand) h and accepts a
// second-order step of up to kSphStep in ln h.
constexpr double kSphBand = 4e-4;
constexpr double kSphStep = 3e-4;

struct SphArgs {
  TreeDev T;
  StatusBlock* wsb;
  BoxScale B;
  double n_ngb;
  long long max_visits;  // node visits per gather
  double* h_out;
  double* rho_out;
  int32_t* ngb_out;
};

// Minimum image of a box-unit difference t (|t| < 1.5): t - rint(t).
__device__ __forceinline__ float sph_mi1(float t) {
  const float r = __fadd_rn(__fadd_rn(t, 12582912.0f), -12582912.0f);
  return __fadd_rn(t, -r);
}

// Compensated (Kahan) addition: the sum is T - C.  The _rn intrinsics keep
// the compiler from reassociating it away.
__device__ __forceinline__ void sph_kahan_add(float& T, float& C, float x) {
  const float y = __fsub_rn(x, C);
  const float t = __fadd_rn(T, y);
  C = __fsub_rn(__fsub_rn(t, T), y);
  T = t;
}

// Float-float arithmetic (a value is hi + lo, |lo| <= ulp(hi) / 2): the
// error-free sum and product of two floats (Knuth's two-sum; the product's
// error from one fused multiply-add) and the products and sums built on
// them, about 2^-46 relative.  The _rn intrinsics keep the compiler from
// contracting or reordering the steps.
struct FF {
  float hi, lo;
};
__device__ __forceinline__ FF ff_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
__device__ __forceinline__ FF ff_quick(float a, float b) {  // |a| >= |b| (or a == 0)
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ FF ff_two_prod(float a, float b) {
  const float p = __fmul_rn(a, b);
  return {p, __fmaf_rn(a, b, -p)};
}
__device__ __forceinline__ FF ff_mul(const FF& a, const FF& b) {
  const FF p = ff_two_prod(a.hi, b.hi);
  return ff_quick(p.hi, __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, p.lo)));
}
__device__ __forceinline__ FF ff_add(const FF& a, const FF& b) {
  const FF s = ff_two_sum(a.hi, b.hi);
  return ff_quick(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}
// max(c - q, 0) for c = 1 or 1/2
__device__ __forceinline__ FF ff_pos_diff(float c, const FF& q) {
  const FF d = ff_two_sum(c, -q.hi);
  const FF r = ff_quick(d.hi, __fsub_rn(d.lo, q.lo));
  return (r.hi > 0.f) ? r : FF{0.f, 0.f};
}

struct SphBufs {
  int* stack;
  int2* queue;
  int* qoff;        // [kSphQueue + 1] slot offsets of the queued leaves
  float4* sa;       // [32] staged candidates: hi part
  float4* sb;       // [32] lo part
  int* sj;          // [32] sorted index
  int (*list)[32];  // [kSphList][lane]
  unsigned char (*img)[32];  // [kSphList][lane] periodic image code of each listed candidate
};

struct SphGroup {
  float cx, cy, cz, ex, ey, ez;  // group box centre and half extents (box units, padded)
};

// Bounding box of the active lanes' targets (hi parts, box units, which are
// non-negative and order like their bit patterns), padded by 1e-6 for the lo
// parts and rounding.  A pass gathers around the lanes it still has to
// serve, so a group whose other lanes have converged reaches fewer leaves.
__device__ __forceinline__ SphGroup active_box(const float3& th, bool act) {
  const uint32_t inf = 0x7f800000u;
  const float lx = __uint_as_float(__reduce_min_sync(0xffffffffu, act ? __float_as_uint(th.x) : inf));
  const float ly = __uint_as_float(__reduce_min_sync(0xffffffffu, act ? __float_as_uint(th.y) : inf));
  const float lz = __uint_as_float(__reduce_min_sync(0xffffffffu, act ? __float_as_uint(th.z) : inf));
  const float hx = __uint_as_float(__reduce_max_sync(0xffffffffu, act ? __float_as_uint(th.x) : 0u));
  const float hy = __uint_as_float(__reduce_max_sync(0xffffffffu, act ? __float_as_uint(th.y) : 0u));
  const float hz = __uint_as_float(__reduce_max_sync(0xffffffffu, act ? __float_as_uint(th.z) : 0u));
  SphGroup G;
  G.cx = 0.5f * (lx + hx);
  G.cy = 0.5f * (ly + hy);
  G.cz = 0.5f * (lz + hz);
  G.ex = 0.5f * (hx - lx) * 1.0001f + 1e-6f;
  G.ey = 0.5f * (hy - ly) * 1.0001f + 1e-6f;
  G.ez = 0.5f * (hz - lz) * 1.0001f + 1e-6f;
  return G;
}

// One gather: every leaf whose cube comes within R (box units) of the group
// box is passed to eval(first, count), in batches.  Warp-uniform control
// flow.  Returns status bits (0 if clean).
template <class Eval>
__device__ uint32_t sph_gather(const SphArgs& A, const SphBufs& W, const SphGroup& G, float R, int nodes_total,
                               int lane, Eval& eval) {
  const TreeDev& T = A.T;
  const float R2 = (R * 1.00001f + 1e-7f) * (R * 1.00001f + 1e-7f);
  const uint32_t lt = (1u << lane) - 1u;
  if (lane == 0) W.stack[0] = (int)(1u << 28);  // the root: node 0, one node
  int sp = 1, nq = 0;
  long long visits = 0;
  __syncwarp();
  for (;;) {
    if (sp > 0 && nq <= kSphQueue - kSphQueueNeed) {
      if (sp > kSphStack - kSphStackNeed) return ST_STACK;
      const int m = sp > kSphDeep ? 1 : min(sp, 32);
      const uint32_t E = (uint32_t)W.stack[max(sp - 1 - lane, 0)];
      __syncwarp();
      const int rcnt = lane < m ? (int)(E >> 28) : 0;
      const int rfirst_l = (int)(E & 0x0fffffffu);
      if (__any_sync(0xffffffffu, lane < m && (rcnt < 1 || rcnt > 8))) return ST_TREELINK;
      int incl = rcnt;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
      }
      const int take = __popc(__ballot_sync(0xffffffffu, lane < m && incl <= 32));
      const int total = __shfl_sync(0xffffffffu, incl, take - 1);
      sp -= take;
      visits += total;
      if (visits > A.max_visits) return ST_WALKCAP;
      // lane s takes node s of the gathered ranges: r = ranges ending at or before s
      int r = 0;
#pragma unroll
      for (int b = 16; b > 0; b >>= 1) {
        const int cand = r + b;
        const int v = __shfl_sync(0xffffffffu, incl, (cand - 1) & 31);
        if (cand <= take && v <= lane) r = cand;
      }
      const int prev = __shfl_sync(0xffffffffu, incl, (r - 1) & 31);
      const int excl = r > 0 ? prev : 0;
      const int rfirst = __shfl_sync(0xffffffffu, rfirst_l, r & 31);
      const bool has = lane < total;
      const int node = has ? rfirst + (lane - excl) : 0;
      if (__any_sync(0xffffffffu, has && (node < 0 || node >= nodes_total))) return ST_TREELINK;
      const float4 NC = T.nC[node];
      const int4 ND = T.nD[node];
      bool keep = false;
      if (has) {
        const float hs = 0.5f * NC.w;
        const float gx = fmaxf(fabsf(sph_mi1(NC.x - G.cx)) - (hs + G.ex), 0.f);
        const float gy = fmaxf(fabsf(sph_mi1(NC.y - G.cy)) - (hs + G.ey), 0.f);
        const float gz = fmaxf(fabsf(sph_mi1(NC.z - G.cz)) - (hs + G.ez), 0.f);
        keep = fmaf(gx, gx, fmaf(gy, gy, gz * gz)) <= R2;
      }
      const bool leaf = meta_leaf(ND.w);
      const int nch = meta_nchild(ND.w);
      bool bad = false;
      if (keep) {
        if (leaf) bad = ND.x < 0 || ND.y < 1 || (int64_t)ND.x + ND.y > T.n;
        else bad = nch <= 0 || nch > 8 || ND.z <= node || ND.z + nch > nodes_total;
      }
      if (__any_sync(0xffffffffu, bad)) return ST_TREELINK;
      const bool push = keep && !leaf;
      const uint32_t pm = __ballot_sync(0xffffffffu, push);
      if (push) W.stack[sp + __popc(pm & lt)] = (int)((uint32_t)ND.z | ((uint32_t)nch << 28));
      sp += __popc(pm);
      const bool q = keep && leaf;
      const uint32_t qm = __ballot_sync(0xffffffffu, q);
      if (q) W.queue[nq + __popc(qm & lt)] = make_int2(ND.x, ND.y);
      nq += __popc(qm);
      __syncwarp();
    } else if (nq > 0) {
      // slot offsets of the queued leaves (warp scan, 32 entries at a time)
      int run = 0;
      for (int b0 = 0; b0 < nq; b0 += 32) {
        const int e = b0 + lane;
        const int c = e < nq ? W.queue[e].y : 0;
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
      // stage the candidates 32 at a time (one coalesced load per lane) and
      // let every lane evaluate them from shared memory
      // and let every lane evaluate them from shared memory; a particle
      // beyond R of the box is not staged (the leaf's cube reached the
      // sphere, the particle does not)
      // Each window of 32 slots finds its slots' leaves without a search:
      // ecur holds the window's first slot, the leaves starting inside the
      // window set bit (start - s0) of one OR-reduced mask (leaves hold at
      // least one particle, so at most 31 start inside it), and slot s0 + l
      // lies in leaf ecur + (number of starts at or before bit l).
      int ecur = 0;
      for (int s0 = 0; s0 < run; s0 += 32) {
        const int ek = ecur + 1 + lane;
        const int sk = ek < nq ? W.qoff[ek] - s0 : 32;
        const uint32_t starts = __reduce_or_sync(0xffffffffu, (sk > 0 && sk < 32) ? (1u << sk) : 0u);
        const int slot = s0 + lane;
        bool stage = false;
        float4 pa = make_float4(0.f, 0.f, 0.f, 0.f), pb = pa;
        int j = 0;
        if (slot < run) {
          const int e = ecur + __popc(starts & ((2u << lane) - 1u));
          j = W.queue[e].x + (slot - W.qoff[e]);
          pa = T.pA[j];
          pb = T.pB[j];
          const float gx = fmaxf(fabsf(sph_mi1(pa.x - G.cx)) - G.ex, 0.f);
          const float gy = fmaxf(fabsf(sph_mi1(pa.y - G.cy)) - G.ey, 0.f);
          const float gz = fmaxf(fabsf(sph_mi1(pa.z - G.cz)) - G.ez, 0.f);
          stage = fmaf(gx, gx, fmaf(gy, gy, gz * gz)) <= R2;
        }
        const uint32_t sm = __ballot_sync(0xffffffffu, stage);
        if (stage) {
          const int at = __popc(sm & lt);
          W.sa[at] = pa;
          W.sb[at] = pb;
          W.sj[at] = j;
        }
        __syncwarp();
        if (sm) eval(W, __popc(sm));
        __syncwarp();
        // the leaf holding the next window's first slot
        int en = ecur + __popc(starts);
        if (en + 1 < nq && W.qoff[en + 1] == s0 + 32) ++en;
        ecur = en;
      }
      nq = 0;
    } else {
      break;
    }
  }
  return 0u;
}

// Split-float squared distance (box units) from a target to a staged particle.
__device__ __forceinline__ float sph_r2_32(const float3& th, const float3& tl, const float4& a, const float4& b) {
  const float dx = sph_mi1(th.x - a.x) + (tl.x - b.x);
  const float dy = sph_mi1(th.y - a.y) + (tl.y - b.y);
  const float dz = sph_mi1(th.z - a.z) + (tl.z - b.z);
  return fmaf(dx, dx, fmaf(dy, dy, dz * dz));
}

// FP32 pass: sums of w(q) and q w'(q) over the particles within h.
struct SphEval32 {
  float3 th, tl;
  float ih2;  // 1 / h^2 (box units)
  float S0, S1;
  // Branch-free: w(q) = 2 u^3 - 8 v^3 and q w'(q) = q (24 v^2 - 6 u^2) with
  // u = max(1 - q, 0), v = max(1/2 - q, 0) (both zero beyond the support),
  // so the warp does not diverge on which lanes hold the candidate.
  __device__ __forceinline__ void operator()(const SphBufs& W, int count) {
#pragma unroll 2
    for (int s = 0; s < count; ++s) {
      const float4 a = W.sa[s];
      const float r2 = sph_r2_32(th, tl, a, W.sb[s]);
      const float x = fmaxf(r2 * ih2, 1e-30f);
      const float q = x * rsqrtf(x);
      const float u = fmaxf(1.0f - q, 0.0f), v = fmaxf(0.5f - q, 0.0f);
      const float u2 = u * u, v2 = v * v;
      S0 += fmaf(2.0f * u2, u, -8.0f * v2 * v);
      const float wq = q * fmaf(24.0f, v2, -6.0f * u2);
      S1 += wq;
    }
  }
};

// Finishing pass: candidates within hb (FP32 test with a margin) go to this
// lane's list with their periodic image; a full list anywhere in the warp is
// flushed, i.e. every lane evaluates its listed candidates in float-float and
// adds w to FP64 sums (sum w, sum m w, which set h and rho to ~1e-12); the
// derivatives, which scale a step below 3e-6 h, are FP32 sums of the same
// neighbours.
struct SphEval64 {
  const SphArgs* A;
  const SphBufs* W;
  int lane;
  int64_t k;           // this lane's sorted index
  float3 th, tl;
  float hb2_32;        // FP32 prefilter radius^2 (box units), with margin
  FF ih2;              // 1 / h^2 (box units)
  double S0, R0;
  // the step's derivatives at this h: sum q w'(q) and sum (m / L^2) q w'(q)
  // (FP32, compensated: C1, Q1), sum q^2 w''(q) and sum (m / L^2) q^2 w''(q)
  float S1, R1, C1, Q1;
  float S2, R2;
  double bq0, bq1;     // q = r / h of the first two neighbours in the band
  int clt, band, cnt;
  __device__ __forceinline__ void flush() {
    const TreeDev& T = A->T;
    const float qhi2 = (float)((1.0 + kSphBand) * (1.0 + kSphBand)), qlo = (float)(1.0 - kSphBand);
    const int top = __reduce_max_sync(0xffffffffu, (unsigned)cnt);
    for (int t = 0; t < top; ++t) {
      if (t < cnt) {
        const int j = W->list[t][lane];
        const int code = W->img[t][lane];
        const float4 a = T.pA[j], b = T.pB[j];
        // d = x_i - x_j - s (box units), s the periodic image found in the
        // listing: the hi parts are multiples of 2^-23 in [0, 1), so their
        // difference minus s is exact; the lo difference is rounded once
        // (2^-48).  d = dh + dl and r^2 = |d|^2 as a float-float.
        const float dh0 = __fsub_rn(__fsub_rn(th.x, a.x), (float)(code % 3 - 1));
        const float dh1 = __fsub_rn(__fsub_rn(th.y, a.y), (float)((code / 3) % 3 - 1));
        const float dh2 = __fsub_rn(__fsub_rn(th.z, a.z), (float)(code / 9 - 1));
        const float dl0 = __fsub_rn(tl.x, b.x), dl1 = __fsub_rn(tl.y, b.y), dl2 = __fsub_rn(tl.z, b.z);
        const FF p0 = ff_two_prod(dh0, dh0), p1 = ff_two_prod(dh1, dh1), p2 = ff_two_prod(dh2, dh2);
        const FF s01 = ff_two_sum(p0.hi, p1.hi), s012 = ff_two_sum(s01.hi, p2.hi);
        // the small terms: the products' errors, 2 dh dl and dl^2
        float c = __fmaf_rn(2.0f * dh0 + dl0, dl0, __fmaf_rn(2.0f * dh1 + dl1, dl1, __fmul_rn(2.0f * dh2 + dl2, dl2)));
        c = __fadd_rn(c, __fadd_rn(__fadd_rn(p0.lo, p1.lo), __fadd_rn(p2.lo, __fadd_rn(s01.lo, s012.lo))));
        const FF q2 = ff_mul(ff_quick(s012.hi, c), ih2);
        if (q2.hi < qhi2) {
          // q = sqrt(q2): the rounded root and one correction,
          // q0 + (q2 - q0^2) / (2 q0), with q0^2 exact
          FF q = {0.f, 0.f};
          const float q0 = __fsqrt_rn(q2.hi);
          if (q0 > 0.f) {
            const FF sq = ff_two_prod(q0, q0);
            const float res = __fadd_rn(__fsub_rn(__fsub_rn(q2.hi, sq.hi), sq.lo), q2.lo);
            q = ff_quick(q0, __fmul_rn(res, __fdiv_rn(0.5f, q0)));
          }
          // w = 2 u^3 - 8 v^3, u = max(1 - q, 0), v = max(1/2 - q, 0)
          const FF u = ff_pos_diff(1.0f, q), v = ff_pos_diff(0.5f, q);
          const FF u3 = ff_mul(ff_mul(u, u), u), v3 = ff_mul(ff_mul(v, v), v);
          const FF w = ff_add(FF{2.0f * u3.hi, 2.0f * u3.lo}, FF{-8.0f * v3.hi, -8.0f * v3.lo});
          const double wd = (double)w.hi + (double)w.lo;
          S0 += wd;
          R0 = fma(T.m64[j], wd, R0);
          const bool in = q.hi < 1.0f || (q.hi == 1.0f && q.lo < 0.0f);
          if (in) {
            // q w'(q) and q^2 w''(q): w' = 18 q^2 - 12 q, w'' = 36 q - 12 for
            // q <= 1/2; w' = -6 u^2, w'' = 12 u (u = 1 - q) beyond
            const float qf = q.hi, uf = 1.0f - qf;
            const bool inner = qf <= 0.5f;
            const float wq = inner ? qf * qf * fmaf(18.0f, qf, -12.0f) : -6.0f * qf * uf * uf;
            const float wqq = inner ? qf * qf * fmaf(36.0f, qf, -12.0f) : 12.0f * qf * qf * uf;
            sph_kahan_add(S1, C1, wq);
            sph_kahan_add(R1, Q1, a.w * wq);
            S2 += wqq;
            R2 = fmaf(a.w, wqq, R2);
          }
          if (j != (int)k) {
            if (in) ++clt;
            if (q.hi >= qlo) {
              const double qd = (double)q.hi + (double)q.lo;
              if (band == 0) bq0 = qd;
              else if (band == 1) bq1 = qd;
              ++band;
            }
          }
        }
      }
    }
    cnt = 0;
    __syncwarp();
  }
  __device__ __forceinline__ void operator()(const SphBufs& Wb, int count) {
    for (int s = 0; s < count; ++s) {
      const float4 a = Wb.sa[s], b = Wb.sb[s];
      const float tx = th.x - a.x, ty = th.y - a.y, tz = th.z - a.z;
      const float nx = tx - sph_mi1(tx), ny = ty - sph_mi1(ty), nz = tz - sph_mi1(tz);  // rint, exact
      const float dx = (tx - nx) + (tl.x - b.x), dy = (ty - ny) + (tl.y - b.y), dz = (tz - nz) + (tl.z - b.z);
      const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
      if (r2 < hb2_32) {
        W->list[cnt][lane] = Wb.sj[s];
        W->img[cnt][lane] = (unsigned char)((int)nx + 1 + 3 * ((int)ny + 1) + 9 * ((int)nz + 1));
        ++cnt;
      }
      if (__any_sync(0xffffffffu, cnt == kSphList)) {
        __syncwarp();
        flush();
      }
    }
  }
};

__global__ void __launch_bounds__(kSphWarps * 32) k_sph_density(SphArgs A) {
  __shared__ int s_stack[kSphWarps][kSphStack];
  __shared__ int2 s_queue[kSphWarps][kSphQueue];
  __shared__ int s_list[kSphWarps][kSphList][32];
  __shared__ unsigned char s_img[kSphWarps][kSphList][32];
  __shared__ int s_qoff[kSphWarps][kSphQueue + 1];
  __shared__ float4 s_sa[kSphWarps][32];
  __shared__ float4 s_sb[kSphWarps][32];
  __shared__ int s_sj[kSphWarps][32];
  const TreeDev& T = A.T;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  if (T.sb->status != 0 || T.sb->magic != kMagicTree) {
    // a failed or missing tree: flag it and write NaN / -1 everywhere
    if (threadIdx.x == 0) set_status(A.wsb, ST_NOTREE);
    for (int64_t kk = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; kk < T.n;
         kk += (int64_t)gridDim.x * blockDim.x) {
      A.h_out[kk] = NAN;
      A.rho_out[kk] = NAN;
      A.ngb_out[kk] = -1;
    }
    return;
  }
  const int64_t g = (int64_t)blockIdx.x * kSphWarps + wib;
  if (g >= T.ngroups) return;
  SphBufs W;
  W.stack = s_stack[wib];
  W.queue = s_queue[wib];
  W.list = s_list[wib];
  W.img = s_img[wib];
  W.qoff = s_qoff[wib];
  W.sa = s_sa[wib];
  W.sb = s_sb[wib];
  W.sj = s_sj[wib];
  int nodes_total = 0;
  for (int l = 0; l < kLevels; ++l) nodes_total += T.sb->level_cnt[l];
  if (nodes_total > T.cap) nodes_total = (int)T.cap;

  const int64_t k = g * kGroup + lane;
  const bool valid = k < T.n;
  const int64_t kc = valid ? k : 0;
  const float4 pa = T.pA[kc], pb = T.pB[kc];
  const float3 th = make_float3(pa.x, pa.y, pa.z), tl = make_float3(pb.x, pb.y, pb.z);
  const float nngb = (float)A.n_ngb;

  // 1. start: the density of the smallest ancestor holding >= N_ngb particles
  float h = 0.5f;
  {
    int p = T.leaf_of[kc];
    for (int up = 0; up < kLevels + 1 && p >= 0 && p < nodes_total; ++up) {
      const int c = T.nD[p].y;
      if ((double)c >= A.n_ngb || T.nParent[p] < 0) {
        const float s = T.nC[p].w;
        h = s * cbrtf(3.0f * nngb / (4.0f * 3.14159265f * (float)c));
        break;
      }
      p = T.nParent[p];
    }
    h = fminf(fmaxf(h, 1e-7f), 0.5f);
  }

  // 2. FP32 Newton passes on ln h
  bool conv = !valid, fail = false;
  float blo = 0.f, bhi = 1e30f;
  uint32_t st = 0;
  for (int pass = 0; pass < kSphPass32 && __any_sync(0xffffffffu, !conv); ++pass) {
    const float Rl = conv ? 0.f : h;
    const float R = __int_as_float((int)__reduce_max_sync(0xffffffffu, (unsigned)__float_as_int(Rl)));
    SphEval32 ev;
    ev.th = th;
    ev.tl = tl;
    ev.ih2 = 1.0f / (h * h);
    ev.S0 = 0.f;
    ev.S1 = 0.f;
    st |= sph_gather(A, W, active_box(th, !conv), R, nodes_total, lane, ev);
    if (st) break;
    if (!conv) {
      const float N = (32.0f / 3.0f) * ev.S0;
      if (N < nngb) blo = h;
      else bhi = h;
      float dl;
      if (ev.S1 < 0.f) dl = (__logf(N) - __logf(nngb)) * ev.S0 / ev.S1;
      else dl = N >= nngb ? -0.7f : 0.7f;
      dl = fminf(fmaxf(dl, -0.7f), 0.7f);
      if (h >= 0.5f && N < nngb) {
        fail = true;  // no root below half the box
        conv = true;
      } else if (fabsf(dl) < kSphConv32) {
        // converged: take the Newton step itself (it may round to h, which
        // is a bracket end by now, so it is not tested against the bracket)
        h = fminf(h * __expf(dl), 0.5f);
        conv = true;
      } else {
        float hn = h * __expf(dl);
        if (blo > 0.f && bhi < 1e30f && !(hn > blo && hn < bhi)) hn = sqrtf(blo * bhi);
        if (hn > 0.5f) hn = 0.5f;
        conv = bhi < 1e30f && bhi - blo < 2e-6f * bhi;
        h = hn;
      }
    }
  }

  // 3. finishing pass(es): Newton step, density and neighbour count
  const double L = A.B.L;
  bool done = !valid || fail;
  double hd = (double)h * L;
  double lo64 = 0.0, hi64 = 0.0;  // FP64 bracket (hi64 = 0: none yet)
  double h_out = NAN, rho_out = NAN;
  int ngb_out = -1;
  for (int pass = 0; pass < kSphPass64 && !st && __any_sync(0xffffffffu, !done); ++pass) {
    SphEval64 ev;
    ev.A = &A;
    ev.W = &W;
    ev.lane = lane;
    ev.k = k;
    ev.th = th;
    ev.tl = tl;
    {
      const double v = (L * L) / (hd * hd);  // 1 / h^2 in box units, as a float-float
      ev.ih2.hi = (float)v;
      ev.ih2.lo = (float)(v - (double)ev.ih2.hi);
    }
    const float hb = (float)(hd * (1.0 + kSphBand) / L);
    ev.hb2_32 = done ? -1.f : hb * hb * 1.0001f + 1e-14f;
    ev.S0 = ev.R0 = 0.0;
    ev.S1 = ev.R1 = ev.C1 = ev.Q1 = 0.f;
    ev.S2 = ev.R2 = 0.f;
    ev.bq0 = ev.bq1 = 0.0;
    ev.clt = ev.band = ev.cnt = 0;
    const float Rl = done ? 0.f : hb;
    const float R = __int_as_float((int)__reduce_max_sync(0xffffffffu, (unsigned)__float_as_int(Rl)));
    st |= sph_gather(A, W, active_box(th, !done), R, nodes_total, lane, ev);
    if (st) break;
    ev.flush();
    if (!done) {
      // Second-order step in d = ln(h / hd): with q' = q e^-d,
      //   sum w(q') = S0 - d S1 + d^2 / 2 (S1 + S2) + O(d^3)
      // (S1 = sum q w', S2 = sum q^2 w''; the spline is C^2, and neighbours
      // entering or leaving the sphere add O(d^3)).  Solve (32/3) of it =
      // N_ngb by Newton steps on the quadratic; its error, ~20 d^3 of N_ngb,
      // is below 1e-9 for the accepted |d| <= kSphStep.
      const double N = (32.0 / 3.0) * ev.S0;
      if (N < A.n_ngb) lo64 = hd;
      else hi64 = hd;
      const double c0 = ev.S0 - (3.0 / 32.0) * A.n_ngb;
      const double s1 = (double)ev.S1 - (double)ev.C1, r1 = (double)ev.R1 - (double)ev.Q1;
      const double c1 = -s1, c2 = 0.5 * (s1 + (double)ev.S2);
      double d;
      if (c1 > 0.0) {
        d = -c0 / c1;
        for (int it = 0; it < 2; ++it) {
          const double den = c1 + 2.0 * c2 * d;
          if (den > 0.0) d -= (c0 + (c1 + c2 * d) * d) / den;
        }
      } else {
        d = N >= A.n_ngb ? -0.69 : 0.69;
      }
      double hn = hd * exp(d);
      const bool small = fabs(d) <= kSphStep;
      if (!small && hi64 > 0.0 && lo64 > 0.0 && !(hn > lo64 && hn < hi64)) hn = 0.5 * (lo64 + hi64);
      // with more than two band neighbours (their distances are not kept)
      // the step must be at the FP64 resolution: no neighbour then lies
      // between hd and hn short of an exact tie
      if (small && (ev.band <= 2 || fabs(d) <= 1e-12)) {
        // the step stays inside the band (kSphBand > kSphStep), so only band
        // neighbours can change side between hd and hn
        const double qn = hn / hd;
        int c = ev.clt;
        if (ev.band >= 1) c += (int)(ev.bq0 < qn) - (int)(ev.bq0 < 1.0);
        if (ev.band >= 2) c += (int)(ev.bq1 < qn) - (int)(ev.bq1 < 1.0);
        // rho at hn from sum m w to second order in d, as sum w above
        const double L2 = L * L;
        const double R0f = ev.R0 + (-d * r1 + 0.5 * d * d * (r1 + (double)ev.R2)) * L2;
        h_out = hn;
        rho_out = 8.0 * R0f / (M_PI * hn * hn * hn);
        ngb_out = c;
        done = true;
      } else {
        hd = hn > 0.5 * L ? 0.5 * L : hn;
      }
    }
  }
  if (st && lane == 0) set_status(A.wsb, st);
  if (valid) {
    if (!done || fail || st) {
      if (!st) set_status(A.wsb, ST_WALKCAP);
      h_out = NAN;
      rho_out = NAN;
      ngb_out = -1;
    }
    const int32_t i = T.order[k];
    A.h_out[i] = h_out;
    A.rho_out[i] = rho_out;
    A.ngb_out[i] = ngb_out;
  }
}

}  // namespace og

extern "C" {

size_t og_sph_ws_bytes(void) { return og::align_up(sizeof(og::StatusBlock)); }

og_status og_sph_density(const og_tree* t, double n_ngb, void* ws, size_t ws_bytes, double* h, double* rho,
                         int32_t* ngb, og_stream stream) {
  if (!t || !t->built || !t->mem) return OG_ETREE;
  if (!ws || !h || !rho || !ngb) return OG_EINVAL;
  if (!std::isfinite(n_ngb) || n_ngb <= 0.0) return OG_EINVAL;
  if ((reinterpret_cast<uintptr_t>(ws) % og::kAlign) != 0) return OG_EINVAL;
  if (ws_bytes < og_sph_ws_bytes()) return OG_ENOSPACE;
  if (t->node_capacity >= (int64_t(1) << 28)) return OG_EINVAL;  // node indices are packed in 28 bits
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  og::SphArgs A;
  A.T = og::tree_view(t);
  A.wsb = static_cast<og::StatusBlock*>(ws);
  A.B = og::box_scale(t->box);
  A.n_ngb = n_ngb;
  A.max_visits = t->max_walk_iters;
  A.h_out = h;
  A.rho_out = rho;
  A.ngb_out = ngb;
  if (cudaMemsetAsync(A.wsb, 0, sizeof(og::StatusBlock), s) != cudaSuccess) return OG_ECUDA;
  const int64_t grid = (t->n_groups + og::kSphWarps - 1) / og::kSphWarps;
  if (grid <= 0) return OG_OK;
  og::k_sph_density<<<(unsigned)grid, og::kSphWarps * 32, 0, s>>>(A);
  return cudaGetLastError() == cudaSuccess ? OG_OK : OG_ECUDA;
}

}  // extern "C"
