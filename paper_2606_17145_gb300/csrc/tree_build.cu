// tree_build.cu -- K3 permute, K4 level-by-level octree build, K5 walk groups.
//
// Nodes are stored level by level (level-major), so the children of a node are
// a contiguous range of the next level.  A node is a maximal run of sorted
// keys sharing the top 3*level bits; it is split (level < 21, more than
// leaf_size members) into the runs of its 8 possible next digits.
//
// Top-down topology: one launch per level.  Eight lanes serve one parent; lane
// d binary-searches the first key whose next digit is >= d inside the
// parent's range, so the child runs come out without touching every key.
// Child slots are taken per block with a single atomic on the level counter.
//
// Bottom-up moments: one launch per level, deepest first.  One thread serves
// one node and sums its children (or a leaf's particles) in FP64 in index
// order, so the result does not depend on scheduling.
#include "og_internal.cuh"

namespace og {


__global__ void k_permute(BuildArgs A, BoxScale B) {
  const TreeDev& T = A.T;
  const double invL2 = B.invL * B.invL;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < T.n; k += (int64_t)gridDim.x * blockDim.x) {
    const int32_t i = A.order[k];
    double w[3];
    float hi[3], lo[3];
    bool ok = true;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const double x = A.pos[3 * (int64_t)i + c];
      ok = ok && finite_bits(x);
      w[c] = wrap_coord(x, B);
      split_box(w[c], B, hi[c], lo[c]);
      T.x64[3 * k + c] = w[c];
    }
    const double m = A.mass[i];
    const double eps = A.eps ? A.eps[i] : A.eps_scalar;
    if (!(ok && positive_finite_bits(m) && positive_finite_bits(eps))) set_status(T.sb, ST_BADINPUT);
    const double h = 2.8 * eps;
    T.m64[k] = m;
    T.h64[k] = h;
    T.order[k] = i;
    // m / L^2 and (h / L)^2 in FP32.  For a power-of-two side with 2^-2e an
    // exact double (invL2 then equals it), m invL2 = m 2^-2e and
    // (h invL)^2 = (h h) 2^-2e wherever the FP32 result is normal, and the
    // rounding to FP32 is done on the integer pipe.
    const bool sq = B.pow2 && B.e >= -511 && B.e <= 537;
    float mw, h2;
    if (!(sq && d2f_scaled((uint64_t)__double_as_longlong(m), 2 * B.e, mw))) mw = (float)(m * invL2);
    const double hh = h * h;
    if (!(sq && d2f_scaled((uint64_t)__double_as_longlong(hh), 2 * B.e, h2))) {
      const double hb = h * B.invL;
      h2 = (float)(hb * hb);
    }
    T.pA[k] = make_float4(hi[0], hi[1], hi[2], mw);
    T.pB[k] = make_float4(lo[0], lo[1], lo[2], h2);
  }
}

__global__ void k_groups(TreeDev T, BoxScale B) {
  // Wrapped positions are non-negative doubles, which order like their bit
  // patterns, and division by L is monotonic: the box in box units is the
  // division of the integer min / max.
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < T.ngroups; g += (int64_t)gridDim.x * blockDim.x) {
    long long lo[3] = {0x7fffffffffffffffll, 0x7fffffffffffffffll, 0x7fffffffffffffffll};
    long long hi[3] = {0, 0, 0};
    const int64_t a = g * kGroup, b = (T.n < a + kGroup ? T.n : a + kGroup);
    for (int64_t k = a; k < b; ++k)
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const long long x = __double_as_longlong(T.x64[3 * k + c]);
        lo[c] = x < lo[c] ? x : lo[c];
        hi[c] = x > hi[c] ? x : hi[c];
      }
    float fl[3], fh[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      fl[c] = __double2float_rd(div_box(__longlong_as_double(lo[c]), B));
      fh[c] = __double2float_ru(div_box(__longlong_as_double(hi[c]), B));
    }
    T.gbox[2 * g] = make_float4(fl[0], fl[1], fl[2], 0.f);
    T.gbox[2 * g + 1] = make_float4(fh[0], fh[1], fh[2], 0.f);
  }
}

__global__ void k_root(TreeDev T, int leaf_size) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    T.sb->magic = kMagicTree;
    for (int l = 0; l < 24; ++l) T.sb->level_cnt[l] = 0;
    T.sb->level_cnt[0] = 1;
    const int leaf = (T.n <= leaf_size) ? 1 : 0;
    T.nD[0] = make_int4(0, (int)T.n, -1, make_meta(0, 0, leaf));
    T.nParent[0] = -1;
  }
}

__device__ __forceinline__ int level_base(const StatusBlock* sb, int level) {
  int b = 0;
  for (int l = 0; l < level; ++l) b += sb->level_cnt[l];
  return b;
}

// Expand level `lev` into level lev + 1.  256 threads = 32 parents per step.
__global__ void __launch_bounds__(256) k_expand(TreeDev T, const uint64_t* __restrict__ keys, int lev, int leaf_size) {
  __shared__ int s_cnt[32];
  __shared__ int s_base;
  const int base = level_base(T.sb, lev);
  const int cnt = T.sb->level_cnt[lev];
  const int next_base = base + cnt;
  if (next_base > T.cap) return;  // capacity exceeded at an upper level (flagged there)
  const int lane = threadIdx.x & 31;
  const int sub = lane & 7;                      // digit handled by this lane
  const int slot = threadIdx.x >> 3;             // parent slot in the block (0..31)
  const int shift = 63 - 3 * (lev + 1);
  for (int step = blockIdx.x * 32; step < cnt; step += gridDim.x * 32) {
    const int p = base + step + slot;
    const bool live = (step + slot) < cnt;
    int4 D = make_int4(0, 0, -1, 0);
    bool split = false;
    if (live) {
      D = T.nD[p];
      split = !meta_leaf(D.w);
    }
    int start = 0, end = 0;
    if (split) {
      // first index in [f, f + c) whose digit at level lev+1 is >= sub
      int lo = D.x, hi = D.x + D.y;
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        const uint32_t dg = (uint32_t)((keys[mid] >> shift) & 7u);
        if (dg < (uint32_t)sub) lo = mid + 1; else hi = mid;
      }
      start = lo;
    }
    const int nxt = __shfl_down_sync(0xffffffffu, start, 1, 8);
    end = (sub == 7) ? D.x + D.y : nxt;
    const bool has = split && end > start;
    const uint32_t seg = (__ballot_sync(0xffffffffu, has) >> (lane & 24)) & 0xffu;
    const int nchild = __popc(seg);
    const int rank = __popc(seg & ((1u << sub) - 1u));
    // block-wide allocation of child slots
    if (sub == 0) s_cnt[slot] = split ? nchild : 0;
    __syncthreads();
    if (threadIdx.x == 0) {
      int run = 0;
      for (int s2 = 0; s2 < 32; ++s2) {
        const int c = s_cnt[s2];
        s_cnt[s2] = run;
        run += c;
      }
      s_base = run ? atomicAdd(&T.sb->level_cnt[lev + 1], run) : 0;
    }
    __syncthreads();
    const int child_first = next_base + s_base + s_cnt[slot];
    if (split) {
      const bool fits = child_first + nchild <= T.cap;
      if (!fits) {
        if (sub == 0) set_status(T.sb, ST_NOSPACE);
      } else {
        if (has) {
          const int c = child_first + rank;
          const int ccount = end - start;
          const int leaf = (ccount <= leaf_size || lev + 1 >= kMaxLevel) ? 1 : 0;
          T.nD[c] = make_int4(start, ccount, -1, make_meta(0, lev + 1, leaf));
          T.nParent[c] = p;
        }
        if (sub == 0) {
          D.z = child_first;
          D.w = make_meta(nchild, lev, 0);
          T.nD[p] = D;
        }
      }
    }
    __syncthreads();
  }
}

// Bottom-up moments for one level, one thread per node.  A leaf sums its
// particles and an internal node its children, in index order; then the
// node's centre of mass, split FP32 copies and cube centre are written.  On
// this GPU an FP64 warp instruction costs the same however many lanes are
// active, so giving each lane its own node (rather than spreading one node
// over several lanes) minimises FP64 instructions per node.
__global__ void __launch_bounds__(256) k_moments(TreeDev T, int lev, BoxScale B) {
  const int base = level_base(T.sb, lev);
  const int cnt = T.sb->level_cnt[lev];
  if (base + cnt > T.cap) return;  // capacity already exceeded (flagged by k_expand)
  const double side = ldexp(B.L, -lev);
  const float side_b = ldexpf(1.0f, -lev);
  const double invL = B.invL, invL2 = B.invL * B.invL;
  for (int step = blockIdx.x * blockDim.x + threadIdx.x; step < cnt; step += gridDim.x * blockDim.x) {
    const int p = base + step;
    const int4 D = T.nD[p];
    double M = 0.0, S0 = 0.0, S1 = 0.0, S2 = 0.0;
    // hmax as an integer max of the bit patterns: softenings are positive
    // (checked by k_permute), and positive doubles order like their bits
    long long Hb = 0;
    if (meta_leaf(D.w)) {
      for (int j = D.x; j < D.x + D.y; ++j) {
        const double m = T.m64[j];
        M += m;
        S0 += m * T.x64[3 * (int64_t)j];
        S1 += m * T.x64[3 * (int64_t)j + 1];
        S2 += m * T.x64[3 * (int64_t)j + 2];
        Hb = max(Hb, __double_as_longlong(T.h64[j]));
        T.leaf_of[j] = p;
      }
    } else {
      const int c1 = D.z + meta_nchild(D.w);
      for (int c = D.z; c < c1; ++c) {
        M += T.mass64[c];
        S0 += T.S64[3 * (int64_t)c];
        S1 += T.S64[3 * (int64_t)c + 1];
        S2 += T.S64[3 * (int64_t)c + 2];
        Hb = max(Hb, __double_as_longlong(T.hmax64[c]));
      }
    }
    const double H = __longlong_as_double(Hb);
    const double invM = 1.0 / M;
    const double com[3] = {S0 * invM, S1 * invM, S2 * invM};
    float hi[3], lo[3];
    double cen[3];
    float cenb[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      if (!(B.pow2 && split_bits((uint64_t)__double_as_longlong(com[c]), B.e, hi[c], lo[c])))
        split_coord(com[c] * invL, hi[c], lo[c]);
      const uint32_t q = quantise(T.x64[3 * (int64_t)D.x + c], B) >> (kMaxLevel - lev);
      // (q + 1/2) side, exact for a power-of-two box: (2q + 1) 2^(e - lev - 1)
      if (!(B.pow2 && double_odd_scaled(2u * q + 1u, B.e - lev - 1, cen[c]))) cen[c] = __dmul_rn((double)q + 0.5, side);
      cenb[c] = ((float)q + 0.5f) * side_b;
    }
    // M / L^2 and (hmax / L)^2 in FP32, as in k_permute
    const bool sq = B.pow2 && B.e >= -511 && B.e <= 537;
    float mw, h2;
    if (!(sq && d2f_scaled((uint64_t)__double_as_longlong(M), 2 * B.e, mw))) mw = (float)(M * invL2);
    const double HH = H * H;
    if (!(sq && d2f_scaled((uint64_t)__double_as_longlong(HH), 2 * B.e, h2))) {
      const double hb = H * invL;
      h2 = (float)(hb * hb);
    }
    T.mass64[p] = M;
    T.hmax64[p] = H;
    T.S64[3 * (int64_t)p] = S0;
    T.S64[3 * (int64_t)p + 1] = S1;
    T.S64[3 * (int64_t)p + 2] = S2;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      T.com64[3 * (int64_t)p + c] = com[c];
      T.cen64[3 * (int64_t)p + c] = cen[c];
    }
    T.nA[p] = make_float4(hi[0], hi[1], hi[2], mw);
    T.nB[p] = make_float4(lo[0], lo[1], lo[2], h2);
    T.nC[p] = make_float4(cenb[0], cenb[1], cenb[2], side_b);
  }
}

cudaError_t launch_tree_build(const BuildArgs& A, cudaStream_t s) {
  const TreeDev& T = A.T;
  int64_t grid = (T.n + 255) / 256;
  if (grid > grid_cap(32)) grid = grid_cap(32);
  const BoxScale B = box_scale(A.L);
  k_permute<<<(unsigned)grid, 256, 0, s>>>(A, B);
  int64_t ggrid = (T.ngroups + 127) / 128;
  if (ggrid > grid_cap(16)) ggrid = grid_cap(16);
  k_groups<<<(unsigned)ggrid, 128, 0, s>>>(T, B);
  k_root<<<1, 32, 0, s>>>(T, A.leaf_size);
  // Grids are fixed (the per-level node count lives on the device); blocks
  // stride over the level.
  const unsigned egrid = grid_cap(8);
  for (int lev = 0; lev < kMaxLevel; ++lev) k_expand<<<egrid, 256, 0, s>>>(T, A.keys, lev, A.leaf_size);
  for (int lev = kMaxLevel; lev >= 0; --lev) k_moments<<<egrid, 256, 0, s>>>(T, lev, B);
  return cudaGetLastError();
}

__global__ void k_copy_nodes(TreeDev T, int64_t m, int32_t* level, int32_t* first, int32_t* count, int32_t* parent,
                             double* mass, double* com, double* hmax, int32_t* child_first, int32_t* nchild) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < m; p += (int64_t)gridDim.x * blockDim.x) {
    const int4 D = T.nD[p];
    if (level) level[p] = meta_level(D.w);
    if (first) first[p] = D.x;
    if (count) count[p] = D.y;
    if (parent) parent[p] = T.nParent[p];
    if (mass) mass[p] = T.mass64[p];
    if (com)
      for (int c = 0; c < 3; ++c) com[3 * p + c] = T.com64[3 * p + c];
    if (hmax) hmax[p] = T.hmax64[p];
    if (child_first) child_first[p] = meta_leaf(D.w) ? -1 : D.z;
    if (nchild) nchild[p] = meta_leaf(D.w) ? 0 : meta_nchild(D.w);
  }
}

cudaError_t launch_copy_nodes(const TreeDev& T, int64_t m, int32_t* level, int32_t* first, int32_t* count,
                              int32_t* parent, double* mass, double* com, double* hmax, int32_t* child_first,
                              int32_t* nchild, cudaStream_t s) {
  if (m <= 0) return cudaSuccess;
  int64_t grid = (m + 255) / 256;
  if (grid > grid_cap(16)) grid = grid_cap(16);
  k_copy_nodes<<<(unsigned)grid, 256, 0, s>>>(T, m, level, first, count, parent, mass, com, hmax, child_first,
                                              nchild);
  return cudaGetLastError();
}

}  // namespace og
