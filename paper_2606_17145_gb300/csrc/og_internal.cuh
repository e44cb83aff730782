// og_internal.cuh -- device-side layout and helpers shared by the CUDA kernels
// of libog.so (not part of the public ABI; see include/og.h).
#pragma once

#include <cmath>
#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

#include "../../include/og.h"
#include "split_coord.cuh"

namespace og {

// Device status bits (OR-ed into the status word of a buffer).
enum : uint32_t {
  ST_BADINPUT = 1u << 0,   // non-finite position
  ST_NOSPACE = 1u << 1,    // node capacity exceeded
  ST_WALKCAP = 1u << 2,    // walk iteration cap
  ST_STACK = 1u << 3,      // traversal stack overflow
  ST_TREELINK = 1u << 4,   // out-of-range node / particle index
  ST_NOTREE = 1u << 5,     // tree status was not clean when the walk started
};

constexpr int kMaxLevel = 21;         // 21 bits per axis
constexpr int kLevels = kMaxLevel + 1;
constexpr int kGroup = 32;            // targets per walk group (one warp)
constexpr size_t kAlign = 256;

// The first 256 bytes of every buffer the library carves.
struct StatusBlock {
  uint32_t status;
  uint32_t magic;
  int32_t level_cnt[24];              // nodes per level (tree buffers)
  unsigned long long counter;         // interaction count / misc
  unsigned long long work;            // dynamic work counter
  int32_t pad[20];
};
static_assert(sizeof(StatusBlock) <= kAlign, "status block fits 256 bytes");

constexpr uint32_t kMagicTree = 0x0637ee01u;
constexpr uint32_t kMagicWs = 0x0637ee02u;

__host__ __device__ inline size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

// Node meta word: nchild (bits 0-7) | level (bits 8-15) | leaf (bit 16).
__host__ __device__ inline int meta_nchild(int m) { return m & 0xff; }
__host__ __device__ inline int meta_level(int m) { return (m >> 8) & 0xff; }
__host__ __device__ inline int meta_leaf(int m) { return (m >> 16) & 1; }
__host__ __device__ inline int make_meta(int nchild, int level, int leaf) {
  return (nchild & 0xff) | ((level & 0xff) << 8) | ((leaf & 1) << 16);
}

// Device view of a tree buffer.  Positions in the FP32 path are in box units
// (xi = x / L) stored as a split float: hi is a multiple of 2^-23 (so hi +/- 1
// and hi_i - hi_j are exact) and lo = xi - hi (|lo| <= 2^-24).
struct TreeDev {
  StatusBlock* sb;
  int64_t n, cap, ngroups;
  double box;
  int leaf_size;
  // particles, Hilbert order
  float4* pA;      // (hi.x, hi.y, hi.z, m / L^2)
  float4* pB;      // (lo.x, lo.y, lo.z, h / L)
  double* x64;     // [n][3] wrapped physical positions
  double* m64;     // [n]
  double* h64;     // [n] softening support h = 2.8 eps
  int32_t* order;  // [n] sorted -> original index
  int32_t* leaf_of;// [n] leaf node of each sorted particle
  // groups of 32
  float4* gbox;    // [2 * ngroups]: min (xyz), max (xyz) in box units, rounded outward
  // nodes
  float4* nA;      // (com_hi xyz, M / L^2)
  float4* nB;      // (com_lo xyz, hmax / L)
  float4* nC;      // (centre xyz, side) in box units (exact)
  int4* nD;        // (first, count, child_first, meta)
  int32_t* nParent;
  double* com64;   // [cap][3]
  double* S64;     // [cap][3] first moments sum(m x)
  double* mass64;  // [cap]
  double* hmax64;  // [cap]
  double* cen64;   // [cap][3] physical geometric centres
};

// Carves a tree buffer.  Returns the total byte count (buf may be null).
inline size_t carve_tree(void* buf, int64_t n, int64_t cap, TreeDev* T) {
  size_t off = 0;
  char* b = static_cast<char*>(buf);
  auto take = [&](size_t bytes) -> void* {
    void* p = b ? b + off : nullptr;
    off = align_up(off + bytes);
    return p;
  };
  int64_t G = (n + kGroup - 1) / kGroup;
  TreeDev t{};
  t.sb = static_cast<StatusBlock*>(take(sizeof(StatusBlock)));
  t.n = n;
  t.cap = cap;
  t.ngroups = G;
  t.pA = static_cast<float4*>(take(sizeof(float4) * n));
  t.pB = static_cast<float4*>(take(sizeof(float4) * n));
  t.x64 = static_cast<double*>(take(sizeof(double) * 3 * n));
  t.m64 = static_cast<double*>(take(sizeof(double) * n));
  t.h64 = static_cast<double*>(take(sizeof(double) * n));
  t.order = static_cast<int32_t*>(take(sizeof(int32_t) * n));
  t.leaf_of = static_cast<int32_t*>(take(sizeof(int32_t) * n));
  t.gbox = static_cast<float4*>(take(sizeof(float4) * 2 * G));
  t.nA = static_cast<float4*>(take(sizeof(float4) * cap));
  t.nB = static_cast<float4*>(take(sizeof(float4) * cap));
  t.nC = static_cast<float4*>(take(sizeof(float4) * cap));
  t.nD = static_cast<int4*>(take(sizeof(int4) * cap));
  t.nParent = static_cast<int32_t*>(take(sizeof(int32_t) * cap));
  t.com64 = static_cast<double*>(take(sizeof(double) * 3 * cap));
  t.S64 = static_cast<double*>(take(sizeof(double) * 3 * cap));
  t.mass64 = static_cast<double*>(take(sizeof(double) * cap));
  t.hmax64 = static_cast<double*>(take(sizeof(double) * cap));
  t.cen64 = static_cast<double*>(take(sizeof(double) * 3 * cap));
  if (T) *T = t;
  return off;
}

inline TreeDev tree_view(const og_tree* t) {
  TreeDev T;
  carve_tree(t->mem, t->n, t->node_capacity, &T);
  T.box = t->box;
  T.leaf_size = t->leaf_size;
  return T;
}

// Keys-sort workspace.
struct SortWs {
  StatusBlock* sb;
  uint64_t* keys_alt;
  int32_t* vals_alt;
  uint32_t* hist;       // [256][nblk]
  uint32_t* digit_tot;  // [256]
  int64_t nblk;
};

constexpr int kSortThreads = 256;
constexpr int kSortItems = 8;
constexpr int kSortTile = kSortThreads * kSortItems;  // 2048 keys per block

inline size_t carve_sort(void* buf, int64_t n, SortWs* W) {
  size_t off = 0;
  char* b = static_cast<char*>(buf);
  auto take = [&](size_t bytes) -> void* {
    void* p = b ? b + off : nullptr;
    off = align_up(off + bytes);
    return p;
  };
  SortWs w{};
  w.nblk = (n + kSortTile - 1) / kSortTile;
  w.sb = static_cast<StatusBlock*>(take(sizeof(StatusBlock)));
  w.keys_alt = static_cast<uint64_t*>(take(sizeof(uint64_t) * n));
  w.vals_alt = static_cast<int32_t*>(take(sizeof(int32_t) * n));
  w.hist = static_cast<uint32_t*>(take(sizeof(uint32_t) * 256 * w.nblk));
  w.digit_tot = static_cast<uint32_t*>(take(sizeof(uint32_t) * 256));
  if (W) *W = w;
  return off;
}

// Adjoint workspace.
struct AdjWs {
  StatusBlock* sb;
  double* Gn;    // [cap][3] per-node sum of J w
  double* Sn;    // [cap]    per-node sum of w . g
  double* Gp;    // [n][3]   per-particle (particle-particle source terms)
  double* Sp;    // [n]
  double* tgt;   // [n][3]   target-side gradient (sorted order)
  double* CG;    // [cap][3] cumulative G from the root
  double* Bn;    // [cap]    cumulative affine term at the node centre
};

inline size_t carve_adj(void* buf, int64_t n, int64_t cap, AdjWs* W) {
  size_t off = 0;
  char* b = static_cast<char*>(buf);
  auto take = [&](size_t bytes) -> void* {
    void* p = b ? b + off : nullptr;
    off = align_up(off + bytes);
    return p;
  };
  AdjWs w{};
  w.sb = static_cast<StatusBlock*>(take(sizeof(StatusBlock)));
  w.Gn = static_cast<double*>(take(sizeof(double) * 3 * cap));
  w.Sn = static_cast<double*>(take(sizeof(double) * cap));
  w.Gp = static_cast<double*>(take(sizeof(double) * 3 * n));
  w.Sp = static_cast<double*>(take(sizeof(double) * n));
  w.tgt = static_cast<double*>(take(sizeof(double) * 3 * n));
  w.CG = static_cast<double*>(take(sizeof(double) * 3 * cap));
  w.Bn = static_cast<double*>(take(sizeof(double) * cap));
  if (W) *W = w;
  return off;
}

__device__ inline void set_status(StatusBlock* sb, uint32_t bits) { atomicOr(&sb->status, bits); }

// Finite: exponent field not all ones.  Positive and finite: the bits, as an
// unsigned integer, lie in [1, 0x7fefffffffffffff].  (Integer tests: the FP64
// pipe is the scarce one.)
__device__ __forceinline__ bool finite_bits(double x) {
  return ((uint64_t)__double_as_longlong(x) & 0x7ff0000000000000ull) != 0x7ff0000000000000ull;
}
__device__ __forceinline__ bool positive_finite_bits(double x) {
  return (uint64_t)__double_as_longlong(x) - 1ull < 0x7fefffffffffffffull;
}

// Split a box-unit coordinate xi in [0, 1] into (hi, lo): hi = k 2^-23 with
// k = rint(xi 2^23), lo = xi - hi rounded to FP32.  This is the definition;
// split_coord takes the integer form where it applies.
__device__ inline void split_coord_f64(double xi, float& hi, float& lo) {
  double k = rint(xi * 8388608.0);
  double h = k * (1.0 / 8388608.0);
  hi = static_cast<float>(h);
  lo = static_cast<float>(xi - h);
}

__device__ inline void split_coord(double xi, float& hi, float& lo) {
  if (!split_bits((uint64_t)__double_as_longlong(xi), 0, hi, lo)) split_coord_f64(xi, hi, lo);
}

// Division by the box side.  When L is a power of two, x / L equals
// x * (1 / L) exactly (both are the correctly rounded value of x 2^-e), so the
// multiply is used; any other L takes the IEEE division.
struct BoxScale {
  double L, invL;
  int pow2;
  int e;  // L = 2^e when pow2
};

inline BoxScale box_scale(double L) {
  int e = 0;
  const double m = std::frexp(L, &e);  // L = m 2^e, m in [0.5, 1)
  return BoxScale{L, 1.0 / L, m == 0.5 ? 1 : 0, e - 1};
}

__device__ inline double div_box(double x, const BoxScale& B) {
  return B.pow2 ? __dmul_rn(x, B.invL) : __ddiv_rn(x, B.L);
}

// (hi, lo) of x / L.  For a power-of-two side, x / L = x 2^-e exactly where
// it is normal, so the integer split reads the bits of x itself.
__device__ inline void split_box(double x, const BoxScale& B, float& hi, float& lo) {
  if (B.pow2 && split_bits((uint64_t)__double_as_longlong(x), B.e, hi, lo)) return;
  split_coord(div_box(x, B), hi, lo);
}

// Periodic wrap into [0, L]: x - L floor(x / L), each operation rounded once
// (no fused multiply-add: the result must be bit-identical to the host form).
__device__ inline double wrap_coord(double x, const BoxScale& B) {
  // power-of-two side and 0 < x < L: x / L is exact and below 1, so the
  // general form returns x itself.  Positive doubles order like their bit
  // patterns, so the range test needs no FP64 compare.
  const long long xb = __double_as_longlong(x);
  if (B.pow2 && xb > 0 && xb < __double_as_longlong(B.L)) return x;
  double fl = floor(div_box(x, B));
  double prod = __dmul_rn(B.L, fl);
  return __dsub_rn(x, prod);
}

__device__ inline uint32_t quantise(double w, const BoxScale& B) {
  if (B.pow2) {
    // w (2^21 / L) = w 2^(21 - e) is exact for a power-of-two side, so its
    // floor is the integer part of the mantissa shifted by the exponent
    const long long wb = __double_as_longlong(w);
    if (wb <= 0) return 0u;                       // +-0 (and negatives)
    const int E = (int)((wb >> 52) & 0x7ff);
    if (E == 0) return 0u;                        // subnormal: far below one cell
    const int sh = E - 1023 + 21 - B.e;           // w 2^(21-e) = 1.f 2^sh
    if (sh < 0) return 0u;
    if (sh >= 21) return 2097151u;                // w >= L: clamp (w is finite here)
    const unsigned long long mant = ((unsigned long long)wb & 0x000fffffffffffffull) | 0x0010000000000000ull;
    return (uint32_t)(mant >> (52 - sh));
  }
  double t = __dmul_rn(div_box(w, B), 2097152.0);
  double fl = floor(t);
  if (fl < 0.0) return 0u;
  if (fl > 2097151.0) return 2097151u;
  return static_cast<uint32_t>(fl);
}

// Arguments of the tree build launches.
struct BuildArgs {
  TreeDev T;
  const uint64_t* keys;
  const int32_t* order;
  const double* pos;
  const double* mass;
  const double* eps;
  double eps_scalar;
  double L;
  int leaf_size;
};

// Arguments of the walk kernels (forward FP32 / FP64, adjoint FP32).
struct WalkArgs {
  TreeDev T;
  StatusBlock* wsb;
  long long max_iters;
  int deep;                    // stack depth above which a step pops one range (<= the compiled bound)
  int64_t g_begin, g_end;      // walk groups [g_begin, g_end) (a key range of targets)
  // FP32, box units
  float rc2, rc2_lo, rc2_hi;   // node tests: rcut^2 and its relative band
  float pp_lo, pp_hi;          // pair cut band
  float th2_lo, th2_hi;        // theta^2 (1 -+ band)
  float lim_lo, lim_hi;        // 0.6 (1 -+ band): containment test
  float grp_rc2;               // group prune threshold (conservative)
  float uni_lim;               // bound for a warp-uniform periodic image
  float t_scale;               // t = r * t_scale - 1  (= u / 1.125 - 1)
  float ex2c;                  // exp(-u^2) = ex2(r2 * ex2c)
  float fp_c;                  // f'(r)/r = fp_c * r * exp(-u^2)
  // FP64, physical units (exact re-checks, FP64 walk)
  double rc2_64, th2_64, box, r_s64, inv2rs64, fp_c64;
  // outputs
  float* accf;
  double* accd;
  int32_t* counts;
  unsigned long long* total;
  // adjoint
  const float* w;
  double* Gn;
  double* Sn;
  double* Gp;
  double* Sp;
  double* tgt;
};

// SM count of the current device (0 on error); grids are sized from it.
int device_sm_count();

// Grid cap: per_sm blocks on every SM of the current device.
inline unsigned grid_cap(int per_sm) {
  const int s = device_sm_count();
  return (unsigned)((s > 0 ? s : 1) * per_sm);
}

cudaError_t launch_keys_sort(const double* pos, int64_t n, double L, uint64_t* keys_out, int32_t* order_out,
                             const SortWs& W, cudaStream_t s);
cudaError_t launch_tree_build(const BuildArgs& A, cudaStream_t s);
// fused (with adjoint): the adjoint walk that also writes accf, counts and
// the interaction total from the same pair evaluations
cudaError_t launch_walk(const WalkArgs& A, int prec, bool adjoint, cudaStream_t s, bool fused = false);
cudaError_t launch_adjoint_push(const TreeDev& T, const AdjWs& W, double L, double* dpos, double* dmass,
                                cudaStream_t s);
cudaError_t launch_copy_nodes(const TreeDev& T, int64_t m, int32_t* level, int32_t* first, int32_t* count,
                              int32_t* parent, double* mass, double* com, double* hmax, int32_t* child_first,
                              int32_t* nchild, cudaStream_t s);

}  // namespace og
