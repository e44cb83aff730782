// keys_sort.cu -- K1 Peano-Hilbert keys and K2 stable LSD radix sort.
//
// K1: one thread per particle.  Position wrap and quantisation use explicitly
// rounded FP64 operations (no contraction) so the integer cell is a pure
// function of the input bits.  The 3-D Hilbert index follows Skilling's
// transpose construction (J. Skilling, "Programming the Hilbert curve", 2004):
// from the most significant bit down, the low bits of axis 0 are inverted or
// exchanged with those of axis i; the axes are then Gray-coded against one
// another and a running parity of the last axis is folded in.  Here the
// parity fold is a bit-parallel suffix XOR and the final interleave uses
// magic-mask bit spreading.
//
// K2: 8 passes of 8-bit digits (63-bit keys).  Each pass is a per-tile digit
// histogram, a per-digit scan over tiles, and a stable scatter that ranks
// equal digits with warp match masks, stages the tile in shared memory in
// digit order and writes contiguous runs.  Stability of every pass gives the
// (key, original index) order.  HBM-bound: ~32 B per key per pass.
#include "og_internal.cuh"

namespace og {

__device__ __forceinline__ uint64_t spread3(uint32_t v) {
  uint64_t x = v & 0x1fffffu;
  x = (x | (x << 32)) & 0x001f00000000ffffull;
  x = (x | (x << 16)) & 0x001f0000ff0000ffull;
  x = (x | (x << 8)) & 0x100f00f00f00f00full;
  x = (x | (x << 4)) & 0x10c30c30c30c30c3ull;
  x = (x | (x << 2)) & 0x1249249249249249ull;
  return x;
}

__device__ __forceinline__ uint64_t hilbert63(uint32_t a, uint32_t b, uint32_t c) {
#pragma unroll
  for (int bit = 20; bit >= 1; --bit) {
    const uint32_t top = 1u << bit;
    const uint32_t low = top - 1u;
    if (a & top) a ^= low;
    if (b & top) {
      a ^= low;
    } else {
      const uint32_t t = (a ^ b) & low;
      a ^= t;
      b ^= t;
    }
    if (c & top) {
      a ^= low;
    } else {
      const uint32_t t = (a ^ c) & low;
      a ^= t;
      c ^= t;
    }
  }
  b ^= a;
  c ^= b;
  // bit p of par = XOR of the bits of c at positions p+1 .. 20
  uint32_t par = (c & 0x1ffffeu) >> 1;
  par ^= par >> 1;
  par ^= par >> 2;
  par ^= par >> 4;
  par ^= par >> 8;
  par ^= par >> 16;
  a ^= par;
  b ^= par;
  c ^= par;
  return (spread3(a) << 2) | (spread3(b) << 1) | spread3(c);
}

__global__ void k_keys(const double* __restrict__ pos, int64_t n, BoxScale B, uint64_t* __restrict__ keys,
                       int32_t* __restrict__ vals, StatusBlock* sb) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double x0 = pos[3 * i], x1 = pos[3 * i + 1], x2 = pos[3 * i + 2];
    uint64_t key = 0;
    if (finite_bits(x0) && finite_bits(x1) && finite_bits(x2)) {
      const uint32_t q0 = quantise(wrap_coord(x0, B), B);
      const uint32_t q1 = quantise(wrap_coord(x1, B), B);
      const uint32_t q2 = quantise(wrap_coord(x2, B), B);
      key = hilbert63(q0, q1, q2);
    } else {
      set_status(sb, ST_BADINPUT);
    }
    keys[i] = key;
    vals[i] = static_cast<int32_t>(i);
  }
}

// Exclusive scan of one value per thread over a block of 256 threads.
__device__ __forceinline__ uint32_t block_exscan256(uint32_t v, uint32_t* s_warp, uint32_t* total) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  uint32_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_warp[w] = x;
  __syncthreads();
  if (w == 0) {
    uint32_t t = lane < 8 ? s_warp[lane] : 0u;
#pragma unroll
    for (int o = 1; o < 8; o <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += y;
    }
    if (lane < 8) s_warp[lane] = t;  // inclusive
  }
  __syncthreads();
  const uint32_t warp_off = w ? s_warp[w - 1] : 0u;
  if (total) *total = s_warp[7];
  const uint32_t r = warp_off + x - v;
  __syncthreads();
  return r;
}

__global__ void __launch_bounds__(kSortThreads) k_sort_hist(const uint64_t* __restrict__ keys, int64_t n, int shift,
                                                            uint32_t* __restrict__ hist, int64_t nblk) {
  __shared__ uint32_t h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  const int64_t base = blockIdx.x * (int64_t)kSortTile;
#pragma unroll
  for (int k = 0; k < kSortItems; ++k) {
    const int64_t idx = base + k * kSortThreads + threadIdx.x;
    if (idx < n) atomicAdd(&h[(keys[idx] >> shift) & 255u], 1u);
  }
  __syncthreads();
  hist[threadIdx.x * nblk + blockIdx.x] = h[threadIdx.x];
}

// One block per digit: exclusive scan over tiles, in place; digit total out.
__global__ void __launch_bounds__(1024) k_sort_scan(uint32_t* hist, int64_t nblk, uint32_t* digit_tot) {
  __shared__ uint32_t s_w[32];
  __shared__ uint32_t s_carry;
  uint32_t* row = hist + blockIdx.x * nblk;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (threadIdx.x == 0) s_carry = 0;
  __syncthreads();
  for (int64_t base = 0; base < nblk; base += 1024) {
    const int64_t i = base + threadIdx.x;
    const uint32_t v = i < nblk ? row[i] : 0u;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) s_w[w] = x;
    __syncthreads();
    if (w == 0) {
      uint32_t t = s_w[lane];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, t, o);
        if (lane >= o) t += y;
      }
      s_w[lane] = t;
    }
    __syncthreads();
    const uint32_t carry = s_carry;
    const uint32_t excl = carry + (w ? s_w[w - 1] : 0u) + x - v;
    if (i < nblk) row[i] = excl;
    __syncthreads();
    if (threadIdx.x == 0) s_carry = carry + s_w[31];
    __syncthreads();
  }
  if (threadIdx.x == 0) digit_tot[blockIdx.x] = s_carry;
}

__global__ void __launch_bounds__(kSortThreads) k_sort_scatter(const uint64_t* __restrict__ kin,
                                                               const int32_t* __restrict__ vin, int64_t n, int shift,
                                                               const uint32_t* __restrict__ hist, int64_t nblk,
                                                               const uint32_t* __restrict__ digit_tot,
                                                               uint64_t* __restrict__ kout, int32_t* __restrict__ vout) {
  __shared__ uint32_t s_wcnt[kSortThreads / 32][256];
  __shared__ uint32_t s_tile_start[256];
  __shared__ uint32_t s_gbase[256];
  __shared__ uint32_t s_scan[8];
  __shared__ uint64_t s_keys[kSortTile];
  __shared__ int32_t s_vals[kSortTile];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t base = blockIdx.x * (int64_t)kSortTile;
  const int tile_n = (int)((n - base) < kSortTile ? (n - base) : kSortTile);
  for (int i = threadIdx.x; i < (kSortThreads / 32) * 256; i += kSortThreads) (&s_wcnt[0][0])[i] = 0u;
  __syncthreads();

  uint64_t key[kSortItems];
  int32_t val[kSortItems];
  uint32_t rank[kSortItems];
  const uint32_t lt = (1u << lane) - 1u;
#pragma unroll
  for (int k = 0; k < kSortItems; ++k) {
    const int li = w * 32 * kSortItems + k * 32 + lane;
    const bool valid = li < tile_n;
    key[k] = valid ? kin[base + li] : 0ull;
    val[k] = valid ? vin[base + li] : 0;
    const uint32_t d = valid ? (uint32_t)((key[k] >> shift) & 255u) : 256u;
    const uint32_t peers = __match_any_sync(0xffffffffu, d);
    const uint32_t before = valid ? s_wcnt[w][d] : 0u;
    rank[k] = before + __popc(peers & lt);
    __syncwarp();
    if (valid && lane == __ffs(peers) - 1) s_wcnt[w][d] = before + __popc(peers);
    __syncwarp();
  }
  __syncthreads();
  // per digit: offsets of each warp inside the tile's run of that digit
  const int d = threadIdx.x;
  uint32_t run = 0;
#pragma unroll
  for (int ww = 0; ww < kSortThreads / 32; ++ww) {
    const uint32_t c = s_wcnt[ww][d];
    s_wcnt[ww][d] = run;
    run += c;
  }
  uint32_t tot_all;
  const uint32_t tstart = block_exscan256(run, s_scan, &tot_all);
  s_tile_start[d] = tstart;
  const uint32_t dbase = block_exscan256(digit_tot[d], s_scan, nullptr);
  s_gbase[d] = dbase + hist[d * nblk + blockIdx.x];
  __syncthreads();
#pragma unroll
  for (int k = 0; k < kSortItems; ++k) {
    const int li = w * 32 * kSortItems + k * 32 + lane;
    if (li < tile_n) {
      const uint32_t dd = (uint32_t)((key[k] >> shift) & 255u);
      const uint32_t p = s_tile_start[dd] + s_wcnt[w][dd] + rank[k];
      s_keys[p] = key[k];
      s_vals[p] = val[k];
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < tile_n; i += kSortThreads) {
    const uint64_t kk = s_keys[i];
    const uint32_t dd = (uint32_t)((kk >> shift) & 255u);
    const uint32_t o = s_gbase[dd] + (uint32_t)i - s_tile_start[dd];
    kout[o] = kk;
    vout[o] = s_vals[i];
  }
}

cudaError_t launch_keys_sort(const double* pos, int64_t n, double L, uint64_t* keys_out, int32_t* order_out,
                             const SortWs& W, cudaStream_t s) {
  const int kb = 256;
  int64_t kgrid = (n + kb - 1) / kb;
  if (kgrid > grid_cap(64)) kgrid = grid_cap(64);
  k_keys<<<(unsigned)kgrid, kb, 0, s>>>(pos, n, box_scale(L), keys_out, order_out, W.sb);
  uint64_t* kin = keys_out;
  int32_t* vin = order_out;
  uint64_t* ko = W.keys_alt;
  int32_t* vo = W.vals_alt;
  for (int pass = 0; pass < 8; ++pass) {
    const int shift = 8 * pass;
    k_sort_hist<<<(unsigned)W.nblk, kSortThreads, 0, s>>>(kin, n, shift, W.hist, W.nblk);
    k_sort_scan<<<256, 1024, 0, s>>>(W.hist, W.nblk, W.digit_tot);
    k_sort_scatter<<<(unsigned)W.nblk, kSortThreads, 0, s>>>(kin, vin, n, shift, W.hist, W.nblk, W.digit_tot, ko,
                                                             vo);
    uint64_t* tk = kin; kin = ko; ko = tk;
    int32_t* tv = vin; vin = vo; vo = tv;
  }
  return cudaGetLastError();
}

}  // namespace og

// ----------------------------------------------------------------------------
// og_keys_sort_noalloc: the same keys and sort with the workspace in a static
// device array instead of a caller buffer (declared in include/og.h).
#include <cmath>
#include <mutex>

namespace {

constexpr int64_t kNoAllocMaxN = int64_t(1) << 20;
constexpr size_t noalloc_round(size_t x) { return (x + og::kAlign - 1) / og::kAlign * og::kAlign; }
// Same carving as og::carve_sort: status block, alternate keys, alternate
// indices, per-tile digit histograms, digit totals.
constexpr size_t kNoAllocBytes =
    noalloc_round(sizeof(og::StatusBlock)) + noalloc_round(sizeof(uint64_t) * kNoAllocMaxN) +
    noalloc_round(sizeof(int32_t) * kNoAllocMaxN) +
    noalloc_round(sizeof(uint32_t) * 256 * ((kNoAllocMaxN + og::kSortTile - 1) / og::kSortTile)) +
    noalloc_round(sizeof(uint32_t) * 256);

// Held by every GPU that loads the library, until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_sort_ws[kNoAllocBytes];

constexpr int kNoAllocMaxDevices = 256;
std::mutex g_noalloc_mu;
void* g_noalloc_base[kNoAllocMaxDevices] = {};

}  // namespace

extern "C" og_status og_keys_sort_noalloc(const double* pos, int64_t n, double box, uint64_t* keys_sorted,
                                          int32_t* order, og_stream stream) {
  if (!pos || !keys_sorted || !order) return OG_EINVAL;
  if (n < 1 || !std::isfinite(box) || !(box > 0.0)) return OG_EINVAL;
  if (n > kNoAllocMaxN) return OG_ENOSPACE;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNoAllocMaxDevices) return OG_ECUDA;
  void* base = nullptr;
  {
    // First call on this device: look up the device address of the static
    // array (the host-side name is only a stand-in for it).
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_base[dev]) {
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_noalloc_sort_ws) != cudaSuccess || !p) return OG_ECUDA;
      g_noalloc_base[dev] = p;
    }
    base = g_noalloc_base[dev];
  }
  og::SortWs W;
  if (og::carve_sort(base, n, &W) > kNoAllocBytes) return OG_ENOSPACE;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // the array keeps the previous call's contents: the status block starts at zero
  if (cudaMemsetAsync(W.sb, 0, sizeof(og::StatusBlock), s) != cudaSuccess) return OG_ECUDA;
  return og::launch_keys_sort(pos, n, box, keys_sorted, order, W, s) == cudaSuccess ? OG_OK : OG_ECUDA;
}
