// probes.cu -- throughput probes of the SM pipes the walks run on.
//
// The walks are bound by the FP32 pipe, the special-function unit (MUFU:
// rsqrt and ex2) and, in the comparison variant, the FP64 pipe.  These
// kernels measure what each pipe delivers on the device at hand, so that the
// roofline fractions reported for the walks use measured peaks rather than
// unit counts.  Each thread runs kChains independent dependency chains (enough
// instruction-level parallelism to hide the pipe latency at 32 resident warps
// per SM); the grid is 4 blocks of 256 threads per SM.  The caller times a
// launch with CUDA events and divides the returned operation count by it.
#include "og_internal.cuh"

namespace og {
namespace {

constexpr int kChains = 8;
constexpr int kUnroll = 16;
constexpr int kThreads = 256;
constexpr int kBlocksPerSM = 4;

// x <- x a + b, a = 1 - 2^-10, b = 2^-10: every chain converges to 1 and
// stays normal.
__global__ void __launch_bounds__(kThreads) k_probe_ffma(int iters, float a, float b, float* sink) {
  float x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = 1.0f + 1e-3f * (float)(threadIdx.x + c);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u)
#pragma unroll
      for (int c = 0; c < kChains; ++c) x[c] = fmaf(x[c], a, b);
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  if (s == -1.0f) *sink = s;  // never true; keeps the chains alive
}

// The same chains, two per instruction (fma.rn.f32x2).
__global__ void __launch_bounds__(kThreads) k_probe_ffma2(int iters, float a, float b, float* sink) {
  unsigned long long x[kChains];
  const unsigned long long A = ((unsigned long long)__float_as_uint(a) << 32) | __float_as_uint(a);
  const unsigned long long B = ((unsigned long long)__float_as_uint(b) << 32) | __float_as_uint(b);
#pragma unroll
  for (int c = 0; c < kChains; ++c) {
    const float v = 1.0f + 1e-3f * (float)(threadIdx.x + c);
    x[c] = ((unsigned long long)__float_as_uint(v) << 32) | __float_as_uint(v);
  }
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u)
#pragma unroll
      for (int c = 0; c < kChains; ++c) asm("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(x[c]) : "l"(A), "l"(B));
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += __uint_as_float((uint32_t)x[c]) + __uint_as_float((uint32_t)(x[c] >> 32));
  if (s == -1.0f) *sink = s;
}

// x <- ex2(rsqrt(x)): for x in [1, 2], rsqrt(x) is in [0.70, 1] and ex2 of
// that in [1.63, 2], so the chain stays in range with no other instruction.
// Two MUFU operations per step: the walk's mix (one rsqrt, one ex2 per
// interaction).
__global__ void __launch_bounds__(kThreads) k_probe_mufu(int iters, float a, float b, float* sink) {
  (void)a;
  (void)b;
  float x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = 1.5f + 1e-4f * (float)(threadIdx.x + c);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < kUnroll / 2; ++u)
#pragma unroll
      for (int c = 0; c < kChains; ++c) {
        float y;
        asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x[c]));
        asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(x[c]) : "f"(y));
      }
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  if (s == -1.0f) *sink = s;
}

__global__ void __launch_bounds__(kThreads) k_probe_dfma(int iters, float a, float b, float* sink) {
  const double A = a, B = b;
  double x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = 1.0 + 1e-3 * (double)(threadIdx.x + c);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u)
#pragma unroll
      for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], A, B);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  if (s == -1.0) *sink = (float)s;
}

}  // namespace

int device_sm_count() {
  // one entry per device ordinal; concurrent first calls store the same value
  static int cache[64] = {0};
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (dev >= 0 && dev < 64 && cache[dev] > 0) return cache[dev];
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  if (dev >= 0 && dev < 64) cache[dev] = sms;
  return sms;
}

}  // namespace og

using namespace og;

extern "C" og_status og_probe_pipe(int32_t kind, int32_t iters, float* sink, uint64_t* ops, og_stream stream) {
  if (!sink || !ops || iters < 1 || iters > (1 << 24)) return OG_EINVAL;
  const int sms = device_sm_count();
  if (sms <= 0) return OG_ECUDA;
  const unsigned blocks = (unsigned)(sms * kBlocksPerSM);
  const uint64_t threads = (uint64_t)blocks * kThreads;
  const uint64_t per_thread = (uint64_t)iters * kUnroll * kChains;
  const float a = 1.0f - 0.0009765625f, b = 0.0009765625f;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  switch (kind) {
    case OG_PROBE_FFMA:
      k_probe_ffma<<<blocks, kThreads, 0, s>>>(iters, a, b, sink);
      *ops = threads * per_thread;
      break;
    case OG_PROBE_FFMA2:
      k_probe_ffma2<<<blocks, kThreads, 0, s>>>(iters, a, b, sink);
      *ops = 2 * threads * per_thread;
      break;
    case OG_PROBE_MUFU:
      k_probe_mufu<<<blocks, kThreads, 0, s>>>(iters, a, b, sink);
      *ops = threads * per_thread;
      break;
    case OG_PROBE_DFMA:
      k_probe_dfma<<<blocks, kThreads, 0, s>>>(iters, a, b, sink);
      *ops = threads * per_thread;
      break;
    default:
      return OG_EINVAL;
  }
  return cudaGetLastError() == cudaSuccess ? OG_OK : OG_ECUDA;
}
