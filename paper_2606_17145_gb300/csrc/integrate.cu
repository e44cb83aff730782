// integrate.cu -- kick and drift of the leapfrog step (declared in
// include/og.h: og_kick / og_drift).
//
// The paper's step drifts every particle at its start and kicks with the
// gravity once the tree is rebuilt (Sec. 2.1).  In the kick-drift-kick form:
// a half kick with the previous accelerations, a drift, the forces, and a
// second half kick.  These two kernels are the kick and the drift.  Positions
// and velocities stay FP64 on the device between steps.  The kick adds the
// two FP32 acceleration arrays (the walk's short-range and the mesh's
// long-range part) in FP64.
#include <cmath>

#include "og_internal.cuh"

namespace og {

__global__ void k_kick(double* __restrict__ vel, const float* __restrict__ a, const float* __restrict__ b,
                       int64_t n3, double dt) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n3; i += (int64_t)gridDim.x * blockDim.x) {
    const double acc = b ? (double)a[i] + (double)b[i] : (double)a[i];
    vel[i] += dt * acc;
  }
}

__global__ void k_drift(double* __restrict__ pos, const double* __restrict__ vel, int64_t n3, double dt) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n3; i += (int64_t)gridDim.x * blockDim.x)
    pos[i] += dt * vel[i];
}

}  // namespace og

namespace {

constexpr int64_t kIntMaxN = 0x7ffffff0LL;

unsigned int_grid(int64_t items) {
  int64_t g = (items + 255) / 256;
  if (g > og::grid_cap(32)) g = og::grid_cap(32);
  return (unsigned)(g > 0 ? g : 1);
}

}  // namespace

extern "C" {

og_status og_kick(double* vel, const float* acc_a, const float* acc_b, int64_t n, double dt, og_stream stream) {
  if (!vel || !acc_a || n < 1 || n > kIntMaxN || !std::isfinite(dt)) return OG_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  og::k_kick<<<int_grid(3 * n), 256, 0, s>>>(vel, acc_a, acc_b, 3 * n, dt);
  return cudaGetLastError() == cudaSuccess ? OG_OK : OG_ECUDA;
}

og_status og_drift(double* pos, const double* vel, int64_t n, double dt, og_stream stream) {
  if (!pos || !vel || n < 1 || n > kIntMaxN || !std::isfinite(dt)) return OG_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  og::k_drift<<<int_grid(3 * n), 256, 0, s>>>(pos, vel, 3 * n, dt);
  return cudaGetLastError() == cudaSuccess ? OG_OK : OG_ECUDA;
}

}  // extern "C"
