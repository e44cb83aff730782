// pm.cu -- the PM long-range complement of the TreePM split (declared in
// include/og.h: og_pm_plan_create / og_pm_plan_destroy / og_pm_ws_bytes /
// og_pm_accel).
//
// The paper (Sec. 3.1) runs the long-range part on a particle mesh with FFTW
// on the host; here it stays on the device next to the tree.  The scheme is
// the GADGET-2 one, the exact complement of the walk's short-range factor
// f(r) = erfc(r / 2 r_s) + (r / (sqrt(pi) r_s)) exp(-r^2 / 4 r_s^2), G = 1:
//
//   k_pm_deposit   CIC: nodes at x = i D (D = L / N, periodic); along each
//                  axis weight 1 - f on node floor(u), f on floor(u) + 1, with
//                  u = x N / L and f = u - floor(u).  FP32 atomics into the
//                  real mesh (masses, not densities: 1 / D^3 goes into the
//                  Green's function).
//   cuFFT R2C      forward transform of the mesh (FP32).
//   k_pm_green     phi_hat = -4 pi rho_hat exp(-k^2 r_s^2) / (k^2 S), with
//                  S = prod_a sinc^4(kappa_a / N) (the CIC window of the
//                  deposit and of the interpolation) and phi_hat(0) = 0.  The
//                  1 / D^3 of the density and the 1 / N^3 of the inverse
//                  transform combine into 1 / L^3.
//   cuFFT C2R      the potential on the mesh.
//   k_pm_interp    per particle: the four-point central difference
//                  F = -[(2/3)(phi(+1) - phi(-1)) - (1/12)(phi(+2) - phi(-2))] / D
//                  at the 8 CIC nodes, summed with the deposit's weights.
//
// The mesh force is never stored: each particle differentiates the potential
// at its own 8 nodes (72 loads of an L2-resident mesh instead of three more
// N^3 meshes in HBM).  Positions are FP64 until the CIC fraction, which is
// rounded to FP32 once, as in the deposit.
#include <cufft.h>

#include <cmath>
#include <cstring>
#include <new>

#include "og_internal.cuh"

namespace og {

// Lower node index i0 in [0, N) and FP32 fraction f of one coordinate: the
// same arithmetic in the deposit and the interpolation, so both see the same
// weights.  u = (w N) / L; for a power-of-two side the division is the exact
// multiply by 1 / L.  When L and N are both powers of two (log2N >= 0),
// u = w 2^(log2N - e) exactly and floor / fraction come from the bits on the
// integer pipe (the FP64 pipe is the scarce one); the FP64 form is the
// definition and the fallback.
__device__ __forceinline__ void cic_axis(double x, const BoxScale& B, int N, int log2N, int& i0, float& f) {
  const double w = wrap_coord(x, B);
  int i;
  if (!(log2N >= 0 && B.pow2 && cic_bits((uint64_t)__double_as_longlong(w), B.e - log2N, i, f))) {
    const double wn = __dmul_rn(w, (double)N);
    const double u = B.pow2 ? __dmul_rn(wn, B.invL) : __ddiv_rn(wn, B.L);
    i = __double2int_rd(u);
    f = __double2float_rn(__dsub_rn(u, (double)i));
  }
  if (i >= N) i -= N;  // w == L
  if (i < 0) i += N;   // w rounded to -0.x ulp: node N - 1, fraction near 1 (as floor and mod give)
  i0 = i;
}

__global__ void k_pm_deposit(const double* __restrict__ pos, const double* __restrict__ mass, int64_t n,
                             BoxScale B, int N, int log2N, float* __restrict__ R, StatusBlock* sb) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
    const double x0 = pos[3 * p], x1 = pos[3 * p + 1], x2 = pos[3 * p + 2];
    const double m = mass[p];
    if (!(finite_bits(x0) && finite_bits(x1) && finite_bits(x2) && finite_bits(m))) {
      set_status(sb, ST_BADINPUT);
      continue;
    }
    int ix, iy, iz;
    float fx, fy, fz;
    cic_axis(x0, B, N, log2N, ix, fx);
    cic_axis(x1, B, N, log2N, iy, fy);
    cic_axis(x2, B, N, log2N, iz, fz);
    const int jx = ix + 1 == N ? 0 : ix + 1, jy = iy + 1 == N ? 0 : iy + 1, jz = iz + 1 == N ? 0 : iz + 1;
    const float mf = (float)m;
    const float wx[2] = {1.0f - fx, fx}, wy[2] = {1.0f - fy, fy}, wz[2] = {1.0f - fz, fz};
    const int ax[2] = {ix, jx}, ay[2] = {iy, jy}, az[2] = {iz, jz};
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
      for (int b = 0; b < 2; ++b)
#pragma unroll
        for (int c = 0; c < 2; ++c)
          atomicAdd(&R[((int64_t)ax[a] * N + ay[b]) * N + az[c]], mf * (wx[a] * wy[b] * wz[c]));
  }
}

__device__ __forceinline__ float pm_sinc(int k, int N) {
  if (k == 0) return 1.0f;
  const float t = (float)k / (float)N;
  return sinpif(t) / (3.14159265358979323846f * t);
}

// The R2C layout [N][N][N/2 + 1], walked as one flat index: every thread
// takes four coefficients a grid stride apart (four independent loads in
// flight).  Both factors of the Green's function separate over the axes,
// exp(-k^2 r_s^2) / S = prod_a exp(-q^2 k_a^2 r_s^2) / sinc^4(k_a / N), so each
// block first tabulates T(k) = exp(-q^2 k^2 r_s^2) / sinc^4(k / N) for
// k = 0 .. N / 2 in shared memory, and a coefficient costs three table
// loads, two products and one reciprocal.
constexpr int kGreenMaxHalf = 513;  // N / 2 + 1 for N <= 1024
constexpr int kGreenUnroll = 4;

// i / d for i < 2^31, 0 < d and a quotient below 2^21 (here at most N^2):
// the FP32 quotient (relative error below 3 2^-24, so off by less than one)
// corrected on the remainder; the loops stay exact for any error.  A few
// instructions where a 64-bit integer division takes dozens.
__device__ __forceinline__ uint32_t div_u31(uint32_t i, uint32_t d, float inv_d) {
  uint32_t q = (uint32_t)((float)i * inv_d);
  int32_t r = (int32_t)(i - q * d);
  while (r < 0) {
    --q;
    r += (int32_t)d;
  }
  while (r >= (int32_t)d) {
    ++q;
    r -= (int32_t)d;
  }
  return q;
}
__global__ void __launch_bounds__(256) k_pm_green(cufftComplex* __restrict__ C, int N, float inv_box,
                                                  float two_pi_over_box, float r_s) {
  __shared__ float Tk[kGreenMaxHalf];
  const int H = N / 2 + 1;
  const float pi = 3.14159265358979323846f;
  // 1 / D^3 (masses -> density) times 1 / N^3 (inverse transform) = 1 / L^3
  const float c0 = -4.0f * pi * (inv_box * inv_box * inv_box);
  const float q2 = two_pi_over_box * two_pi_over_box;
  for (int k = threadIdx.x; k < H; k += blockDim.x) {
    const float s = pm_sinc(k, N);
    const float s2 = s * s;
    Tk[k] = expf(-q2 * (float)(k * k) * r_s * r_s) / (s2 * s2);
  }
  __syncthreads();
  // N <= 1024: N^2 H < 2^29, so the flat index and its split fit 32 bits
  const uint32_t total = (uint32_t)N * (uint32_t)N * (uint32_t)H;
  const uint32_t stride = gridDim.x * blockDim.x;
  const float inv_H = 1.0f / (float)H, inv_N = 1.0f / (float)N;
  for (uint32_t i0 = blockIdx.x * blockDim.x + threadIdx.x; i0 < total; i0 += kGreenUnroll * stride) {
    cufftComplex v[kGreenUnroll];
    float g[kGreenUnroll];
#pragma unroll
    for (int u = 0; u < kGreenUnroll; ++u) {
      const uint32_t i = i0 + u * stride;
      g[u] = 0.0f;
      if (i < total) {
        v[u] = C[i];
        const uint32_t row = div_u31(i, (uint32_t)H, inv_H);
        const int kz = (int)(i - row * (uint32_t)H);
        const uint32_t ixu = div_u31(row, (uint32_t)N, inv_N);
        const int ix = (int)ixu, iy = (int)(row - ixu * (uint32_t)N);
        const int kx = ix <= N / 2 ? ix : N - ix;  // |k|: T is even
        const int ky = iy <= N / 2 ? iy : N - iy;
        const int k2i = kx * kx + ky * ky + kz * kz;
        if (k2i != 0) g[u] = c0 * Tk[kx] * Tk[ky] * Tk[kz] * __frcp_rn(q2 * (float)k2i);
      }
    }
#pragma unroll
    for (int u = 0; u < kGreenUnroll; ++u) {
      const uint32_t i = i0 + u * stride;
      if (i < total) C[i] = make_float2(v[u].x * g[u], v[u].y * g[u]);
    }
  }
}

__device__ __forceinline__ float pm_phi(const float* __restrict__ P, int N, int x, int y, int z) {
  x = x < 0 ? x + N : (x >= N ? x - N : x);
  y = y < 0 ? y + N : (y >= N ? y - N : y);
  z = z < 0 ? z + N : (z >= N ? z - N : z);
  return __ldg(&P[((int64_t)x * N + y) * N + z]);
}

// -dphi/dx at a node by the four-point central difference (times D).
__device__ __forceinline__ float pm_diff(float m2, float m1, float p1, float p2) {
  return -((2.0f / 3.0f) * (p1 - m1) - (1.0f / 12.0f) * (p2 - m2));
}

__global__ void k_pm_interp(const double* __restrict__ pos, int64_t n, BoxScale B, int N, int log2N, float inv_D,
                            const float* __restrict__ P, float* __restrict__ acc) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
    const double x0 = pos[3 * p], x1 = pos[3 * p + 1], x2 = pos[3 * p + 2];
    float a[3] = {0.0f, 0.0f, 0.0f};
    if (finite_bits(x0) && finite_bits(x1) && finite_bits(x2)) {
      int ix, iy, iz;
      float fx, fy, fz;
      cic_axis(x0, B, N, log2N, ix, fx);
      cic_axis(x1, B, N, log2N, iy, fy);
      cic_axis(x2, B, N, log2N, iz, fz);
      const float wx[2] = {1.0f - fx, fx}, wy[2] = {1.0f - fy, fy}, wz[2] = {1.0f - fz, fz};
#pragma unroll
      for (int b = 0; b < 2; ++b)
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          // x: the 6 potentials ix - 2 .. ix + 3 on the line (iy + b, iz + c)
          float v[6];
#pragma unroll
          for (int s = 0; s < 6; ++s) v[s] = pm_phi(P, N, ix - 2 + s, iy + b, iz + c);
          a[0] += wy[b] * wz[c] * (wx[0] * pm_diff(v[0], v[1], v[3], v[4]) + wx[1] * pm_diff(v[1], v[2], v[4], v[5]));
          // y: the line (ix + b, ., iz + c)
#pragma unroll
          for (int s = 0; s < 6; ++s) v[s] = pm_phi(P, N, ix + b, iy - 2 + s, iz + c);
          a[1] += wx[b] * wz[c] * (wy[0] * pm_diff(v[0], v[1], v[3], v[4]) + wy[1] * pm_diff(v[1], v[2], v[4], v[5]));
          // z: the line (ix + b, iy + c, .)
#pragma unroll
          for (int s = 0; s < 6; ++s) v[s] = pm_phi(P, N, ix + b, iy + c, iz - 2 + s);
          a[2] += wx[b] * wy[c] * (wz[0] * pm_diff(v[0], v[1], v[3], v[4]) + wz[1] * pm_diff(v[1], v[2], v[4], v[5]));
        }
    }
    acc[3 * p] = a[0] * inv_D;
    acc[3 * p + 1] = a[1] * inv_D;
    acc[3 * p + 2] = a[2] * inv_D;
  }
}

}  // namespace og

// ----------------------------------------------------------------------------
// C ABI

struct og_pm_plan {
  int32_t n;
  cufftHandle r2c, c2r;
  size_t work_bytes;
};

namespace {

constexpr int64_t kPmMaxN = 0x7ffffff0LL;

struct PmWs {
  og::StatusBlock* sb;
  float* R;            // [N][N][N]: masses, then the potential
  cufftComplex* C;     // [N][N][N/2 + 1]
  void* work;          // cuFFT work area
};

size_t carve_pm(void* buf, int N, size_t work_bytes, PmWs* W) {
  size_t off = 0;
  char* b = static_cast<char*>(buf);
  auto take = [&](size_t bytes) -> void* {
    void* p = b ? b + off : nullptr;
    off = og::align_up(off + bytes);
    return p;
  };
  PmWs w{};
  const size_t n3 = (size_t)N * N * N, h = (size_t)N * N * (N / 2 + 1);
  w.sb = static_cast<og::StatusBlock*>(take(sizeof(og::StatusBlock)));
  w.R = static_cast<float*>(take(sizeof(float) * n3));
  w.C = static_cast<cufftComplex*>(take(sizeof(cufftComplex) * h));
  w.work = take(work_bytes > 0 ? work_bytes : 1);
  if (W) *W = w;
  return off;
}

bool pm_finite_pos(double x) { return std::isfinite(x) && x > 0.0; }

unsigned pm_grid(int64_t items) {
  int64_t g = (items + 255) / 256;
  if (g > og::grid_cap(32)) g = og::grid_cap(32);
  return (unsigned)(g > 0 ? g : 1);
}

}  // namespace

extern "C" {

og_status og_pm_plan_create(int32_t ngrid, og_pm_plan** plan) {
  if (!plan) return OG_EINVAL;
  *plan = nullptr;
  if (ngrid < 8 || ngrid > 1024) return OG_EINVAL;
  og_pm_plan* p = new (std::nothrow) og_pm_plan;
  if (!p) return OG_ENOSPACE;
  p->n = ngrid;
  p->work_bytes = 0;
  bool have_r2c = false, have_c2r = false;
  size_t w1 = 0, w2 = 0;
  bool ok = cufftCreate(&p->r2c) == CUFFT_SUCCESS;
  have_r2c = ok;
  ok = ok && cufftSetAutoAllocation(p->r2c, 0) == CUFFT_SUCCESS;
  ok = ok && cufftMakePlan3d(p->r2c, ngrid, ngrid, ngrid, CUFFT_R2C, &w1) == CUFFT_SUCCESS;
  if (ok) {
    ok = cufftCreate(&p->c2r) == CUFFT_SUCCESS;
    have_c2r = ok;
  }
  ok = ok && cufftSetAutoAllocation(p->c2r, 0) == CUFFT_SUCCESS;
  ok = ok && cufftMakePlan3d(p->c2r, ngrid, ngrid, ngrid, CUFFT_C2R, &w2) == CUFFT_SUCCESS;
  if (!ok) {
    if (have_r2c) cufftDestroy(p->r2c);
    if (have_c2r) cufftDestroy(p->c2r);
    delete p;
    return OG_ECUDA;
  }
  p->work_bytes = w1 > w2 ? w1 : w2;
  *plan = p;
  return OG_OK;
}

void og_pm_plan_destroy(og_pm_plan* plan) {
  if (!plan) return;
  cufftDestroy(plan->r2c);
  cufftDestroy(plan->c2r);
  delete plan;
}

size_t og_pm_ws_bytes(const og_pm_plan* plan) {
  if (!plan) return 0;
  return carve_pm(nullptr, plan->n, plan->work_bytes, nullptr);
}

og_status og_pm_accel(og_pm_plan* plan, const double* pos, const double* mass, int64_t n, double box, double r_s,
                      void* ws, size_t ws_bytes, float* acc, og_stream stream) {
  if (!plan || !pos || !mass || !ws || !acc) return OG_EINVAL;
  if (n < 1 || n > kPmMaxN || !pm_finite_pos(box) || !pm_finite_pos(r_s)) return OG_EINVAL;
  if ((reinterpret_cast<uintptr_t>(ws) % og::kAlign) != 0) return OG_EINVAL;
  if (ws_bytes < og_pm_ws_bytes(plan)) return OG_ENOSPACE;
  const int N = plan->n;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  PmWs W;
  carve_pm(ws, N, plan->work_bytes, &W);
  if (cudaMemsetAsync(W.sb, 0, sizeof(og::StatusBlock), s) != cudaSuccess) return OG_ECUDA;
  if (cudaMemsetAsync(W.R, 0, sizeof(float) * (size_t)N * N * N, s) != cudaSuccess) return OG_ECUDA;
  const og::BoxScale B = og::box_scale(box);
  int log2N = -1;  // N a power of two: its exponent
  for (int e = 0; e < 11; ++e)
    if (N == (1 << e)) log2N = e;
  og::k_pm_deposit<<<pm_grid(n), 256, 0, s>>>(pos, mass, n, B, N, log2N, W.R, W.sb);
  if (cudaGetLastError() != cudaSuccess) return OG_ECUDA;
  if (cufftSetStream(plan->r2c, s) != CUFFT_SUCCESS || cufftSetWorkArea(plan->r2c, W.work) != CUFFT_SUCCESS ||
      cufftExecR2C(plan->r2c, W.R, W.C) != CUFFT_SUCCESS)
    return OG_ECUDA;
  const int rows = N * N;
  og::k_pm_green<<<(unsigned)(rows < (int)og::grid_cap(8) ? rows : (int)og::grid_cap(8)), 256, 0, s>>>(
      W.C, N, (float)(1.0 / box), (float)(2.0 * M_PI / box), (float)r_s);
  if (cudaGetLastError() != cudaSuccess) return OG_ECUDA;
  if (cufftSetStream(plan->c2r, s) != CUFFT_SUCCESS || cufftSetWorkArea(plan->c2r, W.work) != CUFFT_SUCCESS ||
      cufftExecC2R(plan->c2r, W.C, W.R) != CUFFT_SUCCESS)
    return OG_ECUDA;
  og::k_pm_interp<<<pm_grid(n), 256, 0, s>>>(pos, n, B, N, log2N, (float)(N / box), W.R, acc);
  return cudaGetLastError() == cudaSuccess ? OG_OK : OG_ECUDA;
}

}  // extern "C"
