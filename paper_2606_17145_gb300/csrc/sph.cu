// sph.cu -- SPH density and smoothing length on the device (declared in
// include/og.h: og_sph_ws_bytes / og_sph_density).
//
// The paper's SPH density module iterates each particle's smoothing length
// until its sphere holds a fixed number of neighbours, and gathers the
// neighbours inside a sphere before evaluating them (Sec. 2.1).  The reading
// is GADGET-2's: W is the cubic spline with support h,
// rho_i = sum_j m_j W(r_ij, h_i) (the particle itself included), and h_i is
// the root of the kernel-weighted count
// N_eff(h) = (4 pi / 3) h^3 sum_j W(r_ij, h) = (32 / 3) sum_j w(r_ij / h) = N_ngb.
//
// First version, written for correctness on the existing keys and tree: one
// thread per particle, FP64 distances in box units with the periodic minimum
// image.  A thread gathers every particle within a search radius H from a
// stack walk of the tree (cube-sphere test), widens H until N_eff(H) >= N_ngb
// or narrows it when the gather overflows its list, then bisects h in [0, H]
// over the gathered distances: w(r / h) = 0 for r >= h, so for h <= H the
// gathered set gives the full sum.  Every loop and buffer is bounded; an
// overflow or a failed bracket sets a status bit and writes NaN.
#include <cmath>

#include "og_internal.cuh"

namespace og {

constexpr int kSphList = 256;   // gathered neighbours per particle
constexpr int kSphStack = 8 * (kLevels + 1);  // at most 8 children pushed per level
constexpr int kSphTries = 24;   // search-radius changes
constexpr int kSphBisect = 64;  // bisection steps (2^-64 of the bracket)

__device__ __forceinline__ double sph_w(double q) {
  if (q <= 0.5) return 1.0 - 6.0 * q * q + 6.0 * q * q * q;
  if (q <= 1.0) {
    const double t = 1.0 - q;
    return 2.0 * t * t * t;
  }
  return 0.0;
}

__device__ __forceinline__ double sph_mi(double t) { return t - rint(t); }

struct SphArgs {
  TreeDev T;
  StatusBlock* wsb;
  BoxScale B;
  double n_ngb;
  double h0;  // first search radius, box units
  double* h_out;
  double* rho_out;
  int32_t* ngb_out;
};

// Gather the particles within H (box units) of x into (r, j); returns the
// number found, which exceeds kSphList on overflow (the list then holds the
// first kSphList), or -1 on a corrupt link or a stack overflow.
__device__ int sph_gather(const SphArgs& A, const double x[3], double H, double* r, int* jl) {
  const TreeDev& T = A.T;
  int stack[kSphStack];
  int sp = 0, found = 0;
  stack[sp++] = 0;  // the root
  while (sp > 0) {
    const int p = stack[--sp];
    if (p < 0 || p >= T.cap) return -1;
    const int4 D = T.nD[p];
    const float4 NC = T.nC[p];
    const double hs = 0.5 * (double)NC.w;
    double d2 = 0.0;
    const double c[3] = {(double)NC.x, (double)NC.y, (double)NC.z};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const double g = fabs(sph_mi(x[a] - c[a])) - hs;
      if (g > 0.0) d2 += g * g;
    }
    if (d2 >= H * H) continue;  // the cube lies beyond the sphere
    if (meta_leaf(D.w)) {
      for (int j = D.x; j < D.x + D.y; ++j) {
        if (j < 0 || j >= T.n) return -1;
        double s2 = 0.0;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          const double t = sph_mi(x[a] - div_box(T.x64[3 * (int64_t)j + a], A.B));
          s2 += t * t;
        }
        const double rr = sqrt(s2);
        if (rr < H) {
          if (found < kSphList) {
            r[found] = rr;
            jl[found] = j;
          }
          ++found;
        }
      }
    } else {
      const int nc = meta_nchild(D.w);
      if (sp + nc > kSphStack) return -1;
      for (int c2 = 0; c2 < nc; ++c2) stack[sp++] = D.z + c2;
    }
  }
  return found;
}

__device__ __forceinline__ double sph_neff(const double* r, int cnt, double h) {
  double s = 0.0;
  for (int k = 0; k < cnt; ++k) s += sph_w(r[k] / h);
  return (32.0 / 3.0) * s;
}

__global__ void __launch_bounds__(128) k_sph_density(SphArgs A) {
  const TreeDev& T = A.T;
  if (T.sb->status != 0 || T.sb->magic != kMagicTree) {
    if (blockIdx.x == 0 && threadIdx.x == 0) set_status(A.wsb, ST_NOTREE);
    return;
  }
  double r[kSphList];
  int jl[kSphList];
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < T.n; k += (int64_t)gridDim.x * blockDim.x) {
    const int32_t i = T.order[k];
    double x[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) x[a] = div_box(T.x64[3 * k + a], A.B);
    double H = A.h0 < 0.5 ? A.h0 : 0.5;
    int cnt = -1;
    bool ok = false;
    for (int t = 0; t < kSphTries; ++t) {
      cnt = sph_gather(A, x, H, r, jl);
      if (cnt < 0) break;
      if (cnt > kSphList) {  // too many within H: narrow it
        H *= 0.7;
        continue;
      }
      if (sph_neff(r, cnt, H) >= A.n_ngb) {
        ok = true;
        break;
      }
      if (H >= 0.5) break;  // the minimum image allows no wider sphere
      H = H * 1.6 < 0.5 ? H * 1.6 : 0.5;
    }
    if (!ok) {
      set_status(A.wsb, cnt < 0 ? ST_TREELINK : ST_WALKCAP);
      A.h_out[i] = NAN;
      A.rho_out[i] = NAN;
      A.ngb_out[i] = -1;
      continue;
    }
    // N_eff is increasing in h: bisect [0, H] to the FP64 resolution of H
    double lo = 0.0, hi = H;
    for (int s = 0; s < kSphBisect && hi - lo > 1e-12 * hi; ++s) {
      const double mid = 0.5 * (lo + hi);
      if (sph_neff(r, cnt, mid) < A.n_ngb) lo = mid;
      else hi = mid;
    }
    const double h = hi;
    double rho = 0.0;
    int ngb = 0;
    for (int q = 0; q < cnt; ++q) {
      rho += T.m64[jl[q]] * sph_w(r[q] / h);
      if (r[q] < h && jl[q] != (int)k) ++ngb;
    }
    const double hL = h * A.B.L;
    A.h_out[i] = hL;
    A.rho_out[i] = rho * 8.0 / (M_PI * hL * hL * hL);
    A.ngb_out[i] = ngb;
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
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  og::SphArgs A;
  A.T = og::tree_view(t);
  A.wsb = static_cast<og::StatusBlock*>(ws);
  A.B = og::box_scale(t->box);
  A.n_ngb = n_ngb;
  // the radius that holds n_ngb neighbours at the mean density, in box units
  A.h0 = std::cbrt(3.0 * n_ngb / (4.0 * M_PI * (double)t->n));
  A.h_out = h;
  A.rho_out = rho;
  A.ngb_out = ngb;
  if (cudaMemsetAsync(A.wsb, 0, sizeof(og::StatusBlock), s) != cudaSuccess) return OG_ECUDA;
  int64_t grid = (t->n + 127) / 128;
  if (grid > og::grid_cap(16)) grid = og::grid_cap(16);
  og::k_sph_density<<<(unsigned)grid, 128, 0, s>>>(A);
  return cudaGetLastError() == cudaSuccess ? OG_OK : OG_ECUDA;
}

}  // extern "C"
