// adjoint.cu -- K8: push the per-node source terms of the adjoint walk down
// the tree and assemble dL/dx, dL/dm per particle.
//
// For particle k in leaf l, with node sums G_n = sum J w and S_n = sum w.g of
// every term (i, n) collected by the adjoint walk:
//   dL/dxi_k = target_k - m_k (Gp_k + sum_{n containing k} G_n)
//   dL/dm_k  = Sp_k + sum_{n containing k} (S_n - G_n . (xi_k - X_n))
// The ancestor sums are carried top-down as CG_n = sum G over the path and
// the affine term B_n = value of sum(S - G.(y - X)) at the node centre C_n,
// so every step only involves node-sized differences (no cancellation):
//   B_child = B_parent - CG_parent . (C_child - C_parent)
//             + S_child - G_child . (C_child - X_child).
// Everything here is FP64, in box units (xi = x / L, m' = m / L^2); the final
// scaling to physical units is dL/dx = (.)/L, dL/dm = (.)/L^2.
#include "og_internal.cuh"

namespace og {

__global__ void k_adj_down(TreeDev T, AdjWs W, int lev, double invL) {
  if (T.sb->status != 0) return;  // tree not usable (flagged at build time)
  int base = 0;
  for (int l = 0; l < lev; ++l) base += T.sb->level_cnt[l];
  const int cnt = T.sb->level_cnt[lev];
  if (base + cnt > T.cap) return;
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < cnt; s += gridDim.x * blockDim.x) {
    const int p = base + s;
    const float4 NC = T.nC[p];
    const double C[3] = {(double)NC.x, (double)NC.y, (double)NC.z};
    double G[3], X[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      G[c] = W.Gn[3 * (int64_t)p + c];
      X[c] = T.com64[3 * (int64_t)p + c] * invL;
    }
    double B = W.Sn[p] - (G[0] * (C[0] - X[0]) + G[1] * (C[1] - X[1]) + G[2] * (C[2] - X[2]));
    const int q = T.nParent[p];
    if (q >= 0) {
      const float4 QC = T.nC[q];
      const double Cq[3] = {(double)QC.x, (double)QC.y, (double)QC.z};
      double CGq[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) CGq[c] = W.CG[3 * (int64_t)q + c];
      B += W.Bn[q] - (CGq[0] * (C[0] - Cq[0]) + CGq[1] * (C[1] - Cq[1]) + CGq[2] * (C[2] - Cq[2]));
#pragma unroll
      for (int c = 0; c < 3; ++c) G[c] += CGq[c];
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) W.CG[3 * (int64_t)p + c] = G[c];
    W.Bn[p] = B;
  }
}

__global__ void k_adj_particles(TreeDev T, AdjWs W, double L, double* __restrict__ dpos, double* __restrict__ dmass) {
  if (T.sb->status != 0) return;
  const double invL = 1.0 / L, invL2 = 1.0 / (L * L);
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < T.n; k += (int64_t)gridDim.x * blockDim.x) {
    const int l = T.leaf_of[k];
    const float4 NC = T.nC[l];
    const double C[3] = {(double)NC.x, (double)NC.y, (double)NC.z};
    const double mb = T.m64[k] * invL2;
    double gm = W.Bn[l] + W.Sp[k];
    double gx[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const double cg = W.CG[3 * (int64_t)l + c];
      const double xi = T.x64[3 * k + c] * invL;
      gm -= cg * (xi - C[c]);
      gx[c] = W.tgt[3 * k + c] - mb * (cg + W.Gp[3 * k + c]);
    }
    const int32_t i = T.order[k];
#pragma unroll
    for (int c = 0; c < 3; ++c) dpos[3 * (int64_t)i + c] = gx[c] * invL;
    dmass[i] = gm * invL2;
  }
}

cudaError_t launch_adjoint_push(const TreeDev& T, const AdjWs& W, double L, double* dpos, double* dmass,
                                cudaStream_t s) {
  const unsigned grid = grid_cap(8);
  for (int lev = 0; lev <= kMaxLevel; ++lev) k_adj_down<<<grid, 256, 0, s>>>(T, W, lev, 1.0 / L);
  int64_t pg = (T.n + 255) / 256;
  if (pg > grid_cap(32)) pg = grid_cap(32);
  k_adj_particles<<<(unsigned)pg, 256, 0, s>>>(T, W, L, dpos, dmass);
  return cudaGetLastError();
}

}  // namespace og
