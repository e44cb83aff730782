// og_abi.cu -- the extern "C" entry points of libog.so (declared in
// include/og.h): argument checks, buffer carving, launches.  No allocation,
// no synchronisation (except og_poll_status / og_tree_node_count).
#include <cmath>
#include <cstring>

#include "og_internal.cuh"

using namespace og;

namespace {

constexpr int64_t kMaxN = 0x7ffffff0LL;
constexpr double kNodeBand = 1e-4;
constexpr double kPairBand = 4e-6;

bool aligned(const void* p) { return (reinterpret_cast<uintptr_t>(p) % kAlign) == 0; }

og_status cuda_status(cudaError_t e) { return e == cudaSuccess ? OG_OK : OG_ECUDA; }

int64_t default_capacity(int64_t n) { return 2 * n + 1024; }

bool finite_pos(double x) { return std::isfinite(x) && x > 0.0; }

}  // namespace

extern "C" {

void og_params_default(og_params* p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->leaf_size = 16;
  p->rcut_factor = 4.5;
  p->node_capacity = 0;
  p->max_walk_iters = 0;
}

size_t og_keys_sort_ws_bytes(int64_t n) {
  if (n < 1 || n > kMaxN) return 0;
  return carve_sort(nullptr, n, nullptr);
}

size_t og_tree_bytes(int64_t n, const og_params* p) {
  if (n < 1 || n > kMaxN) return 0;
  og_params q;
  if (p) q = *p; else og_params_default(&q);
  const int64_t cap = q.node_capacity > 0 ? q.node_capacity : default_capacity(n);
  if (cap > kMaxN) return 0;
  return carve_tree(nullptr, n, cap, nullptr);
}

size_t og_accel_ws_bytes(const og_tree* t, og_precision prec) {
  (void)prec;
  if (!t) return 0;
  return align_up(sizeof(StatusBlock));
}

size_t og_adjoint_ws_bytes(const og_tree* t, int recompute_lists) {
  (void)recompute_lists;
  if (!t) return 0;
  return carve_adj(nullptr, t->n, t->node_capacity, nullptr);
}

og_status og_keys_sort(const double* pos, int64_t n, double box, uint64_t* keys_sorted, int32_t* order, void* ws,
                       size_t ws_bytes, og_stream stream) {
  if (!pos || !keys_sorted || !order || !ws) return OG_EINVAL;
  if (n < 1 || n > kMaxN || !finite_pos(box)) return OG_EINVAL;
  if (!aligned(ws)) return OG_EINVAL;
  if (ws_bytes < og_keys_sort_ws_bytes(n)) return OG_ENOSPACE;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  SortWs W;
  carve_sort(ws, n, &W);
  cudaError_t e = cudaMemsetAsync(W.sb, 0, sizeof(StatusBlock), s);
  if (e != cudaSuccess) return OG_ECUDA;
  return cuda_status(launch_keys_sort(pos, n, box, keys_sorted, order, W, s));
}

og_status og_tree_build(const uint64_t* keys_sorted, const int32_t* order, const double* pos, const double* mass,
                        const double* eps, double eps_scalar, int64_t n, double box, const og_params* p,
                        void* tree_mem, size_t tree_bytes, og_tree* tree_out, og_stream stream) {
  if (!keys_sorted || !order || !pos || !mass || !tree_mem || !tree_out) return OG_EINVAL;
  if (n < 1 || n > kMaxN || !finite_pos(box)) return OG_EINVAL;
  if (!eps && !finite_pos(eps_scalar)) return OG_EINVAL;
  og_params q;
  if (p) q = *p; else og_params_default(&q);
  if (q.leaf_size < 1 || q.leaf_size > 32) return OG_EINVAL;
  if (!finite_pos(q.rcut_factor)) return OG_EINVAL;
  if (q.node_capacity < 0 || q.max_walk_iters < 0) return OG_EINVAL;
  if (q.deep_stack < 0 || q.deep_stack > 64) return OG_EINVAL;
  const int64_t cap = q.node_capacity > 0 ? q.node_capacity : default_capacity(n);
  if (cap > kMaxN) return OG_EINVAL;
  if (!aligned(tree_mem)) return OG_EINVAL;
  if (tree_bytes < carve_tree(nullptr, n, cap, nullptr)) return OG_ENOSPACE;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  og_tree t;
  std::memset(&t, 0, sizeof(t));
  t.n = n;
  t.n_groups = (n + kGroup - 1) / kGroup;
  t.node_capacity = cap;
  t.box = box;
  t.rcut_factor = q.rcut_factor;
  t.leaf_size = q.leaf_size;
  t.mem = tree_mem;
  t.mem_bytes = tree_bytes;
  t.max_walk_iters = q.max_walk_iters > 0 ? q.max_walk_iters : (1LL << 24);
  t.deep_stack = q.deep_stack > 0 ? q.deep_stack : 64;
  BuildArgs A;
  A.T = tree_view(&t);
  A.keys = keys_sorted;
  A.order = order;
  A.pos = pos;
  A.mass = mass;
  A.eps = eps;
  A.eps_scalar = eps_scalar;
  A.L = box;
  A.leaf_size = q.leaf_size;
  cudaError_t e = cudaMemsetAsync(A.T.sb, 0, sizeof(StatusBlock), s);
  if (e != cudaSuccess) return OG_ECUDA;
  e = launch_tree_build(A, s);
  if (e != cudaSuccess) return OG_ECUDA;
  t.built = 1;
  *tree_out = t;
  return OG_OK;
}

static og_status walk_common(const og_tree* t, double r_s, double theta, WalkArgs& A) {
  if (!t || !t->built || !t->mem) return OG_ETREE;
  if (t->node_capacity >= (int64_t(1) << 28)) return OG_EINVAL;  // the walk packs node indices in 28 bits
  if (!finite_pos(r_s) || !std::isfinite(theta) || theta < 0.0) return OG_EINVAL;
  const double L = t->box;
  const double rcut = t->rcut_factor * r_s;
  if (!(rcut < 0.5 * L)) return OG_EINVAL;
  std::memset(&A, 0, sizeof(A));
  A.T = tree_view(t);
  A.max_iters = t->max_walk_iters;
  if (t->deep_stack < 1 || t->deep_stack > 64) return OG_EINVAL;
  A.deep = t->deep_stack;
  const double rcb = rcut / L;
  const double rcb2 = rcb * rcb;
  const double nb = std::fmax(kNodeBand, 2e-6 / rcb);
  A.rc2 = (float)rcb2;
  A.rc2_lo = (float)(rcb2 * (1.0 - nb));
  A.rc2_hi = (float)(rcb2 * (1.0 + nb));
  A.pp_lo = (float)(rcb2 * (1.0 - kPairBand));
  A.pp_hi = (float)(rcb2 * (1.0 + kPairBand));
  A.th2_lo = (float)(theta * theta * (1.0 - nb));
  A.th2_hi = (float)(theta * theta * (1.0 + nb));
  A.lim_lo = (float)(0.6 * (1.0 - nb));
  A.lim_hi = (float)(0.6 * (1.0 + nb));
  A.grp_rc2 = (float)(rcb2 * 1.001);
  A.uni_lim = (float)((1.0 - rcb) * (1.0 - 1e-4));
  const double inv2rs_b = L / (2.0 * r_s);
  A.t_scale = (float)(inv2rs_b / 1.125);
  A.ex2c = (float)(-1.4426950408889634 * inv2rs_b * inv2rs_b);
  const double rsb = r_s / L;
  A.fp_c = (float)(-1.0 / (2.0 * std::sqrt(M_PI) * rsb * rsb * rsb));
  A.rc2_64 = rcut * rcut;
  A.th2_64 = theta * theta;
  A.box = L;
  A.r_s64 = r_s;
  A.inv2rs64 = 1.0 / (2.0 * r_s);
  A.fp_c64 = -1.0 / (2.0 * std::sqrt(M_PI) * r_s * r_s * r_s);
  return OG_OK;
}

og_status og_shortrange_accel(const og_tree* t, double r_s, double theta, og_precision prec, void* acc,
                              uint64_t* n_interact, int32_t* counts, void* ws, size_t ws_bytes, og_stream stream) {
  if (!t) return OG_ETREE;
  return og_shortrange_accel_range(t, r_s, theta, prec, 0, t->n_groups, acc, n_interact, counts, ws, ws_bytes,
                                   stream);
}

og_status og_shortrange_accel_range(const og_tree* t, double r_s, double theta, og_precision prec,
                                    int64_t g_begin, int64_t g_end, void* acc, uint64_t* n_interact,
                                    int32_t* counts, void* ws, size_t ws_bytes, og_stream stream) {
  if (!acc || !ws) return OG_EINVAL;
  if (prec != OG_FP32_KAHAN && prec != OG_FP64) return OG_EINVAL;
  WalkArgs A;
  og_status st = walk_common(t, r_s, theta, A);
  if (st != OG_OK) return st;
  if (g_begin < 0 || g_end < g_begin || g_end > t->n_groups) return OG_EINVAL;
  A.g_begin = g_begin;
  A.g_end = g_end;
  if (!aligned(ws)) return OG_EINVAL;
  if (ws_bytes < og_accel_ws_bytes(t, prec)) return OG_ENOSPACE;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  A.wsb = static_cast<StatusBlock*>(ws);
  if (prec == OG_FP64) A.accd = static_cast<double*>(acc);
  else A.accf = static_cast<float*>(acc);
  A.counts = counts;
  A.total = reinterpret_cast<unsigned long long*>(n_interact);
  cudaError_t e = cudaMemsetAsync(ws, 0, sizeof(StatusBlock), s);
  if (e == cudaSuccess && n_interact) e = cudaMemsetAsync(n_interact, 0, sizeof(uint64_t), s);
  if (e != cudaSuccess) return OG_ECUDA;
  return cuda_status(launch_walk(A, (int)prec, false, s));
}

og_status og_shortrange_adjoint(const og_tree* t, double r_s, double theta, og_precision prec, const float* w,
                                double* dpos, double* dmass, int recompute_lists, void* ws, size_t ws_bytes,
                                og_stream stream) {
  if (!t) return OG_ETREE;
  return og_shortrange_adjoint_range(t, r_s, theta, prec, w, 0, t->n_groups, dpos, dmass, recompute_lists, ws,
                                     ws_bytes, stream);
}

// The adjoint walk of groups [g_begin, g_end) and the push-down; with acc
// set, the same walk also writes the forward accelerations (fused).
static og_status adjoint_walk(const og_tree* t, double r_s, double theta, og_precision prec, const float* w,
                              int64_t g_begin, int64_t g_end, float* acc, uint64_t* n_interact, int32_t* counts,
                              double* dpos, double* dmass, int recompute_lists, void* ws, size_t ws_bytes,
                              og_stream stream) {
  if (!w || !dpos || !dmass || !ws) return OG_EINVAL;
  if (prec != OG_FP32_KAHAN) return prec == OG_FP64 ? OG_ENOTIMPL : OG_EINVAL;
  if (recompute_lists != 1) return recompute_lists == 0 ? OG_ENOTIMPL : OG_EINVAL;
  WalkArgs A;
  og_status st = walk_common(t, r_s, theta, A);
  if (st != OG_OK) return st;
  if (g_begin < 0 || g_end < g_begin || g_end > t->n_groups) return OG_EINVAL;
  A.g_begin = g_begin;
  A.g_end = g_end;
  if (!aligned(ws)) return OG_EINVAL;
  const size_t need = og_adjoint_ws_bytes(t, recompute_lists);
  if (ws_bytes < need) return OG_ENOSPACE;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  AdjWs W;
  carve_adj(ws, t->n, t->node_capacity, &W);
  // status block and every accumulator start at zero
  cudaError_t e = cudaMemsetAsync(ws, 0, need, s);
  if (e != cudaSuccess) return OG_ECUDA;
  A.wsb = W.sb;
  A.w = w;
  A.Gn = W.Gn;
  A.Sn = W.Sn;
  A.Gp = W.Gp;
  A.Sp = W.Sp;
  A.tgt = W.tgt;
  if (acc) {
    A.accf = acc;
    A.counts = counts;
    A.total = reinterpret_cast<unsigned long long*>(n_interact);
    if (n_interact) {
      e = cudaMemsetAsync(n_interact, 0, sizeof(uint64_t), s);
      if (e != cudaSuccess) return OG_ECUDA;
    }
  }
  e = launch_walk(A, (int)prec, true, s, acc != nullptr);
  if (e != cudaSuccess) return OG_ECUDA;
  TreeDev T = tree_view(t);
  return cuda_status(launch_adjoint_push(T, W, t->box, dpos, dmass, s));
}

og_status og_shortrange_adjoint_range(const og_tree* t, double r_s, double theta, og_precision prec, const float* w,
                                      int64_t g_begin, int64_t g_end, double* dpos, double* dmass,
                                      int recompute_lists, void* ws, size_t ws_bytes, og_stream stream) {
  return adjoint_walk(t, r_s, theta, prec, w, g_begin, g_end, nullptr, nullptr, nullptr, dpos, dmass,
                      recompute_lists, ws, ws_bytes, stream);
}

og_status og_shortrange_accel_adjoint(const og_tree* t, double r_s, double theta, og_precision prec, const float* w,
                                      float* acc, uint64_t* n_interact, int32_t* counts, double* dpos,
                                      double* dmass, void* ws, size_t ws_bytes, og_stream stream) {
  if (!t) return OG_ETREE;
  if (!acc) return OG_EINVAL;
  return adjoint_walk(t, r_s, theta, prec, w, 0, t->n_groups, acc, n_interact, counts, dpos, dmass, 1, ws,
                      ws_bytes, stream);
}

og_status og_poll_status(const void* buf, og_stream stream) {
  if (!buf) return OG_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (cudaStreamSynchronize(s) != cudaSuccess) return OG_ECUDA;
  uint32_t st = 0;
  if (cudaMemcpy(&st, buf, sizeof(st), cudaMemcpyDeviceToHost) != cudaSuccess) return OG_ECUDA;
  if (st & ST_BADINPUT) return OG_EINVAL;
  if (st & ST_NOSPACE) return OG_ENOSPACE;
  if (st & (ST_TREELINK | ST_NOTREE)) return OG_ETREE;
  if (st & (ST_WALKCAP | ST_STACK)) return OG_EWALK;
  return OG_OK;
}

int64_t og_tree_node_count(const og_tree* t, og_stream stream) {
  if (!t || !t->built || !t->mem) return -1;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (cudaStreamSynchronize(s) != cudaSuccess) return -1;
  StatusBlock sb;
  if (cudaMemcpy(&sb, t->mem, sizeof(sb), cudaMemcpyDeviceToHost) != cudaSuccess) return -1;
  int64_t tot = 0;
  for (int l = 0; l < kLevels; ++l) tot += sb.level_cnt[l];
  return tot;
}

og_status og_tree_copy_nodes(const og_tree* t, int32_t* level, int32_t* first, int32_t* count, int32_t* parent,
                             double* mass, double* com, double* hmax, int32_t* child_first, int32_t* nchild,
                             og_stream stream) {
  if (!t || !t->built || !t->mem) return OG_ETREE;
  const int64_t m = og_tree_node_count(t, stream);
  if (m < 0) return OG_ECUDA;
  if (m > t->node_capacity) return OG_ENOSPACE;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  TreeDev T = tree_view(t);
  return cuda_status(launch_copy_nodes(T, m, level, first, count, parent, mass, com, hmax, child_first, nchild, s));
}

const char* og_status_str(og_status st) {
  switch (st) {
    case OG_OK: return "ok";
    case OG_EINVAL: return "invalid argument or non-finite input";
    case OG_ENOSPACE: return "workspace, tree buffer or node capacity too small";
    case OG_ECUDA: return "CUDA runtime error";
    case OG_EWALK: return "walk iteration cap or traversal stack overflow";
    case OG_ETREE: return "tree missing, not built or corrupt";
    case OG_ENOTIMPL: return "option not implemented";
  }
  return "unknown status";
}

}  // extern "C"
