/*
 * og.h -- C ABI of the GB300 short-range gravity library (libog.so).
 *
 * The library computes the short-range part of a TreePM gravity force in a
 * periodic box, i.e. the Barnes-Hut tree walk the paper ports to GPUs
 * (Sec. 2: a tree walk per active particle; Sec. 3.1: Barnes-Hut for the
 * short-range force, long-range PM on the host), and around it the
 * long-range mesh, the leapfrog step and the SPH density.  The steps are
 *
 *   og_keys_sort          63-bit Peano-Hilbert keys + stable radix sort
 *   og_tree_build         octree with monopole moments, level by level
 *   og_shortrange_accel   warp-coherent Barnes-Hut walk (FP32 + Kahan, or FP64)
 *   og_shortrange_adjoint gradient of L = sum_i w_i . a_i with frozen decisions
 *   og_shortrange_accel_adjoint  both in one walk (w known before the forces)
 *   og_pm_accel           the long-range complement on a particle mesh
 *   og_kick / og_drift    the leapfrog step's kick and drift
 *   og_sph_density        SPH density and smoothing length on the same tree
 *
 * Physics conventions (G = 1, attractive, code units):
 *   a_i = -sum_s m_s K_h(r) f(r) d,  d = x_i - x_s (periodic minimum image),
 *   f(r) = erfc(r / 2 r_s) + (r / (sqrt(pi) r_s)) exp(-r^2 / 4 r_s^2),
 *   contributions only for r < rcut = rcut_factor * r_s (default 4.5),
 *   K_h(r) = 1/r^3 for r >= h, the cubic-spline softened kernel inside,
 *   h = 2.8 eps, pairs use max(h_i, h_j), node terms max(h_i, hmax_node).
 * Opening rule for target i and node n (side s, geometric centre c, COM X):
 *   discard if the node cube is farther than rcut from x_i;
 *   accept (one monopole term) if s^2 < theta^2 |x_i - X|^2, x_i is outside
 *   the cube enlarged 1.2x and the whole cube lies within rcut;
 *   otherwise open (a leaf gives particle-particle terms, self excluded).
 *
 * Memory and ownership.  The caller owns every buffer.  Unless stated
 * otherwise, pointers are DEVICE pointers on the current CUDA device; the
 * og_params and og_tree structs are HOST structs.  The library never
 * allocates or frees device memory (except cuFFT, for its own tables, when
 * og_pm_plan_create makes a plan) and never synchronises, except in
 * og_poll_status / og_tree_node_count.  Every call is asynchronous on the
 * given stream.  Workspaces are sized by the *_ws_bytes / og_tree_bytes
 * helpers and must be 256-byte aligned.
 *
 * Errors.  Host-side argument errors are returned immediately.  Errors found
 * on the device (non-finite positions, node capacity exceeded, walk iteration
 * cap or stack overflow, corrupt links) are recorded in a status word at the
 * start of the workspace / tree buffer and returned by og_poll_status.  No
 * C++ exception crosses this interface.
 */
#ifndef OG_H
#define OG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* A cudaStream_t, passed as an opaque pointer (NULL = the legacy stream). */
typedef void* og_stream;

typedef enum og_status {
  OG_OK = 0,
  OG_EINVAL = 1,    /* bad argument (host check), or non-finite input found on device */
  OG_ENOSPACE = 2,  /* workspace or tree buffer too small (host), node capacity exceeded (device) */
  OG_ECUDA = 3,     /* a CUDA runtime call or kernel launch failed */
  OG_EWALK = 4,     /* walk iteration cap hit or traversal stack overflow (device) */
  OG_ETREE = 5,     /* tree missing, not built, or with out-of-range links (device) */
  OG_ENOTIMPL = 6   /* option not implemented */
} og_status;

typedef enum og_precision {
  OG_FP32_KAHAN = 0, /* FP32 interactions, compensated per-particle sums, output float[n][3] */
  OG_FP64 = 1        /* FP64 throughout, output double[n][3] */
} og_precision;

/* Tunables; the paper fixes none of them.  og_params_default() fills:
 * leaf_size 16, rcut_factor 4.5, node_capacity 0 (= 2n + 1024),
 * max_walk_iters 0 (= 2^24 node visits per 32-particle group). */
typedef struct og_params {
  int32_t leaf_size;       /* B: a node with more than B particles is split (1..32) */
  int32_t deep_stack;      /* walk stack depth above which a step pops a single child range: 0 = 64, the
                              largest allowed; a smaller value only trades speed for a lower stack */
  double rcut_factor;      /* rcut = rcut_factor * r_s */
  int64_t node_capacity;   /* nodes reserved in the tree buffer */
  int64_t max_walk_iters;  /* node-visit cap per group; exceeding it sets OG_EWALK */
} og_params;

void og_params_default(og_params* p);

/* Host header of a tree that lives in a caller-owned device buffer.  Filled
 * by og_tree_build; the fields are read-only for the caller.  The buffer
 * must stay alive and unmodified while the tree is used. */
typedef struct og_tree {
  int64_t n;               /* particles */
  int64_t n_groups;        /* ceil(n / 32): walk groups of Hilbert-consecutive particles */
  int64_t node_capacity;
  double box;              /* periodic box side L */
  double rcut_factor;
  int32_t leaf_size;
  int32_t built;           /* 1 after a successful og_tree_build launch */
  void* mem;               /* device buffer (starts with the status block) */
  size_t mem_bytes;
  int64_t max_walk_iters;
  int32_t deep_stack;      /* from og_params (0 replaced by 64) */
  int32_t reserved1;
} og_tree;

/* Bytes of workspace og_keys_sort needs for n particles. */
size_t og_keys_sort_ws_bytes(int64_t n);

/* Bytes of tree buffer for n particles (p may be NULL for defaults). */
size_t og_tree_bytes(int64_t n, const og_params* p);

/* Bytes of workspace for og_shortrange_accel / og_shortrange_adjoint. */
size_t og_accel_ws_bytes(const og_tree* t, og_precision prec);
size_t og_adjoint_ws_bytes(const og_tree* t, int recompute_lists);

/*
 * og_keys_sort -- Peano-Hilbert keys and their stable sort.
 *
 * The paper builds its tree on the host and offloads it every step (Sec. 2.1,
 * Appendix A); Gadget-family codes order particles along a Peano-Hilbert
 * curve (Sec. 2: the infrastructure inherited from Gadget3).  Here:
 *   w = x - L floor(x / L)            (each axis, FP64, rounded once per op)
 *   q = clamp(floor((w / L) 2^21), 0, 2^21 - 1)
 *   key = 63-bit Hilbert index of (q0, q1, q2) (Skilling's transpose form,
 *         axis 0 most significant within each 3-bit digit)
 * then (key, index) pairs are sorted ascending, ties by original index.
 *
 * pos          device, double[n][3], any real values (wrapped periodically)
 * n            1 <= n <= 2^31 - 1
 * box          L > 0
 * keys_sorted  device out, uint64[n]: keys in ascending order
 * order        device out, int32[n]: order[k] = original index of the k-th key
 * ws, ws_bytes device workspace of at least og_keys_sort_ws_bytes(n)
 * Non-finite positions set OG_EINVAL in the workspace status word.
 */
og_status og_keys_sort(const double* pos, int64_t n, double box, uint64_t* keys_sorted, int32_t* order,
                       void* ws, size_t ws_bytes, og_stream stream);

/*
 * og_tree_build -- octree with monopole moments over the sorted particles.
 *
 * The paper's gravity solver walks a Barnes-Hut tree that the host builds
 * and offloads to the GPU every step (Sec. 2.1, and the offloaded tree
 * structures of Appendix A); here the tree is built on the device from the
 * sorted keys.  A node is a maximal run of sorted keys that share their top 3*level bits
 * (the cell at that level); a node with more than leaf_size particles below
 * level 21 is split into its non-empty octants.  Per node: member range,
 * mass M = sum m (FP64), centre of mass sum(m x)/M (FP64), geometric centre
 * and side L / 2^level, largest member softening length.  Built top-down one
 * level per launch (children by binary search on the keys) and reduced
 * bottom-up one level per launch.  Particles are copied into Hilbert order.
 *
 * keys_sorted, order  outputs of og_keys_sort for the same pos / n / box
 * pos          device, double[n][3] (original order)
 * mass         device, double[n] (original order), > 0
 * eps          device, double[n] softening lengths (original order), or NULL
 *              to use eps_scalar for every particle; eps > 0
 * p            tunables (NULL = defaults); tree_mem/tree_bytes: device buffer
 *              of at least og_tree_bytes(n, p)
 * tree_out     host struct filled on success
 * Capacity overflow sets OG_ENOSPACE in the tree status word.
 */
og_status og_tree_build(const uint64_t* keys_sorted, const int32_t* order, const double* pos, const double* mass,
                        const double* eps, double eps_scalar, int64_t n, double box, const og_params* p,
                        void* tree_mem, size_t tree_bytes, og_tree* tree_out, og_stream stream);

/*
 * og_shortrange_accel -- short-range accelerations by the tree walk.
 *
 * One warp walks the tree for 32 Hilbert-consecutive targets (the grouping
 * idea of Sec. 2 and the 32-wide neighbour chunks of Sec. 2.1), keeping a
 * per-target lane mask so that every target gets exactly its own opening
 * decisions (the same as a per-particle walk).  OG_FP32_KAHAN: displacements
 * are formed to FP64 accuracy from split-float positions and rounded to FP32,
 * interactions run in FP32 on the special-function unit, per-target sums are
 * Kahan-compensated; decisions that FP32 cannot settle are re-taken in FP64.
 * OG_FP64: the same walk in double precision.
 *
 * r_s > 0 with rcut_factor * r_s < box / 2; theta >= 0
 * acc          device out, float[n][3] (FP32_KAHAN) or double[n][3] (FP64),
 *              original particle order
 * n_interact   device out (optional, may be NULL): uint64 total number of
 *              interactions (accepted nodes + particle pairs inside rcut)
 * counts       device out (optional, may be NULL): int32[n] interactions per
 *              particle, original order
 * ws, ws_bytes device workspace of at least og_accel_ws_bytes(t, prec)
 */
og_status og_shortrange_accel(const og_tree* t, double r_s, double theta, og_precision prec, void* acc,
                              uint64_t* n_interact, int32_t* counts, void* ws, size_t ws_bytes, og_stream stream);

/*
 * og_shortrange_adjoint -- dL/dx and dL/dm for L = sum_i w_i . a_i.
 *
 * The paper has no adjoint: this call differentiates the walk of
 * og_shortrange_accel (Sec. 2, 3.1: the Barnes-Hut short-range force) with
 * respect to positions and masses, for a loss linear in the accelerations.
 * The opening, cut and softening decisions of og_shortrange_accel are frozen
 * (recomputed deterministically by the same walk).  With g(d) = -F(r) d and
 * J = dg/dd = -F I - (F'/r) d d^T:
 *   target side  dL/dx_i += sum_s M_s J(d_is) w_i
 *   source side  for every term (i, s) and every particle k in s:
 *                dL/dx_k -= m_k J(d_is) w_i,
 *                dL/dm_k += w_i . g(d_is) - (J(d_is) w_i) . (x_k - X_s)
 * (node centres of mass move with their members).  Source terms are summed
 * per node in FP64 and pushed down the tree level by level.
 *
 * w            device, float[n][3] (original order)
 * dpos         device out, double[n][3]; dmass device out, double[n]
 * recompute_lists  must be 1 (interaction lists are recomputed; storing them
 *              returns OG_ENOTIMPL)
 * prec         OG_FP32_KAHAN (FP32 interactions; FP64 accumulators)
 */
og_status og_shortrange_adjoint(const og_tree* t, double r_s, double theta, og_precision prec, const float* w,
                                double* dpos, double* dmass, int recompute_lists, void* ws, size_t ws_bytes,
                                og_stream stream);

/*
 * og_shortrange_accel_adjoint -- og_shortrange_accel (FP32_KAHAN) and
 * og_shortrange_adjoint in one walk, for a loss L = sum_i w_i . a_i whose
 * weights w are known before the forces (the paper's walk, Sec. 2, 3.1, and
 * its adjoint as documented above).  Each pair's force factor F(r) serves
 * both the forward term and the adjoint terms, so the traversal, staging and
 * cut tests are done once.
 *
 * The walk's decisions, batches and summation order are those of the
 * separate calls, so acc, n_interact and counts equal og_shortrange_accel's
 * and dpos, dmass equal og_shortrange_adjoint's for the same tree.
 *
 * prec         OG_FP32_KAHAN only (OG_FP64: OG_ENOTIMPL)
 * w            device, float[n][3] (original order)
 * acc          device out, float[n][3], original order (required)
 * n_interact   device out (optional, may be NULL): uint64 total interactions
 * counts       device out (optional, may be NULL): int32[n], original order
 * dpos         device out, double[n][3]; dmass device out, double[n]
 * ws, ws_bytes device workspace of at least og_adjoint_ws_bytes(t, 1)
 * Status and errors as for og_shortrange_adjoint (read with og_poll_status
 * on ws).
 */
og_status og_shortrange_accel_adjoint(const og_tree* t, double r_s, double theta, og_precision prec, const float* w,
                                      float* acc, uint64_t* n_interact, int32_t* counts, double* dpos,
                                      double* dmass, void* ws, size_t ws_bytes, og_stream stream);

/*
 * og_shortrange_accel_range / og_shortrange_adjoint_range -- the same walks
 * over the walk groups [g_begin, g_end) only, i.e. over the targets with
 * sorted indices [32 g_begin, min(32 g_end, n)): a contiguous range of
 * Peano-Hilbert keys.
 *
 * The paper distributes the walk over MPI ranks by domain, exchanging the
 * particles a rank's targets need (Sec. 2).  These calls are the per-rank
 * part of a key-range decomposition in which every rank holds the same tree
 * (built from all positions) and walks its own range of groups; the
 * package's KeyRangeDecomposition does the collectives.
 *
 * accel_range: like og_shortrange_accel, but only the range's targets are
 *   written (acc, counts: original order; entries of other particles are
 *   left untouched); n_interact counts the range's interactions.
 * adjoint_range: the gradient of the partial loss L_r = sum over the range's
 *   targets i of w_i . a_i (w of other targets is ignored), for every
 *   particle: dpos and dmass are fully written.  The gradients of the ranges
 *   of a partition of [0, n_groups) add up to og_shortrange_adjoint's.
 * 0 <= g_begin <= g_end <= n_groups, else OG_EINVAL; an empty range writes
 *   nothing (accel) or zero gradients (adjoint).  Everything else as for the
 *   full calls.
 */
og_status og_shortrange_accel_range(const og_tree* t, double r_s, double theta, og_precision prec,
                                    int64_t g_begin, int64_t g_end, void* acc, uint64_t* n_interact,
                                    int32_t* counts, void* ws, size_t ws_bytes, og_stream stream);
og_status og_shortrange_adjoint_range(const og_tree* t, double r_s, double theta, og_precision prec, const float* w,
                                      int64_t g_begin, int64_t g_end, double* dpos, double* dmass,
                                      int recompute_lists, void* ws, size_t ws_bytes, og_stream stream);

/*
 * og_keys_sort_noalloc -- og_keys_sort for callers that cannot allocate.
 *
 * The paper has no counterpart: this is a convenience of this library.  Some
 * callers cannot call cudaMalloc, or are not allowed to: for example a host
 * application that hands all GPU memory to its own pool and forbids libraries
 * to allocate, or a loop that must not stall on an allocation.  This call
 * computes exactly what og_keys_sort computes (same keys, same order) without
 * a caller workspace: its scratch is a static device array of the library,
 * sized for at most 2^20 particles (about 12.5 MiB), which every GPU that
 * loads the library holds until the process exits.
 *
 * pos, n, box, keys_sorted, order, stream: as for og_keys_sort; n > 2^20
 * returns OG_ENOSPACE (use og_keys_sort with a workspace for larger sets).
 * The first call on a device looks up the device address of the static array
 * (cudaGetSymbolAddress); make that first call before any stream capture.
 * All calls share the one array: calls that overlap on the GPU (other streams
 * or threads of the same process on the same device) race and must be
 * ordered by the caller.  The array keeps the previous call's contents; the
 * call clears what must start at zero.  There is no status word the caller
 * can read: non-finite positions get key 0 (they sort first), so check
 * positions beforehand if they may be non-finite.  Nothing is allocated or
 * freed, and the stream is not synchronised.
 */
og_status og_keys_sort_noalloc(const double* pos, int64_t n, double box, uint64_t* keys_sorted, int32_t* order,
                               og_stream stream);

/*
 * PM long-range complement of the TreePM split.
 *
 * The paper (Sec. 3.1) adds long-range forces from a particle mesh, which it
 * solves with FFTW on the host.  Here the mesh is on the device:
 *   CIC deposit onto N^3 nodes at x = i L / N (periodic);
 *   FP32 FFT (cuFFT);
 *   phi_hat = -4 pi rho_hat exp(-k^2 r_s^2) / (k^2 S), with S = prod_a
 *     sinc^4(kappa_a / N) deconvolving the CIC window twice and phi_hat(0) = 0;
 *   inverse FFT;
 *   a four-point central-difference gradient;
 *   CIC interpolation back to the particles.
 * G = 1.  With the same r_s, the short-range walk plus this long-range
 * acceleration is the full periodic force (up to the mesh's discretisation
 * error and the walk's cut at rcut).
 *
 * og_pm_plan_create -- make the cuFFT plans for an N^3 mesh (8 <= ngrid <=
 *   1024; a power of two is fastest).  The plan is host memory plus cuFFT's
 *   own tables, which cuFFT allocates on the current device when the plan is
 *   made (the one place this library lets a callee allocate device memory;
 *   the work area and the meshes are the caller's workspace).  *plan is NULL
 *   on error.  Returns OG_EINVAL for a bad ngrid, OG_ECUDA if cuFFT fails.
 * og_pm_plan_destroy -- release a plan (NULL is ignored).  Not while a call
 *   that uses it may still run on the GPU.
 * og_pm_ws_bytes -- workspace bytes for og_pm_accel with this plan: status
 *   block, real mesh (4 N^3 B), complex mesh (8 N^2 (N/2 + 1) B), cuFFT work
 *   area.  0 for a NULL plan.
 * og_pm_accel -- long-range accelerations.
 *   pos   device double[n][3], any real values (wrapped into [0, box));
 *   mass  device double[n];
 *   n     1 .. 2^31 - 16;  box, r_s > 0 and finite;
 *   ws    device workspace of ws_bytes >= og_pm_ws_bytes(plan), 256-byte
 *         aligned; its first word is a status word (og_poll_status);
 *   acc   device float[n][3] out, in the order of pos.
 *   A plan holds one stream and one work area at a time: calls that share a
 *   plan must not overlap (on different streams or threads).
 *   Host-side argument errors return OG_EINVAL / OG_ENOSPACE.  Non-finite
 *   positions or masses are skipped (acceleration 0) and flagged in the
 *   status word (og_poll_status then returns OG_EINVAL).  The call is
 *   asynchronous and can be captured in a CUDA graph.
 */
typedef struct og_pm_plan og_pm_plan;

og_status og_pm_plan_create(int32_t ngrid, og_pm_plan** plan);
void og_pm_plan_destroy(og_pm_plan* plan);
size_t og_pm_ws_bytes(const og_pm_plan* plan);
og_status og_pm_accel(og_pm_plan* plan, const double* pos, const double* mass, int64_t n, double box, double r_s,
                      void* ws, size_t ws_bytes, float* acc, og_stream stream);

/*
 * Leapfrog kick and drift (the paper's step drifts every particle at its
 * start and kicks with the new gravity, Sec. 2.1).  A kick-drift-kick step
 * is og_kick(dt / 2), og_drift(dt), the forces (og_keys_sort,
 * og_tree_build, og_shortrange_accel, og_pm_accel), og_kick(dt / 2).
 *
 * og_kick  -- vel += dt (acc_a + acc_b), componentwise in FP64.
 *   vel    device double[n][3], updated in place;
 *   acc_a  device float[n][3] (e.g. the FP32 walk's output);
 *   acc_b  device float[n][3] or NULL (e.g. og_pm_accel's output).
 * og_drift -- pos += dt vel; positions are not wrapped (every force call
 *   wraps them itself).
 *   pos    device double[n][3], updated in place;  vel device double[n][3].
 * Both: 1 <= n <= 2^31 - 16, dt finite, else OG_EINVAL; asynchronous on
 * the stream; OG_ECUDA if the launch fails.
 */
og_status og_kick(double* vel, const float* acc_a, const float* acc_b, int64_t n, double dt, og_stream stream);
og_status og_drift(double* pos, const double* vel, int64_t n, double dt, og_stream stream);

/*
 * SPH density and smoothing length on the tree (the paper's SPH density
 * module iterates h until the sphere holds a fixed number of neighbours,
 * Sec. 2.1).  With the cubic spline W of support h:
 *   rho_i = sum_j m_j W(r_ij, h_i), the particle itself included, and
 *   h_i is the root of (4 pi / 3) h^3 sum_j W(r_ij, h) = n_ngb
 *   (periodic minimum image; h < box / 2).
 * og_sph_ws_bytes -- workspace bytes (a status block).
 * og_sph_density  -- t: a tree from og_tree_build (its positions and masses);
 *   n_ngb > 0; ws of ws_bytes >= og_sph_ws_bytes(), 256-byte aligned;
 *   outputs in the original particle order: h double[n], rho double[n],
 *   ngb int32[n] (neighbours strictly inside h, self excluded).
 *   A particle whose h cannot be bracketed below box / 2, or whose
 *   iteration hits its pass caps, gets NaN / -1 and sets a status bit
 *   (og_poll_status returns OG_EWALK; a corrupt tree gives OG_ETREE).
 *   h and rho agree with the FP64 definition to ~1e-11 relative (FP32
 *   iterations, then a step from float-float neighbour sums).
 *   Asynchronous on the stream.
 */
size_t og_sph_ws_bytes(void);
og_status og_sph_density(const og_tree* t, double n_ngb, void* ws, size_t ws_bytes, double* h, double* rho,
                         int32_t* ngb, og_stream stream);

/*
 * og_probe_pipe -- throughput probe of one SM pipe (measurement helper).
 *
 * The paper has no counterpart: the walks are bound by the FP32 pipe, the
 * special-function unit and (the comparison variant) the FP64 pipe, and the
 * roofline fractions reported for them need those pipes' rates as measured on
 * the device, not unit counts.  One launch runs independent dependency chains
 * of one instruction kind on every SM (4 blocks of 256 threads per SM); the
 * caller times it with CUDA events on the stream and divides *ops by the time.
 *
 * kind   OG_PROBE_FFMA  fma.rn.f32 (ops = FMAs; flops = 2 ops)
 *        OG_PROBE_FFMA2 fma.rn.f32x2, two FMAs per instruction (ops = FMAs)
 *        OG_PROBE_MUFU  alternating rsqrt.approx / ex2.approx (ops = MUFU ops)
 *        OG_PROBE_DFMA  fma.rn.f64 (ops = FMAs)
 * iters  1 .. 2^24; each thread performs iters x 128 operations
 *        (x 2 for FFMA2); about 2^12 gives a launch of some milliseconds
 * sink   device float[1]; never written in practice (it keeps the chains live)
 * ops    host out: operations the launch performs
 * Returns OG_EINVAL for a bad kind or iters, OG_ECUDA if the launch fails.
 */
enum { OG_PROBE_FFMA = 0, OG_PROBE_FFMA2 = 1, OG_PROBE_MUFU = 2, OG_PROBE_DFMA = 3 };
og_status og_probe_pipe(int32_t kind, int32_t iters, float* sink, uint64_t* ops, og_stream stream);

/* Synchronise the stream and return the status recorded on the device in a
 * workspace or tree buffer (any buffer sized by the helpers above). */
og_status og_poll_status(const void* buf, og_stream stream);

/* Synchronise and return the number of tree nodes (or -1 on error). */
int64_t og_tree_node_count(const og_tree* t, og_stream stream);

/* Copy node fields into caller device buffers (any may be NULL), nodes in
 * the tree's internal order, first og_tree_node_count() entries valid:
 * level, first (sorted particle index), count, parent (-1 for the root),
 * mass (FP64), com (FP64 [.][3]), hmax (FP64), child_first, nchild. */
og_status og_tree_copy_nodes(const og_tree* t, int32_t* level, int32_t* first, int32_t* count, int32_t* parent,
                             double* mass, double* com, double* hmax, int32_t* child_first, int32_t* nchild,
                             og_stream stream);

const char* og_status_str(og_status s);

#ifdef __cplusplus
}
#endif

#endif /* OG_H */
