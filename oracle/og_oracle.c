/*
 * og_oracle.c -- FP64 single-threaded CPU oracle for the TreePM short-range
 * gravity hot path (Peano-Hilbert keys, octree with monopoles, Barnes-Hut
 * walk with periodic minimum image, cubic-spline softening and the erfc/exp
 * short-range factor cut at rcut; plus the adjoint with frozen decisions).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct
 * reference that the CUDA path is checked against.  Only the test suite, the
 * smoke check and the benchmark's CPU-baseline leg may load it.  It shares no
 * code, header, table or constant generator with the CUDA library.
 *
 * The paper (Sec. 2, Sec. 3.1) names the method -- a Barnes-Hut tree walk
 * for the short-range part of a TreePM split, with the long-range part on a
 * PM grid -- but prints none of its formulas.  The formulas below are the
 * standard GADGET-family ones, each stated where it is used:
 *
 *   short-range factor  f(u) = erfc(u) + (2u/sqrt(pi)) exp(-u^2),  u = r/(2 r_s)
 *   cut                 contributions only for r < rcut (rcut = 4.5 r_s)
 *   softening           cubic-spline (Monaghan-Lattanzio) force kernel K_h(r),
 *                       h = 2.8 eps; K_h = 1/r^3 for r >= h
 *   pair acceleration   a_i += -m_j K_h(r) f(u) d,  d = x_i - x_j (minimum image)
 *   keys                63-bit 3-D Hilbert index of the 2^21-per-axis cell,
 *                       by Skilling's (2004) transpose method
 *   tree                octree over the integer cell grid; a node with more
 *                       than B particles below level 21 is split into octants
 *   opening             discard if the node cube is farther than rcut;
 *                       accept (monopole) if side^2 < theta^2 d^2, the target
 *                       is outside the node cube enlarged 1.2x and the whole
 *                       cube lies inside rcut; else open
 *
 * Parity status per function (pins live in tests/test_oracle_*.py):
 *   orc_keys / orc_sort          pinned (Gray-code order 1, bijection,
 *                                face adjacency, nested prefixes)
 *   orc_kernel_K / orc_kernel_f  pinned (enclosed-mass integral of the spline
 *                                density; closed-form derivative of f)
 *   orc_direct                   pinned (two-body closed form, Newtonian limit,
 *                                momentum, pair count vs an independent k-d tree)
 *   orc_tree_* / orc_walk        pinned (theta = 0 equals the direct sum; exact
 *                                cover of the particle set; node moments)
 *   orc_adjoint / orc_fd         pinned (analytic gradient vs central finite
 *                                differences of the forward sum)
 *
 * Build: gcc -O2 -ffp-contract=off -fPIC -shared (no fused multiply-add, so the
 * FP64 decision formulas are evaluated exactly as written).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_BITS 21
#define ORC_QMAX 2097151u /* 2^21 - 1 */

/* ------------------------------------------------------------------ */
/* periodic wrap, quantisation, Hilbert keys                           */
/* ------------------------------------------------------------------ */

/* x folded into [0, box]: x - box*floor(x/box), each operation rounded once. */
static double orc_wrap(double x, double box) {
  double fl = floor(x / box);
  double prod = box * fl;
  return x - prod;
}

/* Integer cell of a wrapped coordinate on the 2^21 grid, clamped. */
static uint32_t orc_quant(double w, double box) {
  double t = (w / box) * 2097152.0;
  double fl = floor(t);
  if (fl < 0.0) return 0u;
  if (fl > (double)ORC_QMAX) return ORC_QMAX;
  return (uint32_t)fl;
}

/* Hilbert index of integer cell (q0,q1,q2), 21 bits per axis (Skilling 2004,
 * "Programming the Hilbert curve": axes -> transposed index, then the bits of
 * the transposed form are read out most-significant first, axis 0 first). */
static uint64_t orc_hilbert(uint32_t q0, uint32_t q1, uint32_t q2) {
  uint32_t X[3];
  X[0] = q0; X[1] = q1; X[2] = q2;
  /* From the top bit down: where axis i has the bit set, the lower bits of
   * axis 0 are inverted; otherwise the lower bits of axes 0 and i swap. */
  for (uint32_t Q = 1u << (ORC_BITS - 1); Q > 1u; Q >>= 1) {
    uint32_t low = Q - 1u;
    for (int i = 0; i < 3; i++) {
      if (X[i] & Q) {
        X[0] ^= low;
      } else {
        uint32_t swap = (X[0] ^ X[i]) & low;
        X[0] ^= swap;
        X[i] ^= swap;
      }
    }
  }
  /* Gray-code the axes against one another ... */
  X[1] ^= X[0];
  X[2] ^= X[1];
  /* ... then fold in the running parity of the last axis. */
  uint32_t par = 0u;
  for (uint32_t Q = 1u << (ORC_BITS - 1); Q > 1u; Q >>= 1)
    if (X[2] & Q) par ^= (Q - 1u);
  X[0] ^= par; X[1] ^= par; X[2] ^= par;
  uint64_t key = 0;
  for (int b = ORC_BITS - 1; b >= 0; b--) {
    uint64_t d = ((uint64_t)((X[0] >> b) & 1u) << 2) |
                 ((uint64_t)((X[1] >> b) & 1u) << 1) |
                 (uint64_t)((X[2] >> b) & 1u);
    key = (key << 3) | d;
  }
  return key;
}

uint64_t orc_hilbert_cell(uint32_t q0, uint32_t q1, uint32_t q2) {
  return orc_hilbert(q0, q1, q2);
}

/* Hilbert index on a 2^bits grid (bits <= 21) for exhaustive pins: the cell is
 * placed at the top of the 21-bit grid and the index is the top 3*bits bits. */
uint64_t orc_hilbert_grid(uint32_t q0, uint32_t q1, uint32_t q2, int bits) {
  int sh = ORC_BITS - bits;
  return orc_hilbert(q0 << sh, q1 << sh, q2 << sh) >> (3 * sh);
}

/* Keys for n positions.  Returns the number of non-finite inputs (their key
 * is set to 0).  qcell, if not NULL, receives the integer cells [n][3]. */
int64_t orc_keys(const double* pos, int64_t n, double box, uint64_t* keys, uint32_t* qcell) {
  int64_t bad = 0;
  for (int64_t i = 0; i < n; i++) {
    uint32_t q[3];
    int ok = 1;
    for (int a = 0; a < 3; a++) {
      double x = pos[3 * i + a];
      if (!isfinite(x)) { ok = 0; q[a] = 0; continue; }
      q[a] = orc_quant(orc_wrap(x, box), box);
    }
    if (!ok) { bad++; keys[i] = 0; }
    else keys[i] = orc_hilbert(q[0], q[1], q[2]);
    if (qcell) { qcell[3 * i] = q[0]; qcell[3 * i + 1] = q[1]; qcell[3 * i + 2] = q[2]; }
  }
  return bad;
}

typedef struct { uint64_t key; int64_t idx; } orc_kv;

static int orc_kv_cmp(const void* a, const void* b) {
  const orc_kv* x = (const orc_kv*)a;
  const orc_kv* y = (const orc_kv*)b;
  if (x->key < y->key) return -1;
  if (x->key > y->key) return 1;
  if (x->idx < y->idx) return -1;
  if (x->idx > y->idx) return 1;
  return 0;
}

/* Stable sort of keys: ascending key, ties by original index. */
void orc_sort(const uint64_t* keys, int64_t n, uint64_t* keys_sorted, int32_t* order) {
  orc_kv* kv = (orc_kv*)malloc(sizeof(orc_kv) * (size_t)(n > 0 ? n : 1));
  for (int64_t i = 0; i < n; i++) { kv[i].key = keys[i]; kv[i].idx = i; }
  qsort(kv, (size_t)n, sizeof(orc_kv), orc_kv_cmp);
  for (int64_t i = 0; i < n; i++) { keys_sorted[i] = kv[i].key; order[i] = (int32_t)kv[i].idx; }
  free(kv);
}

/* ------------------------------------------------------------------ */
/* force law                                                           */
/* ------------------------------------------------------------------ */

/* Short-range factor f(r) = erfc(u) + (2u/sqrt(pi)) exp(-u^2), u = r/(2 r_s). */
double orc_kernel_f(double r, double r_s) {
  double u = r / (2.0 * r_s);
  return erfc(u) + M_2_SQRTPI * u * exp(-u * u);
}

/* d f / d r = -(r^2 / (2 sqrt(pi) r_s^3)) exp(-u^2), divided by r. */
static double orc_kernel_fp_over_r(double r, double r_s) {
  double u = r / (2.0 * r_s);
  return -(r / (2.0 * sqrt(M_PI) * r_s * r_s * r_s)) * exp(-u * u);
}

/* Softened force kernel: acceleration magnitude per unit mass per unit
 * distance, so a pair contributes -m K_h(r) d.  K_h = 1/r^3 for r >= h; inside
 * h it is the force of the cubic-spline density of support h (v = r/h). */
double orc_kernel_K(double r, double h) {
  if (r >= h) return 1.0 / (r * r * r);
  double v = r / h;
  double h3 = 1.0 / (h * h * h);
  if (v < 0.5) return h3 * (32.0 / 3.0 + v * v * (32.0 * v - 38.4));
  return h3 * (64.0 / 3.0 - 48.0 * v + 38.4 * v * v - (32.0 / 3.0) * v * v * v -
               (1.0 / 15.0) / (v * v * v));
}

/* (d K_h / d r) / r. */
static double orc_kernel_Kp_over_r(double r, double h) {
  if (r >= h) { double r2 = r * r; return -3.0 / (r2 * r2 * r); }
  double v = r / h;
  double h5 = 1.0 / (h * h * h * h * h);
  if (v < 0.5) return h5 * (96.0 * v - 76.8);
  return h5 * (-48.0 / v + 76.8 - 32.0 * v + 0.2 / (v * v * v * v * v));
}

/* Minimum image of one displacement component (box > 2 |component| needed
 * for uniqueness; inputs here lie in (-box, box)). */
static double orc_mi(double t, double box) {
  if (t > 0.5 * box) return t - box;
  if (t < -0.5 * box) return t + box;
  return t;
}

static double orc_norm2(const double d[3]) { return (d[0] * d[0] + d[1] * d[1]) + d[2] * d[2]; }

/* F(r) = K_h(r) f(r): the pair acceleration is -m F d. */
static double orc_F(double r, double h, double r_s) { return orc_kernel_K(r, h) * orc_kernel_f(r, r_s); }

/* (dF/dr)/r. */
static double orc_Fp_over_r(double r, double h, double r_s) {
  return orc_kernel_Kp_over_r(r, h) * orc_kernel_f(r, r_s) + orc_kernel_K(r, h) * orc_kernel_fp_over_r(r, r_s);
}

/* ------------------------------------------------------------------ */
/* direct periodic sum (exact target for theta -> 0)                   */
/* ------------------------------------------------------------------ */

/* a_i = -sum_{j != i, r_ij < rcut} m_j K_{max(h_i,h_j)}(r_ij) f(r_ij) d_ij.
 * A cell list with cells no smaller than rcut visits a superset of all pairs
 * with r < rcut, so the sum is the same as the all-pairs sum. */
void orc_direct(const double* pos, const double* mass, const double* hs, int64_t n, double box,
                double r_s, double rcut, const int64_t* targets, int64_t nt, double* acc, int64_t* ninter) {
  double* x = (double*)malloc(sizeof(double) * 3 * (size_t)n);
  for (int64_t i = 0; i < 3 * n; i++) x[i] = orc_wrap(pos[i], box);
  double rc2 = rcut * rcut;
  int nc = (int)floor(box / rcut);
  if (nc > 256) nc = 256;
  if (nc < 3) {
    for (int64_t t = 0; t < nt; t++) {
      int64_t i = targets[t];
      double a[3] = {0, 0, 0};
      int64_t cnt = 0;
      for (int64_t j = 0; j < n; j++) {
        if (j == i) continue;
        double d[3];
        for (int c = 0; c < 3; c++) d[c] = orc_mi(x[3 * i + c] - x[3 * j + c], box);
        double r2 = orc_norm2(d);
        if (!(r2 < rc2)) continue;
        double h = hs[i] > hs[j] ? hs[i] : hs[j];
        double fac = mass[j] * orc_F(sqrt(r2), h, r_s);
        for (int c = 0; c < 3; c++) a[c] -= fac * d[c];
        cnt++;
      }
      for (int c = 0; c < 3; c++) acc[3 * t + c] = a[c];
      if (ninter) ninter[t] = cnt;
    }
    free(x);
    return;
  }
  int64_t ncell = (int64_t)nc * nc * nc;
  int64_t* head = (int64_t*)malloc(sizeof(int64_t) * (size_t)(ncell + 1));
  int64_t* cellof = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
  int64_t* list = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
  memset(head, 0, sizeof(int64_t) * (size_t)(ncell + 1));
  for (int64_t j = 0; j < n; j++) {
    int c3[3];
    for (int c = 0; c < 3; c++) {
      int v = (int)floor(x[3 * j + c] / box * nc);
      if (v < 0) v = 0;
      if (v >= nc) v = nc - 1;
      c3[c] = v;
    }
    cellof[j] = ((int64_t)c3[0] * nc + c3[1]) * nc + c3[2];
    head[cellof[j] + 1]++;
  }
  for (int64_t c = 0; c < ncell; c++) head[c + 1] += head[c];
  {
    int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)ncell);
    memcpy(fill, head, sizeof(int64_t) * (size_t)ncell);
    for (int64_t j = 0; j < n; j++) list[fill[cellof[j]]++] = j;
    free(fill);
  }
  for (int64_t t = 0; t < nt; t++) {
    int64_t i = targets[t];
    double a[3] = {0, 0, 0};
    int64_t cnt = 0;
    int ci[3];
    ci[0] = (int)(cellof[i] / ((int64_t)nc * nc));
    ci[1] = (int)((cellof[i] / nc) % nc);
    ci[2] = (int)(cellof[i] % nc);
    for (int o0 = -1; o0 <= 1; o0++)
      for (int o1 = -1; o1 <= 1; o1++)
        for (int o2 = -1; o2 <= 1; o2++) {
          int c0 = (ci[0] + o0 + nc) % nc, c1 = (ci[1] + o1 + nc) % nc, c2 = (ci[2] + o2 + nc) % nc;
          int64_t c = ((int64_t)c0 * nc + c1) * nc + c2;
          for (int64_t p = head[c]; p < head[c + 1]; p++) {
            int64_t j = list[p];
            if (j == i) continue;
            double d[3];
            for (int k = 0; k < 3; k++) d[k] = orc_mi(x[3 * i + k] - x[3 * j + k], box);
            double r2 = orc_norm2(d);
            if (!(r2 < rc2)) continue;
            double h = hs[i] > hs[j] ? hs[i] : hs[j];
            double fac = mass[j] * orc_F(sqrt(r2), h, r_s);
            for (int k = 0; k < 3; k++) a[k] -= fac * d[k];
            cnt++;
          }
        }
    for (int c = 0; c < 3; c++) acc[3 * t + c] = a[c];
    if (ninter) ninter[t] = cnt;
  }
  free(head); free(cellof); free(list); free(x);
}

/* ------------------------------------------------------------------ */
/* octree over the integer cell grid                                   */
/* ------------------------------------------------------------------ */

typedef struct {
  int32_t level;
  uint32_t cell[3];     /* integer cell coordinates at this level */
  double side;          /* box / 2^level */
  double cen[3];        /* geometric centre ((cell + 0.5) * side) */
  double mass;          /* sum of member masses */
  double com[3];        /* sum m x / sum m */
  double hmax;          /* largest member softening length h */
  int64_t child0;       /* first child (children are contiguous) */
  int32_t nchild;
  int32_t leaf;
  int64_t pbeg, pend;   /* members: idx[pbeg..pend) */
  int64_t parent;
} orc_node;

typedef struct {
  int64_t n;
  double box;
  int leaf_size;
  double* x;        /* wrapped positions [n][3] */
  double* m;
  double* h;
  uint32_t* q;      /* integer cells [n][3] */
  int64_t* idx;     /* member permutation */
  int64_t* tmp;
  orc_node* nodes;
  int64_t nn, cap;
} orc_tree;

static int64_t orc_new_nodes(orc_tree* T, int64_t k) {
  if (T->nn + k > T->cap) {
    int64_t nc = T->cap * 2 + k + 64;
    T->nodes = (orc_node*)realloc(T->nodes, sizeof(orc_node) * (size_t)nc);
    T->cap = nc;
  }
  int64_t first = T->nn;
  T->nn += k;
  return first;
}

static void orc_fill_node(orc_tree* T, int64_t id) {
  orc_node* nd = &T->nodes[id];
  double M = 0.0, s[3] = {0, 0, 0}, hm = 0.0;
  for (int64_t p = nd->pbeg; p < nd->pend; p++) {
    int64_t j = T->idx[p];
    M += T->m[j];
    for (int c = 0; c < 3; c++) s[c] += T->m[j] * T->x[3 * j + c];
    if (T->h[j] > hm) hm = T->h[j];
  }
  nd->mass = M;
  for (int c = 0; c < 3; c++) nd->com[c] = s[c] / M;
  nd->hmax = hm;
  nd->side = ldexp(T->box, -nd->level);
  for (int c = 0; c < 3; c++) nd->cen[c] = ((double)nd->cell[c] + 0.5) * nd->side;
}

static void orc_build_rec(orc_tree* T, int64_t id) {
  orc_fill_node(T, id);
  orc_node nd = T->nodes[id];
  int64_t cnt = nd.pend - nd.pbeg;
  if (cnt <= T->leaf_size || nd.level >= ORC_BITS) {
    T->nodes[id].leaf = 1;
    T->nodes[id].nchild = 0;
    T->nodes[id].child0 = -1;
    return;
  }
  /* partition members by the octant bit of the next level (stable) */
  int sh = ORC_BITS - 1 - nd.level;
  int64_t bucket[9] = {0};
  for (int64_t p = nd.pbeg; p < nd.pend; p++) {
    int64_t j = T->idx[p];
    int o = (int)(((T->q[3 * j] >> sh) & 1u) | (((T->q[3 * j + 1] >> sh) & 1u) << 1) |
                  (((T->q[3 * j + 2] >> sh) & 1u) << 2));
    bucket[o + 1]++;
  }
  for (int o = 0; o < 8; o++) bucket[o + 1] += bucket[o];
  int64_t fill[8];
  for (int o = 0; o < 8; o++) fill[o] = nd.pbeg + bucket[o];
  for (int64_t p = nd.pbeg; p < nd.pend; p++) {
    int64_t j = T->idx[p];
    int o = (int)(((T->q[3 * j] >> sh) & 1u) | (((T->q[3 * j + 1] >> sh) & 1u) << 1) |
                  (((T->q[3 * j + 2] >> sh) & 1u) << 2));
    T->tmp[fill[o]++] = j;
  }
  memcpy(T->idx + nd.pbeg, T->tmp + nd.pbeg, sizeof(int64_t) * (size_t)cnt);
  int nchild = 0;
  for (int o = 0; o < 8; o++) if (bucket[o + 1] > bucket[o]) nchild++;
  int64_t c0 = orc_new_nodes(T, nchild);
  T->nodes[id].leaf = 0;
  T->nodes[id].child0 = c0;
  T->nodes[id].nchild = nchild;
  int k = 0;
  for (int o = 0; o < 8; o++) {
    if (bucket[o + 1] == bucket[o]) continue;
    orc_node* ch = &T->nodes[c0 + k];
    memset(ch, 0, sizeof(*ch));
    ch->level = nd.level + 1;
    ch->cell[0] = (nd.cell[0] << 1) | (uint32_t)(o & 1);
    ch->cell[1] = (nd.cell[1] << 1) | (uint32_t)((o >> 1) & 1);
    ch->cell[2] = (nd.cell[2] << 1) | (uint32_t)((o >> 2) & 1);
    ch->pbeg = nd.pbeg + bucket[o];
    ch->pend = nd.pbeg + bucket[o + 1];
    ch->parent = id;
    k++;
  }
  for (int i = 0; i < nchild; i++) orc_build_rec(T, c0 + i);
}

/* Build the oracle tree.  h[] are softening lengths (h = 2.8 eps), one per
 * particle.  Returns an opaque handle (free with orc_tree_free). */
void* orc_tree_build(const double* pos, const double* mass, const double* h, int64_t n, double box,
                     int leaf_size) {
  orc_tree* T = (orc_tree*)calloc(1, sizeof(orc_tree));
  T->n = n; T->box = box; T->leaf_size = leaf_size;
  T->x = (double*)malloc(sizeof(double) * 3 * (size_t)n);
  T->m = (double*)malloc(sizeof(double) * (size_t)n);
  T->h = (double*)malloc(sizeof(double) * (size_t)n);
  T->q = (uint32_t*)malloc(sizeof(uint32_t) * 3 * (size_t)n);
  T->idx = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
  T->tmp = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
  for (int64_t i = 0; i < n; i++) {
    for (int c = 0; c < 3; c++) {
      T->x[3 * i + c] = orc_wrap(pos[3 * i + c], box);
      T->q[3 * i + c] = orc_quant(T->x[3 * i + c], box);
    }
    T->m[i] = mass[i];
    T->h[i] = h[i];
    T->idx[i] = i;
  }
  T->cap = 1024;
  T->nodes = (orc_node*)malloc(sizeof(orc_node) * (size_t)T->cap);
  T->nn = 0;
  int64_t root = orc_new_nodes(T, 1);
  memset(&T->nodes[root], 0, sizeof(orc_node));
  T->nodes[root].level = 0;
  T->nodes[root].pbeg = 0;
  T->nodes[root].pend = n;
  T->nodes[root].parent = -1;
  orc_build_rec(T, root);
  free(T->tmp);
  T->tmp = NULL;
  return T;
}

void orc_tree_free(void* h) {
  orc_tree* T = (orc_tree*)h;
  if (!T) return;
  free(T->x); free(T->m); free(T->h); free(T->q); free(T->idx); free(T->tmp); free(T->nodes);
  free(T);
}

int64_t orc_tree_nnodes(void* h) { return ((orc_tree*)h)->nn; }

/* Export node data.  Any output pointer may be NULL. */
void orc_tree_nodes(void* hnd, int32_t* level, uint32_t* cell, int64_t* count, double* mass, double* com,
                    double* hmax, int32_t* leaf, int64_t* parent, int64_t* child0, int32_t* nchild) {
  orc_tree* T = (orc_tree*)hnd;
  for (int64_t k = 0; k < T->nn; k++) {
    orc_node* nd = &T->nodes[k];
    if (level) level[k] = nd->level;
    if (cell) for (int c = 0; c < 3; c++) cell[3 * k + c] = nd->cell[c];
    if (count) count[k] = nd->pend - nd->pbeg;
    if (mass) mass[k] = nd->mass;
    if (com) for (int c = 0; c < 3; c++) com[3 * k + c] = nd->com[c];
    if (hmax) hmax[k] = nd->hmax;
    if (leaf) leaf[k] = nd->leaf;
    if (parent) parent[k] = nd->parent;
    if (child0) child0[k] = nd->child0;
    if (nchild) nchild[k] = nd->nchild;
  }
}

/* Members of node k (particle indices), written to out (size >= count). */
void orc_tree_members(void* hnd, int64_t k, int64_t* out) {
  orc_tree* T = (orc_tree*)hnd;
  orc_node* nd = &T->nodes[k];
  for (int64_t p = nd->pbeg; p < nd->pend; p++) out[p - nd->pbeg] = T->idx[p];
}

/* ------------------------------------------------------------------ */
/* the walk                                                            */
/* ------------------------------------------------------------------ */

/* One interaction of a target: kind 0 = accepted node (id = node index),
 * kind 1 = particle-particle (id = particle index). */
typedef struct { int64_t id; int32_t kind; } orc_item;

typedef struct { orc_item* v; int64_t n, cap; } orc_list;

static void orc_push(orc_list* L, int32_t kind, int64_t id) {
  if (L->n == L->cap) {
    L->cap = L->cap * 2 + 64;
    L->v = (orc_item*)realloc(L->v, sizeof(orc_item) * (size_t)L->cap);
  }
  L->v[L->n].kind = kind;
  L->v[L->n].id = id;
  L->n++;
}

typedef struct {
  const orc_tree* T;
  double theta2, rc2, box;
  int64_t i;
  orc_list* out;     /* interactions (inside the cut) */
  orc_list* cover;   /* optional: every node discarded (kind 2), accepted (kind 0, any distance)
                        and every particle of an opened leaf (kind 1, incl. self and beyond cut) */
} orc_walkctx;

/* The node decisions for target i, in this order:
 *   1. discard: squared distance from x_i to the node cube (minimum image per
 *      axis) greater than rcut^2  -> nothing below this node interacts;
 *   2. accept:  side^2 < theta^2 d^2 (d = x_i - COM, minimum image), x_i is
 *      not inside the cube enlarged 1.2x (|x_i - centre| <= 0.6 side on every
 *      axis) and the farthest point of the cube is closer than rcut (a node
 *      that straddles the cut is opened, so the cut is applied per particle)
 *      -> one monopole interaction if d^2 < rcut^2;
 *   3. open:    a leaf gives particle-particle pairs (self excluded, r < rcut),
 *      an internal node recurses into its children. */
static void orc_visit(orc_walkctx* C, int64_t k) {
  const orc_tree* T = C->T;
  const orc_node* nd = &T->nodes[k];
  const double* xi = &T->x[3 * C->i];
  double box = C->box;
  double half = 0.5 * nd->side;
  double e2 = 0.0, cmax = 0.0;
  double dc[3];
  for (int c = 0; c < 3; c++) {
    dc[c] = fabs(orc_mi(xi[c] - nd->cen[c], box));
    if (dc[c] > cmax) cmax = dc[c];
  }
  {
    double e[3];
    for (int c = 0; c < 3; c++) { e[c] = dc[c] - half; if (e[c] < 0.0) e[c] = 0.0; }
    e2 = (e[0] * e[0] + e[1] * e[1]) + e[2] * e[2];
  }
  if (e2 > C->rc2) {
    if (C->cover) orc_push(C->cover, 2, k);
    return;
  }
  /* squared distance from x_i to the farthest point of the node cube */
  double far2;
  {
    double f[3];
    for (int c = 0; c < 3; c++) f[c] = dc[c] + half;
    far2 = (f[0] * f[0] + f[1] * f[1]) + f[2] * f[2];
  }
  double d[3];
  for (int c = 0; c < 3; c++) d[c] = orc_mi(xi[c] - nd->com[c], box);
  double d2 = orc_norm2(d);
  int inside = cmax <= 0.6 * nd->side;
  if ((nd->side * nd->side) < C->theta2 * d2 && !inside && far2 < C->rc2) {
    if (C->cover) orc_push(C->cover, 0, k);
    if (d2 < C->rc2) orc_push(C->out, 0, k);
    return;
  }
  if (nd->leaf) {
    for (int64_t p = nd->pbeg; p < nd->pend; p++) {
      int64_t j = T->idx[p];
      if (C->cover) orc_push(C->cover, 1, j);
      if (j == C->i) continue;
      double dj[3];
      for (int c = 0; c < 3; c++) dj[c] = orc_mi(xi[c] - T->x[3 * j + c], box);
      if (orc_norm2(dj) < C->rc2) orc_push(C->out, 1, j);
    }
    return;
  }
  for (int32_t c = 0; c < nd->nchild; c++) orc_visit(C, nd->child0 + c);
}

static void orc_walk_list(const orc_tree* T, int64_t i, double theta, double rcut, orc_list* out,
                          orc_list* cover) {
  orc_walkctx C;
  C.T = T; C.theta2 = theta * theta; C.rc2 = rcut * rcut; C.box = T->box; C.i = i;
  C.out = out; C.cover = cover;
  out->n = 0;
  if (cover) cover->n = 0;
  orc_visit(&C, 0);
}

/* Source of an interaction item: position, mass, softening. */
static void orc_item_source(const orc_tree* T, const orc_item* it, const double** X, double* M, double* h) {
  if (it->kind == 0) {
    const orc_node* nd = &T->nodes[it->id];
    *X = nd->com; *M = nd->mass; *h = nd->hmax;
  } else {
    *X = &T->x[3 * it->id]; *M = T->m[it->id]; *h = T->h[it->id];
  }
}

/* Tree-walk accelerations of the given targets. */
void orc_walk(void* hnd, double r_s, double rcut, double theta, const int64_t* targets, int64_t nt,
              double* acc, int64_t* ninter) {
  const orc_tree* T = (const orc_tree*)hnd;
  orc_list L = {0};
  for (int64_t t = 0; t < nt; t++) {
    int64_t i = targets[t];
    orc_walk_list(T, i, theta, rcut, &L, NULL);
    double a[3] = {0, 0, 0};
    const double* xi = &T->x[3 * i];
    for (int64_t q = 0; q < L.n; q++) {
      const double* X; double M, hs;
      orc_item_source(T, &L.v[q], &X, &M, &hs);
      double h = T->h[i] > hs ? T->h[i] : hs;
      double d[3];
      for (int c = 0; c < 3; c++) d[c] = orc_mi(xi[c] - X[c], T->box);
      double fac = M * orc_F(sqrt(orc_norm2(d)), h, r_s);
      for (int c = 0; c < 3; c++) a[c] -= fac * d[c];
    }
    for (int c = 0; c < 3; c++) acc[3 * t + c] = a[c];
    if (ninter) ninter[t] = L.n;
  }
  free(L.v);
}

/* Cover check: for each target, how many times each particle is reached
 * through a discarded node, an accepted node or an opened leaf.  A correct
 * walk reaches every particle exactly once.  Returns the number of
 * (target, particle) pairs reached a number of times other than one. */
int64_t orc_walk_cover_errors(void* hnd, double rcut, double theta, const int64_t* targets, int64_t nt) {
  const orc_tree* T = (const orc_tree*)hnd;
  orc_list L = {0}, Cv = {0};
  int32_t* hits = (int32_t*)malloc(sizeof(int32_t) * (size_t)T->n);
  int64_t bad = 0;
  for (int64_t t = 0; t < nt; t++) {
    memset(hits, 0, sizeof(int32_t) * (size_t)T->n);
    orc_walk_list(T, targets[t], theta, rcut, &L, &Cv);
    for (int64_t q = 0; q < Cv.n; q++) {
      if (Cv.v[q].kind == 1) { hits[Cv.v[q].id]++; continue; }
      const orc_node* nd = &T->nodes[Cv.v[q].id];
      for (int64_t p = nd->pbeg; p < nd->pend; p++) hits[T->idx[p]]++;
    }
    for (int64_t j = 0; j < T->n; j++) if (hits[j] != 1) bad++;
  }
  free(hits); free(L.v); free(Cv.v);
  return bad;
}

/* Interaction lists of the given targets, flattened: for target t the items
 * are out_kind/out_id[off[t] .. off[t+1]).  Call with out_kind == NULL to get
 * the offsets only. */
void orc_walk_lists(void* hnd, double rcut, double theta, const int64_t* targets, int64_t nt, int64_t* off,
                    int32_t* out_kind, int64_t* out_id) {
  const orc_tree* T = (const orc_tree*)hnd;
  orc_list L = {0};
  off[0] = 0;
  for (int64_t t = 0; t < nt; t++) {
    orc_walk_list(T, targets[t], theta, rcut, &L, NULL);
    if (out_kind) {
      for (int64_t q = 0; q < L.n; q++) {
        out_kind[off[t] + q] = L.v[q].kind;
        out_id[off[t] + q] = L.v[q].id;
      }
    }
    off[t + 1] = off[t] + L.n;
  }
  free(L.v);
}

/* ------------------------------------------------------------------ */
/* adjoint: dL/dx, dL/dm of L = sum_i w_i . a_i with frozen decisions  */
/* ------------------------------------------------------------------ */

/* For one interaction with displacement d (target minus source), softening h:
 *   g  = -F(r) d                         (acceleration per unit source mass)
 *   Jw = dg/dd . w = -F w - (F'/r)(d.w) d   (J is symmetric)              */
static void orc_pair_adj(const double d[3], double h, double r_s, const double w[3], double g[3], double Jw[3]) {
  double r = sqrt(orc_norm2(d));
  double F = orc_F(r, h, r_s);
  double Fr = orc_Fp_over_r(r, h, r_s);
  double dw = (d[0] * w[0] + d[1] * w[1]) + d[2] * w[2];
  for (int c = 0; c < 3; c++) {
    g[c] = -F * d[c];
    Jw[c] = -F * w[c] - Fr * dw * d[c];
  }
}

/* Targets whose interactions can involve particle k: for a particle-particle
 * term |x_i - x_k| < rcut; for an accepted node n containing k, the node side
 * is below theta*rcut so |x_i - x_k| < rcut (1 + sqrt(3) theta). */
static void orc_mark_neighbourhood(const orc_tree* T, int64_t k, double R2, uint8_t* mark) {
  for (int64_t i = 0; i < T->n; i++) {
    double d[3];
    for (int c = 0; c < 3; c++) d[c] = orc_mi(T->x[3 * i + c] - T->x[3 * k + c], T->box);
    if (orc_norm2(d) <= R2) mark[i] = 1;
  }
}

/* Nodes containing particle k, from the root down (writes up to 32 ids). */
static int orc_ancestors(const orc_tree* T, int64_t k, int64_t* anc) {
  int na = 0;
  int64_t cur = 0;
  for (;;) {
    anc[na++] = cur;
    const orc_node* nd = &T->nodes[cur];
    if (nd->leaf) break;
    int64_t next = -1;
    for (int32_t c = 0; c < nd->nchild; c++) {
      const orc_node* ch = &T->nodes[nd->child0 + c];
      int sh = ORC_BITS - ch->level;
      if ((T->q[3 * k] >> sh) == ch->cell[0] && (T->q[3 * k + 1] >> sh) == ch->cell[1] &&
          (T->q[3 * k + 2] >> sh) == ch->cell[2]) { next = nd->child0 + c; break; }
    }
    if (next < 0) break;
    cur = next;
  }
  return na;
}

/* Analytic gradient for the sample particles (all particles if samples ==
 * NULL).  w is [n][3] in original order.  Outputs are per sample.
 * dpos_abs / dmass_abs (optional, may be NULL): the same sums taken over the
 * absolute values of their terms, i.e. the scale against which the rounding
 * error of any evaluation of these sums is measured (a sum of terms each
 * computed with relative error e is off by at most e times this scale). */
void orc_adjoint(void* hnd, double r_s, double rcut, double theta, const double* w, const int64_t* samples,
                 int64_t ns, double* dpos, double* dmass, double* dpos_abs, double* dmass_abs) {
  const orc_tree* T = (const orc_tree*)hnd;
  int64_t n = T->n, M = T->nn;
  int all = samples == NULL;
  if (all) ns = n;
  uint8_t* mark = (uint8_t*)calloc((size_t)n, 1);
  int64_t* sidx = (int64_t*)malloc(sizeof(int64_t) * (size_t)(ns > 0 ? ns : 1));
  int64_t* slot = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
  for (int64_t i = 0; i < n; i++) slot[i] = -1;
  double R = rcut * (1.0 + sqrt(3.0) * theta) * (1.0 + 1e-9) + 1e-12;
  for (int64_t s = 0; s < ns; s++) {
    sidx[s] = all ? s : samples[s];
    slot[sidx[s]] = s;
  }
  if (all) memset(mark, 1, (size_t)n);
  else for (int64_t s = 0; s < ns; s++) orc_mark_neighbourhood(T, sidx[s], R * R, mark);
  double* Gn = (double*)calloc((size_t)M * 3, sizeof(double));
  double* Sn = (double*)calloc((size_t)M, sizeof(double));
  double* Gp = (double*)calloc((size_t)n * 3, sizeof(double));
  double* Sp = (double*)calloc((size_t)n, sizeof(double));
  double* tgt = (double*)calloc((size_t)ns * 3, sizeof(double));
  const int want_abs = dpos_abs != NULL || dmass_abs != NULL;
  double* Gna = want_abs ? (double*)calloc((size_t)M * 3, sizeof(double)) : NULL;
  double* Sna = want_abs ? (double*)calloc((size_t)M, sizeof(double)) : NULL;
  double* Gpa = want_abs ? (double*)calloc((size_t)n * 3, sizeof(double)) : NULL;
  double* Spa = want_abs ? (double*)calloc((size_t)n, sizeof(double)) : NULL;
  double* tgta = want_abs ? (double*)calloc((size_t)ns * 3, sizeof(double)) : NULL;
  orc_list L = {0};
  for (int64_t i = 0; i < n; i++) {
    if (!mark[i]) continue;
    orc_walk_list(T, i, theta, rcut, &L, NULL);
    const double* xi = &T->x[3 * i];
    const double* wi = &w[3 * i];
    for (int64_t q = 0; q < L.n; q++) {
      const double* X; double Ms, hs;
      orc_item_source(T, &L.v[q], &X, &Ms, &hs);
      double h = T->h[i] > hs ? T->h[i] : hs;
      double d[3], g[3], Jw[3];
      for (int c = 0; c < 3; c++) d[c] = orc_mi(xi[c] - X[c], T->box);
      orc_pair_adj(d, h, r_s, wi, g, Jw);
      if (slot[i] >= 0) for (int c = 0; c < 3; c++) tgt[3 * slot[i] + c] += Ms * Jw[c];
      double wg = (wi[0] * g[0] + wi[1] * g[1]) + wi[2] * g[2];
      if (L.v[q].kind == 0) {
        int64_t id = L.v[q].id;
        for (int c = 0; c < 3; c++) Gn[3 * id + c] += Jw[c];
        Sn[id] += wg;
      } else {
        int64_t j = L.v[q].id;
        for (int c = 0; c < 3; c++) Gp[3 * j + c] += Jw[c];
        Sp[j] += wg;
      }
      if (want_abs) {
        if (slot[i] >= 0) for (int c = 0; c < 3; c++) tgta[3 * slot[i] + c] += Ms * fabs(Jw[c]);
        double* Ga = L.v[q].kind == 0 ? &Gna[3 * L.v[q].id] : &Gpa[3 * L.v[q].id];
        double* Sa = L.v[q].kind == 0 ? &Sna[L.v[q].id] : &Spa[L.v[q].id];
        for (int c = 0; c < 3; c++) Ga[c] += fabs(Jw[c]);
        *Sa += fabs(wg);
      }
    }
  }
  int64_t anc[64];
  for (int64_t s = 0; s < ns; s++) {
    int64_t k = sidx[s];
    double mk = T->m[k];
    double dx[3], dm = Sp[k];
    for (int c = 0; c < 3; c++) dx[c] = tgt[3 * s + c] - mk * Gp[3 * k + c];
    int na = orc_ancestors(T, k, anc);
    for (int a = 0; a < na; a++) {
      const orc_node* nd = &T->nodes[anc[a]];
      const double* G = &Gn[3 * anc[a]];
      double rel[3];
      for (int c = 0; c < 3; c++) rel[c] = T->x[3 * k + c] - nd->com[c];
      for (int c = 0; c < 3; c++) dx[c] -= mk * G[c];
      dm += Sn[anc[a]] - ((G[0] * rel[0] + G[1] * rel[1]) + G[2] * rel[2]);
    }
    for (int c = 0; c < 3; c++) dpos[3 * s + c] = dx[c];
    dmass[s] = dm;
    if (want_abs) {
      double ax[3], am = Spa[k];
      for (int c = 0; c < 3; c++) ax[c] = tgta[3 * s + c] + mk * Gpa[3 * k + c];
      for (int a = 0; a < na; a++) {
        const orc_node* nd = &T->nodes[anc[a]];
        const double* Ga = &Gna[3 * anc[a]];
        for (int c = 0; c < 3; c++) {
          ax[c] += mk * Ga[c];
          am += Ga[c] * fabs(T->x[3 * k + c] - nd->com[c]);
        }
        am += Sna[anc[a]];
      }
      if (dpos_abs) for (int c = 0; c < 3; c++) dpos_abs[3 * s + c] = ax[c];
      if (dmass_abs) dmass_abs[s] = am;
    }
  }
  free(L.v); free(mark); free(sidx); free(slot); free(Gn); free(Sn); free(Gp); free(Sp); free(tgt);
  free(Gna); free(Sna); free(Gpa); free(Spa); free(tgta);
}

/* Part of the loss that involves particle k, with k moved by dx (3-vector)
 * and its mass changed by dmk, holding every interaction list fixed.  Node
 * masses and centres of mass are updated for the change. */
/* *cross (optional) gets bit 0 if an involved term's distance is on the other
 * side of its softening length h than unperturbed, bit 1 if on the other side
 * of rcut (the frozen lists keep the term either way; the kernel has a kink at
 * h, so a central difference across it is only first-order accurate). */
static double orc_local_loss(const orc_tree* T, int64_t k, const double* w, int64_t* off, int32_t* kind,
                             int64_t* ids, const int64_t* tlist, int64_t nt, double r_s, double rcut,
                             const double dxk[3], double dmk, int* cross) {
  double loss = 0.0;
  double mk = T->m[k];
  for (int64_t t = 0; t < nt; t++) {
    int64_t i = tlist[t];
    const double* wi = &w[3 * i];
    for (int64_t q = off[t]; q < off[t + 1]; q++) {
      orc_item it;
      it.kind = kind[q];
      it.id = ids[q];
      int involves = (i == k);
      const double* X; double Ms, hs;
      orc_item_source(T, &it, &X, &Ms, &hs);
      double dX[3] = {0.0, 0.0, 0.0};   /* change of the source position */
      double Mp = Ms;
      if (it.kind == 1 && it.id == k) {
        involves = 1;
        for (int c = 0; c < 3; c++) dX[c] = dxk[c];
        Mp = Ms + dmk;
      } else if (it.kind == 0 && i != k) {
        const orc_node* nd = &T->nodes[it.id];
        int sh = ORC_BITS - nd->level;
        int in = (T->q[3 * k] >> sh) == nd->cell[0] && (T->q[3 * k + 1] >> sh) == nd->cell[1] &&
                 (T->q[3 * k + 2] >> sh) == nd->cell[2];
        if (in) {
          involves = 1;
          Mp = Ms + dmk;
          for (int c = 0; c < 3; c++) {
            /* X' - X = ((m_k + dm)(x_k + dx - X) - m_k (x_k - X)) / M' */
            double rel = T->x[3 * k + c] - X[c];
            dX[c] = ((mk + dmk) * (rel + dxk[c]) - mk * rel) / Mp;
          }
        }
      }
      if (!involves) continue;
      double h = T->h[i] > hs ? T->h[i] : hs;
      double d[3], dz[3];
      for (int c = 0; c < 3; c++) {
        double d0 = orc_mi(T->x[3 * i + c] - X[c], T->box);
        dz[c] = d0;
        d[c] = d0 + (i == k ? dxk[c] : 0.0) - dX[c];
      }
      double r = sqrt(orc_norm2(d));
      if (cross) {
        double r0 = sqrt(orc_norm2(dz));
        if ((r0 < h) != (r < h)) *cross |= 1;
        if ((r0 < rcut) != (r < rcut)) *cross |= 2;
      }
      double fac = -Mp * orc_F(r, h, r_s);
      loss += fac * ((wi[0] * d[0] + wi[1] * d[1]) + wi[2] * d[2]);
    }
  }
  return loss;
}

/* Central finite differences of the frozen-list loss for the sample
 * particles: position step hx (absolute), mass step hm_rel * m_k.
 * flags (optional, may be NULL): per sample, bit 0 if a position step moves an
 * involved term across its softening length h, bit 1 if across rcut. */
void orc_fd(void* hnd, double r_s, double rcut, double theta, const double* w, const int64_t* samples, int64_t ns,
            double hx, double hm_rel, double* dpos, double* dmass, int32_t* flags) {
  const orc_tree* T = (const orc_tree*)hnd;
  int64_t n = T->n;
  double R = rcut * (1.0 + sqrt(3.0) * theta) * (1.0 + 1e-9) + 1e-12;
  uint8_t* mark = (uint8_t*)malloc((size_t)n);
  int64_t* tl = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
  for (int64_t s = 0; s < ns; s++) {
    int64_t k = samples[s];
    memset(mark, 0, (size_t)n);
    orc_mark_neighbourhood(T, k, R * R, mark);
    int64_t nt = 0;
    for (int64_t i = 0; i < n; i++) if (mark[i]) tl[nt++] = i;
    int64_t* off = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nt + 1));
    orc_walk_lists(hnd, rcut, theta, tl, nt, off, NULL, NULL);
    int32_t* kind = (int32_t*)malloc(sizeof(int32_t) * (size_t)(off[nt] + 1));
    int64_t* ids = (int64_t*)malloc(sizeof(int64_t) * (size_t)(off[nt] + 1));
    orc_walk_lists(hnd, rcut, theta, tl, nt, off, kind, ids);
    int cross = 0;
    for (int c = 0; c < 4; c++) {
      double dp[3] = {0, 0, 0}, dn[3] = {0, 0, 0}, mp = 0.0, mn = 0.0, step;
      if (c < 3) { dp[c] = hx; dn[c] = -hx; step = hx; }
      else { step = hm_rel * T->m[k]; mp = step; mn = -step; }
      double Lp = orc_local_loss(T, k, w, off, kind, ids, tl, nt, r_s, rcut, dp, mp, &cross);
      double Ln = orc_local_loss(T, k, w, off, kind, ids, tl, nt, r_s, rcut, dn, mn, &cross);
      double g = (Lp - Ln) / (2.0 * step);
      if (c < 3) dpos[3 * s + c] = g; else dmass[s] = g;
    }
    if (flags) flags[s] = cross;
    free(off); free(kind); free(ids);
  }
  free(mark); free(tl);
}

/* Full loss L = sum_i w_i . a_i from the tree walk (for consistency tests). */
double orc_loss(void* hnd, double r_s, double rcut, double theta, const double* w) {
  const orc_tree* T = (const orc_tree*)hnd;
  int64_t n = T->n;
  int64_t* tl = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
  double* a = (double*)malloc(sizeof(double) * 3 * (size_t)n);
  for (int64_t i = 0; i < n; i++) tl[i] = i;
  orc_walk(hnd, r_s, rcut, theta, tl, n, a, NULL);
  double L = 0.0;
  for (int64_t i = 0; i < 3 * n; i++) L += w[i] * a[i];
  free(tl); free(a);
  return L;
}
