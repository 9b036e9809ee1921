/*
 * afdps_oracle.c -- plain, slow, FP64 CPU oracle for the multiwalk,
 * indirect-index Barnes-Hut gravity path of "Accelerated FDPS -- Algorithms
 * to Use Accelerators with FDPS" (Iwasawa, Namekata, Nitadori, Nomura, Wang,
 * Tsubouchi, Makino; arXiv 1907.02290).
 *
 * TEST INFRASTRUCTURE. This file is the checker, not the product. Only the
 * test suite, __graft_entry__.smoke() and bench.py's cpu_baseline / reference
 * leg load it. It shares no code, header, table or helper with the CUDA path
 * in paper_1907_02290_gb300/csrc, and neither side includes the other.
 *
 * Every function follows the step of the paper named in its comment, in the
 * paper's order. Where the paper is silent the reading taken is stated at the
 * function and collected in the "Readings" list below.
 *
 * Readings of the paper (silent or ambiguous points), fixed here:
 *  R1 force law: Plummer-softened Newtonian gravity with G = 1,
 *     a_i = sum_j m_j (x_j - x_i) / (|x_j - x_i|^2 + eps^2)^(3/2),
 *     phi_i = -sum_j m_j / (|x_j - x_i|^2 + eps^2)^(1/2), j != i.
 *     (Section 6.2 counts n_op = 23 flops per interaction; consistent.)
 *     A pair with |x_j - x_i|^2 + eps^2 == 0 contributes nothing.
 *  R2 root cell (Section 4.3 "coordinates of the root cell are determined
 *     using the positions of all particles"): centre = (min+max)/2 per axis,
 *     side L = smallest power of two >= 1.000001 * (largest extent); L = 1
 *     when the extent is 0.
 *  R3 Morton key (Section 4.3 step 1; 64-bit key, Section 6.2): 21 bits per
 *     axis, q_d = floor((x_d - (c_d - L/2)) * (2^21 / L)) clamped to
 *     [0, 2^21 - 1]; bit 3k+2 = x bit k, 3k+1 = y bit k, 3k = z bit k.
 *  R4 sort (Section 4.3 step 2, Section 6.2): LSD radix sort, eight passes of
 *     eight-bit digits, stable; equal keys keep caller order.
 *  R5 tree (Section 4.3 step 4): a cell splits while count > n_leaf and its
 *     level < 21; children are the non-empty octants in Morton order, found
 *     per level by binary search on the sorted keys. Cells are built level by
 *     level; the exported numbering is depth-first pre-order (children in
 *     Morton order), which equals ascending (first particle, level).
 *  R6 moments (Section 4.3, bottom-up): monopole M = sum m and centre of mass
 *     COM = S / M with S = sum m x ("center-of-mass approximation",
 *     Section 6.2). Leaves sum their particles in Morton order; internal
 *     cells sum their children in Morton order. A massless cell takes its
 *     geometric centre as COM. Quadrupole (traceless, about the COM):
 *     Q_ab = sum m (3 d_a d_b - |d|^2 delta_ab); parents add the children's
 *     Q shifted by the parallel-axis term.
 *  R7 groups (Section 3, n_grp): i-groups are the maximal cells holding at
 *     most n_grp particles, in depth-first order; a leaf holding more than
 *     n_grp particles (only possible at level 21, or when n_grp < n_leaf) is
 *     cut into consecutive chunks of n_grp.
 *  R8 opening criterion (Section 2 "standard Barnes-Hut scheme", opening
 *     angle theta): a cell of side s is accepted as a superparticle for
 *     group g iff s^2 < theta^2 d^2, with d the distance from the cell's COM
 *     to the group's bounding box (0 inside). Evaluated in IEEE FP32 on
 *     FP32-rounded inputs, no fused multiply-add, in the order written in
 *     mac_accept(), so that any two implementations decide identically.
 *  R9 list order: the walk is depth-first from the root, children in Morton
 *     order; an accepted cell appends its cell id to the SPJ list, an opened
 *     leaf appends all its particles (Morton positions) to the EPJ list.
 *  R10 quadrupole softening: phi_q = -(1/2) r.Q.r / rs^5 with
 *     rs^2 = |r|^2 + eps^2, and a_q = Q r / rs^5 - (5/2)(r.Q.r) r / rs^7,
 *     r = x_i - COM.
 *  R11 integrator: kick-drift-kick leapfrog; force evaluation k of a run is
 *     a construction step when k % n_reuse == 0, else it reuses the lists.
 *
 * The learned opening criterion is not in the paper (the paper uses the
 * opening angle only, Section 2); its definition is fixed here:
 *  R12 features of a (group g, cell c) pair, eight FP32 numbers computed
 *     without contraction in the order written in afo_mac_features(): with
 *     d^2 the squared COM-to-box distance of R8, s the cell side, M and Q
 *     the cell's monopole and quadrupole rounded to FP32, n_c its particle
 *     count, A_g the smallest reference acceleration magnitude among the
 *     group's particles, u the vector from the COM to the box centre and e
 *     the half diagonal of the box:
 *       f0 = log2(s/d)        f1 = log2(M / (d^2 A_g))
 *       f2 = log2(|Q|_F / (M s^2))   f3 = log2(e/d)      f4 = log2(n_c)
 *       f5 = log2(eps/d)      f6 = u.Q.u / (|u|^2 |Q|_F)  f7 = log2(|u|/d)
 *     each clamped to [-32, 32]. log2 is lg2(): the exponent of the FP32
 *     argument plus t*p(t) on its mantissa 1+t, p a fixed quartic (Horner
 *     with fused multiply-adds); 0 or subnormal arguments give -127.
 *  R13 network: 8-32-32-1 perceptron with ReLU on both hidden layers; every
 *     parameter (mu and isd included) is an FP16 value. The inputs are
 *     x_k = RN16((f_k - mu_k) * isd_k) (FP32 subtraction and product, then
 *     rounded to the nearest FP16 value, ties to even); hidden layer 1 is
 *     h1_j = RN16(min(max(b1_j + sum_k W1_jk x_k, 0), 65504)); hidden layer
 *     2 is h2_j = max(b2_j + sum_k W2_jk h1_k, 0); the output is
 *     y = b3 + sum_j w3_j h2_j. Every sum is FP32, here the bias followed by
 *     fused multiply-adds in index order (the products of FP16 values are
 *     exact in FP32). FP16 operands are what the tensor cores take; the
 *     order in which an implementation (a tensor core) sums is not fixed, so
 *     afo_mlp_forward_bound also returns a bound on the difference between
 *     this output and any FP32 summation order's, propagated through the
 *     layers: each sum of n terms within 2 gamma_n of another order's
 *     (gamma_n = n U / (1 - n U), U = 2^-22, allowing two units in the last
 *     place per operation), a first-layer activation within the FP16
 *     roundings of its sum's interval, and the later layers through the
 *     absolute weights. A decision of R14 is fixed by the definition only
 *     when the output lies further than that bound from tau.
 *  R14 learned decision for cell c and group g: open if c contains the
 *     group's first particle; accept if s^2 < theta_lo^2 d^2; open if not
 *     s^2 < theta_hi^2 d^2; otherwise accept iff the network's output is
 *     below tau. Without weights or reference accelerations the walk uses
 *     R8 (the theta criterion is the fallback).
 *  R15 training target of a pair: log2 of max over the group's particles i
 *     of |a_i^cell - a_i^exact| / A_i, where a_i^cell is the cell's
 *     superparticle term (R1, plus R10 with quadrupoles), a_i^exact the
 *     direct sum over the cell's particles and A_i particle i's reference
 *     acceleration magnitude; clamped to [-40, 8].
 *  R16 local essential tree (Section 3 and Section 4.3: the global tree is
 *     built over local particles and the superparticles and particles
 *     imported from other domains): the LET of a tree for a remote domain
 *     box B is what a walk from the root under R8, with B as the group box,
 *     would put on a list: each accepted cell as one superparticle (its
 *     COM and monopole), each opened leaf as its particles; in depth-first
 *     order, children in Morton order.
 *
 * Short-range interactions (Section 2: the same walk with a cell-opening
 * criterion other than the opening angle; Section 4.2: their lists can be
 * kept over steps since particles move a small fraction of their spacing):
 *  R17 neighbour lists (gather form). Every particle i carries a search
 *     radius h_i > 0; the lists are made with a margin skin >= 0. The
 *     search box of group g is, per axis, [min_i (x_i - (h_i + skin)),
 *     max_i (x_i + (h_i + skin))] over its particles, each bound computed
 *     in FP64 (round to nearest) and then rounded outward to FP32 (the lower
 *     bound down, the upper bound up). The tight box of a cell is the
 *     min / max of its particles' coordinates, rounded outward to FP32 the
 *     same way. A cell whose tight box meets the search box (closed
 *     intervals on every axis, compared in FP32) is opened when internal
 *     and listed when a leaf; any other cell is dropped with its subtree.
 *     The list of a group is the particles of its listed leaves, depth
 *     first with children in Morton order, which is ascending Morton
 *     position. Every j within h_i + skin of a particle i of the group is
 *     on the list (up to the FP64 rounding of the bounds).
 *  R18 density over a neighbour list (gather form, the usual first pass of
 *     an SPH step): rho_i = sum_j m_j W(|x_j - x_i|, h_i), the particle
 *     itself included, with the M4 cubic spline of support radius h in
 *     three dimensions, W(r, h) = 8 / (pi h^3) w(r / h),
 *       w(q) = 1 - 6 q^2 + 6 q^3   for 0 <= q <= 1/2,
 *       w(q) = 2 (1 - q)^3         for 1/2 < q < 1,
 *       w(q) = 0                   for q >= 1,
 *     normalised so that its integral over space is 1. Also the smooth
 *     neighbour number nnb_i = (4 pi / 3) h_i^3 sum_j W(|x_j - x_i|, h_i)
 *     = (32 / 3) sum_j w(|x_j - x_i| / h_i), which a uniform medium of
 *     number density n takes to (4 pi / 3) h_i^3 n.
 */
#include <float.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define AFO_LEVELS 21 /* deepest level; 21 key bits per axis */

/* Learned opening criterion (R12-R13): 8 features, two hidden layers of 32.
 * Parameter vector: mu[8] isd[8] W1[32][8] b1[32] W2[32][32] b2[32] w3[32]
 * b3[1]. */
#define AFO_MAC_NF 8
#define AFO_MAC_NH 32
#define AFO_MAC_NP (2 * AFO_MAC_NF + AFO_MAC_NH * AFO_MAC_NF + AFO_MAC_NH + \
                    AFO_MAC_NH * AFO_MAC_NH + AFO_MAC_NH + AFO_MAC_NH + 1)

/* ------------------------------------------------------------------------ */
/* Exact target: softened direct summation (R1).                           */
/* ------------------------------------------------------------------------ */

/* For every target t in tgt[0..n_tgt), sum over all j != tgt[t]. */
void afo_direct_sum(int64_t n, const double *x, const double *y, const double *z,
                    const double *m, double eps, int64_t n_tgt, const int64_t *tgt,
                    double *ax, double *ay, double *az, double *pot) {
  const double eps2 = eps * eps;
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t t = 0; t < n_tgt; t++) {
    const int64_t i = tgt[t];
    double sx = 0.0, sy = 0.0, sz = 0.0, sp = 0.0;
    for (int64_t j = 0; j < n; j++) {
      if (j == i) continue;
      const double dx = x[j] - x[i], dy = y[j] - y[i], dz = z[j] - z[i];
      const double r2 = dx * dx + dy * dy + dz * dz + eps2;
      if (r2 == 0.0) continue;
      const double rinv = 1.0 / sqrt(r2);
      const double mr = m[j] * rinv;
      const double mr3 = mr * rinv * rinv;
      sx += mr3 * dx;
      sy += mr3 * dy;
      sz += mr3 * dz;
      sp -= mr;
    }
    ax[t] = sx;
    ay[t] = sy;
    az[t] = sz;
    pot[t] = sp;
  }
}

/* ------------------------------------------------------------------------ */
/* Root cell (Section 4.3; reading R2).                                     */
/* ------------------------------------------------------------------------ */

/* root[0..2] = centre, root[3] = side L (a power of two). Returns 0, or -1
 * when a coordinate is not finite or when no finite power of two reaches
 * 1.000001 x the extent (finite coordinates whose extent overflows, or
 * an extent above 2^1023 / 1.000001): such a set has no root cell in
 * doubles, and counts as non-finite input. */
int afo_root_cell(int64_t n, const double *x, const double *y, const double *z,
                  double root[4]) {
  double lo[3] = {0.0, 0.0, 0.0}, hi[3] = {0.0, 0.0, 0.0};
  const double *p[3] = {x, y, z};
  for (int64_t i = 0; i < n; i++)
    for (int d = 0; d < 3; d++)
      if (!isfinite(p[d][i])) return -1;
  if (n > 0) {
    for (int d = 0; d < 3; d++) lo[d] = hi[d] = p[d][0];
    for (int64_t i = 1; i < n; i++)
      for (int d = 0; d < 3; d++) {
        if (p[d][i] < lo[d]) lo[d] = p[d][i];
        if (p[d][i] > hi[d]) hi[d] = p[d][i];
      }
  }
  double ext = 0.0;
  for (int d = 0; d < 3; d++) {
    root[d] = (lo[d] + hi[d]) * 0.5;
    const double e = hi[d] - lo[d];
    if (e > ext) ext = e;
  }
  const double target = ext * 1.000001;
  if (!(target <= DBL_MAX)) return -1;
  double L = 1.0;
  if (target > 0.0) {
    /* at most 1024 doublings: L reaches target, or overflows to inf */
    while (L < target) L *= 2.0;
    if (isinf(L)) return -1;
    while (L * 0.5 >= target) L *= 0.5;
  }
  root[3] = L;
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Morton keys (Section 4.3 step 1; reading R3).                            */
/* ------------------------------------------------------------------------ */

static uint32_t grid_coord(double v, double corner, double scale) {
  const double t = floor((v - corner) * scale);
  if (!(t > 0.0)) return 0u;
  if (t > 2097151.0) return 2097151u;
  return (uint32_t)t;
}

/* Interleave one bit at a time: x bit k -> key bit 3k+2, y -> 3k+1, z -> 3k. */
static uint64_t interleave3(uint32_t qx, uint32_t qy, uint32_t qz) {
  uint64_t key = 0;
  for (int k = 0; k < AFO_LEVELS; k++) {
    key |= (uint64_t)((qx >> k) & 1u) << (3 * k + 2);
    key |= (uint64_t)((qy >> k) & 1u) << (3 * k + 1);
    key |= (uint64_t)((qz >> k) & 1u) << (3 * k);
  }
  return key;
}

void afo_morton_keys(int64_t n, const double *x, const double *y, const double *z,
                     const double root[4], uint64_t *keys) {
  const double half = root[3] * 0.5;
  const double cx = root[0] - half, cy = root[1] - half, cz = root[2] - half;
  const double scale = 2097152.0 / root[3]; /* 2^21 / L, a power of two */
  for (int64_t i = 0; i < n; i++)
    keys[i] = interleave3(grid_coord(x[i], cx, scale), grid_coord(y[i], cy, scale),
                          grid_coord(z[i], cz, scale));
}

/* ------------------------------------------------------------------------ */
/* Radix sort of key-index pairs (Section 4.3 step 2, Section 6.2: 8-bit    */
/* chunks, eight passes; each pass is a stable counting sort).              */
/* ------------------------------------------------------------------------ */

void afo_radix_sort(int64_t n, const uint64_t *keys_in, uint64_t *keys_out, int64_t *perm) {
  uint64_t *ka = malloc(sizeof(uint64_t) * (size_t)(n > 0 ? n : 1));
  uint64_t *kb = malloc(sizeof(uint64_t) * (size_t)(n > 0 ? n : 1));
  int64_t *ia = malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
  int64_t *ib = malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
  for (int64_t i = 0; i < n; i++) {
    ka[i] = keys_in[i];
    ia[i] = i;
  }
  for (int pass = 0; pass < 8; pass++) {
    const int shift = 8 * pass;
    int64_t count[257];
    memset(count, 0, sizeof(count));
    for (int64_t i = 0; i < n; i++) count[((ka[i] >> shift) & 255u) + 1]++;
    for (int b = 0; b < 256; b++) count[b + 1] += count[b];
    for (int64_t i = 0; i < n; i++) {
      const int b = (int)((ka[i] >> shift) & 255u);
      const int64_t dst = count[b]++;
      kb[dst] = ka[i];
      ib[dst] = ia[i];
    }
    uint64_t *tk = ka; ka = kb; kb = tk;
    int64_t *ti = ia; ia = ib; ib = ti;
  }
  for (int64_t i = 0; i < n; i++) {
    keys_out[i] = ka[i];
    perm[i] = ia[i];
  }
  free(ka); free(kb); free(ia); free(ib);
}

/* ------------------------------------------------------------------------ */
/* Tree state.                                                              */
/* ------------------------------------------------------------------------ */

typedef struct afo_tree {
  int64_t n;
  int n_leaf, n_grp, quad;
  double theta, eps;
  double root[4];
  uint64_t *keys;   /* sorted keys */
  int64_t *perm;    /* perm[k] = caller index of the k-th particle in Morton order */
  double *xs, *ys, *zs, *ms; /* Morton-ordered EPI/EPJ copies (Section 4.3 step 3) */
  /* cells, exported in depth-first pre-order */
  int64_t n_cells;
  int32_t *level;
  int64_t *first, *count, *parent, *skip;
  int32_t *n_child;
  int64_t *child; /* 8 slots per cell, by octant digit, -1 when empty */
  double *mass, *smom, *com, *qmom; /* M; S = sum m x (3); COM (3); Q (6) */
  /* groups */
  int64_t n_groups;
  int64_t *g_first, *g_count, *g_cell;
  double *g_box; /* min x,y,z then max x,y,z */
  int32_t *g_self;
  /* lists (CSR, one EPJ and one SPJ list per group) */
  int64_t *epj_off, *spj_off;
  int32_t *epj, *spj;
  /* learned opening criterion (R12-R15): on when weights and reference
   * accelerations were given */
  int mac_on, need_q;
  float mac_w[AFO_MAC_NP];
  float mac_lo2, mac_hi2, mac_tau;
  float *amag_s; /* reference |a| per particle, Morton order */
  float *g_amin; /* smallest of them per group */
  /* comparison with another implementation of R14 (afo_relist_band): for a
   * pair whose output lies within the rounding bound of R13 from tau, the
   * decision is read from that implementation's SPJ lists (accepted iff the
   * cell is on the group's list); per group, such pairs and those among
   * them decided otherwise than here */
  const int64_t *ovr_off;
  const int32_t *ovr_spj;
  int64_t *band_cnt, *flip_cnt;
  /* neighbour lists (R17): per-cell tight boxes and per-group search boxes
   * (FP32, min x y z then max x y z), CSR lists of Morton positions */
  float *c_tbox, *g_sbox;
  int64_t *nbr_off;
  int32_t *nbr;
} afo_tree;

static void *xcalloc(size_t count, size_t size) {
  return calloc(count > 0 ? count : 1, size);
}

void afo_free(afo_tree *t) {
  if (!t) return;
  free(t->keys); free(t->perm); free(t->xs); free(t->ys); free(t->zs); free(t->ms);
  free(t->level); free(t->first); free(t->count); free(t->parent); free(t->skip);
  free(t->n_child); free(t->child); free(t->mass); free(t->smom); free(t->com); free(t->qmom);
  free(t->g_first); free(t->g_count); free(t->g_cell); free(t->g_box); free(t->g_self);
  free(t->epj_off); free(t->spj_off); free(t->epj); free(t->spj);
  free(t->amag_s); free(t->g_amin);
  free(t->c_tbox); free(t->g_sbox); free(t->nbr_off); free(t->nbr);
  free(t);
}

/* First index in [lo, hi) with keys[idx] >= v (binary search, Section 4.3). */
static int64_t lower_bound_key(const uint64_t *keys, int64_t lo, int64_t hi, uint64_t v) {
  while (lo < hi) {
    const int64_t mid = lo + (hi - lo) / 2;
    if (keys[mid] < v) lo = mid + 1; else hi = mid;
  }
  return lo;
}

/* Reorder (Section 4.3 step 3): copy FP data into Morton order. */
static void reorder(afo_tree *t, const double *x, const double *y, const double *z,
                    const double *m) {
  for (int64_t k = 0; k < t->n; k++) {
    const int64_t i = t->perm[k];
    t->xs[k] = x[i];
    t->ys[k] = y[i];
    t->zs[k] = z[i];
    t->ms[k] = m[i];
  }
}

/* Link (Section 4.3 step 4, reading R5): build cells level by level, top
 * down; the children of a splitting cell are found by binary search for the
 * boundaries of its eight octants. Then renumber depth-first pre-order. */
static void link_cells(afo_tree *t) {
  const int64_t n = t->n;
  int64_t cap = 64, nc = 0;
  int32_t *lv = malloc(sizeof(int32_t) * cap);
  int64_t *fi = malloc(sizeof(int64_t) * cap), *ct = malloc(sizeof(int64_t) * cap);
  int64_t *pa = malloc(sizeof(int64_t) * cap), *ch = malloc(sizeof(int64_t) * cap * 8);
  if (n > 0) {
    lv[0] = 0; fi[0] = 0; ct[0] = n; pa[0] = -1;
    for (int o = 0; o < 8; o++) ch[o] = -1;
    nc = 1;
  }
  int64_t lvl_begin = 0, lvl_end = nc;
  for (int l = 0; l < AFO_LEVELS && lvl_begin < lvl_end; l++) {
    for (int64_t c = lvl_begin; c < lvl_end; c++) {
      if (ct[c] <= t->n_leaf) continue;
      const uint64_t prefix = t->keys[fi[c]] >> (3 * (AFO_LEVELS - l));
      const int shift = 3 * (AFO_LEVELS - l - 1);
      const int64_t end = fi[c] + ct[c];
      for (int o = 0; o < 8; o++) {
        const uint64_t k0 = ((prefix << 3) | (uint64_t)o) << shift;
        const uint64_t k1 = ((prefix << 3) + (uint64_t)o + 1) << shift;
        const int64_t b0 = lower_bound_key(t->keys, fi[c], end, k0);
        const int64_t b1 = lower_bound_key(t->keys, b0, end, k1);
        if (b1 <= b0) continue;
        if (nc == cap) {
          cap *= 2;
          lv = realloc(lv, sizeof(int32_t) * cap);
          fi = realloc(fi, sizeof(int64_t) * cap);
          ct = realloc(ct, sizeof(int64_t) * cap);
          pa = realloc(pa, sizeof(int64_t) * cap);
          ch = realloc(ch, sizeof(int64_t) * cap * 8);
        }
        lv[nc] = l + 1; fi[nc] = b0; ct[nc] = b1 - b0; pa[nc] = c;
        for (int q = 0; q < 8; q++) ch[nc * 8 + q] = -1;
        ch[c * 8 + o] = nc;
        nc++;
      }
    }
    lvl_begin = lvl_end;
    lvl_end = nc;
  }
  /* Depth-first pre-order numbering (children in Morton order). */
  int64_t *rank = malloc(sizeof(int64_t) * (size_t)(nc > 0 ? nc : 1));
  int64_t *size = malloc(sizeof(int64_t) * (size_t)(nc > 0 ? nc : 1));
  for (int64_t c = nc - 1; c >= 0; c--) { /* deeper levels come later */
    size[c] = 1;
    for (int o = 0; o < 8; o++)
      if (ch[c * 8 + o] >= 0) size[c] += size[ch[c * 8 + o]];
  }
  int64_t *stack = malloc(sizeof(int64_t) * (size_t)(nc > 0 ? nc : 1));
  int64_t sp = 0, next = 0;
  if (nc > 0) stack[sp++] = 0;
  while (sp > 0) {
    const int64_t c = stack[--sp];
    rank[c] = next++;
    for (int o = 7; o >= 0; o--)
      if (ch[c * 8 + o] >= 0) stack[sp++] = ch[c * 8 + o];
  }
  t->n_cells = nc;
  t->level = xcalloc(nc, sizeof(int32_t));
  t->first = xcalloc(nc, sizeof(int64_t));
  t->count = xcalloc(nc, sizeof(int64_t));
  t->parent = xcalloc(nc, sizeof(int64_t));
  t->skip = xcalloc(nc, sizeof(int64_t));
  t->n_child = xcalloc(nc, sizeof(int32_t));
  t->child = xcalloc(nc * 8, sizeof(int64_t));
  for (int64_t c = 0; c < nc; c++) {
    const int64_t r = rank[c];
    t->level[r] = lv[c];
    t->first[r] = fi[c];
    t->count[r] = ct[c];
    t->parent[r] = pa[c] >= 0 ? rank[pa[c]] : -1;
    t->skip[r] = r + size[c];
    int nch = 0;
    for (int o = 0; o < 8; o++) {
      const int64_t cc = ch[c * 8 + o];
      t->child[r * 8 + o] = cc >= 0 ? rank[cc] : -1;
      if (cc >= 0) nch++;
    }
    t->n_child[r] = nch;
  }
  free(lv); free(fi); free(ct); free(pa); free(ch); free(rank); free(size); free(stack);
}

/* Geometric centre of a cell: the root corner plus (q + 1/2) cell sides. */
static void cell_centre(const afo_tree *t, int64_t c, double out[3]) {
  const int l = t->level[c];
  const uint64_t prefix = l > 0 ? t->keys[t->first[c]] >> (3 * (AFO_LEVELS - l)) : 0;
  uint32_t q[3] = {0, 0, 0};
  for (int k = 0; k < l; k++) {
    q[0] |= (uint32_t)((prefix >> (3 * k + 2)) & 1u) << k;
    q[1] |= (uint32_t)((prefix >> (3 * k + 1)) & 1u) << k;
    q[2] |= (uint32_t)((prefix >> (3 * k)) & 1u) << k;
  }
  const double s = ldexp(t->root[3], -l);
  for (int d = 0; d < 3; d++)
    out[d] = (t->root[d] - t->root[3] * 0.5) + ((double)q[d] + 0.5) * s;
}

static int is_leaf(const afo_tree *t, int64_t c) { return t->n_child[c] == 0; }

/* Multipole moments, bottom-up (Section 4.3; reading R6). Pre-order ids are
 * visited from last to first, so every child is done before its parent. */
static void moments(afo_tree *t) {
  const int64_t nc = t->n_cells;
  for (int64_t c = nc - 1; c >= 0; c--) {
    double M = 0.0, S[3] = {0.0, 0.0, 0.0};
    if (is_leaf(t, c)) {
      for (int64_t k = t->first[c]; k < t->first[c] + t->count[c]; k++) {
        M += t->ms[k];
        S[0] += t->ms[k] * t->xs[k];
        S[1] += t->ms[k] * t->ys[k];
        S[2] += t->ms[k] * t->zs[k];
      }
    } else {
      for (int o = 0; o < 8; o++) {
        const int64_t cc = t->child[c * 8 + o];
        if (cc < 0) continue;
        M += t->mass[cc];
        for (int d = 0; d < 3; d++) S[d] += t->smom[cc * 3 + d];
      }
    }
    t->mass[c] = M;
    for (int d = 0; d < 3; d++) t->smom[c * 3 + d] = S[d];
    if (M != 0.0) {
      for (int d = 0; d < 3; d++) t->com[c * 3 + d] = S[d] / M;
    } else {
      cell_centre(t, c, &t->com[c * 3]);
    }
  }
  if (!t->quad && !t->need_q) return; /* R12 reads Q even without R10 */
  for (int64_t c = nc - 1; c >= 0; c--) {
    double Q[6] = {0, 0, 0, 0, 0, 0}; /* xx yy zz xy xz yz */
    const double *g = &t->com[c * 3];
    if (is_leaf(t, c)) {
      for (int64_t k = t->first[c]; k < t->first[c] + t->count[c]; k++) {
        const double d[3] = {t->xs[k] - g[0], t->ys[k] - g[1], t->zs[k] - g[2]};
        const double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
        const double mk = t->ms[k];
        Q[0] += mk * (3.0 * d[0] * d[0] - r2);
        Q[1] += mk * (3.0 * d[1] * d[1] - r2);
        Q[2] += mk * (3.0 * d[2] * d[2] - r2);
        Q[3] += mk * (3.0 * d[0] * d[1]);
        Q[4] += mk * (3.0 * d[0] * d[2]);
        Q[5] += mk * (3.0 * d[1] * d[2]);
      }
    } else {
      for (int o = 0; o < 8; o++) {
        const int64_t cc = t->child[c * 8 + o];
        if (cc < 0) continue;
        const double *gc = &t->com[cc * 3];
        const double D[3] = {gc[0] - g[0], gc[1] - g[1], gc[2] - g[2]};
        const double r2 = D[0] * D[0] + D[1] * D[1] + D[2] * D[2];
        const double mc = t->mass[cc];
        const double *qc = &t->qmom[cc * 6];
        Q[0] += qc[0] + mc * (3.0 * D[0] * D[0] - r2);
        Q[1] += qc[1] + mc * (3.0 * D[1] * D[1] - r2);
        Q[2] += qc[2] + mc * (3.0 * D[2] * D[2] - r2);
        Q[3] += qc[3] + mc * (3.0 * D[0] * D[1]);
        Q[4] += qc[4] + mc * (3.0 * D[0] * D[2]);
        Q[5] += qc[5] + mc * (3.0 * D[1] * D[2]);
      }
    }
    for (int q = 0; q < 6; q++) t->qmom[c * 6 + q] = Q[q];
  }
}

/* i-groups (Section 3, n_grp; reading R7), depth-first. */
static void make_groups(afo_tree *t) {
  int64_t cap = 64, ng = 0;
  int64_t *gf = malloc(sizeof(int64_t) * cap), *gc = malloc(sizeof(int64_t) * cap);
  int64_t *gcell = malloc(sizeof(int64_t) * cap);
  int64_t *stack = malloc(sizeof(int64_t) * (size_t)(t->n_cells > 0 ? t->n_cells : 1));
  int64_t sp = 0;
  if (t->n_cells > 0) stack[sp++] = 0;
  while (sp > 0) {
    const int64_t c = stack[--sp];
    if (t->count[c] <= t->n_grp || is_leaf(t, c)) {
      for (int64_t s = 0; s < t->count[c]; s += t->n_grp) {
        if (ng == cap) {
          cap *= 2;
          gf = realloc(gf, sizeof(int64_t) * cap);
          gc = realloc(gc, sizeof(int64_t) * cap);
          gcell = realloc(gcell, sizeof(int64_t) * cap);
        }
        gf[ng] = t->first[c] + s;
        gc[ng] = (t->count[c] - s) < t->n_grp ? (t->count[c] - s) : t->n_grp;
        gcell[ng] = c;
        ng++;
      }
      continue;
    }
    for (int o = 7; o >= 0; o--)
      if (t->child[c * 8 + o] >= 0) stack[sp++] = t->child[c * 8 + o];
  }
  free(stack);
  t->n_groups = ng;
  t->g_first = gf;
  t->g_count = gc;
  t->g_cell = gcell;
  t->g_box = xcalloc(ng * 6, sizeof(double));
  t->g_self = xcalloc(ng, sizeof(int32_t));
}

/* Tight FP64 bounding box of every group's particles. */
static void group_boxes(afo_tree *t) {
  for (int64_t g = 0; g < t->n_groups; g++) {
    double *b = &t->g_box[g * 6];
    const int64_t f = t->g_first[g];
    b[0] = b[3] = t->xs[f];
    b[1] = b[4] = t->ys[f];
    b[2] = b[5] = t->zs[f];
    for (int64_t k = f + 1; k < f + t->g_count[g]; k++) {
      if (t->xs[k] < b[0]) b[0] = t->xs[k];
      if (t->ys[k] < b[1]) b[1] = t->ys[k];
      if (t->zs[k] < b[2]) b[2] = t->zs[k];
      if (t->xs[k] > b[3]) b[3] = t->xs[k];
      if (t->ys[k] > b[4]) b[4] = t->ys[k];
      if (t->zs[k] > b[5]) b[5] = t->zs[k];
    }
  }
}

/* Opening criterion (reading R8), FP32, no contraction (built with
 * -ffp-contract=off). Returns 1 when the cell is accepted as an SPJ. */
static int mac_accept(const float bmin[3], const float bmax[3], const float com[3],
                      float s2, float theta2) {
  float d[3];
  for (int k = 0; k < 3; k++) {
    d[k] = 0.0f;
    if (com[k] < bmin[k]) d[k] = bmin[k] - com[k];
    else if (com[k] > bmax[k]) d[k] = com[k] - bmax[k];
  }
  float d2 = d[0] * d[0];
  d2 = d2 + d[1] * d[1];
  d2 = d2 + d[2] * d[2];
  const float rhs = theta2 * d2;
  return s2 < rhs;
}

/* ------------------------------------------------------------------------ */
/* Learned opening criterion (not in the paper; readings R12-R15).          */
/* ------------------------------------------------------------------------ */

/* lg2 of R12: exponent plus t * p(t) on the mantissa 1 + t, t in [0, 1).
 * p is a least-squares quartic fit of log2(1 + t) / t (max error 1.8e-5). */
float afo_lg2(float x) {
  if (!(x >= FLT_MIN)) return -127.0f;
  if (x > FLT_MAX) return 128.0f;
  uint32_t b;
  memcpy(&b, &x, sizeof(b));
  const int e = (int)((b >> 23) & 0xffu) - 127;
  const uint32_t mb = (b & 0x7fffffu) | 0x3f800000u;
  float mant;
  memcpy(&mant, &mb, sizeof(mant));
  const float t = mant - 1.0f;
  float p = 0.04526829347014427f;
  p = fmaf(p, t, -0.19351652264595032f);
  p = fmaf(p, t, 0.41524556279182434f);
  p = fmaf(p, t, -0.708865225315094f);
  p = fmaf(p, t, 1.4418798685073853f);
  const float pt = p * t;
  return (float)e + pt;
}

void afo_lg2_batch(int64_t n, const float *x, float *out) {
  for (int64_t i = 0; i < n; i++) out[i] = afo_lg2(x[i]);
}

static float clamp32(float v) { return v < -32.0f ? -32.0f : (v > 32.0f ? 32.0f : v); }

/* Features of R12 from FP32 inputs: the group box, the cell's COM, squared
 * side s2, mass M, quadrupole Q (xx yy zz xy xz yz), particle count, eps^2
 * and the group's smallest reference |a|. */
void afo_mac_features(const float bmin[3], const float bmax[3], const float com[3], float s2,
                      float M, const float Q[6], int64_t count, float eps2, float amin,
                      float f[AFO_MAC_NF]) {
  float d[3], u[3], w[3];
  for (int k = 0; k < 3; k++) {
    d[k] = 0.0f;
    if (com[k] < bmin[k]) d[k] = bmin[k] - com[k];
    else if (com[k] > bmax[k]) d[k] = com[k] - bmax[k];
    const float mid = (bmin[k] + bmax[k]) * 0.5f;
    u[k] = mid - com[k];
    w[k] = bmax[k] - bmin[k];
  }
  float d2 = d[0] * d[0];
  d2 = d2 + d[1] * d[1];
  d2 = d2 + d[2] * d[2];
  float u2 = u[0] * u[0];
  u2 = u2 + u[1] * u[1];
  u2 = u2 + u[2] * u[2];
  float e2 = w[0] * w[0];
  e2 = e2 + w[1] * w[1];
  e2 = e2 + w[2] * w[2];
  e2 = e2 * 0.25f;
  float off = Q[3] * Q[3];
  off = off + Q[4] * Q[4];
  off = off + Q[5] * Q[5];
  float q2 = Q[0] * Q[0];
  q2 = q2 + Q[1] * Q[1];
  q2 = q2 + Q[2] * Q[2];
  q2 = q2 + (off + off);
  float Qu[3];
  Qu[0] = Q[0] * u[0] + Q[3] * u[1];
  Qu[0] = Qu[0] + Q[4] * u[2];
  Qu[1] = Q[3] * u[0] + Q[1] * u[1];
  Qu[1] = Qu[1] + Q[5] * u[2];
  Qu[2] = Q[4] * u[0] + Q[5] * u[1];
  Qu[2] = Qu[2] + Q[2] * u[2];
  float uQu = u[0] * Qu[0] + u[1] * Qu[1];
  uQu = uQu + u[2] * Qu[2];
  const float ld = afo_lg2(d2), ls = afo_lg2(s2), lm = afo_lg2(M);
  f[0] = 0.5f * (ls - ld);
  f[1] = (lm - ld) - afo_lg2(amin);
  f[2] = (0.5f * afo_lg2(q2) - lm) - ls;
  f[3] = 0.5f * (afo_lg2(e2) - ld);
  f[4] = afo_lg2((float)count);
  f[5] = 0.5f * (afo_lg2(eps2) - ld);
  f[6] = 0.0f;
  if (u2 > 0.0f && q2 > 0.0f) {
    const float den = u2 * sqrtf(q2);
    if (den > 0.0f) f[6] = uQu / den;
  }
  f[7] = 0.5f * (afo_lg2(u2) - ld);
  for (int k = 0; k < AFO_MAC_NF; k++) f[k] = clamp32(f[k]);
}

/* RN16 of R13: v rounded to the nearest FP16 value (ties to even), as a
 * float; |v| is at most 65504 here (the callers clamp), NaN stays NaN. */
float afo_rn16(float v) {
  if (v != v) return v;
  const float a = fabsf(v);
  if (a == 0.0f) return v;
  int e;
  frexpf(a, &e); /* a = m 2^e, m in [0.5, 1): the FP16 spacing is 2^(e - 11) */
  const int ex = e - 11 < -24 ? -24 : e - 11; /* subnormals: spacing 2^-24 */
  const float r = ldexpf(nearbyintf(ldexpf(a, -ex)), ex);
  return copysignf(r, v);
}

static double gamma_n(int n) {
  const double U = ldexp(1.0, -22);
  return n * U / (1.0 - n * U);
}

static float clamp_h1(float v) {
  v = fmaxf(v, 0.0f);
  return fminf(v, 65504.0f);
}

/* Network of R13 on one feature vector; p holds FP16-representable values.
 * *bound (may be NULL) receives the bound of R13 on the difference between
 * this output and another FP32 summation order's. */
float afo_mlp_forward_bound(const float *p, const float f[AFO_MAC_NF], double *bound) {
  const float *mu = p, *isd = p + AFO_MAC_NF;
  const float *W1 = p + 2 * AFO_MAC_NF, *b1 = W1 + AFO_MAC_NH * AFO_MAC_NF;
  const float *W2 = b1 + AFO_MAC_NH, *b2 = W2 + AFO_MAC_NH * AFO_MAC_NH;
  const float *w3 = b2 + AFO_MAC_NH, *b3 = w3 + AFO_MAC_NH;
  float x[AFO_MAC_NF], h1[AFO_MAC_NH], h2[AFO_MAC_NH];
  double d1[AFO_MAC_NH], d2[AFO_MAC_NH];
  for (int k = 0; k < AFO_MAC_NF; k++) x[k] = afo_rn16((f[k] - mu[k]) * isd[k]);
  for (int j = 0; j < AFO_MAC_NH; j++) {
    float acc = b1[j];
    double s1 = fabs((double)b1[j]);
    for (int k = 0; k < AFO_MAC_NF; k++) {
      acc = fmaf(W1[j * AFO_MAC_NF + k], x[k], acc);
      s1 += fabs((double)W1[j * AFO_MAC_NF + k] * (double)x[k]);
    }
    h1[j] = afo_rn16(clamp_h1(acc));
    /* another order's sum lies in [acc - e, acc + e]; RN16 and the clamps
     * are monotonic, so its activation lies between these two */
    const double e = 2.0 * gamma_n(AFO_MAC_NF + 1) * s1;
    const float lo = afo_rn16(clamp_h1(nextafterf((float)((double)acc - e), -INFINITY)));
    const float hi = afo_rn16(clamp_h1(nextafterf((float)((double)acc + e), INFINITY)));
    d1[j] = fmax((double)hi - (double)h1[j], (double)h1[j] - (double)lo);
  }
  for (int j = 0; j < AFO_MAC_NH; j++) {
    float acc = b2[j];
    double s2 = fabs((double)b2[j]), dj = 0.0;
    for (int k = 0; k < AFO_MAC_NH; k++) {
      const double w = fabs((double)W2[j * AFO_MAC_NH + k]);
      acc = fmaf(W2[j * AFO_MAC_NH + k], h1[k], acc);
      s2 += w * (fabs((double)h1[k]) + d1[k]);
      dj += w * d1[k];
    }
    h2[j] = acc > 0.0f ? acc : 0.0f;
    d2[j] = dj + 2.0 * gamma_n(AFO_MAC_NH + 1) * s2;
  }
  float y = b3[0];
  double s3 = fabs((double)b3[0]), dy = 0.0;
  for (int k = 0; k < AFO_MAC_NH; k++) {
    y = fmaf(w3[k], h2[k], y);
    s3 += fabs((double)w3[k]) * ((double)h2[k] + d2[k]);
    dy += fabs((double)w3[k]) * d2[k];
  }
  if (bound) *bound = dy + 2.0 * gamma_n(AFO_MAC_NH + 1) * s3;
  return y;
}

float afo_mlp_forward(const float *p, const float f[AFO_MAC_NF]) {
  return afo_mlp_forward_bound(p, f, NULL);
}

void afo_mlp_forward_batch(const float *p, int64_t n, const float *feat, float *out) {
  for (int64_t i = 0; i < n; i++) out[i] = afo_mlp_forward(p, feat + i * AFO_MAC_NF);
}

void afo_mlp_forward_bound_batch(const float *p, int64_t n, const float *feat, float *out,
                                 double *bound) {
  for (int64_t i = 0; i < n; i++)
    out[i] = afo_mlp_forward_bound(p, feat + i * AFO_MAC_NF, &bound[i]);
}

/* Training target of R15 for n_i group particles (xi, yi, zi, reference
 * magnitudes ai) and a cell of n_j particles with monopole M at com and
 * quadrupole Q (used when quad != 0). FP64 throughout. */
double afo_mac_label(int64_t n_i, const double *xi, const double *yi, const double *zi,
                     const double *ai, int64_t n_j, const double *xj, const double *yj,
                     const double *zj, const double *mj, double M, const double com[3],
                     const double Q[6], double eps, int quad) {
  const double eps2 = eps * eps;
  double worst = 0.0;
  for (int64_t i = 0; i < n_i; i++) {
    double ex[3] = {0.0, 0.0, 0.0};
    for (int64_t j = 0; j < n_j; j++) {
      const double dx = xj[j] - xi[i], dy = yj[j] - yi[i], dz = zj[j] - zi[i];
      const double r2 = dx * dx + dy * dy + dz * dz + eps2;
      if (r2 == 0.0) continue;
      const double rinv = 1.0 / sqrt(r2);
      const double mr3 = mj[j] * rinv * rinv * rinv;
      ex[0] += mr3 * dx;
      ex[1] += mr3 * dy;
      ex[2] += mr3 * dz;
    }
    double ap[3] = {0.0, 0.0, 0.0};
    const double dx = com[0] - xi[i], dy = com[1] - yi[i], dz = com[2] - zi[i];
    const double r2 = dx * dx + dy * dy + dz * dz + eps2;
    if (r2 > 0.0) {
      const double rinv = 1.0 / sqrt(r2);
      const double mr3 = M * rinv * rinv * rinv;
      ap[0] = mr3 * dx;
      ap[1] = mr3 * dy;
      ap[2] = mr3 * dz;
      if (quad) { /* R10, r = x_i - COM */
        const double r[3] = {-dx, -dy, -dz};
        const double Qr[3] = {Q[0] * r[0] + Q[3] * r[1] + Q[4] * r[2],
                              Q[3] * r[0] + Q[1] * r[1] + Q[5] * r[2],
                              Q[4] * r[0] + Q[5] * r[1] + Q[2] * r[2]};
        const double rQr = r[0] * Qr[0] + r[1] * Qr[1] + r[2] * Qr[2];
        const double rinv2 = rinv * rinv, rinv5 = rinv2 * rinv2 * rinv, rinv7 = rinv5 * rinv2;
        for (int k = 0; k < 3; k++) ap[k] += Qr[k] * rinv5 - 2.5 * rQr * r[k] * rinv7;
      }
    }
    const double e0 = ap[0] - ex[0], e1 = ap[1] - ex[1], e2 = ap[2] - ex[2];
    const double err = sqrt(e0 * e0 + e1 * e1 + e2 * e2) / ai[i];
    if (err > worst || isnan(err)) worst = err;
  }
  double lab = worst > 0.0 ? log2(worst) : -40.0;
  if (!(lab <= 8.0)) lab = 8.0; /* also NaN (zero reference magnitude) */
  if (lab < -40.0) lab = -40.0;
  return lab;
}

/* FP32 inputs of R12 for cell c as the walk sees them. */
static void cell_inputs(const afo_tree *t, int64_t c, float com[3], float *s2, float *M,
                        float Q[6]) {
  const float s = ldexpf((float)t->root[3], -t->level[c]);
  *s2 = s * s;
  for (int k = 0; k < 3; k++) com[k] = (float)t->com[c * 3 + k];
  *M = (float)t->mass[c];
  for (int q = 0; q < 6; q++) Q[q] = (float)t->qmom[c * 6 + q];
}

static void group_boxf(const afo_tree *t, int64_t g, float bmin[3], float bmax[3]) {
  for (int k = 0; k < 3; k++) {
    bmin[k] = (float)t->g_box[g * 6 + k];
    bmax[k] = (float)t->g_box[g * 6 + 3 + k];
  }
}

static int contains_group(const afo_tree *t, int64_t g, int64_t c) {
  return t->g_first[g] >= t->first[c] && t->g_first[g] < t->first[c] + t->count[c];
}

/* Squared COM-to-box distance of R8 (same operations as mac_accept). */
static float box_d2(const float bmin[3], const float bmax[3], const float com[3]) {
  float d[3];
  for (int k = 0; k < 3; k++) {
    d[k] = 0.0f;
    if (com[k] < bmin[k]) d[k] = bmin[k] - com[k];
    else if (com[k] > bmax[k]) d[k] = com[k] - bmax[k];
  }
  float d2 = d[0] * d[0];
  d2 = d2 + d[1] * d[1];
  d2 = d2 + d[2] * d[2];
  return d2;
}

/* Features of the pair (g, c) in a tree built with reference accelerations. */
void afo_pair_features(const afo_tree *t, int64_t g, int64_t c, float f[AFO_MAC_NF]) {
  float bmin[3], bmax[3], com[3], s2, M, Q[6];
  group_boxf(t, g, bmin, bmax);
  cell_inputs(t, c, com, &s2, &M, Q);
  const float e = (float)t->eps;
  afo_mac_features(bmin, bmax, com, s2, M, Q, t->count[c], e * e,
                   t->g_amin ? t->g_amin[g] : 0.0f, f);
}

/* Learned decision of R14; 1 = accept cell c as a superparticle of g. */
static int learned_accept(const afo_tree *t, int64_t g, int64_t c, const float bmin[3],
                          const float bmax[3], const float com[3], float s2) {
  if (contains_group(t, g, c)) return 0;
  const float d2 = box_d2(bmin, bmax, com);
  const float lo = t->mac_lo2 * d2;
  if (s2 < lo) return 1;
  const float hi = t->mac_hi2 * d2;
  if (!(s2 < hi)) return 0;
  float f[AFO_MAC_NF];
  afo_pair_features(t, g, c, f);
  double bound;
  const float y = afo_mlp_forward_bound(t->mac_w, f, &bound);
  const int own = y < t->mac_tau;
  if (!t->ovr_off || !(fabs((double)y - (double)t->mac_tau) <= bound)) return own;
  int other = 0;
  for (int64_t k = t->ovr_off[g]; k < t->ovr_off[g + 1]; k++)
    if (t->ovr_spj[k] == (int32_t)c) other = 1;
  t->band_cnt[g]++;
  if (other != own) t->flip_cnt[g]++;
  return other;
}

/* Training target of R15 for the pair (g, c). */
double afo_pair_label(const afo_tree *t, int64_t g, int64_t c) {
  const int64_t f = t->g_first[g], fc = t->first[c];
  double ai[1024];
  const int64_t ni = t->g_count[g] < 1024 ? t->g_count[g] : 1024;
  for (int64_t i = 0; i < ni; i++) ai[i] = t->amag_s ? (double)t->amag_s[f + i] : 0.0;
  return afo_mac_label(ni, t->xs + f, t->ys + f, t->zs + f, ai, t->count[c], t->xs + fc,
                       t->ys + fc, t->zs + fc, t->ms + fc, t->mass[c], &t->com[c * 3],
                       &t->qmom[c * 6], t->eps, t->quad);
}

/* LET of reading R16 for the domain box (min x y z, max x y z): writes up
 * to cap elements (x, y, z, m, kind: 0 particle, 1 superparticle) and
 * returns their count. */
int64_t afo_let_export(const afo_tree *t, const double box[6], double theta, int64_t cap,
                       double *x, double *y, double *z, double *m, int32_t *kind) {
  float bmin[3], bmax[3];
  for (int k = 0; k < 3; k++) {
    bmin[k] = (float)box[k];
    bmax[k] = (float)box[3 + k];
  }
  const float theta2 = (float)theta * (float)theta;
  const float L = (float)t->root[3];
  int64_t ne = 0;
  int64_t *stack = malloc(sizeof(int64_t) * (size_t)(8 * t->n_cells + 8));
  int64_t sp = 0;
  if (t->n_cells > 0) stack[sp++] = 0;
  while (sp > 0) {
    const int64_t c = stack[--sp];
    const float s = ldexpf(L, -t->level[c]);
    float com[3];
    for (int k = 0; k < 3; k++) com[k] = (float)t->com[c * 3 + k];
    if (mac_accept(bmin, bmax, com, s * s, theta2)) {
      if (ne < cap) {
        x[ne] = t->com[c * 3];
        y[ne] = t->com[c * 3 + 1];
        z[ne] = t->com[c * 3 + 2];
        m[ne] = t->mass[c];
        kind[ne] = 1;
      }
      ne++;
    } else if (is_leaf(t, c)) {
      for (int64_t k = t->first[c]; k < t->first[c] + t->count[c]; k++) {
        if (ne < cap) {
          x[ne] = t->xs[k];
          y[ne] = t->ys[k];
          z[ne] = t->zs[k];
          m[ne] = t->ms[k];
          kind[ne] = 0;
        }
        ne++;
      }
    } else {
      for (int o = 7; o >= 0; o--)
        if (t->child[c * 8 + o] >= 0) stack[sp++] = t->child[c * 8 + o];
    }
  }
  free(stack);
  return ne;
}

void afo_pair_features_batch(const afo_tree *t, int64_t n, const int64_t *pairs, float *f) {
  for (int64_t i = 0; i < n; i++)
    afo_pair_features(t, pairs[2 * i], pairs[2 * i + 1], f + i * AFO_MAC_NF);
}

void afo_pair_label_batch(const afo_tree *t, int64_t n, const int64_t *pairs, double *out) {
#pragma omp parallel for schedule(dynamic, 8)
  for (int64_t i = 0; i < n; i++) out[i] = afo_pair_label(t, pairs[2 * i], pairs[2 * i + 1]);
}

/* Every (group, cell) pair whose decision R14 leaves to the network, over
 * the walk that opens every other cell not accepted below theta_lo: band
 * cells are recorded and opened. Writes up to cap pairs (group, cell) in
 * group order, depth-first, children in Morton order; returns the count. */
int64_t afo_band_pairs(const afo_tree *t, double theta_lo, double theta_hi, int64_t cap,
                       int64_t *pairs) {
  const float lo2 = (float)theta_lo * (float)theta_lo;
  const float hi2 = (float)theta_hi * (float)theta_hi;
  int64_t np = 0;
  int64_t *stack = malloc(sizeof(int64_t) * (size_t)(8 * t->n_cells + 8));
  for (int64_t g = 0; g < t->n_groups; g++) {
    float bmin[3], bmax[3];
    group_boxf(t, g, bmin, bmax);
    int64_t sp = 0;
    if (t->n_cells > 0) stack[sp++] = 0;
    while (sp > 0) {
      const int64_t c = stack[--sp];
      float com[3], s2, M, Q[6];
      cell_inputs(t, c, com, &s2, &M, Q);
      int open = 1;
      if (!contains_group(t, g, c)) {
        const float d2 = box_d2(bmin, bmax, com);
        const float lo = lo2 * d2, hi = hi2 * d2;
        if (s2 < lo) {
          open = 0;
        } else if (s2 < hi) {
          if (np < cap) {
            pairs[2 * np] = g;
            pairs[2 * np + 1] = c;
          }
          np++;
        }
      }
      if (open && !is_leaf(t, c))
        for (int o = 7; o >= 0; o--)
          if (t->child[c * 8 + o] >= 0) stack[sp++] = t->child[c * 8 + o];
    }
  }
  free(stack);
  return np;
}

/* Barnes' vectorised walk for one group (Section 2, Section 4.1; R8 or
 * R14, R9).
 * With epj/spj NULL it only counts. */
static void walk_group(const afo_tree *t, int64_t g, int32_t *epj, int32_t *spj,
                       int64_t *n_epj, int64_t *n_spj, int32_t *self_in) {
  float bmin[3], bmax[3];
  for (int k = 0; k < 3; k++) {
    bmin[k] = (float)t->g_box[g * 6 + k];
    bmax[k] = (float)t->g_box[g * 6 + 3 + k];
  }
  const float theta2 = (float)t->theta * (float)t->theta;
  const float L = (float)t->root[3];
  int64_t ne = 0, ns = 0;
  int32_t self = 0;
  if (t->band_cnt) t->band_cnt[g] = t->flip_cnt[g] = 0;
  int64_t stack[8 * (AFO_LEVELS + 2)];
  int sp = 0;
  if (t->n_cells > 0) stack[sp++] = 0;
  while (sp > 0) {
    const int64_t c = stack[--sp];
    const float s = ldexpf(L, -t->level[c]);
    const float s2 = s * s;
    float com[3];
    for (int k = 0; k < 3; k++) com[k] = (float)t->com[c * 3 + k];
    const int accept = t->mac_on ? learned_accept(t, g, c, bmin, bmax, com, s2)
                                 : mac_accept(bmin, bmax, com, s2, theta2);
    if (accept) {
      if (spj) spj[ns] = (int32_t)c;
      ns++;
    } else if (is_leaf(t, c)) {
      const int64_t f = t->first[c];
      for (int64_t k = f; k < f + t->count[c]; k++) {
        if (epj) epj[ne] = (int32_t)k;
        ne++;
      }
      if (t->g_first[g] >= f && t->g_first[g] < f + t->count[c]) self = 1;
    } else {
      for (int o = 7; o >= 0; o--)
        if (t->child[c * 8 + o] >= 0) stack[sp++] = t->child[c * 8 + o];
    }
  }
  *n_epj = ne;
  *n_spj = ns;
  *self_in = self;
}

static void make_lists(afo_tree *t) {
  const int64_t ng = t->n_groups;
  int64_t *ce = xcalloc(ng, sizeof(int64_t)), *cs = xcalloc(ng, sizeof(int64_t));
#pragma omp parallel for schedule(dynamic, 4)
  for (int64_t g = 0; g < ng; g++)
    walk_group(t, g, NULL, NULL, &ce[g], &cs[g], &t->g_self[g]);
  t->epj_off = xcalloc(ng + 1, sizeof(int64_t));
  t->spj_off = xcalloc(ng + 1, sizeof(int64_t));
  for (int64_t g = 0; g < ng; g++) {
    t->epj_off[g + 1] = t->epj_off[g] + ce[g];
    t->spj_off[g + 1] = t->spj_off[g] + cs[g];
  }
  t->epj = xcalloc(t->epj_off[ng], sizeof(int32_t));
  t->spj = xcalloc(t->spj_off[ng], sizeof(int32_t));
#pragma omp parallel for schedule(dynamic, 4)
  for (int64_t g = 0; g < ng; g++) {
    int64_t a, b;
    int32_t s;
    walk_group(t, g, t->epj + t->epj_off[g], t->spj + t->spj_off[g], &a, &b, &s);
  }
  free(ce);
  free(cs);
}

/* Construction step (Section 4.3, Section 4.2 "tree construction step"):
 * root, keys, sort, reorder, link, moments, groups and interaction lists.
 * With mac_w (AFO_MAC_NP FP16-valued parameters) and amag (reference |a|
 * per particle, caller order) both given, the lists follow the learned
 * decision of R14 with theta_lo, theta_hi and tau; otherwise R8. Returns
 * NULL on bad input (non-finite coordinates or masses). */
afo_tree *afo_build_mac(int64_t n, const double *x, const double *y, const double *z,
                        const double *m, int n_leaf, int n_grp, double theta, double eps,
                        int quad, const float *mac_w, double theta_lo, double theta_hi,
                        double tau, const float *amag) {
  for (int64_t i = 0; i < n; i++)
    if (!isfinite(m[i])) return NULL;
  afo_tree *t = calloc(1, sizeof(afo_tree));
  t->n = n;
  t->n_leaf = n_leaf;
  t->n_grp = n_grp;
  t->theta = theta;
  t->eps = eps;
  t->quad = quad;
  t->need_q = amag != NULL;
  if (mac_w && amag) {
    t->mac_on = 1;
    memcpy(t->mac_w, mac_w, sizeof(t->mac_w));
    t->mac_lo2 = (float)theta_lo * (float)theta_lo;
    t->mac_hi2 = (float)theta_hi * (float)theta_hi;
    t->mac_tau = (float)tau;
  }
  if (afo_root_cell(n, x, y, z, t->root) != 0) {
    free(t);
    return NULL;
  }
  uint64_t *raw = xcalloc(n, sizeof(uint64_t));
  afo_morton_keys(n, x, y, z, t->root, raw);
  t->keys = xcalloc(n, sizeof(uint64_t));
  t->perm = xcalloc(n, sizeof(int64_t));
  afo_radix_sort(n, raw, t->keys, t->perm);
  free(raw);
  t->xs = xcalloc(n, sizeof(double));
  t->ys = xcalloc(n, sizeof(double));
  t->zs = xcalloc(n, sizeof(double));
  t->ms = xcalloc(n, sizeof(double));
  reorder(t, x, y, z, m);
  link_cells(t);
  t->mass = xcalloc(t->n_cells, sizeof(double));
  t->smom = xcalloc(t->n_cells * 3, sizeof(double));
  t->com = xcalloc(t->n_cells * 3, sizeof(double));
  t->qmom = xcalloc(t->n_cells * 6, sizeof(double));
  moments(t);
  make_groups(t);
  group_boxes(t);
  if (amag) {
    t->amag_s = xcalloc(n, sizeof(float));
    for (int64_t k = 0; k < n; k++) t->amag_s[k] = amag[t->perm[k]];
    t->g_amin = xcalloc(t->n_groups, sizeof(float));
    for (int64_t g = 0; g < t->n_groups; g++) {
      float a = t->amag_s[t->g_first[g]];
      for (int64_t k = t->g_first[g] + 1; k < t->g_first[g] + t->g_count[g]; k++)
        if (t->amag_s[k] < a) a = t->amag_s[k];
      t->g_amin[g] = a;
    }
  }
  make_lists(t);
  return t;
}

afo_tree *afo_build(int64_t n, const double *x, const double *y, const double *z,
                    const double *m, int n_leaf, int n_grp, double theta, double eps,
                    int quad) {
  return afo_build_mac(n, x, y, z, m, n_leaf, n_grp, theta, eps, quad, NULL, 0.0, 0.0, 0.0,
                       NULL);
}

/* Reusing step (Section 4.2): topology and lists are kept; the particle
 * data are reordered with the saved permutation and the moments and group
 * boxes are recomputed from the new positions. */
int afo_update(afo_tree *t, const double *x, const double *y, const double *z,
               const double *m) {
  for (int64_t i = 0; i < t->n; i++)
    if (!isfinite(x[i]) || !isfinite(y[i]) || !isfinite(z[i]) || !isfinite(m[i])) return -1;
  reorder(t, x, y, z, m);
  moments(t);
  group_boxes(t);
  return 0;
}

/* Lists made again on the current topology, moments and group boxes (a
 * MAKE_LIST after reusing steps, without a new tree). */
void afo_relist(afo_tree *t) {
  free(t->epj_off); free(t->spj_off); free(t->epj); free(t->spj);
  make_lists(t);
}

/* Lists made again (as afo_relist) with the learned criterion, taking the
 * decisions of another implementation -- given as its SPJ lists, CSR with
 * spj_off[n_groups + 1], cell ids in this tree's numbering -- for the pairs
 * whose network output lies within the rounding bound of R13 from tau, the
 * pairs where two correct FP32 implementations may decide differently.
 * counts[0] receives the number of such pairs visited, counts[1] those the
 * other implementation decided otherwise than this oracle. The lists then
 * equal the other implementation's exactly iff it agrees on every other
 * pair. */
void afo_relist_band(afo_tree *t, const int64_t *spj_off, const int32_t *spj,
                     int64_t counts[2]) {
  t->ovr_off = spj_off;
  t->ovr_spj = spj;
  t->band_cnt = xcalloc(t->n_groups, sizeof(int64_t));
  t->flip_cnt = xcalloc(t->n_groups, sizeof(int64_t));
  afo_relist(t);
  counts[0] = counts[1] = 0;
  for (int64_t g = 0; g < t->n_groups; g++) {
    counts[0] += t->band_cnt[g];
    counts[1] += t->flip_cnt[g];
  }
  free(t->band_cnt);
  free(t->flip_cnt);
  t->band_cnt = t->flip_cnt = NULL;
  t->ovr_off = NULL;
  t->ovr_spj = NULL;
}

/* Force on the saved lists (Section 5: interaction of the EPJs and SPJs of a
 * group's list with its EPIs), FP64, results in caller order. Only the
 * groups sel[0..n_sel) are evaluated (all groups when sel is NULL); the
 * outputs of other particles are left untouched. */
void afo_force_groups(const afo_tree *t, int64_t n_sel, const int64_t *sel, double *ax,
                      double *ay, double *az, double *pot) {
  const double eps2 = t->eps * t->eps;
  const int64_t ng = sel ? n_sel : t->n_groups;
#pragma omp parallel for schedule(dynamic, 4)
  for (int64_t gs = 0; gs < ng; gs++) {
    const int64_t g = sel ? sel[gs] : gs;
    for (int64_t i = t->g_first[g]; i < t->g_first[g] + t->g_count[g]; i++) {
      const double xi = t->xs[i], yi = t->ys[i], zi = t->zs[i];
      double sx = 0.0, sy = 0.0, sz = 0.0, sp = 0.0;
      for (int64_t e = t->epj_off[g]; e < t->epj_off[g + 1]; e++) {
        const int64_t j = t->epj[e];
        if (j == i) continue;
        const double dx = t->xs[j] - xi, dy = t->ys[j] - yi, dz = t->zs[j] - zi;
        const double r2 = dx * dx + dy * dy + dz * dz + eps2;
        if (r2 == 0.0) continue;
        const double rinv = 1.0 / sqrt(r2);
        const double mr = t->ms[j] * rinv;
        const double mr3 = mr * rinv * rinv;
        sx += mr3 * dx;
        sy += mr3 * dy;
        sz += mr3 * dz;
        sp -= mr;
      }
      for (int64_t e = t->spj_off[g]; e < t->spj_off[g + 1]; e++) {
        const int64_t c = t->spj[e];
        const double *cm = &t->com[c * 3];
        const double dx = cm[0] - xi, dy = cm[1] - yi, dz = cm[2] - zi;
        const double r2 = dx * dx + dy * dy + dz * dz + eps2;
        if (r2 == 0.0) continue;
        const double rinv = 1.0 / sqrt(r2);
        const double mr = t->mass[c] * rinv;
        const double mr3 = mr * rinv * rinv;
        sx += mr3 * dx;
        sy += mr3 * dy;
        sz += mr3 * dz;
        sp -= mr;
        if (t->quad) {
          /* R10 with r = x_i - COM = -(dx, dy, dz). */
          const double *Q = &t->qmom[c * 6];
          const double r[3] = {-dx, -dy, -dz};
          const double Qr[3] = {Q[0] * r[0] + Q[3] * r[1] + Q[4] * r[2],
                                Q[3] * r[0] + Q[1] * r[1] + Q[5] * r[2],
                                Q[4] * r[0] + Q[5] * r[1] + Q[2] * r[2]};
          const double rQr = r[0] * Qr[0] + r[1] * Qr[1] + r[2] * Qr[2];
          const double rinv2 = rinv * rinv;
          const double rinv5 = rinv2 * rinv2 * rinv;
          const double rinv7 = rinv5 * rinv2;
          sx += Qr[0] * rinv5 - 2.5 * rQr * r[0] * rinv7;
          sy += Qr[1] * rinv5 - 2.5 * rQr * r[1] * rinv7;
          sz += Qr[2] * rinv5 - 2.5 * rQr * r[2] * rinv7;
          sp -= 0.5 * rQr * rinv5;
        }
      }
      const int64_t o = t->perm[i];
      ax[o] = sx;
      ay[o] = sy;
      az[o] = sz;
      pot[o] = sp;
    }
  }
}

void afo_force(const afo_tree *t, double *ax, double *ay, double *az, double *pot) {
  afo_force_groups(t, 0, NULL, ax, ay, az, pot);
}

/* Kick-drift-kick leapfrog with list reuse (reading R11). acc holds the
 * accelerations at the start (caller order, ax/ay/az) and is updated. The
 * tree *t is rebuilt on construction steps; *t may be replaced. */
int afo_leapfrog(afo_tree **tp, int64_t n, double *x, double *y, double *z, double *vx,
                 double *vy, double *vz, const double *m, double *ax, double *ay, double *az,
                 double *pot, double dt, int n_steps, int n_reuse, int64_t *eval_counter) {
  for (int s = 0; s < n_steps; s++) {
    for (int64_t i = 0; i < n; i++) {
      vx[i] += ax[i] * (0.5 * dt);
      vy[i] += ay[i] * (0.5 * dt);
      vz[i] += az[i] * (0.5 * dt);
      x[i] += vx[i] * dt;
      y[i] += vy[i] * dt;
      z[i] += vz[i] * dt;
    }
    afo_tree *t = *tp;
    if (*eval_counter % n_reuse == 0) {
      afo_tree *nt = afo_build(n, x, y, z, m, t->n_leaf, t->n_grp, t->theta, t->eps, t->quad);
      if (!nt) return -1;
      afo_free(t);
      *tp = t = nt;
    } else if (afo_update(t, x, y, z, m) != 0) {
      return -1;
    }
    (*eval_counter)++;
    afo_force(t, ax, ay, az, pot);
    for (int64_t i = 0; i < n; i++) {
      vx[i] += ax[i] * (0.5 * dt);
      vy[i] += ay[i] * (0.5 * dt);
      vz[i] += az[i] * (0.5 * dt);
    }
  }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Accessors for the ctypes wrapper.                                        */
/* ------------------------------------------------------------------------ */

void afo_sizes(const afo_tree *t, int64_t out[5]) {
  out[0] = t->n;
  out[1] = t->n_cells;
  out[2] = t->n_groups;
  out[3] = t->n_groups > 0 ? t->epj_off[t->n_groups] : 0;
  out[4] = t->n_groups > 0 ? t->spj_off[t->n_groups] : 0;
}

void afo_get_root(const afo_tree *t, double root[4]) { memcpy(root, t->root, sizeof(t->root)); }

void afo_get_order(const afo_tree *t, uint64_t *keys, int64_t *perm) {
  memcpy(keys, t->keys, sizeof(uint64_t) * (size_t)t->n);
  memcpy(perm, t->perm, sizeof(int64_t) * (size_t)t->n);
}

void afo_get_cells(const afo_tree *t, int32_t *level, int64_t *first, int64_t *count,
                   int64_t *parent, int64_t *skip, int32_t *n_child, int64_t *child) {
  const size_t nc = (size_t)t->n_cells;
  memcpy(level, t->level, sizeof(int32_t) * nc);
  memcpy(first, t->first, sizeof(int64_t) * nc);
  memcpy(count, t->count, sizeof(int64_t) * nc);
  memcpy(parent, t->parent, sizeof(int64_t) * nc);
  memcpy(skip, t->skip, sizeof(int64_t) * nc);
  memcpy(n_child, t->n_child, sizeof(int32_t) * nc);
  memcpy(child, t->child, sizeof(int64_t) * nc * 8);
}

void afo_get_moments(const afo_tree *t, double *mass, double *com, double *quad) {
  const size_t nc = (size_t)t->n_cells;
  memcpy(mass, t->mass, sizeof(double) * nc);
  memcpy(com, t->com, sizeof(double) * nc * 3);
  memcpy(quad, t->qmom, sizeof(double) * nc * 6);
}

void afo_get_groups(const afo_tree *t, int64_t *first, int64_t *count, int64_t *cell,
                    double *box, int32_t *self_in) {
  const size_t ng = (size_t)t->n_groups;
  memcpy(first, t->g_first, sizeof(int64_t) * ng);
  memcpy(count, t->g_count, sizeof(int64_t) * ng);
  memcpy(cell, t->g_cell, sizeof(int64_t) * ng);
  memcpy(box, t->g_box, sizeof(double) * ng * 6);
  memcpy(self_in, t->g_self, sizeof(int32_t) * ng);
}

void afo_get_lists(const afo_tree *t, int64_t *epj_off, int32_t *epj, int64_t *spj_off,
                   int32_t *spj) {
  const size_t ng = (size_t)t->n_groups;
  memcpy(epj_off, t->epj_off, sizeof(int64_t) * (ng + 1));
  memcpy(spj_off, t->spj_off, sizeof(int64_t) * (ng + 1));
  if (ng > 0) {
    memcpy(epj, t->epj, sizeof(int32_t) * (size_t)t->epj_off[ng]);
    memcpy(spj, t->spj, sizeof(int32_t) * (size_t)t->spj_off[ng]);
  }
}

/* ------------------------------------------------------------------------ */
/* Short-range neighbour walk and density (Section 2, Section 4.2;          */
/* readings R17, R18).                                                      */
/* ------------------------------------------------------------------------ */

/* FP64 to FP32 rounded toward -inf / +inf. */
static float f32_down(double v) {
  float f = (float)v;
  if ((double)f > v) f = nextafterf(f, -INFINITY);
  return f;
}

static float f32_up(double v) {
  float f = (float)v;
  if ((double)f < v) f = nextafterf(f, INFINITY);
  return f;
}

static int boxes_meet(const float *a, const float *b) {
  for (int k = 0; k < 3; k++)
    if (a[k] > b[3 + k] || a[3 + k] < b[k]) return 0;
  return 1;
}

/* The neighbour lists of R17 for search radii h (caller order) and margin
 * skin, replacing any earlier ones. Returns 0, or -1 when a radius is not
 * finite or not positive, or skin is not finite or negative. */
int afo_nbr_lists(afo_tree *t, const double *h, double skin) {
  if (!isfinite(skin) || skin < 0.0) return -1;
  for (int64_t i = 0; i < t->n; i++)
    if (!isfinite(h[i]) || !(h[i] > 0.0)) return -1;
  free(t->c_tbox); free(t->g_sbox); free(t->nbr_off); free(t->nbr);
  t->c_tbox = xcalloc(t->n_cells * 6, sizeof(float));
  t->g_sbox = xcalloc(t->n_groups * 6, sizeof(float));
  const double *pos[3] = {t->xs, t->ys, t->zs};
  for (int64_t c = 0; c < t->n_cells; c++) {
    double lo[3], hi[3];
    const int64_t f = t->first[c];
    for (int k = 0; k < 3; k++) lo[k] = hi[k] = pos[k][f];
    for (int64_t i = f + 1; i < f + t->count[c]; i++)
      for (int k = 0; k < 3; k++) {
        if (pos[k][i] < lo[k]) lo[k] = pos[k][i];
        if (pos[k][i] > hi[k]) hi[k] = pos[k][i];
      }
    for (int k = 0; k < 3; k++) {
      t->c_tbox[c * 6 + k] = f32_down(lo[k]);
      t->c_tbox[c * 6 + 3 + k] = f32_up(hi[k]);
    }
  }
  for (int64_t g = 0; g < t->n_groups; g++) {
    double lo[3], hi[3];
    for (int64_t i = t->g_first[g]; i < t->g_first[g] + t->g_count[g]; i++) {
      const double r = h[t->perm[i]] + skin;
      for (int k = 0; k < 3; k++) {
        const double a = pos[k][i] - r, b = pos[k][i] + r;
        if (i == t->g_first[g] || a < lo[k]) lo[k] = a;
        if (i == t->g_first[g] || b > hi[k]) hi[k] = b;
      }
    }
    for (int k = 0; k < 3; k++) {
      t->g_sbox[g * 6 + k] = f32_down(lo[k]);
      t->g_sbox[g * 6 + 3 + k] = f32_up(hi[k]);
    }
  }
  /* the walk, once to count and once to write */
  int64_t *stack = malloc(sizeof(int64_t) * (size_t)(8 * (AFO_LEVELS + 2)));
  t->nbr_off = xcalloc(t->n_groups + 1, sizeof(int64_t));
  for (int pass = 0; pass < 2; pass++) {
    if (pass == 1) t->nbr = xcalloc(t->nbr_off[t->n_groups], sizeof(int32_t));
    for (int64_t g = 0; g < t->n_groups; g++) {
      const float *sb = &t->g_sbox[g * 6];
      int64_t ne = 0;
      int64_t sp = 0;
      if (t->n_cells > 0) stack[sp++] = 0;
      while (sp > 0) {
        const int64_t c = stack[--sp];
        if (!boxes_meet(&t->c_tbox[c * 6], sb)) continue;
        if (is_leaf(t, c)) {
          for (int64_t k = t->first[c]; k < t->first[c] + t->count[c]; k++) {
            if (pass == 1) t->nbr[t->nbr_off[g] + ne] = (int32_t)k;
            ne++;
          }
        } else {
          for (int o = 7; o >= 0; o--)
            if (t->child[c * 8 + o] >= 0) stack[sp++] = t->child[c * 8 + o];
        }
      }
      if (pass == 0) t->nbr_off[g + 1] = t->nbr_off[g] + ne;
    }
  }
  free(stack);
  return 0;
}

/* w(q) of R18. */
static double spline_w(double q) {
  if (q <= 0.5) return 1.0 - 6.0 * q * q + 6.0 * q * q * q;
  if (q < 1.0) {
    const double u = 1.0 - q;
    return 2.0 * u * u * u;
  }
  return 0.0;
}

/* Density and smooth neighbour number of R18 over the neighbour lists
 * (current positions: after afo_update the lists are kept), caller order. */
void afo_sph_density(const afo_tree *t, const double *h, double *rho, double *nnb) {
  const double pi = 3.14159265358979323846;
#pragma omp parallel for schedule(dynamic, 4)
  for (int64_t g = 0; g < t->n_groups; g++) {
    for (int64_t i = t->g_first[g]; i < t->g_first[g] + t->g_count[g]; i++) {
      const double hi = h[t->perm[i]];
      double sm = 0.0, sw = 0.0;
      for (int64_t e = t->nbr_off[g]; e < t->nbr_off[g + 1]; e++) {
        const int64_t j = t->nbr[e];
        const double dx = t->xs[j] - t->xs[i], dy = t->ys[j] - t->ys[i],
                     dz = t->zs[j] - t->zs[i];
        const double w = spline_w(sqrt(dx * dx + dy * dy + dz * dz) / hi);
        sm += t->ms[j] * w;
        sw += w;
      }
      rho[t->perm[i]] = 8.0 / (pi * hi * hi * hi) * sm;
      nnb[t->perm[i]] = 32.0 / 3.0 * sw;
    }
  }
}

/* The same sums over every particle j (the definition, no tree), for the
 * targets tgt[0..n_tgt). */
void afo_sph_density_direct(int64_t n, const double *x, const double *y, const double *z,
                            const double *m, const double *h, int64_t n_tgt,
                            const int64_t *tgt, double *rho, double *nnb) {
  const double pi = 3.14159265358979323846;
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t t = 0; t < n_tgt; t++) {
    const int64_t i = tgt[t];
    const double hi = h[i];
    double sm = 0.0, sw = 0.0;
    for (int64_t j = 0; j < n; j++) {
      const double dx = x[j] - x[i], dy = y[j] - y[i], dz = z[j] - z[i];
      const double w = spline_w(sqrt(dx * dx + dy * dy + dz * dz) / hi);
      sm += m[j] * w;
      sw += w;
    }
    rho[t] = 8.0 / (pi * hi * hi * hi) * sm;
    nnb[t] = 32.0 / 3.0 * sw;
  }
}

int64_t afo_nbr_total(const afo_tree *t) { return t->nbr_off ? t->nbr_off[t->n_groups] : -1; }

void afo_get_nbr(const afo_tree *t, int64_t *off, int32_t *idx, float *tbox, float *sbox) {
  memcpy(off, t->nbr_off, sizeof(int64_t) * (size_t)(t->n_groups + 1));
  memcpy(idx, t->nbr, sizeof(int32_t) * (size_t)t->nbr_off[t->n_groups]);
  memcpy(tbox, t->c_tbox, sizeof(float) * (size_t)(6 * t->n_cells));
  memcpy(sbox, t->g_sbox, sizeof(float) * (size_t)(6 * t->n_groups));
}

int afo_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
