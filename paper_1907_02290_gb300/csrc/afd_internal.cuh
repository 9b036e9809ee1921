// Internal declarations of the sm_103a tree-gravity library: the context,
// device buffers and the host-side launchers of every kernel. Not part of
// the C ABI (include/afdps.h is).
#pragma once

#include <cuda_runtime.h>

#include <cfloat>
#include <cstddef>
#include <cstdint>
#include <vector>

#include "afdps.h"

namespace afd {

constexpr int kLevels = 21;          // 21 key bits per axis, deepest level
constexpr uint32_t kNone = 0xffffffffu;

// A device allocation that only grows.
struct DevBuf {
  void *p = nullptr;
  size_t cap = 0;
};

int reserve(DevBuf &b, size_t bytes);  // AFD_OK or AFD_ERR_OOM
void release(DevBuf &b);
template <class T>
inline T *ptr(const DevBuf &b) {
  return static_cast<T *>(b.p);
}

// Device status word bits (OR-ed by kernels, decoded on the host).
enum : int {
  kStNonFinite = 1,
  kStWalkStack = 2,
  kStWalkIter = 4,
  kStOverflow = 8,
  kStBadRadius = 16,
  kStSpin = 32,  // a bounded wait on another block of the same launch gave up
  kStClimb = 64,  // a bottom-up climb went above the deepest level (a malformed tree)
};
int status_to_error(int bits);

// Half-precision far field: the per-group scale 2^-k, 2^k the smallest power
// of two >= mu (the largest M / d^2 over the group's far-field cells, d the
// distance from the cell's centre of mass to the group's box, a bound on
// every far-field term's magnitude M / rs^2), k clamped to [-100, 100]; 1
// without far-field mass.
__device__ __forceinline__ float far_group_scale(float mu) {
  int k = 0;
  if (mu > 0.0f && mu <= 3.4e38f) {
    const uint32_t b = __float_as_uint(mu);
    k = (int)((b >> 23) & 0xffu) - 127 + ((b & 0x7fffffu) != 0u ? 1 : 0);
    k = k < -100 ? -100 : (k > 100 ? 100 : k);
  } else if (mu > 0.0f) {
    k = 100;
  }
  return __uint_as_float((uint32_t)(127 - k) << 23);
}

// Side of the root cell for a scaled largest extent `target` (1.000001 x the
// extent, Section 4.3 root rule): the smallest power of two >= target; 1 when
// target is not positive (a zero extent) or NaN; +inf when no finite power of
// two reaches it (an infinite coordinate, or an extent that overflows). Read
// off the bits of the double with no loop, so every input ends in a fixed
// number of steps. The callers flag a side that is not finite as non-finite
// input.
__device__ __forceinline__ double root_side(double target) {
  if (!(target > 0.0)) return 1.0;
  const unsigned long long b = (unsigned long long)__double_as_longlong(target);
  const unsigned e = (unsigned)((b >> 52) & 0x7ffu);
  const unsigned long long f = b & 0xfffffffffffffull;
  if (e == 0x7ffu) return __longlong_as_double(0x7ff0000000000000ll);  // +inf
  if (e == 0u) {
    // subnormal target = f x 2^-1074, 0 < f < 2^52: the power of two 2^k >= f
    // as a subnormal, or 2^52 x 2^-1074 = the smallest normal, whose bits are
    // 2^52 as well
    const unsigned long long p = f <= 1ull ? 1ull : 1ull << (64 - __clzll((long long)(f - 1ull)));
    return __longlong_as_double((long long)p);
  }
  if (f == 0ull) return target;  // already a power of two
  if (e + 1u == 0x7ffu) return __longlong_as_double(0x7ff0000000000000ll);  // above 2^1023
  return __longlong_as_double((long long)((unsigned long long)(e + 1u) << 52));
}

// Order-preserving 64-bit key of a double (for finite values: a < b iff
// key(a) < key(b), except that -0 sorts below +0): min / max of positions
// on the integer pipes, exact, instead of on GB300's narrow FP64 pipe.
__device__ __forceinline__ unsigned long long okey(double v) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  return b ^ ((unsigned long long)((long long)b >> 63) | 0x8000000000000000ull);
}
__device__ __forceinline__ double okey_value(unsigned long long k) {
  const unsigned long long b = (k & 0x8000000000000000ull) ? (k ^ 0x8000000000000000ull) : ~k;
  return __longlong_as_double((long long)b);
}
__device__ __forceinline__ unsigned long long warp_min_key(unsigned long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = min(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ unsigned long long warp_max_key(unsigned long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// The key of a coordinate for the box reduction; NaN is left out (the
// neutral keys), and is flagged by the finiteness check.
__device__ __forceinline__ void box_keys(double v, unsigned long long &lo, unsigned long long &hi) {
  if (v != v) return;
  const unsigned long long k = okey(v);
  lo = min(lo, k);
  hi = max(hi, k);
}

// Centre and side of a root cell from the box keys (rule of R2, with the
// side from root_side); returns false when the side is not finite.
__device__ __forceinline__ bool root_from_keys(const unsigned long long *klo,
                                               const unsigned long long *khi, double *r) {
  double ext = 0.0;
  for (int d = 0; d < 3; d++) {
    const double lo = okey_value(klo[d]), hi = okey_value(khi[d]);
    r[d] = __dmul_rn(__dadd_rn(lo, hi), 0.5);
    const double e = __dsub_rn(hi, lo);
    if (e > ext) ext = e;
  }
  const double L = root_side(__dmul_rn(ext, 1.000001));
  r[3] = L;
  return L <= DBL_MAX;
}

}  // namespace afd

// Self-checking build (compile with -DAFD_CHECK=1): the kernels test every
// index that comes from data (list entries, chunk links, tree links) before
// using it, print each violation and skip the access. Off by default.
#ifndef AFD_CHECK
#define AFD_CHECK 0
#endif
#if AFD_CHECK
#include <cstdio>
static __device__ __noinline__ bool afd_check_fail(const char *where, unsigned long long i,
                                                   unsigned long long bound) {
  printf("AFD_CHECK %s: index %llu not below %llu (block %d thread %d)\n", where, i, bound,
         (int)blockIdx.x, (int)threadIdx.x);
  return false;
}
#define AFD_IN(i, bound, where)                                                   \
  ((unsigned long long)(i) < (unsigned long long)(bound)                          \
       ? true                                                                     \
       : afd_check_fail(where, (unsigned long long)(i), (unsigned long long)(bound)))
#else
#define AFD_IN(i, bound, where) true
#endif

struct afd_ctx {
  afd_config cfg{};
  int device = 0;
  cudaStream_t stream = nullptr;

  // sizes of the current tree / lists
  int64_t n = 0;
  int64_t n_cells = 0;
  int64_t n_groups = 0;
  int64_t n_units = 0;
  uint64_t n_epj = 0, n_spj = 0, interactions = 0;
  int max_level = 0;
  bool have_tree = false, have_lists = false, saved = false;

  // root cell and status
  afd::DevBuf root;       // f64[4] centre xyz, L
  afd::DevBuf status;     // i32[1]
  afd::DevBuf red_part;   // root-reduction partials
  afd::DevBuf red_count;  // u32 last-block counter (kept at 0 between launches)
  afd::DevBuf u64acc;     // u64[4] small accumulators

  // keys, sort and reorder
  afd::DevBuf keys, keys2, perm, perm2, sort_cnt, sort_off;
  afd::DevBuf xs, ys, zs, ms;  // FP64 Morton order
  afd::DevBuf mxyz;            // m x, m y, m z (3 x n FP64, Morton order): the leaf products of S
  afd::DevBuf jhi, jlo;        // float4 (hi xyz, m) and (lo xyz, 0) per particle

  // link
  afd::DevBuf lk_d, lk_c, lk_e;  // u8 per particle
  afd::DevBuf lk_cnt, lk_off;    // u32 per particle (+1)

  // cells (depth-first pre-order)
  afd::DevBuf c_level, c_first, c_count, c_skip, c_parent, c_child, c_arrive;
  afd::DevBuf leaf_ord, leaf_aux;  // leaves by particle count, and the bucket counters
  afd::DevBuf c_mass, c_smom, c_com, c_quad;  // f64
  afd::DevBuf s_hi, s_lo, s_q0, s_q1;         // float4 superparticle data
  afd::DevBuf node_f, node_i;                 // walk node data (float4, uint2)
  afd::DevBuf c_block;                        // per cell 8 child walk records (2 x uint4 each)
  // half-precision far field: per cell the negated normalised quadrupole
  // -Q / (M s^2) as three half2 words (xx yy, zz xy, xz yz) and s^2; per
  // group the power-of-two scale of its far-field terms
  afd::DevBuf s_h, g_fscale;
  bool fscale_ok = false;  // g_fscale matches the current lists

  // groups and force work units
  afd::DevBuf g_cnt, g_off;
  afd::DevBuf g_first, g_count, g_cell, g_box, g_boxf, g_self;
  afd::DevBuf u_cnt, u_off, u_info;
  // force-kernel launch order of the units of the work share, longest list
  // work first (u_work, u_hist: its per-unit work and bucket counters)
  afd::DevBuf u_order, u_work, u_hist;
  bool u_order_ok = false;

  // lists (CSR)
  afd::DevBuf l_cnt_e, l_cnt_s, epj_off, spj_off, epj, spj;
  // the non-indirect ablation: list entries' j-data copied into list order
  afd::DevBuf m_ehi, m_elo, m_shi, m_slo;
  // local essential tree export: per-cell marks, element counts and offsets
  afd::DevBuf let_mark, let_cnt, let_off;
  // short-range neighbour lists: per-cell tight boxes (float4 lo, hi) and
  // their bottom-up arrival counters, per-group search boxes (float[6]),
  // per-group counts (and a zero SPJ-count scratch), CSR offsets and lists
  afd::DevBuf c_tbox, nbr_arrive, g_sbox, nbr_cnt, nbr_off, nbr;
  // the walk's view of a cell's children's tight boxes: 8 x (lo, hi) per cell
  afd::DevBuf nbr_blk;
  // the walk's work items: seed cells (flags, offsets, ids), per group its
  // item count and first item, per item its group, seed and CSR offset
  afd::DevBuf nbr_seedf, nbr_seedo, nbr_seeds, nbr_icnt, nbr_igoff, nbr_itg, nbr_itr, nbr_ioff;
  afd::DevBuf nbr_sbb;  // union boxes of blocks of 32 seeds
  // density work items (unit, list segment), per-unit segment counts and
  // first items, partial sums of units with several segments
  afd::DevBuf nbr_seg_cnt, nbr_seg_off, nbr_items, nbr_part;
  // density items' launch order, largest work first (with its work and
  // bucket scratch)
  afd::DevBuf nbr_order, nbr_work, nbr_hist;
  bool nbr_order_ok = false;
  uint64_t n_nbr = 0, nbr_pairs = 0;
  int64_t n_items = 0;
  bool nbr_multi = false;  // some unit has several segments
  bool have_nbr = false;
  // walk record arena: per group leaf-record count and chunk-chain heads;
  // chunks of cell ids / leaf records, chain links, cursors (capacity in chunks)
  afd::DevBuf l_nrec;
  afd::DevBuf arena_s, arena_l, hdr_s, hdr_l, arena_cur;
  uint32_t arena_cap_s = 0, arena_cap_l = 0;
  // limits of the walks' bounded loops (afd_set_walk_limits; 0: defaults)
  uint32_t walk_iter_cap = 0, walk_arena_max = 0;
  int walk_stack_cap = 0;

  // scan scratch
  afd::DevBuf scan_tmp;

  // host-array entry point staging
  afd::DevBuf hx, hy, hz, hm, hacc;

  // pinned host scratch for small reads
  void *pinned = nullptr;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  bool force_timed = false;
  // force-kernel launch shape: warps per block (2, 4, 8), list entries staged
  // per chunk (32, 64); set by afd_set_launch / afd_autotune_launch
  int force_warps = 4, force_chunk = 32;

  // work share of a force step split over several processes (one system,
  // disjoint slices of groups): part share_part of share_parts; the groups
  // [share_g0, share_g1) and their units [share_u0, share_u1) of the current
  // lists, and their interactions. share_parts = 1: everything.
  int share_part = 0, share_parts = 1;
  int64_t share_g0 = 0, share_g1 = 0, share_u0 = 0, share_u1 = 0;
  uint64_t share_inter = 0;

  // independent systems (a forest): particles [sys_off[s], sys_off[s+1]) form
  // system s, with its own root cell and group size. n_sys = 1: one system.
  int n_sys = 1;
  std::vector<int64_t> sys_off_h{0, 0};
  std::vector<int32_t> sys_grp_h;
  afd::DevBuf sys_off_d;   // int64[n_sys + 1]
  afd::DevBuf sys_grp_d;   // u32[n_sys]
  afd::DevBuf sys_of;      // u32 per particle, caller order
  afd::DevBuf sys_s;       // u32 per particle, Morton (sorted) order
  afd::DevBuf root_tiles;  // int4 per reduction tile (system, begin, end, -)
  afd::DevBuf g_root;      // u32 per group: root cell of its system

  int64_t eval_counter = 0;
  int64_t launches = 0;  // kernels queued by this context so far

  // learned opening criterion (afd_mac.cuh): FP16-valued weights, band and
  // threshold, reference |a| per particle (caller order) and its Morton-order
  // copy and per-group minimum for the current tree
  afd::DevBuf mac_w;
  bool mac_ready = false;
  float mac_lo2 = 0.0f, mac_hi2 = 0.0f, mac_tau = 0.0f;
  afd::DevBuf amag, amag_s, g_amin;
  int64_t amag_n = -1;
  bool leaf_ord_ok = false;      // leaf_ord holds the current tree's leaves
  bool moments_current = false;  // the cell moments match the current positions
  bool q_current = false;       // the cell quadrupoles match the current positions
  bool blocks_current = false;  // the walk's child records match them too
  bool walk_learned = false;  // the last walk used the learned criterion
  afd::DevBuf mac_cnt;        // u64[2]: network evaluations, accepted (count pass)
  afd::DevBuf band_cnt, band_off;

  // captured reusing timestep (afd_graph_capture_step / afd_graph_launch)
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t graph_exec = nullptr;
  int64_t graph_launches = 0;  // kernels inside the captured graph
  cudaEvent_t graph_done = nullptr;  // recorded after each replay
};

namespace afd {

// ---- scans (afd_util.cu) ----
// Exclusive scan of n values into out[0..n]; out[n] is the total.
int scan_u32(afd_ctx *c, const uint32_t *in, uint32_t *out, int64_t n);
int scan_u32_to_u64(afd_ctx *c, const uint32_t *in, uint64_t *out, int64_t n);

// ---- tree (afd_tree.cu) ----
int launch_root(afd_ctx *c, const double *x, const double *y, const double *z, const double *m,
                int64_t n);
int launch_keys(afd_ctx *c, const double *x, const double *y, const double *z, int64_t n);
int launch_sort(afd_ctx *c, int64_t n);  // sorts keys/perm in place (result in keys, perm)
int launch_reorder(afd_ctx *c, const double *x, const double *y, const double *z,
                   const double *m, int64_t n);
int launch_link(afd_ctx *c, int64_t n);        // sets c->n_cells, c->max_level (syncs)
// bottom-up moments + superparticle data; quadrupoles when the far field
// uses them or need_q
int launch_moments(afd_ctx *c, bool child_blocks, bool need_q);
int launch_groups(afd_ctx *c);                 // sets c->n_groups, c->n_units (syncs)
int launch_group_boxes(afd_ctx *c);

// ---- walk (afd_walk.cu) ----
int launch_walk(afd_ctx *c);  // lists; sets n_epj, n_spj, interactions (syncs)
// neighbour lists from c_tbox and g_sbox; sets n_nbr, nbr_pairs (syncs)
int launch_nbr_walk(afd_ctx *c);

// ---- learned opening criterion (afd_mac.cu) ----
bool mac_usable(const afd_ctx *c);   // weights, reference |a| and quadrupoles present
int launch_group_amin(afd_ctx *c);   // amag_s and g_amin for the current tree
int launch_amag(afd_ctx *c, const float *acc4);  // reference |a| from a force result

// ---- work share (afd_api.cu) ----
// The groups and units of this context's part of the current lists (syncs
// when the share has more than one part).
int compute_share(afd_ctx *c);

// ---- force (afd_force.cu) ----
int order_units(afd_ctx *c);  // the force launch order of the current lists' units
int launch_force(afd_ctx *c, float *acc4);
int launch_materialize(afd_ctx *c);                    // j-data of every list entry, list order
int launch_force_materialized(afd_ctx *c, float *acc4);  // force kernel reading those copies

// ---- per-system statistics (afd_walk.cu) ----
// inter[s] = sum over system s's groups of n_i (n_epj + n_spj); entries[s] =
// its list entries. Device arrays of n_sys u64, overwritten.
int launch_sys_stats(afd_ctx *c, unsigned long long *inter, unsigned long long *entries);

// ---- integration (afd_api.cu) ----

}  // namespace afd
