// Interaction lists (Barnes' vectorised walk, Section 2; multiwalk,
// Section 3; index lists, Section 4.1). One warp walks the tree for one
// i-group, depth first, children in Morton order:
//   an accepted cell appends its id to the group's SPJ list,
//   an opened leaf appends its particles' Morton positions to the EPJ list,
//   an opened internal cell is replaced by its children.
// The warp keeps a stack of cells whose decision is already known (top =
// next in depth-first order). Each step emits the run of accepted / leaf
// entries at the top, in order, and replaces up to four of the open entries
// among the next 32 by their children -- replacing an entry in place by its
// children keeps the depth-first order, whichever entries are expanded
// first. The children of an expanded cell come from one 256-byte block of
// walk records (written by the moments kernel), eight lanes per cell, so an
// expansion costs one coalesced load. One pass: each group appends its
// accepted cell ids and its opened leaves (first particle, count) to two
// record streams in an arena of 64-record chunks (taken from a global
// cursor; each chunk's header names its group, its first record's index in
// the group's stream and that record's position in the group's list); after
// a scan of the per-group counts a compaction kernel places the chunks
// independently into the CSR lists -- leaf records expanded into particle
// indices -- in the same depth-first order. An arena that proves
// too small is grown to the size the cursors report and the pass repeated.
//
// The opening criterion is evaluated in FP32 without contraction: with d the
// distance from the cell's centre of mass to the group's bounding box (0
// inside) and s the cell side, the cell is accepted iff s^2 < theta^2 d^2,
// computed as ((dx*dx + dy*dy) + dz*dz) and theta2 * d2 in that order.
//
// The short-range neighbour walk (Section 2: the same walk with a criterion
// other than the opening angle) is a third mode of the same kernel: a cell
// whose tight box (FP32, rounded outward) meets the group's search box is
// opened, or listed when a leaf; any other cell is dropped with its
// subtree, so the SPJ stream stays empty and the EPJ stream holds the
// candidate neighbours in ascending Morton position. A cell whose tight
// box lies inside the search box is listed whole, as one record of its
// particle range, which is what its leaves would give in order.
//
// With the learned criterion (afd_mac.cuh) the same walk decides each cell
// by learned_pre() (the band tests in FP32) and, for the cells inside the
// band, by the network, which the warp evaluates for sixteen band cells at a
// time on the tensor cores (mac_mma_rows: each band lane writes its cell's
// FP16 input row to shared memory, then twelve mma.sync instructions run
// both layers with the hidden layer kept in registers). The inference entry
// point runs the same code, so the walk and afd_mlp_forward give the same
// outputs bit for bit.
#include "afd_internal.cuh"
#include "afd_mac.cuh"

#include <algorithm>
#include <cstring>

namespace afd {
namespace {

constexpr int kWalkWarps = 4;
constexpr int kWalkThreads = 32 * kWalkWarps;
constexpr int kStack = 448;  // entries per warp; >= 8 * 23 + 4 * 32 needed
constexpr int kExpand = 4;   // cells expanded per step at most
constexpr uint32_t kOpen = 0u, kAccept = 1u, kLeaf = 2u;
constexpr uint32_t kChunk = 64;  // records per arena chunk

struct WalkArgs {
  int64_t n_groups;
  unsigned long long *queue;  // next group (or item) to take, zeroed before each launch
  const float *boxf;
  const uint32_t *g_first, *g_root;
  const float4 *node_f;
  const uint2 *node_i;
  const uint4 *block;
  float theta2;
  uint32_t *cnt_e, *cnt_s, *gself, *n_lrec;
  // record arena: cell ids (SPJ stream) and leaf records (EPJ stream), and
  // per chunk its header (group, index of its first record in the group's
  // stream, output position of that record in the group's list)
  uint32_t *arena_s, *cursor;
  uint2 *arena_l;
  uint4 *hdr_s, *hdr_l;
  uint32_t cap_s, cap_l;
  int *status;
  uint32_t iter_cap;   // warp steps per group (or item) before the walk gives up
  int stack_cap;       // stack entries per warp a walk may use, 1 .. kStack
  uint32_t n_cells;  // read only by the self-checking build
  // learned criterion
  const float *mac_w, *g_amin;
  const float4 *s_hi, *s_q0, *s_q1;
  float lo2, hi2, tau, eps2;
  unsigned long long *mac_cnt;
  // neighbour walk: per-cell tight boxes (lo, hi) and per cell its
  // children's (8 x (lo, hi), by octant); boxf then holds the groups'
  // search boxes
  const float4 *tbox, *nblk;
  // neighbour walk: n_groups counts work items (group, seed cell); their
  // group and the cell the walk starts from
  const uint32_t *it_group, *it_root;
  // half-precision far field: per group the power-of-two scale of its
  // far-field terms (null: not wanted)
  float *gscale;
};

enum : int { kModeTheta = 0, kModeLearned = 1, kModeNeighbour = 2 };

__device__ __forceinline__ float sep_axis(float c, float lo, float hi) {
  float d = 0.0f;
  if (c < lo) d = __fsub_rn(lo, c);
  else if (c > hi) d = __fsub_rn(c, hi);
  return d;
}

__device__ __forceinline__ uint32_t decide(const float *bmin, const float *bmax, float cx,
                                           float cy, float cz, float s2, bool leaf,
                                           float theta2, float &d2o) {
  const float dx = sep_axis(cx, bmin[0], bmax[0]);
  const float dy = sep_axis(cy, bmin[1], bmax[1]);
  const float dz = sep_axis(cz, bmin[2], bmax[2]);
  float d2 = __fmul_rn(dx, dx);
  d2 = __fadd_rn(d2, __fmul_rn(dy, dy));
  d2 = __fadd_rn(d2, __fmul_rn(dz, dz));
  d2o = d2;
  const float rhs = __fmul_rn(theta2, d2);
  if (s2 < rhs) return kAccept;
  return leaf ? kLeaf : kOpen;
}

// Neighbour decision: kAccept ("drop") when the cell's tight box misses the
// search box (closed intervals on every axis); kLeaf when the cell is a leaf
// or its tight box lies inside the search box -- then every leaf below it is
// listed, and in depth-first order those leaves' particles are exactly the
// cell's range [first, first + count), so one record stands for the whole
// subtree and the list is the same; kOpen otherwise.
__device__ __forceinline__ uint32_t decide_nbr(const float *bmin, const float *bmax, float4 lo,
                                               float4 hi, bool leaf) {
  const bool meet = lo.x <= bmax[0] && hi.x >= bmin[0] && lo.y <= bmax[1] && hi.y >= bmin[1] &&
                    lo.z <= bmax[2] && hi.z >= bmin[2];
  if (!meet) return kAccept;
  const bool inside = lo.x >= bmin[0] && hi.x <= bmax[0] && lo.y >= bmin[1] &&
                      hi.y <= bmax[1] && lo.z >= bmin[2] && hi.z <= bmax[2];
  return (leaf || inside) ? kLeaf : kOpen;
}

// Learned decision without the network: kAccept, kOpen / kLeaf, or kBand
// when the network decides (then f receives the features).
constexpr uint32_t kBand = 3u;
__device__ __forceinline__ uint32_t learned_pre(const WalkArgs &a, const float *bmin,
                                                const float *bmax, float cx, float cy, float cz,
                                                float s2, bool leaf, uint32_t id, uint32_t first,
                                                uint32_t count, uint32_t gfirst,
                                                const MacGroup &G, float *f, float &d2o) {
  const uint32_t closed = leaf ? kLeaf : kOpen;
  if (gfirst >= first && gfirst - first < count) return closed;  // holds the group
  const float dx = sep_axis(cx, bmin[0], bmax[0]);
  const float dy = sep_axis(cy, bmin[1], bmax[1]);
  const float dz = sep_axis(cz, bmin[2], bmax[2]);
  float d2 = __fmul_rn(dx, dx);
  d2 = __fadd_rn(d2, __fmul_rn(dy, dy));
  d2 = __fadd_rn(d2, __fmul_rn(dz, dz));
  d2o = d2;
  if (s2 < __fmul_rn(a.lo2, d2)) return kAccept;
  if (!(s2 < __fmul_rn(a.hi2, d2))) return closed;
  const float4 sh = a.s_hi[id], q0 = a.s_q0[id], q1 = a.s_q1[id];
  mac_features_g(bmin, bmax, cx, cy, cz, s2, sh.w, q0, make_float2(q1.x, q1.y), count, d2, G, f);
  return kBand;
}

// Stack entry: x = cell id (open / accepted) or first particle (leaf);
// y = decision << 30 | particle count (leaf).
__device__ __forceinline__ uint2 make_entry(uint32_t dec, uint32_t id, uint32_t first,
                                            uint32_t count) {
  return dec == kLeaf ? make_uint2(first, (dec << 30) | count) : make_uint2(id, dec << 30);
}

// Warp-uniform state of one record stream of one group.
struct RecStream {
  uint32_t chunk;  // current chunk (kNone before the first)
  uint32_t fill;   // records in it
};

// Append the records of the lanes with `on`, in lane order. A chunk index at
// or above the capacity is not written (the cursor still counts it, which
// tells the host how large the arena must be). The lane whose record opens a
// new chunk writes the chunk's header hv: (group, the record's index in the
// group's stream, its output position in the group's list), so that the
// compaction places every chunk on its own, without following the group's
// chunks in order.
template <class T>
__device__ __forceinline__ void rec_put(RecStream &st, bool on, unsigned m, T rec, T *arena,
                                        uint4 *hdr, uint4 hv, uint32_t *cursor, uint32_t cap,
                                        int lane, unsigned lt) {
  const uint32_t n = __popc(m);  // m: the warp's ballot of `on`
  if (n == 0) return;
  const bool grow = st.fill + n > kChunk;
  uint32_t nc = kNone;
  if (grow) {
    if (lane == 0) {
      const uint32_t c = atomicAdd(cursor, 1u);
      nc = c < cap ? c : kNone;
    }
    nc = __shfl_sync(0xffffffffu, nc, 0);
  }
  if (on) {
    const uint32_t p = st.fill + __popc(m & lt);
    if (p < kChunk) {
      if (st.chunk != kNone) arena[(size_t)st.chunk * kChunk + p] = rec;
    } else if (nc != kNone) {
      arena[(size_t)nc * kChunk + (p - kChunk)] = rec;
      if (p == kChunk) hdr[nc] = hv;
    }
  }
  if (grow) {
    st.chunk = nc;
    st.fill = st.fill + n - kChunk;
  } else {
    st.fill += n;
  }
}

// Per-warp scratch of the network evaluation: the FP16 input rows of the
// (up to) 16 band cells of a round.
struct MacScratch {
  uint4 x16[16];
};

// The next group (neighbour walk: work item) for this warp. The grid holds
// only as many warps as are resident at once, and a warp takes its next
// group when it finishes one: with a fixed group per warp, a block's warp
// slots stay held until its slowest group is walked.
__device__ __forceinline__ int64_t take_group(const WalkArgs &a, int lane) {
  unsigned long long v = 0;
  if (lane == 0) v = atomicAdd(a.queue, 1ull);
  return (int64_t)__shfl_sync(0xffffffffu, v, 0);
}

// The learned walk is compiled for eight resident blocks per SM (64
// registers, no spills): its construction step ran 4% faster than at 72
// registers (3.035 against 3.16 ms on the 2^20 Plummer lists). The other
// modes keep the compiler's own choice (34 and 38 registers; a one-block
// minimum gives them 55 and made the plain construction step 1.6% slower).
// SCALE: the group's far-field scale for the half-precision far field is
// tracked (a separate instantiation, so that the other walks keep their
// registers).
template <int MODE, bool SCALE>
__global__ void __launch_bounds__(kWalkThreads, MODE == kModeLearned ? 8 : 0) k_walk(WalkArgs a) {
  constexpr bool LEARNED = MODE == kModeLearned, NBR = MODE == kModeNeighbour;
  __shared__ uint2 stk_all[kWalkWarps][kStack];
  __shared__ __align__(16) MacFrag mf_all[1];  // unused (and dropped) without LEARNED
  __shared__ __align__(16) MacScratch msc_all[LEARNED ? kWalkWarps : 1];
  MacFrag &mf = mf_all[0];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const unsigned lt = (1u << lane) - 1u;
  uint2 *stk = stk_all[wib];
  MacScratch &msc = msc_all[LEARNED ? wib : 0];
  uint32_t evals = 0, accepts = 0, rounds = 0;
  if (LEARNED) {
    mac_frag_load(mf, a.mac_w, threadIdx.x, kWalkThreads);
    __syncthreads();
  }
  for (int64_t g = take_group(a, lane); g < a.n_groups; g = take_group(a, lane)) {
    float bmin[3], bmax[3];
    const int64_t gb = NBR ? (int64_t)a.it_group[g] : g;  // the box's group
#pragma unroll
    for (int k = 0; k < 3; k++) {
      bmin[k] = a.boxf[gb * 6 + k];
      bmax[k] = a.boxf[gb * 6 + 3 + k];
    }
    const uint32_t gfirst = NBR ? 0u : a.g_first[g];
    MacGroup mg = {0.0f, 0.0f, 0.0f};  // the features' per-group terms (learned walk)
    if (LEARNED) mg = mac_group(bmin, bmax, a.g_amin[g], a.eps2);
    uint64_t ne = 0, ns = 0;
    uint32_t nl = 0;  // leaf records
    float mu = 0.0f;  // largest M / d^2 of this lane's accepted cells (half far field)
    RecStream rs{kNone, kChunk}, rl{kNone, kChunk};
    uint32_t self_pos = 0;  // 1 + EPJ-list position of the group's first particle
    uint32_t root_drop = 0;
    float root_d2 = 0.0f;  // (a root holds its groups: never accepted, no far-field term)
    if (lane == 0) {
      uint32_t root = NBR ? a.it_root[g] : a.g_root[g];
      if (!AFD_IN(root, a.n_cells, "walk root")) root = 0u;
      const float4 nf = a.node_f[root];
      const uint2 ni = a.node_i[root];
      const bool leaf = (ni.y >> 31) != 0;
      const uint32_t cnt = ni.y & 0x7fffffffu;
      // a system's root holds all its groups: the learned rule opens it
      const uint32_t d =
          NBR ? decide_nbr(bmin, bmax, a.tbox[(size_t)root * 2], a.tbox[(size_t)root * 2 + 1], leaf)
          : LEARNED ? (leaf ? kLeaf : kOpen)
                    : decide(bmin, bmax, nf.x, nf.y, nf.z, nf.w, leaf, a.theta2, root_d2);
      stk[0] = make_entry(d, root, ni.x, cnt);
      root_drop = (NBR && d == kAccept) ? 1u : 0u;
    }
    // the neighbour walk drops a root that does not meet the search box
    int sp = NBR ? (__shfl_sync(0xffffffffu, root_drop, 0) ? 0 : 1) : 1;
    uint32_t iters = 0;
    __syncwarp();
    while (sp > 0) {
      if (++iters > a.iter_cap) {
        if (lane == 0) atomicOr(a.status, kStWalkIter);
        break;
      }
      const int nv = sp < 32 ? sp : 32;
      const uint2 e = lane < nv ? stk[sp - 1 - lane] : make_uint2(0u, 0u);
      const uint32_t dec = e.y >> 30;
      const unsigned om = __ballot_sync(0xffffffffu, lane < nv && dec == kOpen);
      const int f = om ? __ffs(om) - 1 : nv;
      // ---- emit the decided run at the top, in order ----
      const bool acc = lane < f && dec == kAccept;
      const bool lf = lane < f && dec == kLeaf;
      const unsigned am = __ballot_sync(0xffffffffu, acc);
      if (am) {  // warp-uniform
        const uint32_t ri = (uint32_t)ns + __popc(am & lt);  // record index = list position
        rec_put(rs, acc, am, e.x, a.arena_s, a.hdr_s, make_uint4((uint32_t)g, ri, ri, 0u),
                a.cursor, a.cap_s, lane, lt);
        ns += __popc(am);
      }
      const unsigned lm = __ballot_sync(0xffffffffu, lf);
      if (lm) {  // warp-uniform: leaves among the emitted run
        const uint32_t lfirst = lf ? e.x : 0u, lcnt = lf ? (e.y & 0x3fffffffu) : 0u;
        const uint32_t tot = __reduce_add_sync(0xffffffffu, lcnt);
        // the group's own first particle: remember its EPJ-list position (the
        // group's particles follow it contiguously)
        const bool own = lf && gfirst >= lfirst && gfirst - lfirst < lcnt;
        // the lanes' list positions (an inclusive scan of the counts) are
        // needed only for the own particle's position and for the header of
        // a new chunk: most steps skip the scan
        uint32_t inc = lcnt;
        if (__any_sync(0xffffffffu, own) || rl.fill + __popc(lm) > kChunk) {
#pragma unroll
          for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += t;
          }
        }
        if (own) self_pos = (uint32_t)(ne + (inc - lcnt) + (gfirst - lfirst)) + 1u;
        rec_put(rl, lf, lm, make_uint2(lfirst, lcnt), a.arena_l, a.hdr_l,
                make_uint4((uint32_t)g, nl + __popc(lm & lt), (uint32_t)(ne + (inc - lcnt)), 0u),
                a.cursor + 1, a.cap_l, lane, lt);
        nl += __popc(lm);
        ne += tot;
      }
      if (!om) {  // nothing open among the top entries: all emitted
        sp -= nv;
        __syncwarp();
        continue;
      }
      // ---- expand the first E open entries among the top nv ----
      int E = __popc(om) < kExpand ? __popc(om) : kExpand;
      // position (lane index) of the q-th open entry
      unsigned rest = om;
      int pos_q[kExpand];
#pragma unroll
      for (int q = 0; q < kExpand; q++) {
        pos_q[q] = rest ? __ffs(rest) - 1 : -1;
        if (rest) rest &= rest - 1;
      }
      int last = pos_q[E - 1];
      // keep the stack bounded: fall back to one expansion near the limit
      if ((sp - (last + 1)) + 8 * E + (last + 1 - f - E) > a.stack_cap) {
        E = 1;
        last = pos_q[0];
      }
      const int q_me = lane >> 3, c_me = lane & 7;
      int p_me = -1;
#pragma unroll
      for (int q = 0; q < kExpand; q++)
        if (q == q_me) p_me = pos_q[q];
      uint32_t cid_me = __shfl_sync(0xffffffffu, e.x, p_me < 0 ? 0 : p_me);
      if (q_me < E && !AFD_IN(cid_me, a.n_cells, "walk expanded cell")) cid_me = 0u;
      bool valid = false, leaf_me = false;
      uint2 child_entry = make_uint2(0u, 0u);
      uint32_t d = 0, c_id = 0, c_first = 0, c_cnt = 0;
      float m_me = 0.0f, d2_me = 0.0f;  // the child's mass and squared distance to the box
      float feat[kMacNF];
#pragma unroll
      for (int k = 0; k < kMacNF; k++) feat[k] = 0.0f;
      if (q_me < E) {
        const uint4 *blk = a.block + ((size_t)cid_me * 8 + c_me) * 2;
        const uint4 nf = blk[0], meta = blk[1];
        // the neighbour walk's child box comes with the child record (one
        // round trip per step)
        float4 nlo = make_float4(0.0f, 0.0f, 0.0f, 0.0f), nhi = nlo;
        if (NBR) {
          nlo = a.nblk[((size_t)cid_me * 8 + c_me) * 2];
          nhi = a.nblk[((size_t)cid_me * 8 + c_me) * 2 + 1];
        }
        valid = meta.z != kNone && AFD_IN(meta.z, a.n_cells, "walk child");
        if (valid) {
          leaf_me = (meta.y >> 31) != 0;
          c_id = meta.z;
          c_first = meta.x;
          c_cnt = meta.y & 0x7fffffffu;
          m_me = __uint_as_float(meta.w);
          const float cx = __uint_as_float(nf.x), cy = __uint_as_float(nf.y),
                      cz = __uint_as_float(nf.z), s2 = __uint_as_float(nf.w);
          if (NBR) {
            d = decide_nbr(bmin, bmax, nlo, nhi, leaf_me);
            valid = d != kAccept;  // a dropped cell takes no stack entry
          } else {
            d = LEARNED ? learned_pre(a, bmin, bmax, cx, cy, cz, s2, leaf_me, c_id, c_first,
                                      c_cnt, gfirst, mg, feat, d2_me)
                        : decide(bmin, bmax, cx, cy, cz, s2, leaf_me, a.theta2, d2_me);
          }
        }
      }
      if (LEARNED) {
        const bool need = valid && d == kBand;
        const unsigned bm = __ballot_sync(0xffffffffu, need);
        if (bm) {  // warp-uniform: the network for every band cell of this step
          const int nb = __popc(bm), rank = __popc(bm & lt);
          float y_me = 0.0f;
          if (lane == 0) rounds++;
          // sixteen band cells per round: their FP16 input rows, then both
          // layers on the tensor cores; lane (row % 8) * 4 returns row's output
          for (int r0 = 0; r0 < nb; r0 += 16) {
            const int rr = rank - r0;
            if (need && rr >= 0 && rr < 16) msc.x16[rr] = mac_row16(mf, feat);
            __syncwarp();
            const float2 y = mac_mma_rows(mf, msc.x16, lane);
            const int src = (rr & 7) * 4;
            const float ylo = __shfl_sync(0xffffffffu, y.x, src);
            const float yhi = __shfl_sync(0xffffffffu, y.y, src);
            if (need && rr >= 0 && rr < 16) y_me = rr < 8 ? ylo : yhi;
            __syncwarp();
          }
          if (need) {
            const bool acc_me = y_me < a.tau;
            evals++;
            accepts += acc_me ? 1u : 0u;
            d = acc_me ? kAccept : (leaf_me ? kLeaf : kOpen);
          }
        }
      }
      // an accepted cell's far-field magnitude bound M / d^2 (d^2 > 0: the
      // criterion accepts only cells away from the box)
      if (SCALE && !NBR && valid && d == kAccept) mu = fmaxf(mu, __fdiv_rn(m_me, d2_me));
      if (valid) child_entry = make_entry(d, c_id, c_first, c_cnt);
      const unsigned vm = __ballot_sync(0xffffffffu, valid);
      // The rewritten positions [f, last] in output order: a position kept
      // (not expanded) counts one, an expanded one its valid children. The
      // offsets come from masks (the same for every lane): kept positions
      // below a lane, plus the children of the expanded positions below it.
      const unsigned upto = last == 31 ? 0xffffffffu : ((2u << last) - 1u);
      unsigned xm = 0u;  // expanded positions
      uint32_t pc[kExpand];
#pragma unroll
      for (int q = 0; q < kExpand; q++) {
        pc[q] = __popc((vm >> (8 * q)) & 0xffu);  // zero for q >= E
        if (q < E) xm |= 1u << pos_q[q];
      }
      const unsigned kept = upto & ~((1u << f) - 1u) & ~xm;
      uint32_t K = __popc(kept);
      uint32_t below = 0u;  // children of the expanded positions below this lane
#pragma unroll
      for (int q = 0; q < kExpand; q++) {
        K += pc[q];
        if (q < E && pos_q[q] < lane) below += pc[q];
      }
      const int spn = sp - (last + 1);
      if (spn + (int)K > a.stack_cap) {
        if (lane == 0) atomicOr(a.status, kStWalkStack);
        break;
      }
      // output offset of this lane's parent position (child lanes): the kept
      // positions below it and the children of the expanded ones before it
      uint32_t off_par = __popc(kept & ((1u << (p_me < 0 ? 0 : p_me)) - 1u));
#pragma unroll
      for (int q = 0; q < kExpand; q++)
        if (q < q_me) off_par += pc[q];
      __syncwarp();
      if ((kept >> lane) & 1u) stk[spn + K - 1 - (__popc(kept & lt) + below)] = e;
      if (valid) {
        const unsigned mine = (vm >> (8 * q_me)) & 0xffu;
        const uint32_t o = off_par + __popc(mine & ((1u << c_me) - 1u));
        stk[spn + K - 1 - o] = child_entry;
      }
      sp = spn + (int)K;
      __syncwarp();
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) self_pos = max(self_pos, __shfl_xor_sync(0xffffffffu, self_pos, o));
    if (SCALE && !NBR) {  // the group's far-field scale from its accepted cells
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) mu = fmaxf(mu, __shfl_xor_sync(0xffffffffu, mu, o));
      if (lane == 0) a.gscale[g] = far_group_scale(mu);
    }
    if (lane == 0) {
      a.cnt_e[g] = (uint32_t)ne;
      a.cnt_s[g] = (uint32_t)ns;
      a.n_lrec[g] = nl;
      if (!NBR) a.gself[g] = self_pos;
    }
    __syncwarp();
  }
  if (LEARNED) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      evals += __shfl_xor_sync(0xffffffffu, evals, o);
      accepts += __shfl_xor_sync(0xffffffffu, accepts, o);
    }
    if (lane == 0 && evals) {
      atomicAdd(&a.mac_cnt[0], (unsigned long long)evals);
      atomicAdd(&a.mac_cnt[1], (unsigned long long)accepts);
      atomicAdd(&a.mac_cnt[2], (unsigned long long)rounds);
    }
  }
}

// interactions = sum over groups of n_i * (n_epj + n_spj)
__global__ void k_interactions(int64_t n_groups, const uint32_t *__restrict__ g_count,
                               const uint32_t *__restrict__ ce, const uint32_t *__restrict__ cs,
                               unsigned long long *out) {
  unsigned long long s = 0;
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < n_groups;
       g += (int64_t)gridDim.x * blockDim.x)
    s += (unsigned long long)g_count[g] * ((unsigned long long)ce[g] + (cs ? cs[g] : 0u));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0 && s) atomicAdd(out, s);
}

// The CSR lists from the record arena, chunk by chunk: cell ids copied,
// leaf records expanded into their particles' Morton positions. A chunk's
// header gives its group, the index of its first record in the group's
// stream (so the number of its records) and that record's output position,
// so the chunks are placed independently of one another, in any order.
struct CompactArgs {
  const uint32_t *cnt_s, *n_lrec, *arena_s;
  const uint2 *arena_l;
  const uint4 *hdr_s, *hdr_l;
  const uint64_t *off_e, *off_s;
  uint32_t *epj, *spj;
  uint32_t nch_s, nch_l;  // chunks in use
  int64_t n_groups;       // read only by the self-checking build
  uint64_t n_epj, n_spj;
};

// Leaf records are expanded 32 at a time. Records of kBigRec or more
// entries (whole subtrees of the neighbour walk, level-21 leaves) are
// written one by one with strided stores; for the others, after an inclusive
// scan of their counts, lane t of each pass over their entries finds its
// record by a binary search of the scanned counts (five shuffles) and writes
// first + offset at the record's output position, so the writes stay
// coalesced whatever the mix of sizes.
constexpr uint32_t kBigRec = 64;

// Each warp takes consecutive chunks, kCompactBatch cell-id chunks (warps
// [0, ceil(nch_s / kCompactBatch))) or kCompactBatchL leaf-record chunks
// (the next warps; a leaf chunk expands to about sixteen times as many
// entries). Lane j loads chunk j's header and its group's count and list
// offset (one coalesced load and two gathers for the batch), then the warp
// copies or expands the chunks one after the other.
constexpr uint32_t kCompactBatch = 32, kCompactBatchL = 4;

__global__ void __launch_bounds__(256) k_compact(CompactArgs a) {
  const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  const int64_t nb_s = ((int64_t)a.nch_s + kCompactBatch - 1) / kCompactBatch;
  if (w < nb_s) {
    const int64_t c0 = w * kCompactBatch;
    const int64_t cl = c0 + lane;
    uint32_t nn = 0u;
    uint64_t o = 0;
    if (cl < (int64_t)a.nch_s) {
      const uint4 h = a.hdr_s[cl];
      if (AFD_IN(h.x, a.n_groups, "compact cell chunk group")) {
        const uint32_t ms = a.cnt_s[h.x];
        nn = h.y < ms ? min(kChunk, ms - h.y) : 0u;
        o = a.off_s[h.x] + h.z;
      }
    }
    const int nc = (int)min((int64_t)kCompactBatch, (int64_t)a.nch_s - c0);
#pragma unroll 2
    for (int j = 0; j < nc; j++) {
      const uint32_t nj = __shfl_sync(0xffffffffu, nn, j);
      const uint64_t oj = __shfl_sync(0xffffffffu, o, j);
      const uint32_t *src = a.arena_s + (size_t)(c0 + j) * kChunk;
      for (uint32_t k = lane; k < nj; k += 32)
        if (AFD_IN(oj + k, a.n_spj, "compact spj write")) a.spj[oj + k] = src[k];
    }
    return;
  }
  const int64_t c0 = (w - nb_s) * kCompactBatchL;
  if (c0 >= (int64_t)a.nch_l) return;
  const int64_t cl = c0 + lane;
  uint32_t nr = 0u;
  uint64_t po = 0;
  if (lane < (int)kCompactBatchL && cl < (int64_t)a.nch_l) {
    const uint4 h = a.hdr_l[cl];
    if (AFD_IN(h.x, a.n_groups, "compact leaf chunk group")) {
      const uint32_t r = a.n_lrec[h.x];
      nr = h.y < r ? min(kChunk, r - h.y) : 0u;
      po = a.off_e[h.x] + h.z;
    }
  }
  const int nc = (int)min((int64_t)kCompactBatchL, (int64_t)a.nch_l - c0);
  for (int jc = 0; jc < nc; jc++) {
    const uint32_t nrec = __shfl_sync(0xffffffffu, nr, jc);
    uint64_t pos = __shfl_sync(0xffffffffu, po, jc);
    const uint2 *recs = a.arena_l + (size_t)(c0 + jc) * kChunk;
    for (uint32_t j0 = 0; j0 < nrec; j0 += 32) {
      const bool on = lane < nrec - j0;
      const uint2 rec = on ? recs[j0 + lane] : make_uint2(0u, 0u);
      uint32_t inc = rec.y;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += t;
      }
      const uint32_t tot = __shfl_sync(0xffffffffu, inc, 31);
      const uint32_t ex = inc - rec.y;
      // records of kBigRec or more entries (whole subtrees of the neighbour
      // walk, level-21 leaves): the warp writes each with strided stores
      const bool big = rec.y >= kBigRec;
      unsigned bm = __ballot_sync(0xffffffffu, big);
      while (bm) {
        const int src = __ffs(bm) - 1;
        bm &= bm - 1;
        const uint32_t f0 = __shfl_sync(0xffffffffu, rec.x, src);
        const uint32_t n0 = __shfl_sync(0xffffffffu, rec.y, src);
        const uint64_t o0 = pos + __shfl_sync(0xffffffffu, ex, src);
        for (uint32_t k = lane; k < n0; k += 32)
          if (AFD_IN(o0 + k, a.n_epj, "compact epj write")) a.epj[o0 + k] = f0 + k;
      }
      // the others: lane t of each pass over their entries finds its record
      // by a binary search of their scanned counts
      uint32_t sn = big ? 0u : rec.y;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(0xffffffffu, sn, o);
        if (lane >= o) sn += t;
      }
      const uint32_t stot = __shfl_sync(0xffffffffu, sn, 31);
      const uint32_t sex = sn - (big ? 0u : rec.y);
      for (uint32_t t0 = 0; t0 < stot; t0 += 32) {
        const uint32_t t = t0 + lane;
        // the record holding entry t: the first whose inclusive count > t
        int q = 0;
#pragma unroll
        for (int b = 16; b > 0; b >>= 1)
          if (__shfl_sync(0xffffffffu, sn, q + b - 1) <= t) q += b;
        const uint32_t f = __shfl_sync(0xffffffffu, rec.x, q & 31);
        const uint32_t se = __shfl_sync(0xffffffffu, sex, q & 31);
        const uint32_t e = __shfl_sync(0xffffffffu, ex, q & 31);
        const uint64_t o = pos + e + (t - se);
        if (t < stot && AFD_IN(o, a.n_epj, "compact epj write")) a.epj[o] = f + (t - se);
      }
      pos += tot;
    }
  }
}

__global__ void k_sys_stats(int64_t n_groups, const uint32_t *__restrict__ g_first,
                            const uint32_t *__restrict__ g_count, const uint32_t *__restrict__ ce,
                            const uint32_t *__restrict__ cs, const uint32_t *__restrict__ sys_s,
                            unsigned long long *inter, unsigned long long *entries) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= n_groups) return;
  const uint32_t sy = sys_s ? sys_s[g_first[g]] : 0u;
  const unsigned long long e = (unsigned long long)ce[g] + cs[g];
  atomicAdd(&inter[sy], e * g_count[g]);
  atomicAdd(&entries[sy], e);
}

}  // namespace

int launch_sys_stats(afd_ctx *c, unsigned long long *inter, unsigned long long *entries) {
  const size_t b = sizeof(unsigned long long) * (size_t)c->n_sys;
  if (cudaMemsetAsync(inter, 0, b, c->stream) != cudaSuccess ||
      cudaMemsetAsync(entries, 0, b, c->stream) != cudaSuccess)
    return AFD_ERR_CUDA;
  if (c->n_groups == 0) return AFD_OK;
  k_sys_stats<<<(unsigned)((c->n_groups + 255) / 256), 256, 0, c->stream>>>(
      c->n_groups, ptr<uint32_t>(c->g_first), ptr<uint32_t>(c->g_count),
      ptr<uint32_t>(c->l_cnt_e), ptr<uint32_t>(c->l_cnt_s),
      c->n_sys > 1 ? ptr<uint32_t>(c->sys_s) : nullptr, inter, entries);
  c->launches++;
  return cudaGetLastError() == cudaSuccess ? AFD_OK : AFD_ERR_CUDA;
}

namespace {

// The walk's outputs: per-group counts, offsets and CSR lists (no SPJ side
// for the neighbour walk), and the totals read back.
struct WalkOut {
  uint32_t *cnt_e, *cnt_s;  // cnt_s: scratch for the neighbour walk (all zero)
  DevBuf *off_e, *off_s, *epj, *spj;  // off_s, spj null for the neighbour walk
  uint64_t n_e = 0, n_s = 0, inter = 0;
};

// Blocks of k_walk<MODE, SCALE> resident at once on the device (at most one
// per four groups): the grid of the dynamically scheduled walk.
template <int MODE, bool SCALE>
int64_t walk_blocks(int64_t ng) {
  static int per_sm = 0;
  if (per_sm == 0) {
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_walk<MODE, SCALE>, kWalkThreads, 0) !=
            cudaSuccess ||
        b < 1)
      b = 1;
    per_sm = b;
  }
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
    sms = 152;
  const int64_t want = (ng + kWalkWarps - 1) / kWalkWarps;
  const int64_t cap = (int64_t)per_sm * sms;
  return want < cap ? want : cap;
}

// One pass of k_walk<mode> into the record arena (grown to the size the
// cursors report and the pass repeated when it was too small), the offset
// scans, the interaction count and the compaction into CSR lists.
// Synchronises once per pass.
int run_walk(afd_ctx *c, WalkArgs &a, int mode, WalkOut &o, int64_t ng) {
  int st;
  const bool nbr = mode == kModeNeighbour;
  // arena capacity in chunks: kept from earlier walks, first guess from the
  // group count (about 1500 cell ids and 130 leaves per group of 256)
  const uint32_t cap_max = c->walk_arena_max > 0 ? c->walk_arena_max : (1u << 30);
  if (c->arena_cap_s == 0) c->arena_cap_s = (uint32_t)std::min<int64_t>(ng * 24 + 4096, 1u << 30);
  if (c->arena_cap_l == 0) c->arena_cap_l = (uint32_t)std::min<int64_t>(ng * 4 + 4096, 1u << 30);
  c->arena_cap_s = std::min(c->arena_cap_s, cap_max);
  c->arena_cap_l = std::min(c->arena_cap_l, cap_max);
  a.cnt_e = o.cnt_e;
  a.cnt_s = o.cnt_s;
  a.n_lrec = ptr<uint32_t>(c->l_nrec);
  a.cursor = ptr<uint32_t>(c->arena_cur);
  a.status = ptr<int>(c->status);
  a.iter_cap = c->walk_iter_cap > 0 ? c->walk_iter_cap : (uint32_t)(2 * c->n_cells + 64);
  a.stack_cap = c->walk_stack_cap > 0 ? c->walk_stack_cap : kStack;
  a.n_cells = (uint32_t)c->n_cells;
  a.n_groups = ng;
  const bool scale = a.gscale != nullptr;
  const int64_t nb = mode == kModeLearned ? (scale ? walk_blocks<kModeLearned, true>(ng)
                                                   : walk_blocks<kModeLearned, false>(ng))
                     : nbr ? walk_blocks<kModeNeighbour, false>(ng)
                           : (scale ? walk_blocks<kModeTheta, true>(ng)
                                    : walk_blocks<kModeTheta, false>(ng));
  a.queue = ptr<unsigned long long>(c->u64acc) + 4;
  unsigned long long *inter = ptr<unsigned long long>(c->u64acc) + 1;
  uint64_t *pin = static_cast<uint64_t *>(c->pinned);
  uint32_t need_s = 0, need_l = 0;  // chunks the walk took from each stream
  for (int attempt = 0;; attempt++) {
    if ((st = reserve(c->arena_s, sizeof(uint32_t) * kChunk * (size_t)c->arena_cap_s))) return st;
    if ((st = reserve(c->arena_l, sizeof(uint2) * kChunk * (size_t)c->arena_cap_l))) return st;
    if ((st = reserve(c->hdr_s, sizeof(uint4) * (size_t)c->arena_cap_s))) return st;
    if ((st = reserve(c->hdr_l, sizeof(uint4) * (size_t)c->arena_cap_l))) return st;
    a.arena_s = ptr<uint32_t>(c->arena_s);
    a.arena_l = ptr<uint2>(c->arena_l);
    a.hdr_s = ptr<uint4>(c->hdr_s);
    a.hdr_l = ptr<uint4>(c->hdr_l);
    a.cap_s = c->arena_cap_s;
    a.cap_l = c->arena_cap_l;
    if (cudaMemsetAsync(c->arena_cur.p, 0, 2 * sizeof(uint32_t), c->stream) != cudaSuccess ||
        cudaMemsetAsync(a.queue, 0, sizeof(unsigned long long), c->stream) != cudaSuccess)
      return AFD_ERR_CUDA;
    if (mode == kModeLearned && cudaMemsetAsync(c->mac_cnt.p, 0, 3 * sizeof(unsigned long long),
                                                c->stream) != cudaSuccess)
      return AFD_ERR_CUDA;
    if (mode == kModeLearned && scale)
      k_walk<kModeLearned, true><<<(unsigned)nb, kWalkThreads, 0, c->stream>>>(a);
    else if (mode == kModeLearned)
      k_walk<kModeLearned, false><<<(unsigned)nb, kWalkThreads, 0, c->stream>>>(a);
    else if (nbr)
      k_walk<kModeNeighbour, false><<<(unsigned)nb, kWalkThreads, 0, c->stream>>>(a);
    else if (scale)
      k_walk<kModeTheta, true><<<(unsigned)nb, kWalkThreads, 0, c->stream>>>(a);
    else
      k_walk<kModeTheta, false><<<(unsigned)nb, kWalkThreads, 0, c->stream>>>(a);
    c->launches++;
    if (cudaGetLastError() != cudaSuccess) return AFD_ERR_CUDA;
    if ((st = scan_u32_to_u64(c, a.cnt_e, ptr<uint64_t>(*o.off_e), ng))) return st;
    if (!nbr && (st = scan_u32_to_u64(c, a.cnt_s, ptr<uint64_t>(*o.off_s), ng))) return st;
    cudaMemsetAsync(inter, 0, sizeof(unsigned long long), c->stream);
    if (!nbr) {  // (the neighbour walk counts its pairs per group afterwards)
      k_interactions<<<152, 256, 0, c->stream>>>(ng, ptr<uint32_t>(c->g_count), a.cnt_e,
                                                  a.cnt_s, inter);
      c->launches++;
    }
    cudaMemcpyAsync(pin, ptr<uint64_t>(*o.off_e) + ng, sizeof(uint64_t), cudaMemcpyDeviceToHost,
                    c->stream);
    if (!nbr)
      cudaMemcpyAsync(pin + 1, ptr<uint64_t>(*o.off_s) + ng, sizeof(uint64_t),
                      cudaMemcpyDeviceToHost, c->stream);
    cudaMemcpyAsync(pin + 2, inter, sizeof(uint64_t), cudaMemcpyDeviceToHost, c->stream);
    cudaMemcpyAsync(pin + 3, c->status.p, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
    cudaMemcpyAsync(pin + 4, c->arena_cur.p, 2 * sizeof(uint32_t), cudaMemcpyDeviceToHost,
                    c->stream);
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) return AFD_ERR_CUDA;
    const int bits = (int)(pin[3] & 0xffffffffu);
    if (bits) {
      cudaMemsetAsync(c->status.p, 0, sizeof(int), c->stream);
      return status_to_error(bits);
    }
    need_s = (uint32_t)(pin[4] & 0xffffffffu);
    need_l = (uint32_t)(pin[4] >> 32);
    if (need_s <= c->arena_cap_s && need_l <= c->arena_cap_l) break;
    // the second pass is sized from the cursors: still too small only at the
    // capacity limit
    if (attempt > 0) return AFD_ERR_LIST_OVERFLOW;
    if (need_s > c->arena_cap_s)
      c->arena_cap_s = (uint32_t)std::min<uint64_t>((uint64_t)need_s * 5 / 4 + 1024, cap_max);
    if (need_l > c->arena_cap_l)
      c->arena_cap_l = (uint32_t)std::min<uint64_t>((uint64_t)need_l * 5 / 4 + 1024, cap_max);
  }
  o.n_e = pin[0];
  o.n_s = nbr ? 0 : pin[1];
  o.inter = pin[2];
  if ((st = reserve(*o.epj, sizeof(uint32_t) * o.n_e))) return st;
  if (!nbr && (st = reserve(*o.spj, sizeof(uint32_t) * o.n_s))) return st;
  CompactArgs k;
  k.n_groups = ng;
  k.cnt_s = a.cnt_s;
  k.n_lrec = a.n_lrec;
  k.arena_s = a.arena_s;
  k.arena_l = a.arena_l;
  k.hdr_s = a.hdr_s;
  k.hdr_l = a.hdr_l;
  k.off_e = ptr<uint64_t>(*o.off_e);
  k.off_s = ptr<uint64_t>(nbr ? *o.off_e : *o.off_s);  // read, never used, without SPJs
  k.epj = ptr<uint32_t>(*o.epj);
  k.spj = nbr ? nullptr : ptr<uint32_t>(*o.spj);
  k.nch_s = nbr ? 0u : need_s;  // the neighbour walk emits no cell ids
  k.nch_l = need_l;
  k.n_epj = o.n_e;
  k.n_spj = o.n_s;
  const uint64_t warps = ((uint64_t)k.nch_s + kCompactBatch - 1) / kCompactBatch +
                         ((uint64_t)k.nch_l + kCompactBatchL - 1) / kCompactBatchL;
  if (warps > 0) {
    k_compact<<<(unsigned)((warps * 32 + 255) / 256), 256, 0, c->stream>>>(k);
    c->launches++;
  }
  return cudaGetLastError() == cudaSuccess ? AFD_OK : AFD_ERR_CUDA;
}

int walk_scratch(afd_ctx *c, int64_t ng) {
  int st;
  if ((st = reserve(c->l_nrec, sizeof(uint32_t) * ng))) return st;
  return reserve(c->arena_cur, 2 * sizeof(uint32_t));
}

WalkArgs base_args(afd_ctx *c) {
  WalkArgs a;
  memset(&a, 0, sizeof(a));
  a.n_groups = c->n_groups;
  a.g_first = ptr<uint32_t>(c->g_first);
  a.g_root = ptr<uint32_t>(c->g_root);
  a.node_f = ptr<float4>(c->node_f);
  a.node_i = ptr<uint2>(c->node_i);
  a.block = ptr<uint4>(c->c_block);
  return a;
}

}  // namespace

int launch_walk(afd_ctx *c) {
  const int64_t ng = c->n_groups;
  int st;
  for (afd::DevBuf *b : {&c->l_cnt_e, &c->l_cnt_s})
    if ((st = reserve(*b, sizeof(uint32_t) * ng))) return st;
  for (afd::DevBuf *b : {&c->epj_off, &c->spj_off})
    if ((st = reserve(*b, sizeof(uint64_t) * (ng + 1)))) return st;
  if ((st = walk_scratch(c, ng))) return st;
  // after reusing steps the walk records, group boxes (and quadrupoles) lag
  // the particles: refresh them before walking
  if (c->n_cells > 0 &&
      (!c->moments_current || !c->blocks_current || (c->cfg.mac && !c->q_current))) {
    if ((st = launch_moments(c, true, c->cfg.mac != 0))) return st;
    if ((st = launch_group_boxes(c))) return st;
  }
  if (ng == 0) {
    c->n_epj = c->n_spj = c->interactions = 0;
    cudaMemsetAsync(c->epj_off.p, 0, sizeof(uint64_t), c->stream);
    cudaMemsetAsync(c->spj_off.p, 0, sizeof(uint64_t), c->stream);
    return cudaGetLastError() == cudaSuccess ? AFD_OK : AFD_ERR_CUDA;
  }
  WalkArgs a = base_args(c);
  a.boxf = ptr<float>(c->g_boxf);
  const float th = (float)c->cfg.theta;
  a.theta2 = th * th;
  a.gself = ptr<uint32_t>(c->g_self);
  const bool learned = mac_usable(c);
  if (learned) {
    if ((st = launch_group_amin(c))) return st;
    if ((st = reserve(c->mac_cnt, 3 * sizeof(unsigned long long)))) return st;
    a.mac_w = ptr<float>(c->mac_w);
    a.g_amin = ptr<float>(c->g_amin);
    a.s_hi = ptr<float4>(c->s_hi);
    a.s_q0 = ptr<float4>(c->s_q0);
    a.s_q1 = ptr<float4>(c->s_q1);
    a.lo2 = c->mac_lo2;
    a.hi2 = c->mac_hi2;
    a.tau = c->mac_tau;
    const float e = (float)c->cfg.eps;
    a.eps2 = e * e;
    a.mac_cnt = ptr<unsigned long long>(c->mac_cnt);
  }
  c->walk_learned = learned;
  WalkOut o;
  o.cnt_e = ptr<uint32_t>(c->l_cnt_e);
  o.cnt_s = ptr<uint32_t>(c->l_cnt_s);
  o.off_e = &c->epj_off;
  o.off_s = &c->spj_off;
  o.epj = &c->epj;
  o.spj = &c->spj;
  // the half-precision far field's per-group scales come with the lists
  c->fscale_ok = false;
  const bool half_far = c->cfg.multipole && c->cfg.far_precision != 0;
  if (half_far) {
    if ((st = reserve(c->g_fscale, sizeof(float) * (size_t)ng))) return st;
    a.gscale = ptr<float>(c->g_fscale);
  }
  if ((st = run_walk(c, a, learned ? kModeLearned : kModeTheta, o, ng))) return st;
  c->fscale_ok = half_far;
  c->n_epj = o.n_e;
  c->n_spj = o.n_s;
  c->interactions = o.inter;
  return AFD_OK;
}

namespace {

// Seeds of the neighbour walk: the maximal cells holding at most K particles
// (and any larger leaf), which in depth-first order partition each system's
// particles. A group's walk is split into one item per seed whose tight box
// meets the group's search box; an item walks the seed's subtree, and the
// items' lists, concatenated in seed order, are the group's list -- the
// leaves a walk from the root would list, in the same order (a seed that
// meets the box has ancestors that meet it too). A group whose box reaches
// across the system so becomes many short walks instead of one long one.
__global__ void k_seed_mark(int64_t n_cells, const uint32_t *__restrict__ count,
                            const uint32_t *__restrict__ parent,
                            const uint32_t *__restrict__ child, uint32_t K,
                            uint32_t *__restrict__ flag) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n_cells) return;
  const uint32_t cn = count[c], p = parent[c];
  bool leaf = true;
#pragma unroll
  for (int o = 0; o < 8; o++) leaf = leaf && child[(size_t)c * 8 + o] == kNone;
  flag[c] = ((cn <= K && (p == kNone || count[p] > K)) || (cn > K && leaf)) ? 1u : 0u;
}

__global__ void k_seed_fill(int64_t n_cells, const uint32_t *__restrict__ flag,
                            const uint32_t *__restrict__ off, uint32_t *__restrict__ seeds) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c < n_cells && flag[c]) seeds[off[c]] = (uint32_t)c;
}

// Union boxes of blocks of 32 consecutive seeds (one warp per block), the
// first filter of k_items.
__global__ void k_seed_blocks(uint32_t n_seeds, const uint32_t *__restrict__ seeds,
                              const float4 *__restrict__ tbox, float4 *__restrict__ bbox) {
  const int64_t b = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (b * 32 >= n_seeds) return;
  const uint64_t k = (uint64_t)b * 32 + lane;
  float4 lo = make_float4(INFINITY, INFINITY, INFINITY, 0.0f);
  float4 hi = make_float4(-INFINITY, -INFINITY, -INFINITY, 0.0f);
  if (k < n_seeds) {
    lo = tbox[(size_t)seeds[k] * 2];
    hi = tbox[(size_t)seeds[k] * 2 + 1];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    lo.x = fminf(lo.x, __shfl_xor_sync(0xffffffffu, lo.x, o));
    lo.y = fminf(lo.y, __shfl_xor_sync(0xffffffffu, lo.y, o));
    lo.z = fminf(lo.z, __shfl_xor_sync(0xffffffffu, lo.z, o));
    hi.x = fmaxf(hi.x, __shfl_xor_sync(0xffffffffu, hi.x, o));
    hi.y = fmaxf(hi.y, __shfl_xor_sync(0xffffffffu, hi.y, o));
    hi.z = fmaxf(hi.z, __shfl_xor_sync(0xffffffffu, hi.z, o));
  }
  if (lane == 0) {
    bbox[b * 2] = make_float4(lo.x, lo.y, lo.z, 0.0f);
    bbox[b * 2 + 1] = make_float4(hi.x, hi.y, hi.z, 0.0f);
  }
}

__device__ __forceinline__ bool box_meets(float4 lo, float4 hi, const float *bmin,
                                          const float *bmax) {
  return lo.x <= bmax[0] && hi.x >= bmin[0] && lo.y <= bmax[1] && hi.y >= bmin[1] &&
         lo.z <= bmax[2] && hi.z >= bmin[2];
}

struct ItemArgs {
  int64_t n_groups;
  const uint32_t *g_root, *skip, *seeds;
  uint32_t n_seeds;
  const float *sbox;
  const float4 *tbox, *bbox;
  uint32_t *cnt;                  // count pass: items per group
  const uint32_t *off;            // fill pass: first item per group
  uint32_t *it_group, *it_root;   // fill pass
};

__device__ __forceinline__ uint32_t lower_seed(const uint32_t *seeds, uint32_t n, uint32_t v) {
  uint32_t lo = 0, hi = n;
  while (lo < hi) {
    const uint32_t mid = (lo + hi) >> 1;
    if (seeds[mid] < v) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// One warp per group: the seeds of its system (cell ids in the root's
// subtree range), their blocks' boxes tested 32 at a time and then the
// seeds of each block that meets the search box; FILL writes the items in
// seed order.
template <bool FILL>
__global__ void __launch_bounds__(256) k_items(ItemArgs a) {
  const int64_t g = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (g >= a.n_groups) return;
  const uint32_t root = a.g_root[g];
  const uint32_t s0 = lower_seed(a.seeds, a.n_seeds, root);
  const uint32_t s1 = lower_seed(a.seeds, a.n_seeds, a.skip[root]);
  float bmin[3], bmax[3];
#pragma unroll
  for (int k = 0; k < 3; k++) {
    bmin[k] = a.sbox[g * 6 + k];
    bmax[k] = a.sbox[g * 6 + 3 + k];
  }
  uint32_t n = 0, o = FILL ? a.off[g] : 0u;
  const uint32_t b0 = s0 / 32, b1 = (s1 + 31) / 32;
  for (uint32_t bb = b0; bb < b1; bb += 32) {
    const uint32_t bl = bb + lane;
    const bool bmeet =
        bl < b1 && box_meets(a.bbox[(size_t)bl * 2], a.bbox[(size_t)bl * 2 + 1], bmin, bmax);
    unsigned bm = __ballot_sync(0xffffffffu, bmeet);
    while (bm) {
      const uint32_t blk = bb + (uint32_t)(__ffs(bm) - 1);
      bm &= bm - 1;
      const uint32_t k = blk * 32 + lane;
      bool meet = false;
      uint32_t sc = 0;
      if (k >= s0 && k < s1) {
        sc = a.seeds[k];
        meet = box_meets(a.tbox[(size_t)sc * 2], a.tbox[(size_t)sc * 2 + 1], bmin, bmax);
      }
      const unsigned m = __ballot_sync(0xffffffffu, meet);
      if (FILL && meet) {
        const uint32_t at = o + n + __popc(m & ((1u << lane) - 1u));
        a.it_group[at] = (uint32_t)g;
        a.it_root[at] = sc;
      }
      n += __popc(m);
    }
  }
  if (!FILL && lane == 0) a.cnt[g] = n;
}

// Group offsets from the item offsets, and the candidate pairs
// sum_g n_g * list length.
__global__ void k_group_lists(int64_t n_groups, const uint32_t *__restrict__ item_off,
                              const uint64_t *__restrict__ ioff,
                              const uint32_t *__restrict__ g_count, uint64_t *__restrict__ off,
                              unsigned long long *pairs) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  unsigned long long s = 0;
  if (g < n_groups) {
    const uint64_t b = ioff[item_off[g]], e = ioff[item_off[g + 1]];
    off[g] = b;
    if (g == n_groups - 1) off[n_groups] = e;
    s = (unsigned long long)g_count[g] * (e - b);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0 && s) atomicAdd(pairs, s);
}

inline unsigned nblocks256(int64_t n) { return (unsigned)((n + 255) / 256); }

}  // namespace

int launch_nbr_walk(afd_ctx *c) {
  const int64_t ng = c->n_groups, nc = c->n_cells;
  int st;
  if ((st = reserve(c->nbr_off, sizeof(uint64_t) * (ng + 1)))) return st;
  if (ng == 0) {
    c->n_nbr = c->nbr_pairs = 0;
    cudaMemsetAsync(c->nbr_off.p, 0, sizeof(uint64_t), c->stream);
    return cudaGetLastError() == cudaSuccess ? AFD_OK : AFD_ERR_CUDA;
  }
  uint32_t *pin = static_cast<uint32_t *>(c->pinned);
  // seeds
  const uint32_t K = (uint32_t)std::max<int64_t>(4 * (int64_t)c->cfg.n_grp, c->n / 256);
  if ((st = reserve(c->nbr_seedf, sizeof(uint32_t) * (size_t)nc))) return st;
  if ((st = reserve(c->nbr_seedo, sizeof(uint32_t) * (size_t)(nc + 1)))) return st;
  k_seed_mark<<<nblocks256(nc), 256, 0, c->stream>>>(nc, ptr<uint32_t>(c->c_count),
                                                     ptr<uint32_t>(c->c_parent),
                                                     ptr<uint32_t>(c->c_child), K,
                                                     ptr<uint32_t>(c->nbr_seedf));
  c->launches++;
  if ((st = scan_u32(c, ptr<uint32_t>(c->nbr_seedf), ptr<uint32_t>(c->nbr_seedo), nc))) return st;
  if (cudaMemcpyAsync(pin, ptr<uint32_t>(c->nbr_seedo) + nc, sizeof(uint32_t),
                      cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
      cudaStreamSynchronize(c->stream) != cudaSuccess)
    return AFD_ERR_CUDA;
  const uint32_t n_seeds = pin[0];
  if ((st = reserve(c->nbr_seeds, sizeof(uint32_t) * (size_t)n_seeds))) return st;
  k_seed_fill<<<nblocks256(nc), 256, 0, c->stream>>>(nc, ptr<uint32_t>(c->nbr_seedf),
                                                     ptr<uint32_t>(c->nbr_seedo),
                                                     ptr<uint32_t>(c->nbr_seeds));
  c->launches++;
  const int64_t nsb = ((int64_t)n_seeds + 31) / 32;
  if ((st = reserve(c->nbr_sbb, sizeof(float4) * 2 * (size_t)std::max<int64_t>(nsb, 1))))
    return st;
  if (nsb > 0) {
    k_seed_blocks<<<nblocks256(nsb * 32), 256, 0, c->stream>>>(
        n_seeds, ptr<uint32_t>(c->nbr_seeds), ptr<float4>(c->c_tbox), ptr<float4>(c->nbr_sbb));
    c->launches++;
  }
  // items: per group the seeds its search box meets, in seed order
  if ((st = reserve(c->nbr_icnt, sizeof(uint32_t) * (size_t)ng))) return st;
  if ((st = reserve(c->nbr_igoff, sizeof(uint32_t) * (size_t)(ng + 1)))) return st;
  ItemArgs ia;
  ia.n_groups = ng;
  ia.g_root = ptr<uint32_t>(c->g_root);
  ia.skip = ptr<uint32_t>(c->c_skip);
  ia.seeds = ptr<uint32_t>(c->nbr_seeds);
  ia.n_seeds = n_seeds;
  ia.sbox = ptr<float>(c->g_sbox);
  ia.tbox = ptr<float4>(c->c_tbox);
  ia.bbox = ptr<float4>(c->nbr_sbb);
  ia.cnt = ptr<uint32_t>(c->nbr_icnt);
  ia.off = ptr<uint32_t>(c->nbr_igoff);
  ia.it_group = ia.it_root = nullptr;
  k_items<false><<<nblocks256(ng * 32), 256, 0, c->stream>>>(ia);
  c->launches++;
  if ((st = scan_u32(c, ia.cnt, ptr<uint32_t>(c->nbr_igoff), ng))) return st;
  if (cudaMemcpyAsync(pin, ptr<uint32_t>(c->nbr_igoff) + ng, sizeof(uint32_t),
                      cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
      cudaStreamSynchronize(c->stream) != cudaSuccess)
    return AFD_ERR_CUDA;
  const int64_t ni = pin[0];
  if ((st = reserve(c->nbr_itg, sizeof(uint32_t) * (size_t)std::max<int64_t>(ni, 1)))) return st;
  if ((st = reserve(c->nbr_itr, sizeof(uint32_t) * (size_t)std::max<int64_t>(ni, 1)))) return st;
  ia.it_group = ptr<uint32_t>(c->nbr_itg);
  ia.it_root = ptr<uint32_t>(c->nbr_itr);
  k_items<true><<<nblocks256(ng * 32), 256, 0, c->stream>>>(ia);
  c->launches++;
  if (cudaGetLastError() != cudaSuccess) return AFD_ERR_CUDA;
  // the walk over the items, into per-item CSR lists = per-group lists
  if ((st = reserve(c->nbr_cnt, sizeof(uint32_t) * 2 * (size_t)std::max<int64_t>(ni, 1))))
    return st;
  if ((st = reserve(c->nbr_ioff, sizeof(uint64_t) * (size_t)(ni + 1)))) return st;
  if ((st = walk_scratch(c, ni))) return st;
  unsigned long long *pairs = ptr<unsigned long long>(c->u64acc) + 3;
  if (cudaMemsetAsync(pairs, 0, sizeof(unsigned long long), c->stream) != cudaSuccess)
    return AFD_ERR_CUDA;
  uint64_t n_e = 0;
  if (ni > 0) {
    WalkArgs a = base_args(c);
    a.boxf = ptr<float>(c->g_sbox);
    a.tbox = ptr<float4>(c->c_tbox);
    a.nblk = ptr<float4>(c->nbr_blk);
    a.it_group = ia.it_group;
    a.it_root = ia.it_root;
    WalkOut o;
    o.cnt_e = ptr<uint32_t>(c->nbr_cnt);
    o.cnt_s = ptr<uint32_t>(c->nbr_cnt) + ni;
    o.off_e = &c->nbr_ioff;
    o.off_s = nullptr;
    o.epj = &c->nbr;
    o.spj = nullptr;
    if ((st = run_walk(c, a, kModeNeighbour, o, ni))) return st;
    n_e = o.n_e;
  } else if (cudaMemsetAsync(c->nbr_ioff.p, 0, sizeof(uint64_t), c->stream) != cudaSuccess) {
    return AFD_ERR_CUDA;
  }
  k_group_lists<<<nblocks256(ng), 256, 0, c->stream>>>(
      ng, ptr<uint32_t>(c->nbr_igoff), ptr<uint64_t>(c->nbr_ioff), ptr<uint32_t>(c->g_count),
      ptr<uint64_t>(c->nbr_off), pairs);
  c->launches++;
  uint64_t *pin64 = static_cast<uint64_t *>(c->pinned);
  if (cudaMemcpyAsync(pin64, pairs, sizeof(uint64_t), cudaMemcpyDeviceToHost, c->stream) !=
          cudaSuccess ||
      cudaStreamSynchronize(c->stream) != cudaSuccess)
    return AFD_ERR_CUDA;
  c->n_nbr = n_e;
  c->nbr_pairs = pin64[0];
  return AFD_OK;
}

}  // namespace afd

extern "C" int afd_set_walk_limits(afd_ctx *c, int64_t iter_cap, int32_t stack_cap,
                                   int64_t arena_chunks_max) {
  if (!c || iter_cap < 0 || iter_cap > 0xffffffffll || stack_cap < 0 ||
      stack_cap > afd::kStack || arena_chunks_max < 0 || arena_chunks_max > (1ll << 30))
    return AFD_ERR_ARG;
  c->walk_iter_cap = (uint32_t)iter_cap;
  c->walk_stack_cap = stack_cap;
  c->walk_arena_max = (uint32_t)arena_chunks_max;
  return AFD_OK;
}
