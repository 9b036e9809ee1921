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
// cursor, linked per group); after a scan of the per-group counts a
// compaction kernel writes the CSR lists -- leaf records expanded into
// particle indices -- in the same depth-first order. An arena that proves
// too small is grown to the size the cursors report and the pass repeated.
//
// The opening criterion is evaluated in FP32 without contraction: with d the
// distance from the cell's centre of mass to the group's bounding box (0
// inside) and s the cell side, the cell is accepted iff s^2 < theta^2 d^2,
// computed as ((dx*dx + dy*dy) + dz*dz) and theta2 * d2 in that order.
//
// With the learned criterion (afd_mac.cuh) the same walk decides each cell
// by learned_pre() (the band tests in FP32) and, for the cells inside the
// band, by the network, which the whole warp evaluates for four band cells
// at a time: lane j computes hidden unit j of both layers (its weights read
// from shared memory, the cells' inputs and hidden values broadcast from
// shared memory, one packed FMA covering two cells), and the 32 output
// products are summed by an xor butterfly, which adds them in exactly the
// defined pairwise-halving order. The arithmetic per unit is mac_mlp_t's, so
// the decisions are the same bit for bit; the warp needs few registers and
// no lane sits idle in the layers.
#include "afd_internal.cuh"
#include "afd_mac.cuh"

#include <algorithm>

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
  const float *boxf;
  const uint32_t *g_first, *g_root;
  const float4 *node_f;
  const uint2 *node_i;
  const uint4 *block;
  float theta2;
  uint32_t *cnt_e, *cnt_s, *gself, *n_lrec;
  // record arena: cell ids (SPJ stream) and leaf records (EPJ stream)
  uint32_t *arena_s, *next_s, *next_l, *head_s, *head_l, *cursor;
  uint2 *arena_l;
  uint32_t cap_s, cap_l;
  int *status;
  uint32_t iter_cap;
  uint32_t n_cells;  // read only by the self-checking build
  // learned criterion
  const float *mac_w, *g_amin;
  const float4 *s_hi, *s_q0, *s_q1;
  float lo2, hi2, tau, eps2;
  unsigned long long *mac_cnt;
};

__device__ __forceinline__ float sep_axis(float c, float lo, float hi) {
  float d = 0.0f;
  if (c < lo) d = __fsub_rn(lo, c);
  else if (c > hi) d = __fsub_rn(c, hi);
  return d;
}

__device__ __forceinline__ uint32_t decide(const float *bmin, const float *bmax, float cx,
                                           float cy, float cz, float s2, bool leaf,
                                           float theta2) {
  const float dx = sep_axis(cx, bmin[0], bmax[0]);
  const float dy = sep_axis(cy, bmin[1], bmax[1]);
  const float dz = sep_axis(cz, bmin[2], bmax[2]);
  float d2 = __fmul_rn(dx, dx);
  d2 = __fadd_rn(d2, __fmul_rn(dy, dy));
  d2 = __fadd_rn(d2, __fmul_rn(dz, dz));
  const float rhs = __fmul_rn(theta2, d2);
  if (s2 < rhs) return kAccept;
  return leaf ? kLeaf : kOpen;
}

// Learned decision without the network: kAccept, kOpen / kLeaf, or kBand
// when the network decides (then f receives the features).
constexpr uint32_t kBand = 3u;
__device__ __forceinline__ uint32_t learned_pre(const WalkArgs &a, const float *bmin,
                                                const float *bmax, float cx, float cy, float cz,
                                                float s2, bool leaf, uint32_t id, uint32_t first,
                                                uint32_t count, uint32_t gfirst, float amin,
                                                float *f) {
  const uint32_t closed = leaf ? kLeaf : kOpen;
  if (gfirst >= first && gfirst - first < count) return closed;  // holds the group
  const float dx = sep_axis(cx, bmin[0], bmax[0]);
  const float dy = sep_axis(cy, bmin[1], bmax[1]);
  const float dz = sep_axis(cz, bmin[2], bmax[2]);
  float d2 = __fmul_rn(dx, dx);
  d2 = __fadd_rn(d2, __fmul_rn(dy, dy));
  d2 = __fadd_rn(d2, __fmul_rn(dz, dz));
  if (s2 < __fmul_rn(a.lo2, d2)) return kAccept;
  if (!(s2 < __fmul_rn(a.hi2, d2))) return closed;
  const float4 sh = a.s_hi[id], q0 = a.s_q0[id], q1 = a.s_q1[id];
  mac_features(bmin, bmax, cx, cy, cz, s2, sh.w, q0, make_float2(q1.x, q1.y), count, a.eps2,
               amin, f);
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
// tells the host how large the arena must be).
template <class T>
__device__ __forceinline__ void rec_put(RecStream &st, bool on, T rec, T *arena, uint32_t *next,
                                        uint32_t *cursor, uint32_t cap, uint32_t *head,
                                        int lane, unsigned lt) {
  const unsigned m = __ballot_sync(0xffffffffu, on);
  const uint32_t n = __popc(m);
  if (n == 0) return;
  const bool grow = st.fill + n > kChunk;
  uint32_t nc = kNone;
  if (grow) {
    if (lane == 0) {
      const uint32_t c = atomicAdd(cursor, 1u);
      nc = c < cap ? c : kNone;
      if (st.chunk == kNone) *head = nc;
      else next[st.chunk] = nc;
    }
    nc = __shfl_sync(0xffffffffu, nc, 0);
  }
  if (on) {
    const uint32_t p = st.fill + __popc(m & lt);
    if (p < kChunk) {
      if (st.chunk != kNone) arena[(size_t)st.chunk * kChunk + p] = rec;
    } else if (nc != kNone) {
      arena[(size_t)nc * kChunk + (p - kChunk)] = rec;
    }
  }
  if (grow) {
    st.chunk = nc;
    st.fill = st.fill + n - kChunk;
  } else {
    st.fill += n;
  }
}

// The network's weights as the walk reads them: per hidden unit (lane) a
// padded row, so that four consecutive weights are one 16-byte load without
// bank conflicts; the vectors in their own small array.
constexpr int kW1Row = 12, kW2Row = 36;
struct MacWeights {
  float w1[kMacNH][kW1Row];  // W1[j][k], k < 8
  float w2[kMacNH][kW2Row];  // W2[j][k], k < 32
  float vec[2 * kMacNF + 3 * kMacNH + 4];  // mu, isd, b1, b2, w3, b3
};
constexpr int kVecB1 = 2 * kMacNF, kVecB2 = kVecB1 + kMacNH, kVecW3 = kVecB2 + kMacNH,
              kVecB3 = kVecW3 + kMacNH;

// Per-warp scratch of the warp-wide network evaluation.
struct MacScratch {
  float4 xin[8][kMacNF];  // inputs: [band cell / 4][k] -> 4 cells
  float4 hin[kMacNH];     // hidden layer 1 of the current 4 cells: [unit]
};

template <bool LEARNED>
__global__ void __launch_bounds__(kWalkThreads) k_walk(WalkArgs a) {
  __shared__ uint2 stk_all[kWalkWarps][kStack];
  __shared__ __align__(16) MacWeights mw_all[1];  // unused (and dropped) without LEARNED
  __shared__ __align__(16) MacScratch msc_all[LEARNED ? kWalkWarps : 1];
  MacWeights &mw = mw_all[0];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const unsigned lt = (1u << lane) - 1u;
  uint2 *stk = stk_all[wib];
  MacScratch &msc = msc_all[LEARNED ? wib : 0];
  uint32_t evals = 0, accepts = 0, rounds = 0;
  if (LEARNED) {
    for (int i = threadIdx.x; i < kMacNH * kMacNF; i += kWalkThreads)
      mw.w1[i / kMacNF][i % kMacNF] = a.mac_w[kMacOffW1 + i];
    for (int i = threadIdx.x; i < kMacNH * kMacNH; i += kWalkThreads)
      mw.w2[i / kMacNH][i % kMacNH] = a.mac_w[kMacOffW2 + i];
    for (int i = threadIdx.x; i < 2 * kMacNF; i += kWalkThreads) mw.vec[i] = a.mac_w[i];
    for (int i = threadIdx.x; i < kMacNH; i += kWalkThreads) {
      mw.vec[kVecB1 + i] = a.mac_w[kMacOffB1 + i];
      mw.vec[kVecB2 + i] = a.mac_w[kMacOffB2 + i];
      mw.vec[kVecW3 + i] = a.mac_w[kMacOffW3 + i];
    }
    if (threadIdx.x == 0) mw.vec[kVecB3] = a.mac_w[kMacOffB3];
    __syncthreads();
  }
  for (int64_t g = (int64_t)blockIdx.x * kWalkWarps + wib; g < a.n_groups;
       g += (int64_t)gridDim.x * kWalkWarps) {
    float bmin[3], bmax[3];
#pragma unroll
    for (int k = 0; k < 3; k++) {
      bmin[k] = a.boxf[g * 6 + k];
      bmax[k] = a.boxf[g * 6 + 3 + k];
    }
    const uint32_t gfirst = a.g_first[g];
    const float amin = LEARNED ? a.g_amin[g] : 0.0f;
    uint64_t ne = 0, ns = 0;
    uint32_t nl = 0;  // leaf records
    RecStream rs{kNone, kChunk}, rl{kNone, kChunk};
    uint32_t self_pos = 0;  // 1 + EPJ-list position of the group's first particle
    if (lane == 0) {
      uint32_t root = a.g_root[g];
      if (!AFD_IN(root, a.n_cells, "walk root")) root = 0u;
      const float4 nf = a.node_f[root];
      const uint2 ni = a.node_i[root];
      const bool leaf = (ni.y >> 31) != 0;
      const uint32_t cnt = ni.y & 0x7fffffffu;
      // a system's root holds all its groups: the learned rule opens it
      const uint32_t d = LEARNED ? (leaf ? kLeaf : kOpen)
                                 : decide(bmin, bmax, nf.x, nf.y, nf.z, nf.w, leaf, a.theta2);
      stk[0] = make_entry(d, root, ni.x, cnt);
    }
    int sp = 1;
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
      rec_put(rs, acc, e.x, a.arena_s, a.next_s, a.cursor, a.cap_s, a.head_s + g, lane, lt);
      ns += __popc(am);
      const uint32_t lfirst = lf ? e.x : 0u, lcnt = lf ? (e.y & 0x3fffffffu) : 0u;
      uint32_t inc = lcnt;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += t;
      }
      const uint32_t tot = __shfl_sync(0xffffffffu, inc, 31);
      // the group's own first particle: remember its EPJ-list position (the
      // group's particles follow it contiguously)
      if (lf && gfirst >= lfirst && gfirst - lfirst < lcnt)
        self_pos = (uint32_t)(ne + (inc - lcnt) + (gfirst - lfirst)) + 1u;
      rec_put(rl, lf, make_uint2(lfirst, lcnt), a.arena_l, a.next_l, a.cursor + 1, a.cap_l,
              a.head_l + g, lane, lt);
      nl += __popc(__ballot_sync(0xffffffffu, lf));
      ne += tot;
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
      if ((sp - (last + 1)) + 8 * E + (last + 1 - f - E) > kStack) {
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
      float feat[kMacNF];
#pragma unroll
      for (int k = 0; k < kMacNF; k++) feat[k] = 0.0f;
      if (q_me < E) {
        const uint4 *blk = a.block + ((size_t)cid_me * 8 + c_me) * 2;
        const uint4 nf = blk[0], meta = blk[1];
        valid = meta.z != kNone && AFD_IN(meta.z, a.n_cells, "walk child");
        if (valid) {
          leaf_me = (meta.y >> 31) != 0;
          c_id = meta.z;
          c_first = meta.x;
          c_cnt = meta.y & 0x7fffffffu;
          const float cx = __uint_as_float(nf.x), cy = __uint_as_float(nf.y),
                      cz = __uint_as_float(nf.z), s2 = __uint_as_float(nf.w);
          d = LEARNED ? learned_pre(a, bmin, bmax, cx, cy, cz, s2, leaf_me, c_id, c_first, c_cnt,
                                    gfirst, amin, feat)
                      : decide(bmin, bmax, cx, cy, cz, s2, leaf_me, a.theta2);
        }
      }
      if (LEARNED) {
        const bool need = valid && d == kBand;
        const unsigned bm = __ballot_sync(0xffffffffu, need);
        if (bm) {  // warp-uniform: the network for every band cell of this step
          const int nb = __popc(bm), rank = __popc(bm & lt);
          float y_me = 0.0f;
          if (lane == 0) rounds++;
          float *xin = reinterpret_cast<float *>(msc.xin);
          if (need)
#pragma unroll
            for (int k = 0; k < kMacNF; k++)
              xin[((rank >> 2) * kMacNF + k) * 4 + (rank & 3)] =
                  __fmul_rn(__fsub_rn(feat[k], mw.vec[k]), mw.vec[kMacNF + k]);
          __syncwarp();
          for (int g4 = 0; g4 < nb; g4 += 4) {
            // layer 1, unit = lane, cells g4 .. g4 + 3 (pairs (0,1), (2,3))
            const float b1 = mw.vec[kVecB1 + lane];
            unsigned long long A01 = mac_pk(b1, b1), A23 = A01;
#pragma unroll
            for (int kq = 0; kq < kMacNF / 4; kq++) {
              const float4 w4 = *reinterpret_cast<const float4 *>(&mw.w1[lane][4 * kq]);
              const float wk[4] = {w4.x, w4.y, w4.z, w4.w};
#pragma unroll
              for (int i = 0; i < 4; i++) {
                const float4 x = msc.xin[g4 >> 2][4 * kq + i];
                const unsigned long long W = mac_pk(wk[i], wk[i]);
                A01 = mac_fma2(W, mac_pk(x.x, x.y), A01);
                A23 = mac_fma2(W, mac_pk(x.z, x.w), A23);
              }
            }
            float h[4] = {mac_lo(A01), mac_hi(A01), mac_lo(A23), mac_hi(A23)};
#pragma unroll
            for (int c = 0; c < 4; c++) h[c] = h[c] > 0.0f ? h[c] : 0.0f;
            msc.hin[lane] = make_float4(h[0], h[1], h[2], h[3]);
            __syncwarp();
            // layer 2, unit = lane
            const float b2 = mw.vec[kVecB2 + lane];
            unsigned long long B01 = mac_pk(b2, b2), B23 = B01;
#pragma unroll 2
            for (int kq = 0; kq < kMacNH / 4; kq++) {
              const float4 w4 = *reinterpret_cast<const float4 *>(&mw.w2[lane][4 * kq]);
              const float wk[4] = {w4.x, w4.y, w4.z, w4.w};
#pragma unroll
              for (int i = 0; i < 4; i++) {
                const float4 hk = msc.hin[4 * kq + i];
                const unsigned long long W = mac_pk(wk[i], wk[i]);
                B01 = mac_fma2(W, mac_pk(hk.x, hk.y), B01);
                B23 = mac_fma2(W, mac_pk(hk.z, hk.w), B23);
              }
            }
            // output: products w3_j h2_j, xor butterfly (= pairwise halving), + b3
            const float w3 = mw.vec[kVecW3 + lane];
            float o[4] = {mac_lo(B01), mac_hi(B01), mac_lo(B23), mac_hi(B23)};
#pragma unroll
            for (int c = 0; c < 4; c++) o[c] = __fmul_rn(w3, o[c] > 0.0f ? o[c] : 0.0f);
#pragma unroll
            for (int off = kMacNH / 2; off > 0; off >>= 1)
#pragma unroll
              for (int c = 0; c < 4; c++) o[c] = __fadd_rn(o[c], __shfl_xor_sync(0xffffffffu, o[c], off));
            const float b3 = mw.vec[kVecB3];
#pragma unroll
            for (int c = 0; c < 4; c++)
              if (need && rank == g4 + c) y_me = __fadd_rn(o[c], b3);
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
      if (valid) child_entry = make_entry(d, c_id, c_first, c_cnt);
      const unsigned vm = __ballot_sync(0xffffffffu, valid);
      // output count of each rewritten position [f, last]: children or itself
      int expanded_q = -1;
#pragma unroll
      for (int q = 0; q < kExpand; q++)
        if (q < E && pos_q[q] == lane) expanded_q = q;
      uint32_t cnt = 0;
      if (lane >= f && lane <= last)
        cnt = expanded_q >= 0 ? __popc((vm >> (8 * expanded_q)) & 0xffu) : 1u;
      uint32_t oinc = cnt;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(0xffffffffu, oinc, o);
        if (lane >= o) oinc += t;
      }
      const uint32_t K = __shfl_sync(0xffffffffu, oinc, 31);
      const uint32_t off_me = oinc - cnt;
      const int spn = sp - (last + 1);
      if (spn + (int)K > kStack) {
        if (lane == 0) atomicOr(a.status, kStWalkStack);
        break;
      }
      // output offset of this lane's parent position (child lanes)
      const uint32_t off_par = __shfl_sync(0xffffffffu, off_me, p_me < 0 ? 0 : p_me);
      __syncwarp();
      if (lane >= f && lane <= last && expanded_q < 0) stk[spn + K - 1 - off_me] = e;
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
    if (lane == 0) {
      a.cnt_e[g] = (uint32_t)ne;
      a.cnt_s[g] = (uint32_t)ns;
      a.n_lrec[g] = nl;
      a.gself[g] = self_pos;
      if (ns == 0) a.head_s[g] = kNone;
      if (nl == 0) a.head_l[g] = kNone;
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
    s += (unsigned long long)g_count[g] * ((unsigned long long)ce[g] + cs[g]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0 && s) atomicAdd(out, s);
}

// The CSR lists from the record arena, one warp per group: cell ids copied,
// leaf records expanded into their particles' Morton positions.
struct CompactArgs {
  int64_t n_groups;
  const uint32_t *cnt_s, *n_lrec, *head_s, *head_l, *next_s, *next_l, *arena_s;
  const uint2 *arena_l;
  const uint64_t *off_e, *off_s;
  uint32_t *epj, *spj;
  uint32_t cap_s, cap_l;  // read only by the self-checking build
  uint64_t n_epj, n_spj;
};

constexpr int kCompactBuf = 1024;  // staged EPJ entries per warp

__global__ void __launch_bounds__(256) k_compact(CompactArgs a) {
  __shared__ uint32_t buf_all[8][kCompactBuf];
  const int64_t g = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  uint32_t *buf = buf_all[threadIdx.x >> 5];
  if (g >= a.n_groups) return;
  const uint32_t ms = a.cnt_s[g];
  uint32_t c = a.head_s[g];
  const uint64_t os = a.off_s[g];
  for (uint32_t i0 = 0; i0 < ms; i0 += kChunk) {
    if (!AFD_IN(c, a.cap_s, "compact cell chunk")) return;
    const uint32_t nn = min(kChunk, ms - i0);
    for (uint32_t k = lane; k < nn; k += 32)
      if (AFD_IN(os + i0 + k, a.n_spj, "compact spj write"))
        a.spj[os + i0 + k] = a.arena_s[(size_t)c * kChunk + k];
    if (i0 + kChunk < ms) c = a.next_s[c];
  }
  const uint32_t r = a.n_lrec[g];
  c = a.head_l[g];
  uint64_t pos = a.off_e[g];
  for (uint32_t i0 = 0; i0 < r; i0 += kChunk) {
    if (!AFD_IN(c, a.cap_l, "compact leaf chunk")) return;
    const uint32_t nrec = min(kChunk, r - i0);
    for (uint32_t j0 = 0; j0 < nrec; j0 += 32) {
      const bool on = lane < nrec - j0;
      const uint2 rec = on ? a.arena_l[(size_t)c * kChunk + j0 + lane] : make_uint2(0u, 0u);
      uint32_t inc = rec.y;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += t;
      }
      const uint32_t tot = __shfl_sync(0xffffffffu, inc, 31);
      const uint32_t ex = inc - rec.y;
      if (tot <= (uint32_t)kCompactBuf) {
        // each lane expands its own leaf into shared memory, then the warp
        // stores the run with coalesced writes
        for (uint32_t k = 0; k < rec.y; k++) buf[ex + k] = rec.x + k;
        __syncwarp();
        for (uint32_t i = lane; i < tot; i += 32)
          if (AFD_IN(pos + i, a.n_epj, "compact epj write")) a.epj[pos + i] = buf[i];
        __syncwarp();
      } else {  // very large leaves (level 21): one leaf at a time
        unsigned lm = __ballot_sync(0xffffffffu, on && rec.y > 0);
        while (lm) {
          const int src = __ffs(lm) - 1;
          lm &= lm - 1;
          const uint32_t f0 = __shfl_sync(0xffffffffu, rec.x, src);
          const uint32_t c0 = __shfl_sync(0xffffffffu, rec.y, src);
          const uint32_t x0 = __shfl_sync(0xffffffffu, ex, src);
          for (uint32_t k = lane; k < c0; k += 32)
            if (AFD_IN(pos + x0 + k, a.n_epj, "compact epj write")) a.epj[pos + x0 + k] = f0 + k;
        }
      }
      pos += tot;
    }
    if (i0 + kChunk < r) c = a.next_l[c];
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

int launch_walk(afd_ctx *c) {
  const int64_t ng = c->n_groups;
  int st;
  for (afd::DevBuf *b : {&c->l_cnt_e, &c->l_cnt_s, &c->l_nrec, &c->l_head_s, &c->l_head_l})
    if ((st = reserve(*b, sizeof(uint32_t) * ng))) return st;
  for (afd::DevBuf *b : {&c->epj_off, &c->spj_off})
    if ((st = reserve(*b, sizeof(uint64_t) * (ng + 1)))) return st;
  if ((st = reserve(c->arena_cur, 2 * sizeof(uint32_t)))) return st;
  // after reusing steps the walk records, group boxes (and quadrupoles) lag
  // the particles: refresh them before walking
  if (c->n_cells > 0 && (!c->blocks_current || (c->cfg.mac && !c->q_current))) {
    if ((st = launch_moments(c, true, c->cfg.mac != 0))) return st;
    if ((st = launch_group_boxes(c))) return st;
  }
  if (ng == 0) {
    c->n_epj = c->n_spj = c->interactions = 0;
    cudaMemsetAsync(c->epj_off.p, 0, sizeof(uint64_t), c->stream);
    cudaMemsetAsync(c->spj_off.p, 0, sizeof(uint64_t), c->stream);
    return cudaGetLastError() == cudaSuccess ? AFD_OK : AFD_ERR_CUDA;
  }
  // arena capacity in chunks: kept from earlier walks, first guess from the
  // group count (about 1500 cell ids and 130 leaves per group of 256)
  if (c->arena_cap_s == 0) c->arena_cap_s = (uint32_t)std::min<int64_t>(ng * 24 + 4096, 1u << 30);
  if (c->arena_cap_l == 0) c->arena_cap_l = (uint32_t)std::min<int64_t>(ng * 4 + 4096, 1u << 30);
  WalkArgs a;
  a.n_groups = ng;
  a.boxf = ptr<float>(c->g_boxf);
  a.g_first = ptr<uint32_t>(c->g_first);
  a.g_root = ptr<uint32_t>(c->g_root);
  a.node_f = ptr<float4>(c->node_f);
  a.node_i = ptr<uint2>(c->node_i);
  a.block = ptr<uint4>(c->c_block);
  const float th = (float)c->cfg.theta;
  a.theta2 = th * th;
  a.cnt_e = ptr<uint32_t>(c->l_cnt_e);
  a.cnt_s = ptr<uint32_t>(c->l_cnt_s);
  a.n_lrec = ptr<uint32_t>(c->l_nrec);
  a.head_s = ptr<uint32_t>(c->l_head_s);
  a.head_l = ptr<uint32_t>(c->l_head_l);
  a.gself = ptr<uint32_t>(c->g_self);
  a.cursor = ptr<uint32_t>(c->arena_cur);
  a.status = ptr<int>(c->status);
  a.iter_cap = (uint32_t)(2 * c->n_cells + 64);
  a.n_cells = (uint32_t)c->n_cells;
  const bool learned = mac_usable(c);
  a.mac_w = nullptr;
  a.g_amin = nullptr;
  a.s_hi = a.s_q0 = a.s_q1 = nullptr;
  a.lo2 = a.hi2 = a.tau = a.eps2 = 0.0f;
  a.mac_cnt = nullptr;
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
  int64_t nb = (ng + kWalkWarps - 1) / kWalkWarps;
  if (nb > 152 * 32) nb = 152 * 32;
  unsigned long long *inter = ptr<unsigned long long>(c->u64acc) + 1;
  uint64_t *pin = static_cast<uint64_t *>(c->pinned);
  for (int attempt = 0;; attempt++) {
    if ((st = reserve(c->arena_s, sizeof(uint32_t) * kChunk * (size_t)c->arena_cap_s))) return st;
    if ((st = reserve(c->arena_l, sizeof(uint2) * kChunk * (size_t)c->arena_cap_l))) return st;
    if ((st = reserve(c->next_s, sizeof(uint32_t) * (size_t)c->arena_cap_s))) return st;
    if ((st = reserve(c->next_l, sizeof(uint32_t) * (size_t)c->arena_cap_l))) return st;
    a.arena_s = ptr<uint32_t>(c->arena_s);
    a.arena_l = ptr<uint2>(c->arena_l);
    a.next_s = ptr<uint32_t>(c->next_s);
    a.next_l = ptr<uint32_t>(c->next_l);
    a.cap_s = c->arena_cap_s;
    a.cap_l = c->arena_cap_l;
    if (cudaMemsetAsync(c->arena_cur.p, 0, 2 * sizeof(uint32_t), c->stream) != cudaSuccess)
      return AFD_ERR_CUDA;
    if (learned && cudaMemsetAsync(c->mac_cnt.p, 0, 3 * sizeof(unsigned long long),
                                   c->stream) != cudaSuccess)
      return AFD_ERR_CUDA;
    if (learned) k_walk<true><<<(unsigned)nb, kWalkThreads, 0, c->stream>>>(a);
    else k_walk<false><<<(unsigned)nb, kWalkThreads, 0, c->stream>>>(a);
    c->launches++;
    if (cudaGetLastError() != cudaSuccess) return AFD_ERR_CUDA;
    if ((st = scan_u32_to_u64(c, a.cnt_e, ptr<uint64_t>(c->epj_off), ng))) return st;
    if ((st = scan_u32_to_u64(c, a.cnt_s, ptr<uint64_t>(c->spj_off), ng))) return st;
    cudaMemsetAsync(inter, 0, sizeof(unsigned long long), c->stream);
    k_interactions<<<152, 256, 0, c->stream>>>(ng, ptr<uint32_t>(c->g_count), a.cnt_e, a.cnt_s,
                                                inter);
    c->launches++;
    cudaMemcpyAsync(pin, ptr<uint64_t>(c->epj_off) + ng, sizeof(uint64_t), cudaMemcpyDeviceToHost,
                    c->stream);
    cudaMemcpyAsync(pin + 1, ptr<uint64_t>(c->spj_off) + ng, sizeof(uint64_t),
                    cudaMemcpyDeviceToHost, c->stream);
    cudaMemcpyAsync(pin + 2, inter, sizeof(uint64_t), cudaMemcpyDeviceToHost, c->stream);
    cudaMemcpyAsync(pin + 3, c->status.p, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
    cudaMemcpyAsync(pin + 4, c->arena_cur.p, 2 * sizeof(uint32_t), cudaMemcpyDeviceToHost,
                    c->stream);
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) return AFD_ERR_CUDA;
    const int bits = (int)(pin[3] & 0xffffffffu);
    if (bits) return status_to_error(bits);
    const uint32_t need_s = (uint32_t)(pin[4] & 0xffffffffu), need_l = (uint32_t)(pin[4] >> 32);
    if (need_s <= c->arena_cap_s && need_l <= c->arena_cap_l) break;
    if (attempt > 0) return AFD_ERR_LIST_OVERFLOW;  // cannot happen: sized from the cursors
    if (need_s > c->arena_cap_s)
      c->arena_cap_s = (uint32_t)std::min<uint64_t>((uint64_t)need_s * 5 / 4 + 1024, 1u << 30);
    if (need_l > c->arena_cap_l)
      c->arena_cap_l = (uint32_t)std::min<uint64_t>((uint64_t)need_l * 5 / 4 + 1024, 1u << 30);
  }
  c->n_epj = pin[0];
  c->n_spj = pin[1];
  c->interactions = pin[2];
  if ((st = reserve(c->epj, sizeof(uint32_t) * c->n_epj))) return st;
  if ((st = reserve(c->spj, sizeof(uint32_t) * c->n_spj))) return st;
  CompactArgs k;
  k.n_groups = ng;
  k.cnt_s = a.cnt_s;
  k.n_lrec = a.n_lrec;
  k.head_s = a.head_s;
  k.head_l = a.head_l;
  k.next_s = a.next_s;
  k.next_l = a.next_l;
  k.arena_s = a.arena_s;
  k.arena_l = a.arena_l;
  k.off_e = ptr<uint64_t>(c->epj_off);
  k.off_s = ptr<uint64_t>(c->spj_off);
  k.epj = ptr<uint32_t>(c->epj);
  k.spj = ptr<uint32_t>(c->spj);
  k.cap_s = c->arena_cap_s;
  k.cap_l = c->arena_cap_l;
  k.n_epj = c->n_epj;
  k.n_spj = c->n_spj;
  k_compact<<<(unsigned)((ng * 32 + 255) / 256), 256, 0, c->stream>>>(k);
  c->launches++;
  return cudaGetLastError() == cudaSuccess ? AFD_OK : AFD_ERR_CUDA;
}

}  // namespace afd
