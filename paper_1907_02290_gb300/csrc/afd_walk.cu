// Interaction lists (Barnes' vectorised walk, Section 2; multiwalk,
// Section 3; index lists, Section 4.1). One warp walks the tree for one
// i-group, depth first, children in Morton order:
//   an accepted cell appends its id to the group's SPJ list,
//   an opened leaf appends its particles' Morton positions to the EPJ list,
//   an opened internal cell is replaced by its children.
// The warp keeps a stack of cells whose decision is already known. Each
// step either emits the run of accepted / leaf entries at the top of the
// stack in order, or expands the open cell at the top, deciding its (up to
// eight) children in parallel. Emission therefore follows depth-first
// order exactly. Two passes: counts, then (after a scan) the fill.
//
// The opening criterion is evaluated in FP32 without contraction: with d the
// distance from the cell's centre of mass to the group's bounding box (0
// inside) and s the cell side, the cell is accepted iff s^2 < theta^2 d^2,
// computed as ((dx*dx + dy*dy) + dz*dz) and theta2 * d2 in that order.
#include "afd_internal.cuh"

namespace afd {
namespace {

constexpr int kWalkWarps = 4;
constexpr int kWalkThreads = 32 * kWalkWarps;
constexpr int kStack = 8 * (kLevels + 2);
constexpr uint32_t kOpen = 0u, kAccept = 1u, kLeaf = 2u;

struct WalkArgs {
  int64_t n_groups;
  const float *boxf;
  const uint32_t *g_first;
  const float4 *node_f;
  const uint2 *node_i;
  const uint32_t *child;
  float theta2;
  uint32_t *cnt_e, *cnt_s, *gself;
  const uint64_t *off_e, *off_s;
  uint32_t *epj, *spj;
  int *status;
  uint32_t iter_cap;
};

__device__ __forceinline__ float sep_axis(float c, float lo, float hi) {
  float d = 0.0f;
  if (c < lo) d = __fsub_rn(lo, c);
  else if (c > hi) d = __fsub_rn(c, hi);
  return d;
}

__device__ __forceinline__ uint32_t decide(const float *bmin, const float *bmax, float4 nf,
                                           uint2 ni, float theta2) {
  const float dx = sep_axis(nf.x, bmin[0], bmax[0]);
  const float dy = sep_axis(nf.y, bmin[1], bmax[1]);
  const float dz = sep_axis(nf.z, bmin[2], bmax[2]);
  float d2 = __fmul_rn(dx, dx);
  d2 = __fadd_rn(d2, __fmul_rn(dy, dy));
  d2 = __fadd_rn(d2, __fmul_rn(dz, dz));
  const float rhs = __fmul_rn(theta2, d2);
  if (nf.w < rhs) return kAccept;
  return (ni.y >> 31) ? kLeaf : kOpen;
}

template <bool FILL>
__global__ void __launch_bounds__(kWalkThreads) k_walk(WalkArgs a) {
  __shared__ uint32_t stk_all[kWalkWarps][kStack];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const unsigned lt = (1u << lane) - 1u;
  uint32_t *stk = stk_all[wib];
  for (int64_t g = (int64_t)blockIdx.x * kWalkWarps + wib; g < a.n_groups;
       g += (int64_t)gridDim.x * kWalkWarps) {
    float bmin[3], bmax[3];
#pragma unroll
    for (int k = 0; k < 3; k++) {
      bmin[k] = a.boxf[g * 6 + k];
      bmax[k] = a.boxf[g * 6 + 3 + k];
    }
    const uint32_t gfirst = a.g_first[g];
    const uint64_t be = FILL ? a.off_e[g] : 0, bs = FILL ? a.off_s[g] : 0;
    uint64_t ne = 0, ns = 0;
    bool self = false;
    if (lane == 0) stk[0] = 0u | (decide(bmin, bmax, a.node_f[0], a.node_i[0], a.theta2) << 30);
    int sp = 1;
    uint32_t iters = 0;
    __syncwarp();
    while (sp > 0) {
      if (++iters > a.iter_cap) {
        if (lane == 0) atomicOr(a.status, kStWalkIter);
        break;
      }
      const int nv = sp < 32 ? sp : 32;
      const uint32_t e = lane < nv ? stk[sp - 1 - lane] : 0u;
      const uint32_t dec = e >> 30, cid = e & 0x3fffffffu;
      const unsigned om = __ballot_sync(0xffffffffu, lane < nv && dec == kOpen);
      const int f = om ? __ffs(om) - 1 : nv;
      const bool emit = lane < f;
      const bool acc = emit && dec == kAccept;
      const bool lf = emit && dec == kLeaf;
      const unsigned am = __ballot_sync(0xffffffffu, acc);
      if (FILL && acc) a.spj[bs + ns + __popc(am & lt)] = cid;
      ns += __popc(am);
      uint32_t lfirst = 0, lcnt = 0;
      if (lf) {
        const uint2 ni = a.node_i[cid];
        lfirst = ni.x;
        lcnt = ni.y & 0x7fffffffu;
        if (gfirst >= lfirst && gfirst - lfirst < lcnt) self = true;
      }
      uint32_t inc = lcnt;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += t;
      }
      const uint32_t tot = __shfl_sync(0xffffffffu, inc, 31);
      if (FILL) {
        const uint32_t ex = inc - lcnt;
        unsigned lm = __ballot_sync(0xffffffffu, lf);
        while (lm) {
          const int src = __ffs(lm) - 1;
          lm &= lm - 1;
          const uint32_t f0 = __shfl_sync(0xffffffffu, lfirst, src);
          const uint32_t c0 = __shfl_sync(0xffffffffu, lcnt, src);
          const uint32_t x0 = __shfl_sync(0xffffffffu, ex, src);
          for (uint32_t k = lane; k < c0; k += 32) a.epj[be + ne + x0 + k] = f0 + k;
        }
      }
      ne += tot;
      sp -= f;
      if (f < nv) {
        const uint32_t c = __shfl_sync(0xffffffffu, cid, f);
        sp -= 1;
        const uint32_t ch = lane < 8 ? a.child[(size_t)c * 8 + lane] : kNone;
        const bool valid = ch != kNone;
        uint32_t d = 0;
        if (valid) d = decide(bmin, bmax, a.node_f[ch], a.node_i[ch], a.theta2);
        const unsigned vm = __ballot_sync(0xffffffffu, valid);
        const int nvc = __popc(vm);
        if (sp + nvc > kStack) {
          if (lane == 0) atomicOr(a.status, kStWalkStack);
          break;
        }
        __syncwarp();
        if (valid) stk[sp + nvc - 1 - __popc(vm & lt)] = ch | (d << 30);
        sp += nvc;
      }
      __syncwarp();
    }
    self = __any_sync(0xffffffffu, self);
    if (!FILL && lane == 0) {
      a.cnt_e[g] = (uint32_t)ne;
      a.cnt_s[g] = (uint32_t)ns;
      a.gself[g] = self ? 1u : 0u;
    }
    __syncwarp();
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

}  // namespace

int launch_walk(afd_ctx *c) {
  const int64_t ng = c->n_groups;
  int st;
  for (afd::DevBuf *b : {&c->l_cnt_e, &c->l_cnt_s})
    if ((st = reserve(*b, sizeof(uint32_t) * ng))) return st;
  for (afd::DevBuf *b : {&c->epj_off, &c->spj_off})
    if ((st = reserve(*b, sizeof(uint64_t) * (ng + 1)))) return st;
  if (ng == 0) {
    c->n_epj = c->n_spj = c->interactions = 0;
    cudaMemsetAsync(c->epj_off.p, 0, sizeof(uint64_t), c->stream);
    cudaMemsetAsync(c->spj_off.p, 0, sizeof(uint64_t), c->stream);
    return cudaGetLastError() == cudaSuccess ? AFD_OK : AFD_ERR_CUDA;
  }
  if (c->n_cells >= (int64_t)1 << 30) return AFD_ERR_LIST_OVERFLOW;
  WalkArgs a;
  a.n_groups = ng;
  a.boxf = ptr<float>(c->g_boxf);
  a.g_first = ptr<uint32_t>(c->g_first);
  a.node_f = ptr<float4>(c->node_f);
  a.node_i = ptr<uint2>(c->node_i);
  a.child = ptr<uint32_t>(c->c_child);
  const float th = (float)c->cfg.theta;
  a.theta2 = th * th;
  a.cnt_e = ptr<uint32_t>(c->l_cnt_e);
  a.cnt_s = ptr<uint32_t>(c->l_cnt_s);
  a.gself = ptr<uint32_t>(c->g_self);
  a.off_e = ptr<uint64_t>(c->epj_off);
  a.off_s = ptr<uint64_t>(c->spj_off);
  a.epj = nullptr;
  a.spj = nullptr;
  a.status = ptr<int>(c->status);
  a.iter_cap = (uint32_t)(2 * c->n_cells + 64);
  int64_t nb = (ng + kWalkWarps - 1) / kWalkWarps;
  if (nb > 152 * 32) nb = 152 * 32;
  k_walk<false><<<(unsigned)nb, kWalkThreads, 0, c->stream>>>(a);
  c->launches++;
  if (cudaGetLastError() != cudaSuccess) return AFD_ERR_CUDA;
  if ((st = scan_u32_to_u64(c, a.cnt_e, ptr<uint64_t>(c->epj_off), ng))) return st;
  if ((st = scan_u32_to_u64(c, a.cnt_s, ptr<uint64_t>(c->spj_off), ng))) return st;
  unsigned long long *inter = ptr<unsigned long long>(c->u64acc) + 1;
  cudaMemsetAsync(inter, 0, sizeof(unsigned long long), c->stream);
  k_interactions<<<152, 256, 0, c->stream>>>(ng, ptr<uint32_t>(c->g_count), a.cnt_e, a.cnt_s,
                                              inter);
  c->launches++;
  uint64_t *pin = static_cast<uint64_t *>(c->pinned);
  cudaMemcpyAsync(pin, ptr<uint64_t>(c->epj_off) + ng, sizeof(uint64_t), cudaMemcpyDeviceToHost,
                  c->stream);
  cudaMemcpyAsync(pin + 1, ptr<uint64_t>(c->spj_off) + ng, sizeof(uint64_t),
                  cudaMemcpyDeviceToHost, c->stream);
  cudaMemcpyAsync(pin + 2, inter, sizeof(uint64_t), cudaMemcpyDeviceToHost, c->stream);
  cudaMemcpyAsync(pin + 3, c->status.p, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) return AFD_ERR_CUDA;
  const int bits = (int)(pin[3] & 0xffffffffu);
  if (bits) return status_to_error(bits);
  c->n_epj = pin[0];
  c->n_spj = pin[1];
  c->interactions = pin[2];
  if ((st = reserve(c->epj, sizeof(uint32_t) * c->n_epj))) return st;
  if ((st = reserve(c->spj, sizeof(uint32_t) * c->n_spj))) return st;
  a.epj = ptr<uint32_t>(c->epj);
  a.spj = ptr<uint32_t>(c->spj);
  k_walk<true><<<(unsigned)nb, kWalkThreads, 0, c->stream>>>(a);
  c->launches++;
  return cudaGetLastError() == cudaSuccess ? AFD_OK : AFD_ERR_CUDA;
}

}  // namespace afd
