// Local essential tree (Section 3; Section 4.3: the global tree is built over
// the local particles and what other domains export). The LET of this
// context's tree for a remote domain box is what the theta walk, with that
// box as the group box, puts on a list: accepted cells as superparticles
// (COM, monopole) and the particles of opened leaves, in depth-first order.
//
// One warp walks the tree (the cells a step pops, up to 32, are decided in
// parallel) and marks each exported cell; a scan over the cell ids -- the
// depth-first pre-order -- then gives every exported element its position,
// so the export comes out in depth-first order whatever order the walk
// visited the cells in.
#include <cmath>

#include "afd_internal.cuh"

namespace afd {
namespace {

constexpr int kLetStack = 8192;  // cell ids on the walking warp's stack

struct LetArgs {
  float bmin[3], bmax[3], theta2;
  const float4 *node_f;
  const uint2 *node_i;
  const uint32_t *child;
  uint32_t *mark;  // per cell: 0 no, 1 superparticle, 2 leaf particles
  int *status;
  uint32_t iter_cap, n_cells;
};

__device__ __forceinline__ float let_sep(float c, float lo, float hi) {
  float d = 0.0f;
  if (c < lo) d = __fsub_rn(lo, c);
  else if (c > hi) d = __fsub_rn(c, hi);
  return d;
}

__global__ void __launch_bounds__(32) k_let_mark(LetArgs a) {
  __shared__ uint32_t stk[kLetStack];
  const int lane = threadIdx.x;
  if (lane == 0) stk[0] = 0u;  // the root
  int sp = 1;
  uint32_t iters = 0;
  __syncwarp();
  while (sp > 0) {
    if (++iters > a.iter_cap) {
      if (lane == 0) atomicOr(a.status, kStWalkIter);
      break;
    }
    const int nv = sp < 32 ? sp : 32;
    uint32_t c = lane < nv ? stk[sp - 1 - lane] : 0u;
    bool open = false;
    if (lane < nv && AFD_IN(c, a.n_cells, "let cell")) {
      const float4 nf = a.node_f[c];
      const uint2 ni = a.node_i[c];
      const bool leaf = (ni.y >> 31) != 0;
      // the opening criterion of the walk (theta, the box as the group box)
      const float dx = let_sep(nf.x, a.bmin[0], a.bmax[0]);
      const float dy = let_sep(nf.y, a.bmin[1], a.bmax[1]);
      const float dz = let_sep(nf.z, a.bmin[2], a.bmax[2]);
      float d2 = __fmul_rn(dx, dx);
      d2 = __fadd_rn(d2, __fmul_rn(dy, dy));
      d2 = __fadd_rn(d2, __fmul_rn(dz, dz));
      if (nf.w < __fmul_rn(a.theta2, d2)) a.mark[c] = 1u;
      else if (leaf) a.mark[c] = 2u;
      else open = true;
    }
    uint32_t ch[8];
    uint32_t nch = 0;
    if (open) {
      const uint4 c0 = reinterpret_cast<const uint4 *>(a.child)[2 * (size_t)c];
      const uint4 c1 = reinterpret_cast<const uint4 *>(a.child)[2 * (size_t)c + 1];
      const uint32_t all[8] = {c0.x, c0.y, c0.z, c0.w, c1.x, c1.y, c1.z, c1.w};
#pragma unroll
      for (int o = 0; o < 8; o++)
        if (all[o] != kNone) ch[nch++] = all[o];
    }
    uint32_t inc = nch;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t t = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += t;
    }
    const uint32_t K = __shfl_sync(0xffffffffu, inc, 31);
    const int spn = sp - nv;
    if (spn + (int)K > kLetStack) {
      if (lane == 0) atomicOr(a.status, kStWalkStack);
      break;
    }
    __syncwarp();
    const uint32_t o0 = inc - nch;
#pragma unroll
    for (int o = 0; o < 8; o++)
      if ((uint32_t)o < nch) stk[spn + o0 + o] = ch[o];
    sp = spn + (int)K;
    __syncwarp();
  }
}

// Elements per cell: 1 for a superparticle, the particle count for a leaf.
__global__ void k_let_count(int64_t nc, const uint32_t *__restrict__ mark,
                            const uint32_t *__restrict__ count, uint32_t *__restrict__ cnt) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nc) return;
  const uint32_t k = mark[c];
  cnt[c] = k == 1u ? 1u : (k == 2u ? count[c] : 0u);
}

struct EmitArgs {
  int64_t nc;
  uint64_t cap;
  const uint32_t *mark, *first, *count;
  const uint64_t *off;
  const double *com, *mass, *xs, *ys, *zs, *ms;
  double *x, *y, *z, *m;
  uint32_t *kind;
};

__global__ void k_let_emit(EmitArgs a) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= a.nc) return;
  const uint32_t k = a.mark[c];
  if (k == 0u) return;
  uint64_t o = a.off[c];
  if (k == 1u) {
    if (o < a.cap) {
      a.x[o] = a.com[3 * c];
      a.y[o] = a.com[3 * c + 1];
      a.z[o] = a.com[3 * c + 2];
      a.m[o] = a.mass[c];
      if (a.kind) a.kind[o] = 1u;
    }
    return;
  }
  const uint32_t f = a.first[c], e = f + a.count[c];
  for (uint32_t j = f; j < e; j++, o++) {
    if (o >= a.cap) break;
    a.x[o] = a.xs[j];
    a.y[o] = a.ys[j];
    a.z[o] = a.zs[j];
    a.m[o] = a.ms[j];
    if (a.kind) a.kind[o] = 0u;
  }
}

}  // namespace
}  // namespace afd

using namespace afd;

extern "C" int afd_let_export(afd_ctx *c, const double *box, double theta, int64_t cap, double *x,
                              double *y, double *z, double *m, uint32_t *kind, int64_t *n_out) {
  if (!c || !box || !n_out || cap < 0 || !std::isfinite(theta) || theta < 0.0) return AFD_ERR_ARG;
  if (cap > 0 && (!x || !y || !z || !m)) return AFD_ERR_ARG;
  for (int k = 0; k < 6; k++)
    if (!std::isfinite(box[k])) return AFD_ERR_ARG;
  if (!c->have_tree) return AFD_ERR_NO_TREE;
  if (c->n_sys != 1) return AFD_ERR_ARG;  // one system: the tree of one domain
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != c->device && cudaSetDevice(c->device) != cudaSuccess) return AFD_ERR_CUDA;
  struct Restore {
    int d;
    ~Restore() {
      if (d >= 0) cudaSetDevice(d);
    }
  } restore{prev != c->device ? prev : -1};
  *n_out = 0;
  const int64_t nc = c->n_cells;
  if (nc == 0) return AFD_OK;
  int st;  // (node_f, node_i hold the current moments after reusing steps too)
  if ((st = reserve(c->let_mark, sizeof(uint32_t) * (size_t)nc)) ||
      (st = reserve(c->let_cnt, sizeof(uint32_t) * (size_t)nc)) ||
      (st = reserve(c->let_off, sizeof(uint64_t) * (size_t)(nc + 1))))
    return st;
  if (cudaMemsetAsync(c->let_mark.p, 0, sizeof(uint32_t) * (size_t)nc, c->stream) != cudaSuccess)
    return AFD_ERR_CUDA;
  LetArgs a;
  for (int k = 0; k < 3; k++) {
    a.bmin[k] = (float)box[k];
    a.bmax[k] = (float)box[3 + k];
  }
  const float th = (float)theta;
  a.theta2 = th * th;
  a.node_f = ptr<float4>(c->node_f);
  a.node_i = ptr<uint2>(c->node_i);
  a.child = ptr<uint32_t>(c->c_child);
  a.mark = ptr<uint32_t>(c->let_mark);
  a.status = ptr<int>(c->status);
  a.iter_cap = (uint32_t)(nc + 64);
  a.n_cells = (uint32_t)nc;
  k_let_mark<<<1, 32, 0, c->stream>>>(a);
  const unsigned nb = (unsigned)((nc + 255) / 256);
  k_let_count<<<nb, 256, 0, c->stream>>>(nc, a.mark, ptr<uint32_t>(c->c_count),
                                         ptr<uint32_t>(c->let_cnt));
  c->launches += 2;
  if (cudaGetLastError() != cudaSuccess) return AFD_ERR_CUDA;
  if ((st = scan_u32_to_u64(c, ptr<uint32_t>(c->let_cnt), ptr<uint64_t>(c->let_off), nc)))
    return st;
  uint64_t *pin = static_cast<uint64_t *>(c->pinned) + 1;  // word 0 holds the status
  int *pst = static_cast<int *>(c->pinned);
  if (cudaMemcpyAsync(pin, ptr<uint64_t>(c->let_off) + nc, sizeof(uint64_t),
                      cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
      cudaMemcpyAsync(pst, c->status.p, sizeof(int), cudaMemcpyDeviceToHost, c->stream) !=
          cudaSuccess ||
      cudaStreamSynchronize(c->stream) != cudaSuccess)
    return AFD_ERR_CUDA;
  if (pst[0]) {
    cudaMemsetAsync(c->status.p, 0, sizeof(int), c->stream);
    return status_to_error(pst[0]);
  }
  const int64_t total = (int64_t)pin[0];
  *n_out = total;
  if (cap == 0 || total == 0) return AFD_OK;
  EmitArgs e;
  e.nc = nc;
  e.cap = (uint64_t)cap;
  e.mark = a.mark;
  e.first = ptr<uint32_t>(c->c_first);
  e.count = ptr<uint32_t>(c->c_count);
  e.off = ptr<uint64_t>(c->let_off);
  e.com = ptr<double>(c->c_com);
  e.mass = ptr<double>(c->c_mass);
  e.xs = ptr<double>(c->xs);
  e.ys = ptr<double>(c->ys);
  e.zs = ptr<double>(c->zs);
  e.ms = ptr<double>(c->ms);
  e.x = x;
  e.y = y;
  e.z = z;
  e.m = m;
  e.kind = kind;
  k_let_emit<<<nb, 256, 0, c->stream>>>(e);
  c->launches++;
  if (cudaGetLastError() != cudaSuccess) return AFD_ERR_CUDA;
  return cudaStreamSynchronize(c->stream) == cudaSuccess ? AFD_OK : AFD_ERR_CUDA;
}
