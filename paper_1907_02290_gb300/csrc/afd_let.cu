// Local essential tree (Section 3; Section 4.3: the global tree is built over
// the local particles and what other domains export). The LET of this
// context's tree for a remote domain box is what the theta walk, with that
// box as the group box, puts on a list: accepted cells as superparticles
// (COM, monopole) and the particles of opened leaves, in depth-first order.
//
// The walk reaches a cell iff it opens every ancestor, so the export is
// marked without walking: one thread per cell tests the criterion on the
// cell's ancestors (at most 21) and on the cell itself. A scan over the cell
// ids -- the depth-first pre-order -- then gives every exported element its
// position, so the export comes out in the walk's depth-first order.
#include <cmath>

#include "afd_internal.cuh"

namespace afd {
namespace {

struct LetArgs {
  float bmin[3], bmax[3], theta2;
  const float4 *node_f;
  const uint2 *node_i;
  const uint32_t *parent;
  uint32_t *mark;  // per cell: 0 no, 1 superparticle, 2 leaf particles
  uint32_t n_cells;
};

__device__ __forceinline__ float let_sep(float c, float lo, float hi) {
  float d = 0.0f;
  if (c < lo) d = __fsub_rn(lo, c);
  else if (c > hi) d = __fsub_rn(c, hi);
  return d;
}

// The opening criterion of the walk (theta, the box as the group box).
__device__ __forceinline__ bool let_accept(const LetArgs &a, uint32_t c) {
  const float4 nf = a.node_f[c];
  const float dx = let_sep(nf.x, a.bmin[0], a.bmax[0]);
  const float dy = let_sep(nf.y, a.bmin[1], a.bmax[1]);
  const float dz = let_sep(nf.z, a.bmin[2], a.bmax[2]);
  float d2 = __fmul_rn(dx, dx);
  d2 = __fadd_rn(d2, __fmul_rn(dy, dy));
  d2 = __fadd_rn(d2, __fmul_rn(dz, dz));
  return nf.w < __fmul_rn(a.theta2, d2);
}

// One thread per cell. The walk reaches a cell iff it opens every ancestor,
// i.e. accepts none of them; a reached cell is exported as a superparticle
// if accepted, as its particles if a leaf (mark 1, 2; 0 otherwise).
__global__ void __launch_bounds__(256) k_let_mark(LetArgs a) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)a.n_cells) return;
  const uint32_t c = (uint32_t)t;
  uint32_t p = a.parent[c];
  for (int up = 0; p != kNone && up <= kLevels; up++) {
    if (!AFD_IN(p, a.n_cells, "let parent")) break;
    if (let_accept(a, p)) {
      a.mark[c] = 0u;
      return;
    }
    p = a.parent[p];
  }
  const bool leaf = (a.node_i[c].y >> 31) != 0;
  a.mark[c] = let_accept(a, c) ? 1u : (leaf ? 2u : 0u);
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
  int st;
  // after reusing steps that kept only neighbour lists the moments lag
  if (!c->moments_current && (st = launch_moments(c, false, false))) return st;
  if ((st = reserve(c->let_mark, sizeof(uint32_t) * (size_t)nc)) ||
      (st = reserve(c->let_cnt, sizeof(uint32_t) * (size_t)nc)) ||
      (st = reserve(c->let_off, sizeof(uint64_t) * (size_t)(nc + 1))))
    return st;
  LetArgs a;
  for (int k = 0; k < 3; k++) {
    a.bmin[k] = (float)box[k];
    a.bmax[k] = (float)box[3 + k];
  }
  const float th = (float)theta;
  a.theta2 = th * th;
  a.node_f = ptr<float4>(c->node_f);
  a.node_i = ptr<uint2>(c->node_i);
  a.parent = ptr<uint32_t>(c->c_parent);
  a.mark = ptr<uint32_t>(c->let_mark);
  a.n_cells = (uint32_t)nc;
  const unsigned nb = (unsigned)((nc + 255) / 256);
  k_let_mark<<<nb, 256, 0, c->stream>>>(a);
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
