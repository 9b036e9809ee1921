// C ABI entry points (include/afdps.h), the kick/drift kernels of the
// leapfrog and the FP64 energy reduction.
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "afd_internal.cuh"

using namespace afd;

namespace {

// Makes the context's device current for the duration of a call and
// restores the caller's device afterwards.
struct DeviceGuard {
  int prev = -1;
  bool ok = false;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    ok = cudaSetDevice(dev) == cudaSuccess;
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

#define TRY(x)                    \
  do {                            \
    int _s = (x);                 \
    if (_s != AFD_OK) return _s;  \
  } while (0)

inline int cuda_ok(cudaError_t e) {
  if (e == cudaSuccess) return AFD_OK;
  cudaGetLastError();
  return AFD_ERR_CUDA;
}

constexpr int kThreads = 256;

__global__ void k_kick_drift(double *__restrict__ x, double *__restrict__ y,
                             double *__restrict__ z, double *__restrict__ vx,
                             double *__restrict__ vy, double *__restrict__ vz,
                             const float4 *__restrict__ acc, int64_t n, double dtk, double dtd) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float4 a = acc[i];
  const double ux = vx[i] + (double)a.x * dtk;
  const double uy = vy[i] + (double)a.y * dtk;
  const double uz = vz[i] + (double)a.z * dtk;
  vx[i] = ux;
  vy[i] = uy;
  vz[i] = uz;
  x[i] += ux * dtd;
  y[i] += uy * dtd;
  z[i] += uz * dtd;
}

__global__ void k_kick(double *__restrict__ vx, double *__restrict__ vy, double *__restrict__ vz,
                       const float4 *__restrict__ acc, int64_t n, double dtk) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float4 a = acc[i];
  vx[i] += (double)a.x * dtk;
  vy[i] += (double)a.y * dtk;
  vz[i] += (double)a.z * dtk;
}

// FP64 energies with a fixed reduction order: block b sums a fixed slice,
// the last block sums the block partials in block order.
constexpr int kEnergyBlocks = 304;

__global__ void k_energy(const double *__restrict__ vx, const double *__restrict__ vy,
                         const double *__restrict__ vz, const double *__restrict__ m,
                         const float4 *__restrict__ acc, int64_t n, double *__restrict__ part,
                         unsigned *__restrict__ counter, double *__restrict__ out) {
  double k = 0.0, w = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double v2 = vx[i] * vx[i] + vy[i] * vy[i] + vz[i] * vz[i];
    k += 0.5 * m[i] * v2;
    w += 0.5 * m[i] * (double)acc[i].w;
  }
  __shared__ double sk[kThreads], sw[kThreads];
  __shared__ bool last;
  sk[threadIdx.x] = k;
  sw[threadIdx.x] = w;
  __syncthreads();
  for (int s = kThreads / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      sk[threadIdx.x] += sk[threadIdx.x + s];
      sw[threadIdx.x] += sw[threadIdx.x + s];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = sk[0];
    part[2 * blockIdx.x + 1] = sw[0];
    __threadfence();
    last = atomicAdd(counter, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last || threadIdx.x != 0) return;
  __threadfence();
  double K = 0.0, W = 0.0;
  for (unsigned b = 0; b < gridDim.x; b++) {
    K += __ldcg(&part[2 * b]);
    W += __ldcg(&part[2 * b + 1]);
  }
  out[0] = K;
  out[1] = W;
  *counter = 0u;
}

int read_status(afd_ctx *c) {
  int *pin = static_cast<int *>(c->pinned);
  if (cudaMemcpyAsync(pin, c->status.p, sizeof(int), cudaMemcpyDeviceToHost, c->stream) !=
          cudaSuccess ||
      cudaStreamSynchronize(c->stream) != cudaSuccess) {
    cudaGetLastError();
    return AFD_ERR_CUDA;
  }
  const int bits = *pin;
  if (bits) cudaMemsetAsync(c->status.p, 0, sizeof(int), c->stream);
  return status_to_error(bits);
}

int tree_build(afd_ctx *c, const double *x, const double *y, const double *z, const double *m,
               int64_t n) {
  if (n < 0 || n >= ((int64_t)1 << 30)) return AFD_ERR_ARG;
  if (n > 0 && (!x || !y || !z || !m)) return AFD_ERR_ARG;
  if (c->n_sys > 1 && n != c->sys_off_h[c->n_sys]) return AFD_ERR_SHAPE;
  c->have_tree = c->have_lists = c->saved = c->have_nbr = c->u_order_ok = false;
  c->n = n;
  TRY(launch_root(c, x, y, z, m, n));
  TRY(launch_keys(c, x, y, z, n));
  TRY(launch_sort(c, n));
  TRY(launch_reorder(c, x, y, z, m, n));
  TRY(launch_link(c, n));
  TRY(read_status(c));
  TRY(launch_moments(c, true, c->cfg.mac != 0));
  TRY(launch_groups(c));
  TRY(launch_group_boxes(c));
  c->have_tree = true;
  return AFD_OK;
}

int make_lists(afd_ctx *c, int mode) {
  if (mode != AFD_MAKE_LIST && mode != AFD_MAKE_LIST_FOR_REUSE) return AFD_ERR_ARG;
  if (!c->have_tree) return AFD_ERR_NO_TREE;
  c->have_lists = c->saved = c->u_order_ok = false;
  TRY(launch_walk(c));
  if (c->share_parts > 1) TRY(compute_share(c));
  TRY(order_units(c));
  c->have_lists = true;
  c->saved = mode == AFD_MAKE_LIST_FOR_REUSE;
  return AFD_OK;
}

int reuse(afd_ctx *c, const double *x, const double *y, const double *z, const double *m) {
  // kept gravity lists or neighbour lists (both survive the move)
  if (!(c->saved && c->have_lists) && !c->have_nbr) return AFD_ERR_NO_SAVED_LIST;
  if (c->n > 0 && (!x || !y || !z || !m)) return AFD_ERR_ARG;
  if (!c->saved) c->have_lists = false;  // gravity lists not made for reuse end here
  TRY(launch_reorder(c, x, y, z, m, c->n));
  if (c->have_lists) {
    TRY(launch_moments(c, false, false));  // lists are kept: no criterion runs
  } else {
    // only neighbour lists are kept, and the density needs positions alone:
    // the moments wait until something reads them
    c->moments_current = c->blocks_current = c->q_current = false;
  }
  return AFD_OK;
}

int calc_force(afd_ctx *c, float *acc4) {
  if (!c->have_lists) return c->have_tree ? AFD_ERR_NO_SAVED_LIST : AFD_ERR_NO_TREE;
  if (c->n > 0 && !acc4) return AFD_ERR_ARG;
  TRY(launch_force(c, acc4));
  // the learned opening criterion scales cells by these magnitudes at the
  // next construction step (with a work share the other parts' rows are not
  // here yet: the caller passes the combined forces to afd_mac_set_reference)
  if (c->cfg.mac && c->share_parts == 1) TRY(launch_amag(c, acc4));
  return AFD_OK;
}

int calc_force_all(afd_ctx *c, const double *x, const double *y, const double *z,
                   const double *m, int64_t n, float *acc4, int mode) {
  if (mode == AFD_REUSE_LIST) {
    if (!c->saved) return AFD_ERR_NO_SAVED_LIST;
    if (n != c->n) return AFD_ERR_SHAPE;
    TRY(reuse(c, x, y, z, m));
  } else {
    TRY(tree_build(c, x, y, z, m, n));
    TRY(make_lists(c, mode));
  }
  return calc_force(c, acc4);
}

inline unsigned nblocks(int64_t n) { return (unsigned)((n + kThreads - 1) / kThreads); }

int kick_drift_launch(afd_ctx *c, double *x, double *y, double *z, double *vx, double *vy,
                      double *vz, const float *acc4, int64_t n, double dtk, double dtd) {
  if (n == 0) return AFD_OK;
  k_kick_drift<<<nblocks(n), kThreads, 0, c->stream>>>(
      x, y, z, vx, vy, vz, reinterpret_cast<const float4 *>(acc4), n, dtk, dtd);
  c->launches++;
  return cuda_ok(cudaGetLastError());
}

int kick_launch(afd_ctx *c, double *vx, double *vy, double *vz, const float *acc4, int64_t n,
                double dtk) {
  if (n == 0) return AFD_OK;
  k_kick<<<nblocks(n), kThreads, 0, c->stream>>>(vx, vy, vz,
                                                 reinterpret_cast<const float4 *>(acc4), n, dtk);
  c->launches++;
  return cuda_ok(cudaGetLastError());
}

void graph_release(afd_ctx *c) {
  // a replay still running finishes before its graph goes
  if (c->graph_exec && c->graph_done) cudaEventSynchronize(c->graph_done);
  if (c->graph_exec) cudaGraphExecDestroy(c->graph_exec);
  if (c->graph) cudaGraphDestroy(c->graph);
  c->graph_exec = nullptr;
  c->graph = nullptr;
}

}  // namespace

namespace afd {

// Contiguous parts of a work array: bounds[p] is the first index k whose
// prefix sum (work[0] + ... + work[k - 1]) reaches total * p / parts, so each
// part's work is within one element's work of total / parts. All-zero work
// is split by count.
void partition_work(const uint64_t *work, int64_t n, int parts, int64_t *bounds) {
  uint64_t total = 0;
  for (int64_t i = 0; i < n; i++) total += work[i];
  const bool by_count = total == 0;
  if (by_count) total = (uint64_t)n;
  bounds[0] = 0;
  int64_t k = 0;
  uint64_t prefix = 0;
  for (int p = 1; p < parts; p++) {
    const unsigned __int128 target = (unsigned __int128)total * (unsigned)p;
    while (k < n && (unsigned __int128)prefix * (unsigned)parts < target) {
      prefix += by_count ? 1u : work[k];
      k++;
    }
    bounds[p] = k;
  }
  bounds[parts] = n;
}

int compute_share(afd_ctx *c) {
  const int64_t ng = c->n_groups;
  c->share_g0 = c->share_g1 = c->share_u0 = c->share_u1 = 0;
  c->share_inter = 0;
  if (ng == 0) return AFD_OK;
  std::vector<uint32_t> ce(ng), cs(ng), gc(ng), uo(ng + 1);
  const size_t b = sizeof(uint32_t) * (size_t)ng;
  if (cudaMemcpyAsync(ce.data(), c->l_cnt_e.p, b, cudaMemcpyDeviceToHost, c->stream) !=
          cudaSuccess ||
      cudaMemcpyAsync(cs.data(), c->l_cnt_s.p, b, cudaMemcpyDeviceToHost, c->stream) !=
          cudaSuccess ||
      cudaMemcpyAsync(gc.data(), c->g_count.p, b, cudaMemcpyDeviceToHost, c->stream) !=
          cudaSuccess ||
      cudaMemcpyAsync(uo.data(), c->u_off.p, b + sizeof(uint32_t), cudaMemcpyDeviceToHost,
                      c->stream) != cudaSuccess ||
      cudaStreamSynchronize(c->stream) != cudaSuccess)
    return AFD_ERR_CUDA;
  std::vector<uint64_t> w(ng);
  for (int64_t g = 0; g < ng; g++) w[g] = (uint64_t)gc[g] * ((uint64_t)ce[g] + cs[g]);
  std::vector<int64_t> bounds(c->share_parts + 1);
  partition_work(w.data(), ng, c->share_parts, bounds.data());
  c->share_g0 = bounds[c->share_part];
  c->share_g1 = bounds[c->share_part + 1];
  c->share_u0 = uo[c->share_g0];
  c->share_u1 = uo[c->share_g1];
  for (int64_t g = c->share_g0; g < c->share_g1; g++) c->share_inter += w[g];
  return AFD_OK;
}

}  // namespace afd

extern "C" {

int afd_partition_work(const uint64_t *work, int64_t n, int parts, int64_t *bounds) {
  if (n < 0 || parts < 1 || !bounds || (n > 0 && !work)) return AFD_ERR_ARG;
  partition_work(work, n, parts, bounds);
  return AFD_OK;
}

int afd_set_work_share(afd_ctx *c, int part, int parts) {
  if (!c || parts < 1 || part < 0 || part >= parts) return AFD_ERR_ARG;
  DeviceGuard g(c->device);
  c->share_part = part;
  c->share_parts = parts;
  if (c->have_lists) {
    if (parts > 1) TRY(compute_share(c));
    return order_units(c);
  }
  return AFD_OK;
}

int afd_get_work_share(afd_ctx *c, int64_t *out) {
  if (!c || !out) return AFD_ERR_ARG;
  const bool all = c->share_parts == 1 || !c->have_lists;
  out[0] = c->share_part;
  out[1] = c->share_parts;
  out[2] = all ? 0 : c->share_g0;
  out[3] = all ? (c->have_tree ? c->n_groups : 0) : c->share_g1;
  out[4] = all ? (c->have_lists ? (int64_t)c->interactions : 0) : (int64_t)c->share_inter;
  return AFD_OK;
}


int afd_create(afd_ctx **out, const afd_config *cfg, int device, void *stream) {
  if (!out || !cfg) return AFD_ERR_ARG;
  *out = nullptr;
  if (!std::isfinite(cfg->eps) || cfg->eps < 0.0 || !std::isfinite(cfg->theta) ||
      cfg->theta < 0.0 || cfg->n_leaf < 1 || cfg->n_grp < 1 || cfg->n_grp > 1024 ||
      (cfg->multipole != 0 && cfg->multipole != 1) || cfg->far_precision < 0 ||
      cfg->far_precision > 2 || (cfg->mac != 0 && cfg->mac != 1) || cfg->reserved != 0)
    return AFD_ERR_ARG;
  DeviceGuard g(device);
  if (!g.ok) return AFD_ERR_CUDA;
  afd_ctx *c = new (std::nothrow) afd_ctx();
  if (!c) return AFD_ERR_OOM;
  c->cfg = *cfg;
  c->device = device;
  c->stream = static_cast<cudaStream_t>(stream);
  if (cudaMallocHost(&c->pinned, 256) != cudaSuccess || cudaEventCreate(&c->ev0) != cudaSuccess ||
      cudaEventCreate(&c->ev1) != cudaSuccess || reserve(c->status, 16) != AFD_OK ||
      reserve(c->red_count, 16) != AFD_OK || reserve(c->u64acc, 64) != AFD_OK ||
      cudaMemset(c->status.p, 0, 16) != cudaSuccess ||
      cudaMemset(c->red_count.p, 0, 16) != cudaSuccess) {
    cudaGetLastError();
    afd_destroy(c);
    return AFD_ERR_CUDA;
  }
  *out = c;
  return AFD_OK;
}

void afd_destroy(afd_ctx *c) {
  if (!c) return;
  DeviceGuard g(c->device);
  cudaStreamSynchronize(c->stream);
  graph_release(c);
  if (c->graph_done) cudaEventDestroy(c->graph_done);
  c->graph_done = nullptr;
  DevBuf *bufs[] = {&c->root, &c->status, &c->red_part, &c->red_count, &c->u64acc, &c->keys,
                    &c->keys2, &c->perm, &c->perm2, &c->sort_cnt, &c->sort_off, &c->xs, &c->ys,
                    &c->zs, &c->ms, &c->jhi, &c->jlo, &c->lk_d, &c->lk_c, &c->lk_e, &c->lk_cnt,
                    &c->lk_off, &c->c_level, &c->c_first, &c->c_count, &c->c_skip, &c->c_parent,
                    &c->c_child, &c->c_arrive, &c->leaf_ord, &c->leaf_aux, &c->c_mass, &c->c_smom, &c->c_com, &c->c_quad,
                    &c->s_hi, &c->s_lo, &c->s_q0, &c->s_q1, &c->node_f, &c->node_i, &c->c_block, &c->g_cnt,
                    &c->g_off, &c->g_first, &c->g_count, &c->g_cell, &c->g_box, &c->g_boxf,
                    &c->g_self, &c->u_cnt, &c->u_off, &c->u_info, &c->l_cnt_e,
                    &c->l_cnt_s, &c->epj_off, &c->spj_off, &c->epj, &c->spj, &c->scan_tmp,
                    &c->hx, &c->hy, &c->hz, &c->hm, &c->hacc, &c->sys_off_d,
                    &c->sys_grp_d, &c->sys_of, &c->sys_s, &c->root_tiles, &c->g_root,
                    &c->mac_w, &c->amag, &c->amag_s, &c->g_amin, &c->mac_cnt,
                    &c->band_cnt, &c->band_off, &c->l_nrec,
                    &c->arena_s, &c->arena_l, &c->hdr_s, &c->hdr_l, &c->arena_cur,
                    &c->m_ehi, &c->m_elo, &c->m_shi, &c->m_slo, &c->let_mark,
                    &c->let_cnt, &c->let_off, &c->c_tbox, &c->nbr_arrive, &c->g_sbox,
                    &c->nbr_cnt, &c->nbr_off, &c->nbr, &c->nbr_blk, &c->nbr_seg_cnt,
                    &c->nbr_seg_off, &c->nbr_items, &c->nbr_part, &c->nbr_seedf,
                    &c->nbr_seedo, &c->nbr_seeds, &c->nbr_icnt, &c->nbr_igoff, &c->nbr_itg,
                    &c->nbr_itr, &c->nbr_ioff, &c->nbr_sbb, &c->mxyz, &c->u_order,
                    &c->u_work, &c->u_hist, &c->nbr_order, &c->nbr_work, &c->nbr_hist,
                    &c->s_h, &c->g_fscale};
  for (DevBuf *b : bufs) release(*b);
  if (c->pinned) cudaFreeHost(c->pinned);
  if (c->ev0) cudaEventDestroy(c->ev0);
  if (c->ev1) cudaEventDestroy(c->ev1);
  delete c;
}

int afd_set_systems(afd_ctx *c, const int64_t *sys_off, int n_sys, const int32_t *n_grp) {
  if (!c || !sys_off || n_sys < 1 || n_sys > 65535) return AFD_ERR_ARG;
  if (sys_off[0] != 0 || sys_off[n_sys] >= ((int64_t)1 << 30)) return AFD_ERR_ARG;
  for (int s = 0; s < n_sys; s++)
    if (sys_off[s + 1] < sys_off[s]) return AFD_ERR_ARG;
  if (n_grp)
    for (int s = 0; s < n_sys; s++)
      if (n_grp[s] < 1 || n_grp[s] > 1024) return AFD_ERR_ARG;
  DeviceGuard g(c->device);
  c->have_tree = c->have_lists = c->saved = c->u_order_ok = false;
  c->n_sys = n_sys;
  c->sys_off_h.assign(sys_off, sys_off + n_sys + 1);
  if (n_grp) c->sys_grp_h.assign(n_grp, n_grp + n_sys);
  else c->sys_grp_h.clear();
  TRY(reserve(c->sys_off_d, sizeof(int64_t) * (size_t)(n_sys + 1)));
  TRY(cuda_ok(cudaMemcpy(c->sys_off_d.p, sys_off, sizeof(int64_t) * (size_t)(n_sys + 1),
                         cudaMemcpyHostToDevice)));
  if (n_grp) {
    std::vector<uint32_t> gs(n_grp, n_grp + n_sys);
    TRY(reserve(c->sys_grp_d, sizeof(uint32_t) * (size_t)n_sys));
    TRY(cuda_ok(cudaMemcpy(c->sys_grp_d.p, gs.data(), sizeof(uint32_t) * (size_t)n_sys,
                           cudaMemcpyHostToDevice)));
  }
  return AFD_OK;
}

int afd_set_stream(afd_ctx *c, void *stream) {
  if (!c) return AFD_ERR_ARG;
  c->stream = static_cast<cudaStream_t>(stream);
  return AFD_OK;
}

int afd_tree_build(afd_ctx *c, const double *x, const double *y, const double *z,
                   const double *m, int64_t n) {
  if (!c) return AFD_ERR_ARG;
  DeviceGuard g(c->device);
  return tree_build(c, x, y, z, m, n);
}

int afd_make_interaction_lists(afd_ctx *c, int mode) {
  if (!c) return AFD_ERR_ARG;
  DeviceGuard g(c->device);
  return make_lists(c, mode);
}

int afd_reuse_lists(afd_ctx *c, const double *x, const double *y, const double *z,
                    const double *m) {
  if (!c) return AFD_ERR_ARG;
  DeviceGuard g(c->device);
  return reuse(c, x, y, z, m);
}

int afd_calc_force(afd_ctx *c, float *acc4) {
  if (!c) return AFD_ERR_ARG;
  DeviceGuard g(c->device);
  return calc_force(c, acc4);
}

int afd_calc_force_all(afd_ctx *c, const double *x, const double *y, const double *z,
                       const double *m, int64_t n, float *acc4, int mode) {
  if (!c) return AFD_ERR_ARG;
  if (mode < AFD_MAKE_LIST || mode > AFD_REUSE_LIST) return AFD_ERR_ARG;
  DeviceGuard g(c->device);
  return calc_force_all(c, x, y, z, m, n, acc4, mode);
}

int afd_calc_force_all_host(afd_ctx *c, const double *x, const double *y, const double *z,
                            const double *m, int64_t n, float *acc4_host, int mode) {
  if (!c || n < 0) return AFD_ERR_ARG;
  if (n > 0 && (!x || !y || !z || !m || !acc4_host)) return AFD_ERR_ARG;
  if (mode < AFD_MAKE_LIST || mode > AFD_REUSE_LIST) return AFD_ERR_ARG;
  DeviceGuard g(c->device);
  const size_t bd = sizeof(double) * (size_t)n;
  TRY(reserve(c->hx, bd));
  TRY(reserve(c->hy, bd));
  TRY(reserve(c->hz, bd));
  TRY(reserve(c->hm, bd));
  TRY(reserve(c->hacc, sizeof(float4) * (size_t)n));
  if (n > 0) {
    TRY(cuda_ok(cudaMemcpyAsync(c->hx.p, x, bd, cudaMemcpyHostToDevice, c->stream)));
    TRY(cuda_ok(cudaMemcpyAsync(c->hy.p, y, bd, cudaMemcpyHostToDevice, c->stream)));
    TRY(cuda_ok(cudaMemcpyAsync(c->hz.p, z, bd, cudaMemcpyHostToDevice, c->stream)));
    TRY(cuda_ok(cudaMemcpyAsync(c->hm.p, m, bd, cudaMemcpyHostToDevice, c->stream)));
  }
  // Pinned (page-locked, mapped) output: the force kernel writes the
  // accelerations straight into it over the host link while it runs, instead
  // of a copy after it. Not with the learned criterion (its |a| pass reads
  // the forces back) nor with a work share.
  float *dev_out = ptr<float>(c->hacc);
  bool direct = false;
  if (n > 0 && !c->cfg.mac && c->share_parts == 1) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, acc4_host) == cudaSuccess &&
        at.type == cudaMemoryTypeHost && at.devicePointer != nullptr) {
      dev_out = static_cast<float *>(at.devicePointer);
      direct = true;
    } else {
      cudaGetLastError();
    }
  }
  TRY(calc_force_all(c, ptr<double>(c->hx), ptr<double>(c->hy), ptr<double>(c->hz),
                     ptr<double>(c->hm), n, dev_out, mode));
  if (n > 0 && !direct)
    TRY(cuda_ok(cudaMemcpyAsync(acc4_host, c->hacc.p, sizeof(float4) * (size_t)n,
                                cudaMemcpyDeviceToHost, c->stream)));
  TRY(cuda_ok(cudaStreamSynchronize(c->stream)));
  return read_status(c);
}

int afd_kick_drift(afd_ctx *c, double *x, double *y, double *z, double *vx, double *vy,
                   double *vz, const float *acc4, int64_t n, double dt_kick, double dt_drift) {
  if (!c || n < 0) return AFD_ERR_ARG;
  if (n == 0) return AFD_OK;
  if (!x || !y || !z || !vx || !vy || !vz || !acc4) return AFD_ERR_ARG;
  DeviceGuard g(c->device);
  return kick_drift_launch(c, x, y, z, vx, vy, vz, acc4, n, dt_kick, dt_drift);
}

int afd_kick(afd_ctx *c, double *vx, double *vy, double *vz, const float *acc4, int64_t n,
             double dt_kick) {
  if (!c || n < 0) return AFD_ERR_ARG;
  if (n == 0) return AFD_OK;
  if (!vx || !vy || !vz || !acc4) return AFD_ERR_ARG;
  DeviceGuard g(c->device);
  return kick_launch(c, vx, vy, vz, acc4, n, dt_kick);
}

int afd_leapfrog(afd_ctx *c, double *x, double *y, double *z, double *vx, double *vy,
                 double *vz, const double *m, int64_t n, float *acc4, double dt, int n_steps,
                 int n_reuse) {
  if (!c || n < 0 || n_steps < 0 || n_reuse < 1) return AFD_ERR_ARG;
  DeviceGuard g(c->device);
  for (int s = 0; s < n_steps; s++) {
    TRY(afd_kick_drift(c, x, y, z, vx, vy, vz, acc4, n, 0.5 * dt, dt));
    const int64_t k = (int64_t)s + 1;
    const bool rebuild = (k % n_reuse == 0) || !c->saved || c->n != n;
    TRY(calc_force_all(c, x, y, z, m, n, acc4,
                       rebuild ? AFD_MAKE_LIST_FOR_REUSE : AFD_REUSE_LIST));
    TRY(afd_kick(c, vx, vy, vz, acc4, n, 0.5 * dt));
  }
  return AFD_OK;
}

int afd_energy(afd_ctx *c, const double *vx, const double *vy, const double *vz,
               const double *m, const float *acc4, int64_t n, double *out) {
  if (!c || !out || n < 0) return AFD_ERR_ARG;
  out[0] = out[1] = 0.0;
  if (n == 0) return AFD_OK;
  if (!vx || !vy || !vz || !m || !acc4) return AFD_ERR_ARG;
  DeviceGuard g(c->device);
  TRY(reserve(c->red_part, sizeof(double) * 2 * kEnergyBlocks + 64));
  double *part = ptr<double>(c->red_part);
  double *res = part + 2 * kEnergyBlocks;
  int64_t nb = (n + kThreads - 1) / kThreads;
  if (nb > kEnergyBlocks) nb = kEnergyBlocks;
  k_energy<<<(unsigned)nb, kThreads, 0, c->stream>>>(vx, vy, vz, m,
                                                     reinterpret_cast<const float4 *>(acc4), n,
                                                     part, ptr<unsigned>(c->red_count), res);
  c->launches++;
  TRY(cuda_ok(cudaGetLastError()));
  double *pin = static_cast<double *>(c->pinned);
  TRY(cuda_ok(cudaMemcpyAsync(pin, res, 2 * sizeof(double), cudaMemcpyDeviceToHost, c->stream)));
  TRY(cuda_ok(cudaStreamSynchronize(c->stream)));
  out[0] = pin[0];
  out[1] = pin[1];
  return AFD_OK;
}

int afd_system_stats(afd_ctx *c, int64_t *inter, int64_t *entries) {
  if (!c || !inter || !entries) return AFD_ERR_ARG;
  if (!c->have_lists) return c->have_tree ? AFD_ERR_NO_SAVED_LIST : AFD_ERR_NO_TREE;
  DeviceGuard g(c->device);
  DevBuf tmp;
  const size_t b = sizeof(unsigned long long) * (size_t)c->n_sys;
  int st = reserve(tmp, 2 * b);
  if (st == AFD_OK) {
    unsigned long long *d = ptr<unsigned long long>(tmp);
    st = launch_sys_stats(c, d, d + c->n_sys);
    if (st == AFD_OK) st = cuda_ok(cudaStreamSynchronize(c->stream));
    if (st == AFD_OK) st = cuda_ok(cudaMemcpy(inter, d, b, cudaMemcpyDeviceToHost));
    if (st == AFD_OK) st = cuda_ok(cudaMemcpy(entries, d + c->n_sys, b, cudaMemcpyDeviceToHost));
  }
  release(tmp);
  return st;
}

int afd_graph_capture_step(afd_ctx *c, double *x, double *y, double *z, double *vx, double *vy,
                           double *vz, const double *m, float *acc4, double dt) {
  if (!c) return AFD_ERR_ARG;
  if (!c->saved || !c->have_lists) return AFD_ERR_NO_SAVED_LIST;
  if (c->stream == nullptr) return AFD_ERR_ARG;  // the legacy stream cannot be captured
  DeviceGuard g(c->device);
  graph_release(c);
  const int64_t n = c->n;
  if (c->cfg.mac) TRY(reserve(c->amag, sizeof(float) * (size_t)n));  // no allocation in capture
  if (!c->graph_done &&
      cudaEventCreateWithFlags(&c->graph_done, cudaEventDisableTiming) != cudaSuccess)
    return AFD_ERR_CUDA;
  // earlier work on the stream may still run: the capture records launches
  // only, and a replay is ordered after it on the stream
  if (cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaGetLastError();
    return AFD_ERR_CUDA;
  }
  const int64_t l0 = c->launches;
  int st = kick_drift_launch(c, x, y, z, vx, vy, vz, acc4, n, 0.5 * dt, dt);
  if (st == AFD_OK) st = reuse(c, x, y, z, m);
  if (st == AFD_OK) st = calc_force(c, acc4);
  if (st == AFD_OK) st = kick_launch(c, vx, vy, vz, acc4, n, 0.5 * dt);
  cudaGraph_t graph = nullptr;
  const cudaError_t ec = cudaStreamEndCapture(c->stream, &graph);
  if (st != AFD_OK || ec != cudaSuccess) {
    cudaGetLastError();
    if (graph) cudaGraphDestroy(graph);
    return st != AFD_OK ? st : AFD_ERR_CUDA;
  }
  c->graph = graph;
  if (cudaGraphInstantiate(&c->graph_exec, graph, 0) != cudaSuccess) {
    cudaGetLastError();
    graph_release(c);
    return AFD_ERR_CUDA;
  }
  c->graph_launches = c->launches - l0;
  c->launches = l0;
  return AFD_OK;
}

int afd_graph_launch(afd_ctx *c) {
  if (!c) return AFD_ERR_ARG;
  if (!c->graph_exec) return AFD_ERR_NO_SAVED_LIST;
  DeviceGuard g(c->device);
  TRY(cuda_ok(cudaGraphLaunch(c->graph_exec, c->stream)));
  TRY(cuda_ok(cudaEventRecord(c->graph_done, c->stream)));
  c->launches += c->graph_launches;
  return AFD_OK;
}

int afd_autotune_n_grp(afd_ctx *c, const double *x, const double *y, const double *z,
                       const double *m, int64_t n, const int32_t *cand, int n_cand, int n_reuse,
                       float *acc4, int32_t *best) {
  if (!c || !cand || n_cand < 1 || n_reuse < 1 || !best || (n > 0 && !acc4)) return AFD_ERR_ARG;
  for (int k = 0; k < n_cand; k++)
    if (cand[k] < 1 || cand[k] > 1024) return AFD_ERR_ARG;
  DeviceGuard g(c->device);
  const int ns = c->n_sys;
  const std::vector<int64_t> off = c->sys_off_h;
  std::vector<double> cost((size_t)ns * n_cand, 0.0);
  std::vector<int64_t> inter(ns), entries(ns);
  cudaEvent_t e[4];
  for (auto &ev : e)
    if (cudaEventCreate(&ev) != cudaSuccess) return AFD_ERR_CUDA;
  int st = AFD_OK;
  for (int k = 0; k < n_cand && st == AFD_OK; k++) {
    std::vector<int32_t> grp(ns, cand[k]);
    if (ns > 1) st = afd_set_systems(c, off.data(), ns, grp.data());
    else c->cfg.n_grp = cand[k];
    for (int rep = 0; rep < 2 && st == AFD_OK; rep++) {  // the first pass warms up
      cudaEventRecord(e[0], c->stream);
      st = tree_build(c, x, y, z, m, n);
      if (st == AFD_OK) st = make_lists(c, AFD_MAKE_LIST_FOR_REUSE);
      cudaEventRecord(e[1], c->stream);
      if (st == AFD_OK) st = calc_force(c, acc4);
      cudaEventRecord(e[2], c->stream);
    }
    if (st != AFD_OK) break;
    float t_build = 0.f, t_force = 0.f;
    cudaEventSynchronize(e[2]);
    cudaEventElapsedTime(&t_build, e[0], e[1]);
    cudaEventElapsedTime(&t_force, e[1], e[2]);
    st = afd_system_stats(c, inter.data(), entries.data());
    if (st != AFD_OK) break;
    double it = 0, en = 0;
    for (int s2 = 0; s2 < ns; s2++) {
      it += (double)inter[s2];
      en += (double)entries[s2];
    }
    for (int s2 = 0; s2 < ns; s2++) {
      // measured times shared out by each system's list entries / interactions
      const double cb = en > 0 ? t_build * (double)entries[s2] / en : 0.0;
      const double cf = it > 0 ? t_force * (double)inter[s2] / it : 0.0;
      cost[(size_t)s2 * n_cand + k] = cb / n_reuse + cf;
    }
  }
  for (auto &ev : e) cudaEventDestroy(ev);
  if (st != AFD_OK) return st;
  for (int s2 = 0; s2 < ns; s2++) {
    int kb = 0;
    for (int k = 1; k < n_cand; k++)
      if (cost[(size_t)s2 * n_cand + k] < cost[(size_t)s2 * n_cand + kb]) kb = k;
    best[s2] = cand[kb];
  }
  if (ns > 1) return afd_set_systems(c, off.data(), ns, best);
  c->cfg.n_grp = best[0];
  c->have_tree = c->have_lists = c->saved = c->u_order_ok = false;
  return AFD_OK;
}

int afd_set_launch(afd_ctx *c, int warps_per_block, int chunk) {
  if (!c || (warps_per_block != 2 && warps_per_block != 4 && warps_per_block != 8) ||
      (chunk != 32 && chunk != 64))
    return AFD_ERR_ARG;
  c->force_warps = warps_per_block;
  c->force_chunk = chunk;
  return AFD_OK;
}

int afd_get_launch(afd_ctx *c, int *warps_per_block, int *chunk) {
  if (!c || !warps_per_block || !chunk) return AFD_ERR_ARG;
  *warps_per_block = c->force_warps;
  *chunk = c->force_chunk;
  return AFD_OK;
}

int afd_autotune_launch(afd_ctx *c, float *acc4, int reps, float *ms_out) {
  if (!c || reps < 1 || (c->n > 0 && !acc4)) return AFD_ERR_ARG;
  if (!c->have_lists) return c->have_tree ? AFD_ERR_NO_SAVED_LIST : AFD_ERR_NO_TREE;
  DeviceGuard g(c->device);
  const int shapes[3] = {2, 4, 8}, chunks[2] = {32, 64};
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return AFD_ERR_CUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return AFD_ERR_CUDA;
  }
  int st = AFD_OK, bw = c->force_warps, bc = c->force_chunk;
  float best = 1e30f;
  for (int ci = 0; ci < 2 && st == AFD_OK; ci++)
    for (int wi = 0; wi < 3 && st == AFD_OK; wi++) {
      c->force_warps = shapes[wi];
      c->force_chunk = chunks[ci];
      st = launch_force(c, acc4);  // warm-up (and the one-time attribute set)
      if (st != AFD_OK) break;
      cudaEventRecord(e0, c->stream);
      for (int r = 0; r < reps && st == AFD_OK; r++) st = launch_force(c, acc4);
      cudaEventRecord(e1, c->stream);
      float ms = 0.0f;
      if (st == AFD_OK && (cudaEventSynchronize(e1) != cudaSuccess ||
                           cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
        st = AFD_ERR_CUDA;
      if (ms_out) ms_out[ci * 3 + wi] = ms / (float)reps;
      if (st == AFD_OK && ms < best) {
        best = ms;
        bw = shapes[wi];
        bc = chunks[ci];
      }
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  c->force_warps = bw;
  c->force_chunk = bc;
  return st;
}

int afd_calc_force_materialized(afd_ctx *c, float *acc4, float *ms_out) {
  if (!c || (c->n > 0 && !acc4)) return AFD_ERR_ARG;
  if (!c->have_lists) return c->have_tree ? AFD_ERR_NO_SAVED_LIST : AFD_ERR_NO_TREE;
  if (c->cfg.multipole) return AFD_ERR_ARG;  // monopole lists only
  DeviceGuard g(c->device);
  cudaEvent_t e[3];
  for (auto &ev : e)
    if (cudaEventCreate(&ev) != cudaSuccess) return AFD_ERR_CUDA;
  cudaEventRecord(e[0], c->stream);
  int st = launch_materialize(c);
  cudaEventRecord(e[1], c->stream);
  if (st == AFD_OK) st = launch_force_materialized(c, acc4);
  cudaEventRecord(e[2], c->stream);
  if (st == AFD_OK && cudaEventSynchronize(e[2]) != cudaSuccess) st = AFD_ERR_CUDA;
  if (st == AFD_OK && ms_out) {
    cudaEventElapsedTime(&ms_out[0], e[0], e[1]);
    cudaEventElapsedTime(&ms_out[1], e[1], e[2]);
  }
  for (auto &ev : e) cudaEventDestroy(ev);
  return st;
}

int afd_sync(afd_ctx *c) {
  if (!c) return AFD_ERR_ARG;
  DeviceGuard g(c->device);
  return read_status(c);
}

int afd_stats(afd_ctx *c, int64_t *out) {
  if (!c || !out) return AFD_ERR_ARG;
  out[0] = c->have_tree ? c->n : 0;
  out[1] = c->have_tree ? c->n_cells : 0;
  out[2] = c->have_tree ? c->n_groups : 0;
  out[3] = c->have_lists ? (int64_t)c->n_epj : 0;
  out[4] = c->have_lists ? (int64_t)c->n_spj : 0;
  out[5] = c->have_lists ? (int64_t)c->interactions : 0;
  out[6] = c->saved ? 1 : 0;
  out[7] = c->have_tree ? c->max_level : 0;
  out[8] = c->launches;
  out[9] = c->n_units;
  return AFD_OK;
}

int afd_export(afd_ctx *c, int what, void *host_buf, size_t *bytes) {
  if (!c || !bytes) return AFD_ERR_ARG;
  const void *src = nullptr;
  size_t sz = 0;
  const size_t n = (size_t)c->n, nc = (size_t)c->n_cells, ng = (size_t)c->n_groups;
  const bool tree = c->have_tree, lists = c->have_lists;
  switch (what) {
    case AFD_EXPORT_ROOT: src = c->root.p; sz = tree ? 4 * sizeof(double) * c->n_sys : 0; break;
    case AFD_EXPORT_KEYS: src = c->keys.p; sz = tree ? n * 8 : 0; break;
    case AFD_EXPORT_PERM: src = c->perm.p; sz = tree ? n * 4 : 0; break;
    case AFD_EXPORT_CELL_LEVEL: src = c->c_level.p; sz = tree ? nc * 4 : 0; break;
    case AFD_EXPORT_CELL_FIRST: src = c->c_first.p; sz = tree ? nc * 4 : 0; break;
    case AFD_EXPORT_CELL_COUNT: src = c->c_count.p; sz = tree ? nc * 4 : 0; break;
    case AFD_EXPORT_CELL_SKIP: src = c->c_skip.p; sz = tree ? nc * 4 : 0; break;
    case AFD_EXPORT_CELL_PARENT: src = c->c_parent.p; sz = tree ? nc * 4 : 0; break;
    case AFD_EXPORT_CELL_CHILD: src = c->c_child.p; sz = tree ? nc * 32 : 0; break;
    case AFD_EXPORT_CELL_MASS: src = c->c_mass.p; sz = tree ? nc * 8 : 0; break;
    case AFD_EXPORT_CELL_COM: src = c->c_com.p; sz = tree ? nc * 24 : 0; break;
    case AFD_EXPORT_CELL_QUAD: src = c->c_quad.p; sz = tree ? nc * 48 : 0; break;
    case AFD_EXPORT_GROUP_FIRST: src = c->g_first.p; sz = tree ? ng * 4 : 0; break;
    case AFD_EXPORT_GROUP_COUNT: src = c->g_count.p; sz = tree ? ng * 4 : 0; break;
    case AFD_EXPORT_GROUP_BOX: src = c->g_box.p; sz = tree ? ng * 48 : 0; break;
    case AFD_EXPORT_GROUP_SELF: src = c->g_self.p; sz = lists ? ng * 4 : 0; break;
    case AFD_EXPORT_EPJ_OFF: src = c->epj_off.p; sz = lists ? (ng + 1) * 8 : 0; break;
    case AFD_EXPORT_EPJ_IDX: src = c->epj.p; sz = lists ? (size_t)c->n_epj * 4 : 0; break;
    case AFD_EXPORT_SPJ_OFF: src = c->spj_off.p; sz = lists ? (ng + 1) * 8 : 0; break;
    case AFD_EXPORT_SPJ_IDX: src = c->spj.p; sz = lists ? (size_t)c->n_spj * 4 : 0; break;
    case AFD_EXPORT_NBR_OFF: src = c->nbr_off.p; sz = c->have_nbr ? (ng + 1) * 8 : 0; break;
    case AFD_EXPORT_NBR_IDX: src = c->nbr.p; sz = c->have_nbr ? (size_t)c->n_nbr * 4 : 0; break;
    case AFD_EXPORT_CELL_TBOX: src = c->c_tbox.p; sz = c->have_nbr ? nc * 32 : 0; break;
    case AFD_EXPORT_GROUP_SBOX: src = c->g_sbox.p; sz = c->have_nbr ? ng * 24 : 0; break;
    default: return AFD_ERR_ARG;
  }
  if (!host_buf) {
    *bytes = sz;
    return AFD_OK;
  }
  if (*bytes < sz) return AFD_ERR_ARG;
  *bytes = sz;
  if (sz == 0) return AFD_OK;
  DeviceGuard g(c->device);
  TRY(cuda_ok(cudaStreamSynchronize(c->stream)));
  return cuda_ok(cudaMemcpy(host_buf, src, sz, cudaMemcpyDeviceToHost));
}

int afd_last_force_ms(afd_ctx *c, float *ms) {
  if (!c || !ms) return AFD_ERR_ARG;
  *ms = 0.0f;
  if (!c->force_timed) return AFD_OK;
  DeviceGuard g(c->device);
  TRY(cuda_ok(cudaEventSynchronize(c->ev1)));
  return cuda_ok(cudaEventElapsedTime(ms, c->ev0, c->ev1));
}

const char *afd_error_string(int status) {
  switch (status) {
    case AFD_OK: return "ok";
    case AFD_ERR_ARG: return "invalid argument";
    case AFD_ERR_CUDA: return "CUDA runtime error";
    case AFD_ERR_NONFINITE: return "non-finite particle coordinate or mass";
    case AFD_ERR_NO_SAVED_LIST: return "no interaction lists saved for reuse";
    case AFD_ERR_SHAPE: return "particle count differs from the saved tree";
    case AFD_ERR_LIST_OVERFLOW: return "list or cell count exceeds 32-bit indexing";
    case AFD_ERR_TIMEOUT: return "bounded device wait or walk iteration limit reached";
    case AFD_ERR_NO_TREE: return "no tree built";
    case AFD_ERR_OOM: return "device allocation failed";
    case AFD_ERR_WALK_STACK: return "tree walk overflowed its stack";
    case AFD_ERR_TOO_LARGE: return "problem size above the static scratch limit (n <= 2^31 - 1)";
    case AFD_ERR_NO_REFERENCE:
      return "no reference accelerations for the current particles (learned opening criterion)";
    case AFD_ERR_BAD_RADIUS: return "search radius not finite and positive";
    default: return "unknown status";
  }
}

}  // extern "C"
