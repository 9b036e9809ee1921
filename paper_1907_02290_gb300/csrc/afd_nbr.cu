// Short-range neighbour walk and gather density (Section 2: short-range
// interactions such as SPH use the tree walk with a cell-opening criterion
// other than the opening angle; Section 4.2: their lists can be kept over
// several steps).
//
// Lists. Every cell gets its tight bounding box (k_nbr_tbox: leaves from
// their particles in FP64, rounded outward to FP32; internal cells from
// their children, bottom-up -- a finished cell counts itself at its parent
// and the last child to arrive combines the parent, writing its children's
// boxes by octant into a 256-byte block beside the walk's child records, so
// that an expansion step of the walk loads both at once). Every group gets its
// search box (k_nbr_sbox: per axis the min of x_i - (h_i + skin) and the
// max of x_i + (h_i + skin) over its particles, FP64 bounds rounded
// outward). The walk of afd_walk.cu in its neighbour mode then lists the
// particles of every leaf whose tight box meets the search box; cells that
// miss it are dropped with their subtrees, and a cell inside it is listed
// whole as its contiguous particle range. Outward rounding is monotone, so
// a parent's FP32 box contains its children's and the walk finds exactly
// the leaves a scan over all leaves would. Each group's walk is split into
// items, one per seed cell its search box meets (afd_walk.cu), so that a
// group whose box reaches across the system is walked by many warps.
//
// Density (k_density). Work item = (force work unit, segment of at most
// kSegLen list entries): a unit is a group's chunk of up to 32 particles (a
// chunk of r <= 16 splits the warp into S = 2 or 4 j-streams, lane = stream *
// (32 / S) + particle, as in the force kernel), and long lists -- sparse outer
// groups whose search boxes reach far -- are spread over several warps. One
// warp per item walks its segment 32 entries at a time: each lane gathers one
// j by index (hi/lo float4 pair) one chunk ahead and forms its coordinates
// relative to the group's first particle; the entries inside the unit's reach
// box (x_i -+ h_i over the unit's particles: the group's list is made for the
// whole group's search box) are staged with their masses in shared memory,
// compacted, the rest of the chunk padded far away and massless (two buffers,
// one __syncwarp per chunk; coordinates in separate arrays, each j-stream's
// entries consecutive). Every lane then tests its i against the chunk's j's of
// its stream four at a time -- two 16-byte loads per coordinate give two
// packed f32x2 pairs; r^2 and q^2 = r^2 / h_i^2 are 7 FP32 operations per pair
// in 3.5 issue slots -- and evaluates the spline for the four only when one of
// them has q^2 < 1: 1 / h_i and 8 / (pi h_i^3) in FP32, q by one sqrt.approx,
// w = 2 ((1 - q)^3 - 4 max(1/2 - q, 0)^3) in packed arithmetic. Sums per
// chunk, chunk sums added to the item's totals, then across streams. A unit of
// one segment writes its particles' results; a unit of several writes partial
// sums per item, which k_density_fin adds in segment order -- the result does
// not depend on scheduling.
#include <cfloat>
#include <cmath>
#include <cstring>

#include "afd_f32x2.cuh"
#include "afd_internal.cuh"
#include "afd_order.cuh"

namespace afd {
namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ int child_count(const uint32_t *child, uint32_t c) {
  int k = 0;
#pragma unroll
  for (int o = 0; o < 8; o++) k += __ldg(&child[(size_t)c * 8 + o]) != kNone ? 1 : 0;
  return k;
}

struct TboxArgs {
  int64_t n_cells;
  const uint32_t *first, *count, *parent, *child;
  const double *xs, *ys, *zs;
  float4 *tb;  // 2 per cell: (min x y z, 0), (max x y z, 0)
  float4 *blk;  // 16 per cell: its 8 children's boxes by octant (empty: lo > hi)
  uint32_t *arrive;
  uint64_t n_part;  // read only by the self-checking build
  int *status;      // kStClimb if the climb outruns the tree's depth
};

__global__ void __launch_bounds__(kThreads) k_nbr_tbox(TboxArgs a) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= a.n_cells) return;
  uint32_t c = (uint32_t)t;
  if (child_count(a.child, c) != 0) return;
  {
    const uint32_t f = a.first[c], e = f + a.count[c];
    if (e > f && !AFD_IN(e - 1, a.n_part, "tbox leaf range")) return;
    double lo[3] = {a.xs[f], a.ys[f], a.zs[f]}, hi[3] = {lo[0], lo[1], lo[2]};
    for (uint32_t k = f + 1; k < e; k++) {
      const double v[3] = {a.xs[k], a.ys[k], a.zs[k]};
#pragma unroll
      for (int d = 0; d < 3; d++) {
        lo[d] = fmin(lo[d], v[d]);
        hi[d] = fmax(hi[d], v[d]);
      }
    }
    a.tb[(size_t)c * 2] = make_float4(__double2float_rd(lo[0]), __double2float_rd(lo[1]),
                                      __double2float_rd(lo[2]), 0.0f);
    a.tb[(size_t)c * 2 + 1] = make_float4(__double2float_ru(hi[0]), __double2float_ru(hi[1]),
                                          __double2float_ru(hi[2]), 0.0f);
  }
  // a leaf of level l reaches the root in l climbs (at most kLevels)
  for (int round = 0;; round++) {
    const uint32_t p = a.parent[c];
    if (p == kNone) break;
    if (round > kLevels) {
      atomicOr(a.status, kStClimb);
      break;
    }
    if (!AFD_IN(p, a.n_cells, "tbox parent")) break;
    __threadfence();
    const unsigned old = atomicAdd(&a.arrive[p], 1u);
    if ((int)old != child_count(a.child, p) - 1) break;
    __threadfence();
    float4 lo = make_float4(INFINITY, INFINITY, INFINITY, 0.0f);
    float4 hi = make_float4(-INFINITY, -INFINITY, -INFINITY, 0.0f);
    for (int o = 0; o < 8; o++) {
      const uint32_t cc = __ldg(&a.child[(size_t)p * 8 + o]);
      float4 l = make_float4(INFINITY, INFINITY, INFINITY, 0.0f);
      float4 h = make_float4(-INFINITY, -INFINITY, -INFINITY, 0.0f);
      if (cc != kNone && AFD_IN(cc, a.n_cells, "tbox child")) {
        l = __ldcg(&a.tb[(size_t)cc * 2]);
        h = __ldcg(&a.tb[(size_t)cc * 2 + 1]);
        lo = make_float4(fminf(lo.x, l.x), fminf(lo.y, l.y), fminf(lo.z, l.z), 0.0f);
        hi = make_float4(fmaxf(hi.x, h.x), fmaxf(hi.y, h.y), fmaxf(hi.z, h.z), 0.0f);
      }
      a.blk[((size_t)p * 8 + o) * 2] = l;
      a.blk[((size_t)p * 8 + o) * 2 + 1] = h;
    }
    a.tb[(size_t)p * 2] = lo;
    a.tb[(size_t)p * 2 + 1] = hi;
    c = p;
  }
}

__device__ __forceinline__ float warp_minf(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ float warp_maxf(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

__device__ __forceinline__ bool radius_ok(double h) { return h > 0.0 && h <= DBL_MAX; }

// One warp per group: its search box.
__global__ void __launch_bounds__(kThreads) k_nbr_sbox(int64_t n_groups,
                                                       const uint32_t *__restrict__ g_first,
                                                       const uint32_t *__restrict__ g_count,
                                                       const uint32_t *__restrict__ perm,
                                                       const double *__restrict__ xs,
                                                       const double *__restrict__ ys,
                                                       const double *__restrict__ zs,
                                                       const double *__restrict__ h, double skin,
                                                       float *__restrict__ sbox, int *status,
                                                       uint64_t n_part) {
  const int64_t g = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (g >= n_groups) return;
  const uint32_t f = g_first[g], e = f + g_count[g];
  float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  bool bad = false;
  for (uint32_t k = f + lane; k < e; k += 32) {
    uint32_t o = perm[k];
    if (!AFD_IN(o, n_part, "sbox perm")) o = 0;
    const double hk = h[o];
    if (!radius_ok(hk)) {
      bad = true;
      continue;
    }
    const double r = __dadd_rn(hk, skin);
    const double v[3] = {xs[k], ys[k], zs[k]};
#pragma unroll
    for (int d = 0; d < 3; d++) {
      lo[d] = fminf(lo[d], __double2float_rd(__dsub_rn(v[d], r)));
      hi[d] = fmaxf(hi[d], __double2float_ru(__dadd_rn(v[d], r)));
    }
  }
  if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(status, kStBadRadius);
#pragma unroll
  for (int d = 0; d < 3; d++) {
    lo[d] = warp_minf(lo[d]);
    hi[d] = warp_maxf(hi[d]);
  }
  if (lane == 0)
#pragma unroll
    for (int d = 0; d < 3; d++) {
      sbox[g * 6 + d] = lo[d];
      sbox[g * 6 + 3 + d] = hi[d];
    }
}


__device__ __forceinline__ float sqrt_approx(float x) {
  float r;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// w / 2 of the spline for two pairs from their q^2 clamped to 1 (so that
// pairs beyond the support give 0), in packed arithmetic: with
// u = 1 - q and v = max(1/2 - q, 0), w = 2 (u^3 - 4 v^3), which is
// 1 - 6 q^2 + 6 q^3 for q <= 1/2 and 2 (1 - q)^3 above; the factor 2 is
// applied to the sums.
__device__ __forceinline__ f2 spline_half2(float c0, float c1) {
  const f2 one = pk(1.0f, 1.0f), m4 = pk(-4.0f, -4.0f);
  const float q0 = sqrt_approx(c0), q1 = sqrt_approx(c1);
  const f2 U = sub2(one, pk(q0, q1));
  const f2 V = pk(fmaxf(0.5f - q0, 0.0f), fmaxf(0.5f - q1, 0.0f));
  const f2 U3 = mul2(mul2(U, U), U), V3 = mul2(mul2(V, V), V);
  return fma2(V3, m4, U3);
}

// Density work item = (force work unit, segment of at most kSegLen list
// entries): long lists (sparse outer groups whose search boxes reach far)
// are spread over several warps instead of holding one warp for the whole
// kernel.
constexpr uint32_t kSegLen = 4096;
constexpr int kDensWarps = 8;
constexpr float kFar = 1e18f;  // staging pad: a massless j far outside any support

struct DensArgs {
  int64_t n_items;
  const uint2 *items;        // (unit, segment)
  const uint32_t *order;     // launch order of the items (null: index order)
  const uint32_t *seg_cnt;   // per unit: its segments
  const uint32_t *seg_off;   // per unit: its first item
  const uint2 *u_info;
  const uint32_t *g_first, *g_count;
  const float4 *jhi, *jlo;  // particles, Morton order (hi xyz + mass, lo xyz)
  const uint64_t *off;
  const uint32_t *idx;
  const uint32_t *perm;
  const double *h;  // caller order
  float *rho, *nnb;  // caller order; nnb may be null
  float2 *part;      // per item and lane: partial sums of a multi-segment unit
  int *status;
  // sizes, read only by the self-checking build
  uint64_t n, n_groups, n_list, n_units;
};

struct IParticle {
  uint32_t i, oi;
  bool act, bad;
  float xi, yi, zi, h, hinv, hinv2;
  float4 oh, ol;
};

__device__ __forceinline__ IParticle i_particle(const DensArgs &a, uint32_t g, uint32_t ioff,
                                                int p) {
  IParticle r;
  const uint32_t gf = a.g_first[g], gc = a.g_count[g];
  r.act = ioff + p < gc;
  r.i = gf + (r.act ? ioff + p : 0u);
  if (!AFD_IN(r.i, a.n, "density i")) r.i = 0;
  r.oh = a.jhi[gf];
  r.ol = a.jlo[gf];
  const float4 ih = a.jhi[r.i], il = a.jlo[r.i];
  r.xi = __fadd_rn(__fsub_rn(ih.x, r.oh.x), __fsub_rn(il.x, r.ol.x));
  r.yi = __fadd_rn(__fsub_rn(ih.y, r.oh.y), __fsub_rn(il.y, r.ol.y));
  r.zi = __fadd_rn(__fsub_rn(ih.z, r.oh.z), __fsub_rn(il.z, r.ol.z));
  r.oi = a.perm[r.i];
  if (!AFD_IN(r.oi, a.n, "density perm")) r.oi = 0;
  double hh = a.h[r.oi];
  r.bad = !radius_ok(hh);
  if (r.bad) hh = 1.0;
  r.h = __double2float_rn(hh);
  r.hinv = __frcp_rn(r.h);
  r.hinv2 = r.hinv * r.hinv;
  return r;
}

__device__ __forceinline__ void density_out(const DensArgs &a, const IParticle &ip, float tm,
                                            float tw) {
  // tm, tw are the sums of m_j w / 2 and w / 2
  const float sixteen_over_pi = 5.092958178940651f;  // 2 x 8 / pi
  a.rho[ip.oi] = ip.bad ? NAN : sixteen_over_pi * (ip.hinv2 * ip.hinv) * tm;
  if (a.nnb) a.nnb[ip.oi] = ip.bad ? NAN : (64.0f / 3.0f) * tw;
  if (ip.bad) atomicOr(a.status, kStBadRadius);
}

// Staging area of one warp: two buffers of 32 entries, coordinates and
// masses in separate arrays. Entry e of a chunk goes to slot (e % S) * W +
// e / S, so each j-stream's entries are consecutive and four of them are one
// 16-byte load: two packed pairs.
struct DensStage {
  float x[2][32], y[2][32], z[2][32], m[2][32];
};

template <int S>
__device__ __forceinline__ void density_item(const DensArgs &a, DensStage &st, int lane,
                                             int64_t item) {
  constexpr int W = 32 / S;
  const uint2 it = a.items[item];
  if (!AFD_IN(it.x, a.n_units, "density item unit")) return;
  const uint2 info = a.u_info[it.x];
  if (!AFD_IN(info.x, a.n_groups, "density unit group")) return;
  const uint32_t g = info.x, ioff = info.y & 0xffffu;
  const int p = lane & (W - 1), s = lane / W;
  const int slot = (lane % S) * W + lane / S;  // where this lane stages its entry
  const IParticle ip = i_particle(a, g, ioff, p);
  const f2 X = pk(ip.xi, ip.xi), Y = pk(ip.yi, ip.yi), Z = pk(ip.zi, ip.zi);
  const f2 H2 = pk(ip.hinv2, ip.hinv2);
  const uint64_t b0 = a.off[g] + (uint64_t)it.y * kSegLen;
  const uint64_t e = a.off[g + 1], b1 = e < b0 + kSegLen ? e : b0 + kSegLen;
  // the first chunk's gather
  float4 ph = make_float4(kFar, kFar, kFar, 0.0f), pl = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
  if (b0 + lane < b1) {
    uint32_t j = 0;
    if (AFD_IN(b0 + lane, a.n_list, "density list")) j = a.idx[b0 + lane];
    if (!AFD_IN(j, a.n, "density j")) j = 0;
    ph = a.jhi[j];
    pl = a.jlo[j];
  }
  // the unit's reach box: x_i -+ h_i over its particles, widened by a
  // relative 1e-5 (rounding slack; a pair dropped by it has q > 1 - 1e-5,
  // where w < 1e-14)
  float rb[6];
  {
    const bool use = ip.act && !ip.bad;
    const float hr = use ? ip.h * 1.00001f : 0.0f;
    rb[0] = use ? ip.xi - hr : INFINITY;
    rb[1] = use ? ip.yi - hr : INFINITY;
    rb[2] = use ? ip.zi - hr : INFINITY;
    rb[3] = use ? ip.xi + hr : -INFINITY;
    rb[4] = use ? ip.yi + hr : -INFINITY;
    rb[5] = use ? ip.zi + hr : -INFINITY;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
      for (int d = 0; d < 3; d++) {
        rb[d] = fminf(rb[d], __shfl_xor_sync(0xffffffffu, rb[d], o));
        rb[3 + d] = fmaxf(rb[3 + d], __shfl_xor_sync(0xffffffffu, rb[3 + d], o));
      }
  }
  const unsigned lt = (1u << lane) - 1u;
  float tm = 0.0f, tw = 0.0f;
  int buf = 0;
  for (uint64_t base = b0; base < b1; base += 32) {
    // stage the chunk's entries that reach the unit, compacted (relative
    // coordinates, mass), and pad the rest far away and massless
    const float rx = __fadd_rn(__fsub_rn(ph.x, ip.oh.x), __fsub_rn(pl.x, ip.ol.x));
    const float ry = __fadd_rn(__fsub_rn(ph.y, ip.oh.y), __fsub_rn(pl.y, ip.ol.y));
    const float rz = __fadd_rn(__fsub_rn(ph.z, ip.oh.z), __fsub_rn(pl.z, ip.ol.z));
    const bool keep = base + lane < b1 && rx >= rb[0] && rx <= rb[3] && ry >= rb[1] &&
                      ry <= rb[4] && rz >= rb[2] && rz <= rb[5];
    const unsigned km = __ballot_sync(0xffffffffu, keep);
    const int nkeep = __popc(km);
    if (keep) {
      const int e = __popc(km & lt);
      const int sl = (e % S) * W + e / S;
      st.x[buf][sl] = rx;
      st.y[buf][sl] = ry;
      st.z[buf][sl] = rz;
      st.m[buf][sl] = ph.w;
    }
    if (lane >= nkeep) {
      st.x[buf][slot] = kFar;
      st.y[buf][slot] = kFar;
      st.z[buf][slot] = kFar;
      st.m[buf][slot] = 0.0f;
    }
    __syncwarp();
    // the next chunk's gather, in flight while this one is evaluated
    const uint64_t nx = base + 32 + lane;
    if (nx < b1) {
      uint32_t j = 0;
      if (AFD_IN(nx, a.n_list, "density list")) j = a.idx[nx];
      if (!AFD_IN(j, a.n, "density j")) j = 0;
      ph = a.jhi[j];
      pl = a.jlo[j];
    }
    f2 cm2 = pk(0.0f, 0.0f), cw2 = cm2;  // per chunk, halves of the sums in two lanes
    // each stream's kept entries, four at a time (the pads make up the last four)
    const int kk = (((nkeep + S - 1) / S) + 3) & ~3;
    for (int k = 0; k < kk; k += 4) {
      const ulonglong2 xs = *reinterpret_cast<const ulonglong2 *>(&st.x[buf][s * W + k]);
      const ulonglong2 ys = *reinterpret_cast<const ulonglong2 *>(&st.y[buf][s * W + k]);
      const ulonglong2 zs = *reinterpret_cast<const ulonglong2 *>(&st.z[buf][s * W + k]);
      const f2 dx0 = sub2(xs.x, X), dy0 = sub2(ys.x, Y), dz0 = sub2(zs.x, Z);
      const f2 dx1 = sub2(xs.y, X), dy1 = sub2(ys.y, Y), dz1 = sub2(zs.y, Z);
      const f2 q0 = mul2(fma2(dz0, dz0, fma2(dy0, dy0, mul2(dx0, dx0))), H2);
      const f2 q1 = mul2(fma2(dz1, dz1, fma2(dy1, dy1, mul2(dx1, dx1))), H2);
      float qa, qb, qc, qd;
      upk(q0, qa, qb);
      upk(q1, qc, qd);
      if (fminf(fminf(qa, qb), fminf(qc, qd)) < 1.0f) {  // one of the four is inside
        const ulonglong2 ms = *reinterpret_cast<const ulonglong2 *>(&st.m[buf][s * W + k]);
        const f2 w01 = spline_half2(fminf(qa, 1.0f), fminf(qb, 1.0f));
        const f2 w23 = spline_half2(fminf(qc, 1.0f), fminf(qd, 1.0f));
        cm2 = fma2(ms.x, w01, cm2);
        cm2 = fma2(ms.y, w23, cm2);
        cw2 = add2(cw2, add2(w01, w23));
      }
    }
    float m0, m1, w0, w1;
    upk(cm2, m0, m1);
    upk(cw2, w0, w1);
    tm += m0 + m1;
    tw += w0 + w1;
    buf ^= 1;
  }
#pragma unroll
  for (int o = W; o < 32; o <<= 1) {
    tm += __shfl_xor_sync(0xffffffffu, tm, o);
    tw += __shfl_xor_sync(0xffffffffu, tw, o);
  }
  if (s != 0) return;
  if (a.seg_cnt[it.x] == 1) {
    if (ip.act) density_out(a, ip, tm, tw);
  } else {
    a.part[(size_t)item * 32 + p] = make_float2(tm, tw);
  }
}

__global__ void __launch_bounds__(kDensWarps * 32) k_density(DensArgs a) {
  __shared__ __align__(16) DensStage stage[kDensWarps];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t k = (int64_t)blockIdx.x * kDensWarps + w;
  if (k >= a.n_items) return;
  const int64_t item = a.order ? (int64_t)a.order[k] : k;
  if (!AFD_IN(item, (uint64_t)a.n_items, "density item order")) return;
  const uint32_t u = a.items[item].x;
  if (!AFD_IN(u, a.n_units, "density item unit")) return;
  const int sidx = (int)((a.u_info[u].y >> 16) & 3u);
  if (sidx == 0) density_item<1>(a, stage[w], lane, item);
  else if (sidx == 1) density_item<2>(a, stage[w], lane, item);
  else density_item<4>(a, stage[w], lane, item);
}

// Units of several segments: their partial sums added in segment order.
__global__ void __launch_bounds__(kThreads) k_density_fin(DensArgs a) {
  const int64_t u = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int p = threadIdx.x & 31;
  if (u >= (int64_t)a.n_units) return;
  const uint32_t ns = a.seg_cnt[u];
  if (ns <= 1) return;
  const uint2 info = a.u_info[u];
  if (!AFD_IN(info.x, a.n_groups, "density unit group")) return;
  const uint32_t ioff = info.y & 0xffffu;
  if (ioff + p >= a.g_count[info.x]) return;
  const IParticle ip = i_particle(a, info.x, ioff, p);
  float tm = 0.0f, tw = 0.0f;
  const uint32_t i0 = a.seg_off[u];
  for (uint32_t k = 0; k < ns; k++) {
    const float2 v = a.part[(size_t)(i0 + k) * 32 + p];
    tm += v.x;
    tw += v.y;
  }
  density_out(a, ip, tm, tw);
}

// Items of each unit: ceil(list length / kSegLen), at least one.
__global__ void k_seg_count(int64_t n_units, const uint2 *__restrict__ u_info,
                            const uint64_t *__restrict__ off, uint32_t *__restrict__ seg_cnt) {
  const int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (u >= n_units) return;
  const uint32_t g = u_info[u].x;
  const uint64_t len = off[g + 1] - off[g];
  const uint64_t ns = (len + kSegLen - 1) / kSegLen;
  seg_cnt[u] = ns > 0 ? (uint32_t)ns : 1u;
}

__global__ void k_seg_fill(int64_t n_units, const uint32_t *__restrict__ seg_cnt,
                           const uint32_t *__restrict__ seg_off, uint2 *__restrict__ items) {
  const int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (u >= n_units) return;
  for (uint32_t k = 0; k < seg_cnt[u]; k++) items[seg_off[u] + k] = make_uint2((uint32_t)u, k);
}

// Work of each density item: its segment's list entries per j-stream (the
// reach-box test runs over every entry); the items are launched largest
// work first (afd_order.cuh).
__global__ void k_dens_work(int64_t n_items, const uint2 *__restrict__ items,
                            const uint2 *__restrict__ u_info, const uint64_t *__restrict__ off,
                            uint32_t *__restrict__ work, uint32_t *__restrict__ hist) {
  uint32_t wmax = 0, cnt = 0;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n_items;
       k += (int64_t)gridDim.x * blockDim.x) {
    const uint2 it = items[k];
    const uint2 info = u_info[it.x];
    const uint32_t g = info.x;
    const uint64_t b0 = off[g] + (uint64_t)it.y * kSegLen, e = off[g + 1];
    const uint64_t len = e > b0 ? (e - b0 < kSegLen ? e - b0 : kSegLen) : 0u;
    const uint32_t w = (uint32_t)(len >> ((info.y >> 16) & 3u));
    work[k] = w;
    wmax = max(wmax, w);
    cnt++;
  }
  order_reduce(hist, wmax, cnt);
}

inline unsigned blocks_for(int64_t threads) { return (unsigned)((threads + kThreads - 1) / kThreads); }

int nbr_boxes(afd_ctx *c, const double *h, double skin) {
  const int64_t nc = c->n_cells, ng = c->n_groups;
  int st;
  if ((st = reserve(c->c_tbox, sizeof(float4) * 2 * (size_t)nc))) return st;
  if ((st = reserve(c->nbr_blk, sizeof(float4) * 16 * (size_t)nc))) return st;
  if ((st = reserve(c->nbr_arrive, sizeof(uint32_t) * (size_t)nc))) return st;
  if ((st = reserve(c->g_sbox, sizeof(float) * 6 * (size_t)ng))) return st;
  if (nc == 0) return AFD_OK;
  if (cudaMemsetAsync(c->nbr_arrive.p, 0, sizeof(uint32_t) * (size_t)nc, c->stream) != cudaSuccess)
    return AFD_ERR_CUDA;
  TboxArgs a;
  a.n_cells = nc;
  a.first = ptr<uint32_t>(c->c_first);
  a.count = ptr<uint32_t>(c->c_count);
  a.parent = ptr<uint32_t>(c->c_parent);
  a.child = ptr<uint32_t>(c->c_child);
  a.xs = ptr<double>(c->xs);
  a.ys = ptr<double>(c->ys);
  a.zs = ptr<double>(c->zs);
  a.tb = ptr<float4>(c->c_tbox);
  a.blk = ptr<float4>(c->nbr_blk);
  a.arrive = ptr<uint32_t>(c->nbr_arrive);
  a.n_part = (uint64_t)c->n;
  a.status = ptr<int>(c->status);
  k_nbr_tbox<<<blocks_for(nc), kThreads, 0, c->stream>>>(a);
  c->launches++;
  if (ng > 0) {
    k_nbr_sbox<<<blocks_for(ng * 32), kThreads, 0, c->stream>>>(
        ng, ptr<uint32_t>(c->g_first), ptr<uint32_t>(c->g_count), ptr<uint32_t>(c->perm),
        ptr<double>(c->xs), ptr<double>(c->ys), ptr<double>(c->zs), h, skin,
        ptr<float>(c->g_sbox), ptr<int>(c->status), (uint64_t)c->n);
    c->launches++;
  }
  return cudaGetLastError() == cudaSuccess ? AFD_OK : AFD_ERR_CUDA;
}

// Density work items of the current lists (synchronises once).
int nbr_items(afd_ctx *c) {
  const int64_t nu = c->n_units;
  int st;
  c->n_items = 0;
  c->nbr_multi = false;
  c->nbr_order_ok = false;
  if (nu == 0) return AFD_OK;
  if ((st = reserve(c->nbr_seg_cnt, sizeof(uint32_t) * (size_t)nu))) return st;
  if ((st = reserve(c->nbr_seg_off, sizeof(uint32_t) * (size_t)(nu + 1)))) return st;
  const uint32_t *cnt = ptr<uint32_t>(c->nbr_seg_cnt);
  uint32_t *off = ptr<uint32_t>(c->nbr_seg_off);
  k_seg_count<<<blocks_for(nu), kThreads, 0, c->stream>>>(nu, ptr<uint2>(c->u_info),
                                                          ptr<uint64_t>(c->nbr_off),
                                                          ptr<uint32_t>(c->nbr_seg_cnt));
  c->launches++;
  if (cudaGetLastError() != cudaSuccess) return AFD_ERR_CUDA;
  if ((st = scan_u32(c, cnt, off, nu))) return st;
  uint32_t *pin = static_cast<uint32_t *>(c->pinned);
  if (cudaMemcpyAsync(pin, off + nu, sizeof(uint32_t), cudaMemcpyDeviceToHost, c->stream) !=
          cudaSuccess ||
      cudaStreamSynchronize(c->stream) != cudaSuccess)
    return AFD_ERR_CUDA;
  c->n_items = pin[0];
  c->nbr_multi = c->n_items > nu;
  if ((st = reserve(c->nbr_items, sizeof(uint2) * (size_t)c->n_items))) return st;
  if (c->nbr_multi &&
      (st = reserve(c->nbr_part, sizeof(float2) * 32 * (size_t)c->n_items)))
    return st;
  k_seg_fill<<<blocks_for(nu), kThreads, 0, c->stream>>>(nu, cnt, off, ptr<uint2>(c->nbr_items));
  c->launches++;
  if (cudaGetLastError() != cudaSuccess) return AFD_ERR_CUDA;
  // the items' launch order, largest work first
  const int64_t ni = c->n_items;
  if (ni >= (int64_t)kOrderFlag) return AFD_OK;  // item ids need bit 31: index order
  if ((st = reserve(c->nbr_order, sizeof(uint32_t) * (size_t)ni))) return st;
  if ((st = reserve(c->nbr_work, sizeof(uint32_t) * (size_t)ni))) return st;
  if ((st = reserve(c->nbr_hist, sizeof(uint32_t) * (kOrderBuckets + 2)))) return st;
  uint32_t *hist = ptr<uint32_t>(c->nbr_hist), *work = ptr<uint32_t>(c->nbr_work);
  if (cudaMemsetAsync(hist, 0, sizeof(uint32_t) * (kOrderBuckets + 2), c->stream) != cudaSuccess)
    return AFD_ERR_CUDA;
  const int64_t want = (ni + kThreads - 1) / kThreads;
  k_dens_work<<<(unsigned)(want < 152 * 8 ? want : 152 * 8), kThreads, 0, c->stream>>>(
      ni, ptr<uint2>(c->nbr_items), ptr<uint2>(c->u_info), ptr<uint64_t>(c->nbr_off), work, hist);
  c->launches++;
  if (order_by_work(c->stream, ni, 0, work, hist, ptr<uint32_t>(c->nbr_order), &c->launches) !=
      cudaSuccess)
    return AFD_ERR_CUDA;
  c->nbr_order_ok = true;
  return AFD_OK;
}

// Make the device current for the call and restore the caller's afterwards.
struct DeviceScope {
  int prev = -1;
  bool ok = true;
  explicit DeviceScope(int dev) {
    int cur = 0;
    cudaGetDevice(&cur);
    if (cur != dev) {
      ok = cudaSetDevice(dev) == cudaSuccess;
      prev = cur;
    }
  }
  ~DeviceScope() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

}  // namespace
}  // namespace afd

using namespace afd;

extern "C" {

int afd_make_neighbour_lists(afd_ctx *c, const double *h, double skin) {
  if (!c) return AFD_ERR_ARG;
  if (!(skin >= 0.0) || !(skin <= DBL_MAX)) return AFD_ERR_ARG;
  if (!c->have_tree) return AFD_ERR_NO_TREE;
  if (c->n > 0 && !h) return AFD_ERR_ARG;
  DeviceScope scope(c->device);
  if (!scope.ok) return AFD_ERR_CUDA;
  c->have_nbr = false;
  int st;
  if ((st = nbr_boxes(c, h, skin))) return st;
  if ((st = launch_nbr_walk(c))) return st;  // reads (and clears) the status word
  if ((st = nbr_items(c))) return st;
  c->have_nbr = true;
  return AFD_OK;
}

int afd_calc_density(afd_ctx *c, const double *h, float *rho, float *nnb) {
  if (!c) return AFD_ERR_ARG;
  if (!c->have_nbr) return c->have_tree ? AFD_ERR_NO_SAVED_LIST : AFD_ERR_NO_TREE;
  if (c->n > 0 && (!h || !rho)) return AFD_ERR_ARG;
  if (c->n == 0 || c->n_units == 0) return AFD_OK;
  DeviceScope scope(c->device);
  if (!scope.ok) return AFD_ERR_CUDA;
  DensArgs a;
  a.n_items = c->n_items;
  a.items = ptr<uint2>(c->nbr_items);
  a.order = c->nbr_order_ok ? ptr<uint32_t>(c->nbr_order) : nullptr;
  a.seg_cnt = ptr<uint32_t>(c->nbr_seg_cnt);
  a.seg_off = ptr<uint32_t>(c->nbr_seg_off);
  a.u_info = ptr<uint2>(c->u_info);
  a.g_first = ptr<uint32_t>(c->g_first);
  a.g_count = ptr<uint32_t>(c->g_count);
  a.jhi = ptr<float4>(c->jhi);
  a.jlo = ptr<float4>(c->jlo);
  a.off = ptr<uint64_t>(c->nbr_off);
  a.idx = ptr<uint32_t>(c->nbr);
  a.perm = ptr<uint32_t>(c->perm);
  a.h = h;
  a.rho = rho;
  a.nnb = nnb;
  a.part = c->nbr_multi ? ptr<float2>(c->nbr_part) : nullptr;
  a.status = ptr<int>(c->status);
  a.n = (uint64_t)c->n;
  a.n_groups = (uint64_t)c->n_groups;
  a.n_list = c->n_nbr;
  a.n_units = (uint64_t)c->n_units;
  const unsigned nb = (unsigned)((c->n_items + kDensWarps - 1) / kDensWarps);
  k_density<<<nb, kDensWarps * 32, 0, c->stream>>>(a);
  c->launches++;
  if (c->nbr_multi) {
    k_density_fin<<<blocks_for(c->n_units * 32), kThreads, 0, c->stream>>>(a);
    c->launches++;
  }
  return cudaGetLastError() == cudaSuccess ? AFD_OK : AFD_ERR_CUDA;
}

int afd_neighbour_stats(afd_ctx *c, int64_t *out) {
  if (!c || !out) return AFD_ERR_ARG;
  out[0] = c->have_nbr ? (int64_t)c->n_nbr : 0;
  out[1] = c->have_nbr ? (int64_t)c->nbr_pairs : 0;
  return AFD_OK;
}

}  // extern "C"
