// Force kernel (Section 5: the indirect-index dispatch; Eq. kernel of
// Section 6.2). Work unit = (i-group, chunk of 32 of its particles); one
// warp per unit. The warp walks the group's EPJ list, then its SPJ list, 32
// entries at a time: each lane gathers one j by index (float4 hi + float4 lo
// of a particle or of a cell's centre of mass), forms its coordinates
// relative to the group centre, stages them in shared memory, and then every
// lane runs the 32 interactions against its own i-particle.
//
// Precision. Positions are FP64 in memory. Group-relative coordinates are
// formed from hi/lo FP32 pairs, (x_hi - c_hi) + (x_lo - c_lo): when x and c
// are close the hi difference is exact (Sterbenz) and the result equals the
// FP64 difference rounded to FP32 up to the tiny lo terms; when they are far
// apart the relative rounding error is that of one FP32 operation. The
// pairwise term is FP32 with a hardware reciprocal square root. Each chunk's
// 32 terms are summed in FP32 and the chunk sums are accumulated with Kahan
// compensation.
//
// Per interaction: 3 FADD (dx), 3 FFMA (r^2), 1 MUFU.RSQ, 3 FMUL, 3 FFMA (a),
// 1 FADD (phi) -- 23 flops by the paper's convention (Section 6.2, n_op).
#include "afd_internal.cuh"

namespace afd {
namespace {

constexpr int kForceWarps = 4;
constexpr int kForceThreads = 32 * kForceWarps;

struct ForceArgs {
  int64_t n_units;
  const uint32_t *u_group, *u_off;
  const uint32_t *g_first, *g_count, *g_self;
  const float4 *g_chi, *g_clo;
  const float4 *jhi, *jlo;  // particles, Morton order
  const float4 *shi, *slo;  // cells
  const float4 *sq0, *sq1;  // cell quadrupoles
  const uint64_t *off_e, *off_s;
  const uint32_t *epj, *spj;
  const uint32_t *perm;
  float eps2;
  float4 *out;
};

__device__ __forceinline__ float rsqrt_fast(float x) {
  float r;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ void kahan_add(float &s, float &c, float v) {
  const float y = v - c;
  const float t = s + y;
  c = (t - s) - y;
  s = t;
}

struct Acc {
  float x = 0.f, y = 0.f, z = 0.f, p = 0.f;     // running sums
  float cx = 0.f, cy = 0.f, cz = 0.f, cp = 0.f; // Kahan compensation
};

template <bool GUARD>
__device__ __forceinline__ void interact(float4 j, float xi, float yi, float zi, float eps2,
                                         float &px, float &py, float &pz, float &pp) {
  const float dx = j.x - xi, dy = j.y - yi, dz = j.z - zi;
  const float r2 = fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, eps2)));
  float rinv = rsqrt_fast(r2);
  if (GUARD) rinv = r2 > 0.0f ? rinv : 0.0f;
  const float mr = j.w * rinv;
  const float mr3 = mr * rinv * rinv;
  px = fmaf(mr3, dx, px);
  py = fmaf(mr3, dy, py);
  pz = fmaf(mr3, dz, pz);
  pp += mr;
}

// Quadrupole term of one cell (Q about its COM, r = x_i - COM = -d):
//   phi -= (1/2) r.Q.r / rs^5,  a += Q r / rs^5 - (5/2) (r.Q.r) r / rs^7.
template <bool GUARD>
__device__ __forceinline__ void interact_quad(float4 j, float4 q0, float4 q1, float xi, float yi,
                                              float zi, float eps2, float &px, float &py,
                                              float &pz, float &pp) {
  const float dx = j.x - xi, dy = j.y - yi, dz = j.z - zi;
  const float r2 = fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, eps2)));
  float rinv = rsqrt_fast(r2);
  if (GUARD) rinv = r2 > 0.0f ? rinv : 0.0f;
  const float rinv2 = rinv * rinv;
  const float mr = j.w * rinv;
  const float mr3 = mr * rinv2;
  // monopole
  px = fmaf(mr3, dx, px);
  py = fmaf(mr3, dy, py);
  pz = fmaf(mr3, dz, pz);
  pp += mr;
  // quadrupole with r = -d: Q r = -(Q d), r.Q.r = d.Q.d
  const float qdx = fmaf(q0.x, dx, fmaf(q0.w, dy, q1.x * dz));
  const float qdy = fmaf(q0.w, dx, fmaf(q0.y, dy, q1.y * dz));
  const float qdz = fmaf(q1.x, dx, fmaf(q1.y, dy, q0.z * dz));
  const float dqd = fmaf(dx, qdx, fmaf(dy, qdy, dz * qdz));
  const float rinv5 = rinv2 * rinv2 * rinv;
  const float rinv7 = rinv5 * rinv2;
  // a = -(Q d)/rs^5 + (5/2)(d.Q.d) d / rs^7
  const float t = 2.5f * dqd * rinv7;
  px = fmaf(t, dx, fmaf(-rinv5, qdx, px));
  py = fmaf(t, dy, fmaf(-rinv5, qdy, py));
  pz = fmaf(t, dz, fmaf(-rinv5, qdz, pz));
  pp = fmaf(0.5f * dqd, rinv5, pp);
}

template <bool GUARD, bool QUAD>
__global__ void __launch_bounds__(kForceThreads) k_force(ForceArgs a) {
  __shared__ float4 jbuf[kForceWarps][32];
  __shared__ float4 qbuf0[QUAD ? kForceWarps : 1][32];
  __shared__ float4 qbuf1[QUAD ? kForceWarps : 1][32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t u = (int64_t)blockIdx.x * kForceWarps + w;
  if (u >= a.n_units) return;
  const uint32_t g = a.u_group[u];
  const uint32_t chunk = (uint32_t)u - a.u_off[g];
  const uint32_t gf = a.g_first[g], gc = a.g_count[g];
  const uint32_t il = chunk * 32u + lane;
  const bool active = il < gc;
  const uint32_t i = gf + il;
  const float4 ch = a.g_chi[g], cl = a.g_clo[g];
  float xi = 0.f, yi = 0.f, zi = 0.f, mi = 0.f;
  if (active) {
    const float4 h = a.jhi[i], l = a.jlo[i];
    xi = (h.x - ch.x) + (l.x - cl.x);
    yi = (h.y - ch.y) + (l.y - cl.y);
    zi = (h.z - ch.z) + (l.z - cl.z);
    mi = h.w;
  }
  Acc acc;
  const float eps2 = a.eps2;
  // ---- EPJ list: particles ----
  {
    const uint64_t o0 = a.off_e[g], o1 = a.off_e[g + 1];
    for (uint64_t base = o0; base < o1; base += 32) {
      const uint64_t k = base + lane;
      float4 r = make_float4(1e18f, 1e18f, 1e18f, 0.0f);
      if (k < o1) {
        const uint32_t j = a.epj[k];
        const float4 h = a.jhi[j], l = a.jlo[j];
        r = make_float4((h.x - ch.x) + (l.x - cl.x), (h.y - ch.y) + (l.y - cl.y),
                        (h.z - ch.z) + (l.z - cl.z), h.w);
      }
      __syncwarp();
      jbuf[w][lane] = r;
      __syncwarp();
      float px = 0.f, py = 0.f, pz = 0.f, pp = 0.f;
#pragma unroll 8
      for (int t = 0; t < 32; t++) interact<GUARD>(jbuf[w][t], xi, yi, zi, eps2, px, py, pz, pp);
      kahan_add(acc.x, acc.cx, px);
      kahan_add(acc.y, acc.cy, py);
      kahan_add(acc.z, acc.cz, pz);
      kahan_add(acc.p, acc.cp, pp);
    }
  }
  // ---- SPJ list: cells (monopole, optionally quadrupole) ----
  {
    const uint64_t o0 = a.off_s[g], o1 = a.off_s[g + 1];
    for (uint64_t base = o0; base < o1; base += 32) {
      const uint64_t k = base + lane;
      float4 r = make_float4(1e18f, 1e18f, 1e18f, 0.0f);
      float4 q0 = make_float4(0.f, 0.f, 0.f, 0.f), q1 = q0;
      if (k < o1) {
        const uint32_t j = a.spj[k];
        const float4 h = a.shi[j], l = a.slo[j];
        r = make_float4((h.x - ch.x) + (l.x - cl.x), (h.y - ch.y) + (l.y - cl.y),
                        (h.z - ch.z) + (l.z - cl.z), h.w);
        if (QUAD) {
          q0 = a.sq0[j];
          q1 = a.sq1[j];
        }
      }
      __syncwarp();
      jbuf[w][lane] = r;
      if (QUAD) {
        qbuf0[w][lane] = q0;
        qbuf1[w][lane] = q1;
      }
      __syncwarp();
      float px = 0.f, py = 0.f, pz = 0.f, pp = 0.f;
      if (QUAD) {
#pragma unroll 4
        for (int t = 0; t < 32; t++)
          interact_quad<GUARD>(jbuf[w][t], qbuf0[w][t], qbuf1[w][t], xi, yi, zi, eps2, px, py, pz, pp);
      } else {
#pragma unroll 8
        for (int t = 0; t < 32; t++) interact<GUARD>(jbuf[w][t], xi, yi, zi, eps2, px, py, pz, pp);
      }
      kahan_add(acc.x, acc.cx, px);
      kahan_add(acc.y, acc.cy, py);
      kahan_add(acc.z, acc.cz, pz);
      kahan_add(acc.p, acc.cp, pp);
    }
  }
  if (!active) return;
  // Remove the self pair (dx = 0 exactly, so it added m_i / eps to phi only).
  if (!GUARD && a.g_self[g]) {
    const float r2 = fmaf(0.0f, 0.0f, fmaf(0.0f, 0.0f, fmaf(0.0f, 0.0f, eps2)));
    kahan_add(acc.p, acc.cp, -(mi * rsqrt_fast(r2)));
  }
  a.out[a.perm[i]] = make_float4(acc.x, acc.y, acc.z, -acc.p);
}

}  // namespace

int launch_force(afd_ctx *c, float *acc4) {
  if (c->n == 0 || c->n_units == 0) return AFD_OK;
  ForceArgs a;
  a.n_units = c->n_units;
  a.u_group = ptr<uint32_t>(c->u_group);
  a.u_off = ptr<uint32_t>(c->u_off);
  a.g_first = ptr<uint32_t>(c->g_first);
  a.g_count = ptr<uint32_t>(c->g_count);
  a.g_self = ptr<uint32_t>(c->g_self);
  a.g_chi = ptr<float4>(c->g_chi);
  a.g_clo = ptr<float4>(c->g_clo);
  a.jhi = ptr<float4>(c->jhi);
  a.jlo = ptr<float4>(c->jlo);
  a.shi = ptr<float4>(c->s_hi);
  a.slo = ptr<float4>(c->s_lo);
  a.sq0 = ptr<float4>(c->s_q0);
  a.sq1 = ptr<float4>(c->s_q1);
  a.off_e = ptr<uint64_t>(c->epj_off);
  a.off_s = ptr<uint64_t>(c->spj_off);
  a.epj = ptr<uint32_t>(c->epj);
  a.spj = ptr<uint32_t>(c->spj);
  a.perm = ptr<uint32_t>(c->perm);
  const float e = (float)c->cfg.eps;
  a.eps2 = e * e;
  a.out = reinterpret_cast<float4 *>(acc4);
  const unsigned nb = (unsigned)((c->n_units + kForceWarps - 1) / kForceWarps);
  const bool guard = !(a.eps2 > 0.0f);
  cudaEventRecord(c->ev0, c->stream);
  if (c->cfg.multipole) {
    if (guard) k_force<true, true><<<nb, kForceThreads, 0, c->stream>>>(a);
    else k_force<false, true><<<nb, kForceThreads, 0, c->stream>>>(a);
  } else if (guard) {
    k_force<true, false><<<nb, kForceThreads, 0, c->stream>>>(a);
  } else {
    k_force<false, false><<<nb, kForceThreads, 0, c->stream>>>(a);
  }
  c->launches++;
  cudaEventRecord(c->ev1, c->stream);
  c->force_timed = true;
  return cudaGetLastError() == cudaSuccess ? AFD_OK : AFD_ERR_CUDA;
}

}  // namespace afd
