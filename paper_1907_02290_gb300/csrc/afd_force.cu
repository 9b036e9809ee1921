// Force kernel (Section 5: the indirect-index dispatch; Eq. kernel of
// Section 6.2). Work unit = (i-group, chunk of 32 of its particles); a warp
// takes one work item: a unit, or two consecutive units of one group (a full
// one and the next if that holds more than 16 particles), which share the
// group's list, each lane then holding two i-particles. The warp walks the group's EPJ list, then its SPJ list, 32 or
// 64 entries at a time (a launch choice): each lane gathers its j's by index
// (float4 hi + float4 lo of a particle or of a cell's centre of mass), forms
// their coordinates relative to the group origin, stages them in shared
// memory, and then every lane runs the chunk's interactions against its own
// i-particle(s). The gathers of the next chunk are issued before the current
// chunk is computed. The items are launched largest list work first.
//
// Packed arithmetic: each lane evaluates two j's (an even and an odd slot
// of the chunk) against an i in one pass of f32x2 instructions -- 13
// packed FP32 operations and two MUFU.RSQ per two interactions -- which
// halves the issue slots of the scalar loop.
//
// Self pairs: a group's own particles form one contiguous run of its EPJ
// list (recorded by the walk); in the chunks holding that run each lane gives
// its own pair zero mass, so nothing has to be subtracted afterwards.
//
// Precision. Positions are FP64 in memory. Coordinates relative to the
// group origin (the centre of mass of the group's cell) are formed from
// hi/lo FP32 pairs, (x_hi - c_hi) + (x_lo - c_lo): when x and c are close
// the hi difference is exact (Sterbenz) and the result equals the FP64
// difference rounded to FP32 up to the tiny lo terms; when they are far
// apart the relative rounding error is that of one FP32 operation. The
// terms are summed in packed FP32 accumulators (with one i-particle per
// lane, two of them over alternate j-pairs), and every 128 packed pairs the
// partial sums are folded into Kahan-compensated accumulators.
//
// Per interaction: 3 FADD (dx), 3 FFMA (r^2), 1 MUFU.RSQ, 3 FMUL, 3 FFMA (a),
// 1 FADD (phi) -- 23 flops by the paper's convention (Section 6.2, n_op).
#include "afd_f32x2.cuh"
#include "afd_internal.cuh"
#include "afd_order.cuh"

namespace afd {
namespace {

#ifndef AFD_FORCE_MAX_REGS
#define AFD_FORCE_MAX_REGS 96  // register budget of the monopole kernel (5 blocks of 4 warps per SM)
#endif
#ifndef AFD_FORCE_ILP2
#define AFD_FORCE_ILP2 1  // two independent accumulator chains per lane
#endif
#ifndef AFD_FORCE_FLUSH_PAIRS
#define AFD_FORCE_FLUSH_PAIRS 128  // pair-iterations per lane between Kahan flushes
#endif
#ifndef AFD_FORCE_PAIRS
#define AFD_FORCE_PAIRS 1  // two units of a group per warp
#endif
#ifndef AFD_FORCE_UNIT_IPT2
#define AFD_FORCE_UNIT_IPT2 1  // units of their own also two i-particles per lane
#endif
#ifndef AFD_FORCE_QUAD_IPT2
#define AFD_FORCE_QUAD_IPT2 1  // the quadrupole kernel also two i-particles per lane
#endif
#ifndef AFD_FORCE_QUAD_REGS
#define AFD_FORCE_QUAD_REGS 112  // register budget of the quadrupole kernel
#endif
#ifndef AFD_FORCE_PERSISTENT
#define AFD_FORCE_PERSISTENT 0  // warps take units from an atomic queue
#endif


struct ForceArgs {
  int64_t n_units;  // the launch covers units [u_base, n_units)
  const uint32_t *u_order;  // their launch order (null: index order)
  const uint32_t *n_items;  // entries of the launch order (device)
  int64_t u_base;
  unsigned long long *queue;  // work counter of the persistent variant (zeroed per launch)
  const uint2 *u_info;
  const uint32_t *g_first, *g_count, *g_self, *g_cell;
  const float4 *jhi, *jlo;  // j-particles, Morton order (or materialised lists)
  const float4 *ihi, *ilo;  // i-particles, Morton order
  const float4 *ohi, *olo;  // cells, for the group origin
  const float4 *shi, *slo;  // cells
  const float4 *sq0, *sq1;  // cell quadrupoles
  const uint4 *sh;          // half-precision far field: -Q/(M s^2) as half2 words, s^2
  const float *gscale;      // half-precision far field: per-group power-of-two scale
  const uint64_t *off_e, *off_s;
  const uint32_t *epj, *spj;
  const uint32_t *perm;
  float eps2;
  float4 *out;
  // sizes, read only by the self-checking build
  uint64_t n, n_cells, n_groups, n_epj, n_spj;
};

__device__ __forceinline__ float rsqrt_fast(float x) {
  float r;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// One lane, one i-particle, two j's (an even and an odd slot of the chunk)
// per packed instruction: 13 f32x2 operations and 2 MUFU.RSQ for two
// interactions.
template <bool GUARD>
__device__ __forceinline__ void interact2(float4 a, float4 b, f2 XI, f2 YI, f2 ZI, f2 E2, f2 &AX,
                                          f2 &AY, f2 &AZ, f2 &PP) {
  const f2 DX = sub2(pk(a.x, a.y), XI);
  const f2 DY = sub2(pk(a.z, a.w), YI);
  const f2 DZ = sub2(pk(b.x, b.y), ZI);
  const f2 R2 = fma2(DX, DX, fma2(DY, DY, fma2(DZ, DZ, E2)));
  float r0, r1;
  upk(R2, r0, r1);
  float q0 = rsqrt_fast(r0), q1 = rsqrt_fast(r1);
  if (GUARD) {
    q0 = r0 > 0.0f ? q0 : 0.0f;
    q1 = r1 > 0.0f ? q1 : 0.0f;
  }
  const f2 RI = pk(q0, q1);
  const f2 MR = mul2(pk(b.z, b.w), RI);
  const f2 MR3 = mul2(mul2(MR, RI), RI);
  AX = fma2(MR3, DX, AX);
  AY = fma2(MR3, DY, AY);
  AZ = fma2(MR3, DZ, AZ);
  PP = add2(PP, MR);
}

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"(smem_addr(dst)), "l"(src));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N));
}

// Monopole + quadrupole of two cells (even, odd) against one i, packed.
// With d = COM - x_i (so r = x_i - COM = -d): Q r = -(Q d), r.Q.r = d.Q.d,
//   a += M d / rs^3 - (Q d) / rs^5 + (5/2)(d.Q.d) d / rs^7,
//   phi_sum += M / rs + (1/2)(d.Q.d) / rs^5   (phi = -phi_sum).
template <bool GUARD>
__device__ __forceinline__ void interact_quad2(float4 a, float4 b, float4 qa, float4 qb,
                                               float4 qc, f2 XI, f2 YI, f2 ZI, f2 E2, f2 &AX,
                                               f2 &AY, f2 &AZ, f2 &PP) {
  const f2 DX = sub2(pk(a.x, a.y), XI);
  const f2 DY = sub2(pk(a.z, a.w), YI);
  const f2 DZ = sub2(pk(b.x, b.y), ZI);
  const f2 R2 = fma2(DX, DX, fma2(DY, DY, fma2(DZ, DZ, E2)));
  float r0, r1;
  upk(R2, r0, r1);
  float q0 = rsqrt_fast(r0), q1 = rsqrt_fast(r1);
  if (GUARD) {
    q0 = r0 > 0.0f ? q0 : 0.0f;
    q1 = r1 > 0.0f ? q1 : 0.0f;
  }
  const f2 RI = pk(q0, q1);
  const f2 RI2 = mul2(RI, RI);
  const f2 MR = mul2(pk(b.z, b.w), RI);
  const f2 MR3 = mul2(MR, RI2);
  const f2 QXX = pk(qa.x, qa.y), QYY = pk(qa.z, qa.w), QZZ = pk(qb.x, qb.y);
  const f2 QXY = pk(qb.z, qb.w), QXZ = pk(qc.x, qc.y), QYZ = pk(qc.z, qc.w);
  const f2 QDX = fma2(QXX, DX, fma2(QXY, DY, mul2(QXZ, DZ)));
  const f2 QDY = fma2(QXY, DX, fma2(QYY, DY, mul2(QYZ, DZ)));
  const f2 QDZ = fma2(QXZ, DX, fma2(QYZ, DY, mul2(QZZ, DZ)));
  const f2 DQD = fma2(DX, QDX, fma2(DY, QDY, mul2(DZ, QDZ)));
  const f2 RI5 = mul2(mul2(RI2, RI2), RI);
  const f2 RI7 = mul2(RI5, RI2);
  const f2 K = fma2(mul2(pk(2.5f, 2.5f), DQD), RI7, MR3);  // M/rs^3 + 2.5 dQd/rs^7
  const f2 NRI5 = sub2(pk(0.0f, 0.0f), RI5);
  AX = fma2(K, DX, fma2(NRI5, QDX, AX));
  AY = fma2(K, DY, fma2(NRI5, QDY, AY));
  AZ = fma2(K, DZ, fma2(NRI5, QDZ, AZ));
  PP = fma2(mul2(pk(0.5f, 0.5f), DQD), RI5, add2(PP, MR));
}

// ---- packed half precision (BF16 or FP16) for the far field
template <int FAR>  // 1: bf16x2, 2: f16x2
__device__ __forceinline__ uint32_t h2_from_f2(f2 v) {
  float a, b;
  upk(v, a, b);
  uint32_t r;
  if (FAR == 1) asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(b), "f"(a));
  else asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(b), "f"(a));
  return r;
}
template <int FAR>
__device__ __forceinline__ uint32_t hfma2(uint32_t a, uint32_t b, uint32_t c) {
  uint32_t d;
  if (FAR == 1) asm("fma.rn.bf16x2 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
  else asm("fma.rn.f16x2 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
  return d;
}
template <int FAR>
__device__ __forceinline__ uint32_t hmul2(uint32_t a, uint32_t b) {
  uint32_t d;
  if (FAR == 1) asm("mul.rn.bf16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
  else asm("mul.rn.f16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
  return d;
}
template <int FAR>
__device__ __forceinline__ uint32_t hconst2(float v) {
  return h2_from_f2<FAR>(pk(v, v));
}
// c + a b for the two halves of half-precision pairs a, b (BF16 or FP16)
// into the FP32 pair c: the product of two such values is exact in FP32,
// so each half is one rounding to FP32 (mixed-precision FMA), with no
// half-precision product or conversion between.
template <int FAR>
__device__ __forceinline__ f2 fma_h2_f32(uint32_t a, uint32_t b, f2 c) {
  float c0, c1;
  upk(c, c0, c1);
  if (FAR == 1)
    asm("{.reg .b16 a0, a1, b0, b1;\n\t"
        "mov.b32 {a0, a1}, %2;\n\t"
        "mov.b32 {b0, b1}, %3;\n\t"
        "fma.rn.f32.bf16 %0, a0, b0, %0;\n\t"
        "fma.rn.f32.bf16 %1, a1, b1, %1;}"
        : "+f"(c0), "+f"(c1)
        : "r"(a), "r"(b));
  else
    asm("{.reg .b16 a0, a1, b0, b1;\n\t"
        "mov.b32 {a0, a1}, %2;\n\t"
        "mov.b32 {b0, b1}, %3;\n\t"
        "fma.rn.f32.f16 %0, a0, b0, %0;\n\t"
        "fma.rn.f32.f16 %1, a1, b1, %1;}"
        : "+f"(c0), "+f"(c1)
        : "r"(a), "r"(b));
  return pk(c0, c1);
}

// Monopole + quadrupole of two cells (even, odd) against one i, the whole
// far-field term formed in half precision. With d = COM - x_i, rs^2 = |d|^2 +
// eps^2, u = d / rs (|u| <= 1), sigma = s^2 / rs^2 (< theta^2 for an
// accepted cell), the dimensionless shape Qn = Q / (M s^2), P = -Qn u (from
// the cell's stored -Qn) and T = u.P = -u.Qn.u, the monopole plus the
// softened quadrupole term (Q r / rs^5 - 2.5 (r.Q.r) r / rs^7 with r = -d,
// and -0.5 r.Q.r / rs^5) are
//   a = (M / rs^2) [u + sigma (P - 2.5 T u)],
//   phi_sum = (M / rs) (1 - 0.5 sigma T)           (phi = -phi_sum).
// The geometry (d, rs, u, sigma) is FP32; u, sigma, the shape and the
// magnitude M' / rs^2 are rounded to half precision and the bracket is
// half-precision arithmetic; its product with the magnitude goes straight
// into the FP32 sums by a mixed-precision FMA (fma_h2_f32; likewise the
// potential's quadrupole correction with M' / rs rounded to half). The
// group's scale (computed by the list walk): M' = M 2^-k_g carries the
// group's power-of-two scale (2^k_g >= the largest M / d^2 over the group's
// far-field cells), so every magnitude is at most about 1 and the FP16
// range (2^16 above that, 2^-24 below) holds the group's terms; the
// accumulators are multiplied by 2^k_g when folded. The monopole potential
// M' / rs stays FP32.
template <bool GUARD, int FAR>
__device__ __forceinline__ void interact_far_half(float4 a, float4 b, uint4 qa, uint2 qb, f2 S2,
                                                  f2 XI, f2 YI, f2 ZI, f2 E2, f2 &AX, f2 &AY,
                                                  f2 &AZ, f2 &PP) {
  const f2 DX = sub2(pk(a.x, a.y), XI);
  const f2 DY = sub2(pk(a.z, a.w), YI);
  const f2 DZ = sub2(pk(b.x, b.y), ZI);
  const f2 R2 = fma2(DX, DX, fma2(DY, DY, fma2(DZ, DZ, E2)));
  float r0, r1;
  upk(R2, r0, r1);
  float q0 = rsqrt_fast(r0), q1 = rsqrt_fast(r1);
  if (GUARD) {
    q0 = r0 > 0.0f ? q0 : 0.0f;
    q1 = r1 > 0.0f ? q1 : 0.0f;
  }
  const f2 RI = pk(q0, q1);
  const f2 MR = mul2(pk(b.z, b.w), RI);  // M' / rs
  const f2 RI2 = mul2(RI, RI);
  const uint32_t MU = h2_from_f2<FAR>(mul2(MR, RI));   // M' / rs^2
  const uint32_t SG = h2_from_f2<FAR>(mul2(S2, RI2));  // s^2 / rs^2
  const uint32_t UX = h2_from_f2<FAR>(mul2(DX, RI));
  const uint32_t UY = h2_from_f2<FAR>(mul2(DY, RI));
  const uint32_t UZ = h2_from_f2<FAR>(mul2(DZ, RI));
  // qa = (xx, yy, zz, xy), qb = (xz, yz) of -Q / (M s^2), each an (even, odd) pair
  const uint32_t PX = hfma2<FAR>(qa.x, UX, hfma2<FAR>(qa.w, UY, hmul2<FAR>(qb.x, UZ)));
  const uint32_t PY = hfma2<FAR>(qa.w, UX, hfma2<FAR>(qa.y, UY, hmul2<FAR>(qb.y, UZ)));
  const uint32_t PZ = hfma2<FAR>(qb.x, UX, hfma2<FAR>(qb.y, UY, hmul2<FAR>(qa.z, UZ)));
  const uint32_t T = hfma2<FAR>(UX, PX, hfma2<FAR>(UY, PY, hmul2<FAR>(UZ, PZ)));
  const uint32_t C = hmul2<FAR>(hconst2<FAR>(-2.5f), T);
  const uint32_t BX = hfma2<FAR>(SG, hfma2<FAR>(C, UX, PX), UX);
  const uint32_t BY = hfma2<FAR>(SG, hfma2<FAR>(C, UY, PY), UY);
  const uint32_t BZ = hfma2<FAR>(SG, hfma2<FAR>(C, UZ, PZ), UZ);
  // the products accumulated straight into the FP32 sums
  AX = fma_h2_f32<FAR>(MU, BX, AX);
  AY = fma_h2_f32<FAR>(MU, BY, AY);
  AZ = fma_h2_f32<FAR>(MU, BZ, AZ);
  const uint32_t PQ = hmul2<FAR>(hmul2<FAR>(hconst2<FAR>(-0.5f), SG), T);
  // the quadrupole correction (M' / rs) PQ, M' / rs rounded to half precision
  PP = fma_h2_f32<FAR>(h2_from_f2<FAR>(MR), PQ, add2(PP, MR));
}

// Shared-memory staging of one warp: raw j data of two chunks in flight
// (double buffer filled by cp.async) and the packed pair layout of the chunk
// being computed:
//   P0[p] = (x_2p, x_2p+1, y_2p, y_2p+1), P1[p] = (z_2p, z_2p+1, m_2p, m_2p+1).
// CH: list entries per staged chunk (32 or 64, a launch choice); each lane
// stages CH / 32 entries; CH / 2 packed pairs per chunk.
template <bool QUAD, int CH>
struct WarpStage {
  static constexpr int kPairs = CH / 2;
  float4 rh[2][CH], rl[2][CH];
  // quadrupoles (FP32), or (half-precision far field) in rq0 the cell's
  // half record
  float4 rq0[QUAD ? 2 : 1][QUAD ? CH : 1], rq1[QUAD ? 2 : 1][QUAD ? CH : 1];
  float4 P0[kPairs], P1[kPairs];
  // quadrupole pairs: QA = (xx, yy), QB = (zz, xy), QC = (xz, yz), each (even, odd)
  float4 QA[QUAD ? kPairs : 1], QB[QUAD ? kPairs : 1], QC[QUAD ? kPairs : 1];
  // half-precision far field: negated normalised quadrupole pairs (xx, yy, zz, xy),
  // (xz, yz) as (even, odd) half2 words, and the cell side squared of both cells
  uint4 HA[QUAD ? kPairs : 1];
  uint2 HB[QUAD ? kPairs : 1];
  float2 S2[QUAD ? kPairs : 1];
  float4 ch, cl;  // origin of the relative coordinates (hi, lo)
};

// Per-lane state: IPT i-particles (coordinates duplicated in both halves of
// a packed pair) and eps^2.
template <int IPT>
struct Lane {
  int lane, stream;
  f2 XI[IPT], YI[IPT], ZI[IPT];
  f2 E2;
};

// Kahan-compensated running sums of one i-particle (both packed streams folded).
struct Sums {
  float v[4], c[4];  // sx sy sz sp; their compensations
};
__device__ __forceinline__ void sums_init(Sums &s) {
#pragma unroll
  for (int k = 0; k < 4; k++) s.v[k] = s.c[k] = 0.0f;
}
__device__ __forceinline__ void kahan_fold_k(Sums &s, int k, f2 v) {
  float v0, v1;
  upk(v, v0, v1);
  const float y = (v0 + v1) - s.c[k];
  const float t = s.v[k] + y;
  s.c[k] = (t - s.v[k]) - y;
  s.v[k] = t;
}
__device__ __forceinline__ float sums_value(const Sums &s, int k) { return s.v[k] - s.c[k]; }

// Issue the asynchronous gather of list entries [base, base + CH) into
// buffer b: lane l copies entries base + l + 32 r (lanes past the end copy
// nothing). j[r] are the entries' indices.
// With the half-precision far field a far-field entry is 32 bytes: the
// cell's (COM hi, M) and its half record; the COM's lo part is left out (it
// moves the relative coordinate by 2^-24 of the COM's magnitude, far below
// half precision).
template <bool QUAD, int FAR, int CH>
__device__ __forceinline__ void gather(WarpStage<QUAD, CH> &st, int b, int lane, uint64_t base,
                                       uint64_t o1, const uint32_t *j, const float4 *hi,
                                       const float4 *lo, const float4 *sq0, const float4 *sq1,
                                       const uint4 *sh, bool quad_list) {
#pragma unroll
  for (int r = 0; r < CH / 32; r++) {
    const int slot = lane + 32 * r;
    if (base + slot < o1) {
      cp_async16(&st.rh[b][slot], hi + j[r]);
      if (QUAD && quad_list && FAR) {
        cp_async16(&st.rq0[b][slot], sh + j[r]);
      } else {
        cp_async16(&st.rl[b][slot], lo + j[r]);
        if (QUAD && quad_list) {
          cp_async16(&st.rq0[b][slot], sq0 + j[r]);
          cp_async16(&st.rq1[b][slot], sq1 + j[r]);
        }
      }
    }
  }
  cp_async_commit();
}

template <int CH>
__device__ __forceinline__ void load_idx(uint32_t *j, const uint32_t *idx, uint64_t base,
                                         uint64_t o1, int lane, uint64_t jbound) {
#pragma unroll
  for (int r = 0; r < CH / 32; r++) {
    const uint64_t k = base + lane + 32 * r;
    // idx null: the j-data are materialised in list order (the non-indirect
    // ablation), so the entry's own position is its index
    j[r] = k < o1 ? (idx ? idx[k] : (uint32_t)k) : 0u;
    if (!AFD_IN(j[r], jbound, "force list entry")) j[r] = 0u;
  }
}

// One list (EPJ or SPJ) of one group for one warp with S j-streams.
// With the half-precision far field (FAR, quadrupole SPJ list) the masses
// are scaled by the group's power of two gsc on staging and the partial
// sums multiplied back by 1 / gsc (exact) when folded.
template <bool GUARD, bool QUAD, int FAR, int S, int IPT, int CH>
__device__ __forceinline__ void run_list(WarpStage<QUAD, CH> &st, const Lane<IPT> &ln, Sums *sm,
                                         const uint32_t *idx, uint64_t o0, uint64_t o1,
                                         const float4 *hi, const float4 *lo, const float4 *sq0,
                                         const float4 *sq1, const uint4 *sh, bool quad_list,
                                         float eps2, const int64_t *self_at, uint64_t nlist,
                                         uint64_t jbound, float gsc) {
  if (o0 >= o1) return;
  if (!AFD_IN(o1 - 1, nlist, "force list range")) return;
  constexpr int kChunk = CH, kPer = CH / 32, kPairs = CH / 2;
  const int lane = ln.lane;
  const f2 Z0 = pk(0.0f, 0.0f);
  // prologue: chunk 0 in flight, indices of chunk 1 in registers
  uint32_t j0[kPer], jn[kPer];
  load_idx<CH>(j0, idx, o0, o1, lane, jbound);
  const bool half_far = QUAD && FAR && quad_list;
  const f2 unscale = pk(1.0f / gsc, 1.0f / gsc);  // powers of two: exact
  gather<QUAD, FAR, CH>(st, 0, lane, o0, o1, j0, hi, lo, sq0, sq1, sh, quad_list);
  load_idx<CH>(jn, idx, o0 + kChunk, o1, lane, jbound);
  f2 AX[IPT], AY[IPT], AZ[IPT], PP[IPT];
#pragma unroll
  for (int q = 0; q < IPT; q++) AX[q] = AY[q] = AZ[q] = PP[q] = Z0;
  int pending = 0;  // pair-iterations accumulated since the last Kahan flush
  int b = 0;
  for (uint64_t base = o0; base < o1; base += kChunk) {
    // next chunk in flight, indices of the one after in registers
    const uint64_t nb = base + kChunk;
    gather<QUAD, FAR, CH>(st, b ^ 1, lane, nb, o1, jn, hi, lo, sq0, sq1, sh, quad_list);
    load_idx<CH>(jn, idx, nb + kChunk, o1, lane, jbound);
    cp_async_wait<1>();  // this lane's copies of the current chunk have landed
    float rx[kPer], ry[kPer], rz[kPer], rm[kPer];
    const float4 ch = st.ch, cl = st.cl;
#pragma unroll
    for (int r = 0; r < kPer; r++) {
      // relative coordinates of this lane's j (far, massless padding past the end)
      const int slot = lane + 32 * r;
      rx[r] = ry[r] = rz[r] = 1e18f;
      rm[r] = 0.0f;
      if (base + slot < o1) {
        const float4 h = st.rh[b][slot];
        if (half_far) {  // COM hi only; the mass carries the group's scale
          rx[r] = (h.x - ch.x) - cl.x;
          ry[r] = (h.y - ch.y) - cl.y;
          rz[r] = (h.z - ch.z) - cl.z;
          rm[r] = h.w * gsc;
        } else {
          const float4 l = st.rl[b][slot];
          rx[r] = (h.x - ch.x) + (l.x - cl.x);
          ry[r] = (h.y - ch.y) + (l.y - cl.y);
          rz[r] = (h.z - ch.z) + (l.z - cl.z);
          rm[r] = h.w;
        }
      }
    }
    __syncwarp();
#pragma unroll
    for (int r = 0; r < kPer; r++) {
      const int slot = lane + 32 * r;
      float *p0 = reinterpret_cast<float *>(&st.P0[slot >> 1]);
      float *p1 = reinterpret_cast<float *>(&st.P1[slot >> 1]);
      const int e = slot & 1;
      p0[e] = rx[r];
      p0[2 + e] = ry[r];
      p1[e] = rz[r];
      p1[2 + e] = rm[r];
      if (QUAD && quad_list && FAR) {
        // the cell's half record: (xx, yy), (zz, xy), (xz, yz) of -Qn as
        // half2 words, s^2; this lane's half of each (even, odd) pair
        const bool v = base + slot < o1;
        const uint4 rec = v ? *reinterpret_cast<const uint4 *>(&st.rq0[b][slot])
                            : make_uint4(0u, 0u, 0u, 0u);
        unsigned short *ha = reinterpret_cast<unsigned short *>(&st.HA[slot >> 1]);
        unsigned short *hb = reinterpret_cast<unsigned short *>(&st.HB[slot >> 1]);
        ha[0 + e] = (unsigned short)(rec.x & 0xffffu);  // xx
        ha[2 + e] = (unsigned short)(rec.x >> 16);      // yy
        ha[4 + e] = (unsigned short)(rec.y & 0xffffu);  // zz
        ha[6 + e] = (unsigned short)(rec.y >> 16);      // xy
        hb[0 + e] = (unsigned short)(rec.z & 0xffffu);  // xz
        hb[2 + e] = (unsigned short)(rec.z >> 16);      // yz
        reinterpret_cast<float *>(&st.S2[slot >> 1])[e] = __uint_as_float(rec.w);
      } else if (QUAD && quad_list) {
        const bool v = base + slot < o1;
        const float4 q0 = v ? st.rq0[b][slot] : make_float4(0.f, 0.f, 0.f, 0.f);
        const float4 q1 = v ? st.rq1[b][slot] : make_float4(0.f, 0.f, 0.f, 0.f);
        float *qa = reinterpret_cast<float *>(&st.QA[slot >> 1]);
        float *qb = reinterpret_cast<float *>(&st.QB[slot >> 1]);
        float *qc = reinterpret_cast<float *>(&st.QC[slot >> 1]);
        qa[e] = q0.x;      // xx
        qa[2 + e] = q0.y;  // yy
        qb[e] = q0.z;      // zz
        qb[2 + e] = q0.w;  // xy
        qc[e] = q1.x;      // xz
        qc[2 + e] = q1.y;  // yz
      }
    }
    __syncwarp();
    // does some lane's own particle sit in this chunk? (every lane votes)
    bool self_here = false;
#pragma unroll
    for (int q = 0; q < IPT; q++)
      self_here |= self_at[q] >= (int64_t)base && self_at[q] < (int64_t)base + kChunk;
    const bool any_self = __any_sync(0xffffffffu, self_here);
    if (QUAD && quad_list && FAR) {
#pragma unroll (IPT == 1 ? 4 : 2)
      for (int t = ln.stream; t < kPairs; t += S) {
        const float4 p0 = st.P0[t], p1 = st.P1[t];
        const uint4 ha = st.HA[t];
        const uint2 hb = st.HB[t];
        const f2 s2 = pk(st.S2[t].x, st.S2[t].y);
#pragma unroll
        for (int q = 0; q < IPT; q++)
          interact_far_half<GUARD, FAR ? FAR : 1>(p0, p1, ha, hb, s2, ln.XI[q], ln.YI[q],
                                                  ln.ZI[q], ln.E2, AX[q], AY[q], AZ[q], PP[q]);
      }
    } else if (QUAD && quad_list) {
#pragma unroll (IPT == 1 ? 4 : 2)
      for (int t = ln.stream; t < kPairs; t += S) {
        const float4 p0 = st.P0[t], p1 = st.P1[t], qa = st.QA[t], qb = st.QB[t], qc = st.QC[t];
#pragma unroll
        for (int q = 0; q < IPT; q++)
          interact_quad2<GUARD>(p0, p1, qa, qb, qc, ln.XI[q], ln.YI[q], ln.ZI[q], ln.E2, AX[q],
                                AY[q], AZ[q], PP[q]);
      }
    } else if (any_self) {
      // a chunk holding some lane's own particle: that pair gets zero mass
      int ts[IPT];
#pragma unroll
      for (int q = 0; q < IPT; q++) {
        const bool h = self_at[q] >= (int64_t)base && self_at[q] < (int64_t)base + kChunk;
        ts[q] = h ? (int)(self_at[q] - (int64_t)base) : -1;
      }
#pragma unroll
      for (int t = ln.stream; t < kPairs; t += S) {
        const float4 p0 = st.P0[t], p1 = st.P1[t];
#pragma unroll
        for (int q = 0; q < IPT; q++) {
          float4 p1q = p1;
          if (ts[q] == 2 * t) p1q.z = 0.0f;
          if (ts[q] == 2 * t + 1) p1q.w = 0.0f;
          interact2<GUARD>(p0, p1q, ln.XI[q], ln.YI[q], ln.ZI[q], ln.E2, AX[q], AY[q], AZ[q],
                           PP[q]);
        }
      }
    } else if (IPT == 2) {
      // two i-particles per lane: each staged pair serves both (two chains)
#pragma unroll 2
      for (int t = ln.stream; t < kPairs; t += S) {
        const float4 p0 = st.P0[t], p1 = st.P1[t];
#pragma unroll
        for (int q = 0; q < IPT; q++)
          interact2<GUARD>(p0, p1, ln.XI[q], ln.YI[q], ln.ZI[q], ln.E2, AX[q], AY[q], AZ[q],
                           PP[q]);
      }
    } else if (AFD_FORCE_ILP2 && S == 1) {
      f2 BX = Z0, BY = Z0, BZ = Z0, BP = Z0;
#pragma unroll
      for (int t = 0; t < kPairs; t += 2) {
        interact2<GUARD>(st.P0[t], st.P1[t], ln.XI[0], ln.YI[0], ln.ZI[0], ln.E2, AX[0], AY[0],
                         AZ[0], PP[0]);
        interact2<GUARD>(st.P0[t + 1], st.P1[t + 1], ln.XI[0], ln.YI[0], ln.ZI[0], ln.E2, BX, BY,
                         BZ, BP);
      }
      AX[0] = add2(AX[0], BX);
      AY[0] = add2(AY[0], BY);
      AZ[0] = add2(AZ[0], BZ);
      PP[0] = add2(PP[0], BP);
    } else {
#pragma unroll
      for (int t = ln.stream; t < kPairs; t += S)
        interact2<GUARD>(st.P0[t], st.P1[t], ln.XI[0], ln.YI[0], ln.ZI[0], ln.E2, AX[0], AY[0],
                         AZ[0], PP[0]);
    }
    pending += kPairs / S;
    if (pending >= AFD_FORCE_FLUSH_PAIRS || nb >= o1) {
#pragma unroll
      for (int q = 0; q < IPT; q++) {
        if (half_far) {
          AX[q] = mul2(AX[q], unscale);
          AY[q] = mul2(AY[q], unscale);
          AZ[q] = mul2(AZ[q], unscale);
          PP[q] = mul2(PP[q], unscale);
        }
        kahan_fold_k(sm[q], 0, AX[q]);
        kahan_fold_k(sm[q], 1, AY[q]);
        kahan_fold_k(sm[q], 2, AZ[q]);
        kahan_fold_k(sm[q], 3, PP[q]);
        AX[q] = AY[q] = AZ[q] = PP[q] = Z0;
      }
      pending = 0;
    }
    b ^= 1;
  }
  cp_async_wait<0>();
  __syncwarp();
}

template <bool GUARD, bool QUAD, int FAR, int S, int IPT, int CH>
__device__ __forceinline__ void run_unit(WarpStage<QUAD, CH> &st, const ForceArgs &a, uint32_t g,
                                         const Lane<IPT> &ln, Sums *sm, const int64_t *self_at) {
  run_list<GUARD, QUAD, FAR, S, IPT, CH>(st, ln, sm, a.epj, a.off_e[g], a.off_e[g + 1], a.jhi,
                                         a.jlo, nullptr, nullptr, nullptr, false, a.eps2,
                                         self_at, a.n_epj, a.epj ? a.n : a.n_epj, 1.0f);
  int64_t none[IPT];
#pragma unroll
  for (int q = 0; q < IPT; q++) none[q] = -1;
  const float gsc = (QUAD && FAR) ? a.gscale[g] : 1.0f;
  run_list<GUARD, QUAD, FAR, S, IPT, CH>(st, ln, sm, a.spj, a.off_s[g], a.off_s[g + 1], a.shi,
                                         a.slo, a.sq0, a.sq1, a.sh, QUAD, a.eps2, none, a.n_spj,
                                         a.spj ? a.n_cells : a.n_spj, gsc);
}

// One work unit with IPT particles per lane and S j-streams: set up the
// lanes' i-particles, run both lists, combine the streams and write.
template <bool GUARD, bool QUAD, int FAR, int S, int IPT, int CH>
__device__ __forceinline__ void unit_body(const ForceArgs &a, WarpStage<QUAD, CH> &st, int lane,
                                          uint32_t g, uint32_t ioff) {
  constexpr int W = 32 / S;
  Lane<IPT> ln;
  ln.lane = lane;
  ln.stream = lane / W;
  const uint32_t gf = a.g_first[g], gc = a.g_count[g];
  // origin of the relative coordinates: the group cell's centre of mass
  uint32_t gcell = a.g_cell[g];
  if (!AFD_IN(gcell, a.n_cells, "force group cell")) gcell = 0u;
  const float4 ch = a.ohi[gcell], cl = a.olo[gcell];
  if (lane == 0) {
    st.ch = ch;
    st.cl = cl;
  }
  uint32_t il[IPT];
  bool active[IPT];
#pragma unroll
  for (int q = 0; q < IPT; q++) {
    il[q] = ioff + (uint32_t)(q * W + (lane & (W - 1)));
    active[q] = il[q] < gc && AFD_IN(gf + il[q], a.n, "force i-particle");
    float xi = 0.f, yi = 0.f, zi = 0.f;
    if (active[q]) {
      const float4 h = a.ihi[gf + il[q]], l = a.ilo[gf + il[q]];
      xi = (h.x - ch.x) + (l.x - cl.x);
      yi = (h.y - ch.y) + (l.y - cl.y);
      zi = (h.z - ch.z) + (l.z - cl.z);
    }
    ln.XI[q] = pk(xi, xi);
    ln.YI[q] = pk(yi, yi);
    ln.ZI[q] = pk(zi, zi);
  }
  ln.E2 = pk(a.eps2, a.eps2);
  Sums sm[IPT];
#pragma unroll
  for (int q = 0; q < IPT; q++) sums_init(sm[q]);
  __syncwarp();
  // EPJ-list positions of this lane's own particles (-1: not on the list)
  const uint32_t gs = a.g_self[g];
  int64_t self_at[IPT];
#pragma unroll
  for (int q = 0; q < IPT; q++)
    self_at[q] =
        (gs && active[q]) ? (int64_t)a.off_e[g] + (int64_t)(gs - 1u) + (int64_t)il[q] : -1;
  run_unit<GUARD, QUAD, FAR, S, IPT, CH>(st, a, g, ln, sm, self_at);
#pragma unroll
  for (int q = 0; q < IPT; q++) {
    float ax = sums_value(sm[q], 0), ay = sums_value(sm[q], 1), az = sums_value(sm[q], 2);
    float pot = sums_value(sm[q], 3);
    // combine the j-streams of each particle
#pragma unroll
    for (int o = W; o < 32; o <<= 1) {
      ax += __shfl_xor_sync(0xffffffffu, ax, o);
      ay += __shfl_xor_sync(0xffffffffu, ay, o);
      az += __shfl_xor_sync(0xffffffffu, az, o);
      pot += __shfl_xor_sync(0xffffffffu, pot, o);
    }
    if (active[q] && ln.stream == 0) {
      const uint32_t o = a.perm[gf + il[q]];
      if (AFD_IN(o, a.n, "force output")) a.out[o] = make_float4(ax, ay, az, -pot);
    }
  }
}

// Work unit u: group g = info.x; info.y holds the first particle offset
// (bits 0-15) and log2 of the j-stream split S (bits 16-17): S = 1 << sidx
// streams of W = 32 >> sidx particles, lane = stream * W + particle. The
// monopole kernel runs such a unit as 2 S streams of W / 2 lanes, each lane
// with two of the unit's particles (the same lanes busy, every staged
// j-pair serving two i-particles); a pair item (a full unit and the next)
// as one stream of 32 lanes with two particles each.
template <bool GUARD, bool QUAD, int FAR, int CH>
__device__ __forceinline__ void force_unit(const ForceArgs &a, WarpStage<QUAD, CH> &st, int lane,
                                           int64_t u, bool pair) {
  const uint2 info = a.u_info[u];
  if (!AFD_IN(info.x, a.n_groups, "force unit group")) return;
  const uint32_t g = info.x, ioff = info.y & 0xffffu;
  const int sidx = (int)((info.y >> 16) & 3u);
  if (!QUAD || AFD_FORCE_QUAD_IPT2) {
    if (pair) {
      unit_body<GUARD, QUAD, FAR, 1, 2, CH>(a, st, lane, g, ioff);
      return;
    }
    if (AFD_FORCE_UNIT_IPT2) {
      if (sidx == 0) unit_body<GUARD, QUAD, FAR, 2, 2, CH>(a, st, lane, g, ioff);
      else if (sidx == 1) unit_body<GUARD, QUAD, FAR, 4, 2, CH>(a, st, lane, g, ioff);
      else unit_body<GUARD, QUAD, FAR, 8, 2, CH>(a, st, lane, g, ioff);
      return;
    }
  }
  if (sidx == 0) unit_body<GUARD, QUAD, FAR, 1, 1, CH>(a, st, lane, g, ioff);
  else if (sidx == 1) unit_body<GUARD, QUAD, FAR, 2, 1, CH>(a, st, lane, g, ioff);
  else unit_body<GUARD, QUAD, FAR, 4, 1, CH>(a, st, lane, g, ioff);
}

// The work item at launch position k: without a launch order, unit
// u_base + k; with one, entry k of the order (false: past the last item).
// An entry is a unit index, bit 31 set when the warp also takes the group's
// next unit (two i-particles per lane).
__device__ __forceinline__ bool launch_item(const ForceArgs &a, int64_t k, int64_t &u, bool &pair) {
  pair = false;
  if (!a.u_order) {
    u = a.u_base + k;
    return u < a.n_units;
  }
  if (k >= (int64_t)*a.n_items) return false;
  const uint32_t e = a.u_order[k];
  u = (int64_t)(e & 0x7fffffffu);
  pair = (e >> 31) != 0u;
  return AFD_IN(u, (uint64_t)a.n_units, "force unit order");
}

// Block shape is a launch choice (2, 4 or 8 warps): each warp's staging area
// lives in dynamic shared memory. The register budget is the same for every
// shape: 96 per thread with FP32 monopoles, 112 with quadrupoles (two
// i-particles per lane in both; 104 and 128 measured slower).
constexpr int kForceMaxThreads = 256;

template <bool GUARD, bool QUAD, int FAR, int CH>
__global__ void __launch_bounds__(kForceMaxThreads) __maxnreg__(QUAD ? AFD_FORCE_QUAD_REGS : AFD_FORCE_MAX_REGS)
    k_force(ForceArgs a) {
  extern __shared__ __align__(16) unsigned char force_smem[];
  WarpStage<QUAD, CH> *stage = reinterpret_cast<WarpStage<QUAD, CH> *>(force_smem);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (AFD_FORCE_PERSISTENT) {
    for (;;) {
      unsigned long long k = 0;
      if (lane == 0) k = atomicAdd(a.queue, 1ull);
      k = __shfl_sync(0xffffffffu, k, 0);
      int64_t u;
      bool pair;
      if ((int64_t)k + a.u_base >= a.n_units || !launch_item(a, (int64_t)k, u, pair)) return;
      force_unit<GUARD, QUAD, FAR, CH>(a, stage[w], lane, u, pair);
      __syncwarp();
    }
  } else {
    const int64_t k = (int64_t)blockIdx.x * nw + w;
    int64_t u;
    bool pair;
    if (a.u_base + k >= a.n_units || !launch_item(a, k, u, pair)) return;
    force_unit<GUARD, QUAD, FAR, CH>(a, stage[w], lane, u, pair);
  }
}

template <bool GUARD, bool QUAD, int FAR, int CH>
int launch_k_force(const ForceArgs &a, unsigned nb, int warps, cudaStream_t s) {
  const size_t smem = sizeof(WarpStage<QUAD, CH>) * (size_t)warps;
  static bool attr_set[8] = {false, false, false, false, false, false, false, false};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev >= 0 && dev < 8 && !attr_set[dev]) {
    if (cudaFuncSetAttribute(k_force<GUARD, QUAD, FAR, CH>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(sizeof(WarpStage<QUAD, CH>) * 8)) != cudaSuccess)
      return AFD_ERR_CUDA;
    attr_set[dev] = true;
  }
  k_force<GUARD, QUAD, FAR, CH><<<nb, 32 * warps, smem, s>>>(a);
  return AFD_OK;
}

}  // namespace

namespace {

// Half-precision far field, per cell: the negated dimensionless quadrupole
// shape -Q / (M s^2) (FP64 quotient, rounded to BF16 / FP16) packed as half2
// words (xx, yy), (zz, xy), (xz, yz), and s^2 (FP32). A massless cell gets
// a zero shape.
template <int FAR>
__global__ void __launch_bounds__(256) k_far_half(int64_t nc, const double *__restrict__ quad,
                                                  const double *__restrict__ mass,
                                                  const float4 *__restrict__ node_f,
                                                  uint4 *__restrict__ s_h) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nc) return;
  const float s2 = node_f[c].w;
  const double den = __dmul_rn(mass[c], (double)s2);
  const double inv = den > 0.0 ? -1.0 / den : 0.0;
  float q[6];
#pragma unroll
  for (int k = 0; k < 6; k++) q[k] = __double2float_rn(__dmul_rn(quad[c * 6 + k], inv));
  s_h[c] = make_uint4(h2_from_f2<FAR>(pk(q[0], q[1])), h2_from_f2<FAR>(pk(q[2], q[3])),
                      h2_from_f2<FAR>(pk(q[4], q[5])), __float_as_uint(s2));
}


// Non-indirect ablation: copy every list entry's j-data into list order.
__global__ void k_materialize(uint64_t n, const uint32_t *__restrict__ idx,
                              const float4 *__restrict__ hi, const float4 *__restrict__ lo,
                              float4 *__restrict__ ohi, float4 *__restrict__ olo) {
  for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
       k += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t j = idx[k];
    ohi[k] = hi[j];
    olo[k] = lo[j];
  }
}

// Launch order of the force work items. A warp takes one item: a unit, or
// two consecutive units of one group -- a full one and the
// next when that holds more than 16 particles -- which share the group's
// list: each lane then carries two i-particles (lanes past the second
// unit's end only one), and every staged j-pair serves up to 64 particles
// instead of 32. Measured without the list traffic, a staged j-pair shared
// by two i-particles keeps the FP32 pipe 0.82 busy against 0.72 for one
// (the quadrupole loop: 9.1e11 against 8.6e11 interactions per second). An item's warp streams its
// group's whole list (split over S j-streams for the last, partial unit), so
// its time follows the list work L * IPT / S; the items are launched largest
// work first (afd_order.cuh). Every item writes its own particles.

// The item unit u starts: its work, kOrderFlag when it takes the group's
// next unit too, or kNoItem when the previous unit took it.
__device__ __forceinline__ uint32_t unit_item(const uint2 *u_info, const uint32_t *g_count,
                                              const uint64_t *off_e, const uint64_t *off_s,
                                              int64_t u, bool pairs) {
  const uint2 info = u_info[u];
  const uint32_t g = info.x, ioff = info.y & 0xffffu;
  const uint32_t sidx = (info.y >> 16) & 3u;
  bool pair = false;
  if (pairs && sidx == 0u) {
    // a unit in an even slot takes the next unit too when that one holds
    // more than 16 particles (fewer are cheaper as a unit of their own, split
    // into j-streams); the next unit then starts no item
    const uint32_t cn = g_count[g];
    if ((ioff & 32u) != 0u && cn - ioff > 16u) return kNoItem;
    pair = (ioff & 32u) == 0u && cn - ioff > 48u;
  }
  const uint64_t L = (off_e[g + 1] - off_e[g]) + (off_s[g + 1] - off_s[g]);
  uint64_t w = pair ? 2u * L : (L >> sidx);
  if (w > kOrderWorkMax) w = kOrderWorkMax;
  return (uint32_t)w | (pair ? kOrderFlag : 0u);
}

__global__ void k_unit_work(int64_t u0, int64_t nu, const uint2 *__restrict__ u_info,
                            const uint32_t *__restrict__ g_count,
                            const uint64_t *__restrict__ off_e, const uint64_t *__restrict__ off_s,
                            bool pairs, uint32_t *__restrict__ work, uint32_t *__restrict__ hist) {
  uint32_t wmax = 0, items = 0;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < nu;
       k += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t w = unit_item(u_info, g_count, off_e, off_s, u0 + k, pairs);
    work[k] = w;
    if (w != kNoItem) {
      wmax = max(wmax, w & ~kOrderFlag);
      items++;
    }
  }
  order_reduce(hist, wmax, items);
}

}  // namespace

int order_units(afd_ctx *c) {
  c->u_order_ok = false;
  const int64_t u0 = c->share_parts > 1 ? c->share_u0 : 0;
  const int64_t u1 = c->share_parts > 1 ? c->share_u1 : c->n_units;
  const int64_t nu = u1 - u0;
  if (nu <= 0) return AFD_OK;
  if (c->n_units >= (int64_t)kOrderFlag) return AFD_OK;  // unit ids need bit 31: index order
  if (reserve(c->u_order, sizeof(uint32_t) * (size_t)nu) != AFD_OK ||
      reserve(c->u_work, sizeof(uint32_t) * (size_t)nu) != AFD_OK ||
      reserve(c->u_hist, sizeof(uint32_t) * (kOrderBuckets + 2)) != AFD_OK)
    return AFD_ERR_OOM;
  uint32_t *hist = ptr<uint32_t>(c->u_hist), *work = ptr<uint32_t>(c->u_work);
  if (cudaMemsetAsync(hist, 0, sizeof(uint32_t) * (kOrderBuckets + 2), c->stream) != cudaSuccess)
    return AFD_ERR_CUDA;
  // two i-particles per lane, with monopole or quadrupole far fields
  const bool pairs = AFD_FORCE_PAIRS && (!c->cfg.multipole || AFD_FORCE_QUAD_IPT2);
  constexpr int kT = 256;
  const int64_t want = (nu + kT - 1) / kT;
  const unsigned nb = (unsigned)(want < 152 * 8 ? want : 152 * 8);
  k_unit_work<<<nb, kT, 0, c->stream>>>(u0, nu, ptr<uint2>(c->u_info), ptr<uint32_t>(c->g_count),
                                        ptr<uint64_t>(c->epj_off), ptr<uint64_t>(c->spj_off),
                                        pairs, work, hist);
  c->launches++;
  if (order_by_work(c->stream, nu, u0, work, hist, ptr<uint32_t>(c->u_order), &c->launches) !=
      cudaSuccess)
    return AFD_ERR_CUDA;
  c->u_order_ok = true;
  return AFD_OK;
}

int launch_force_impl(afd_ctx *c, float *acc4, bool materialized);

int launch_force(afd_ctx *c, float *acc4) { return launch_force_impl(c, acc4, false); }

int launch_materialize(afd_ctx *c) {
  const size_t ne = (size_t)c->n_epj, ns = (size_t)c->n_spj;
  for (afd::DevBuf *b : {&c->m_ehi, &c->m_elo})
    if (reserve(*b, sizeof(float4) * ne) != AFD_OK) return AFD_ERR_OOM;
  for (afd::DevBuf *b : {&c->m_shi, &c->m_slo})
    if (reserve(*b, sizeof(float4) * ns) != AFD_OK) return AFD_ERR_OOM;
  if (ne)
    k_materialize<<<152 * 16, 256, 0, c->stream>>>(ne, ptr<uint32_t>(c->epj), ptr<float4>(c->jhi),
                                                   ptr<float4>(c->jlo), ptr<float4>(c->m_ehi),
                                                   ptr<float4>(c->m_elo));
  if (ns)
    k_materialize<<<152 * 16, 256, 0, c->stream>>>(ns, ptr<uint32_t>(c->spj), ptr<float4>(c->s_hi),
                                                   ptr<float4>(c->s_lo), ptr<float4>(c->m_shi),
                                                   ptr<float4>(c->m_slo));
  c->launches += (ne ? 1 : 0) + (ns ? 1 : 0);
  return cudaGetLastError() == cudaSuccess ? AFD_OK : AFD_ERR_CUDA;
}

int launch_force_materialized(afd_ctx *c, float *acc4) {
  return launch_force_impl(c, acc4, true);
}

int launch_force_impl(afd_ctx *c, float *acc4, bool materialized) {
  if (c->n == 0 || c->n_units == 0) return AFD_OK;
  // the units of this context's work share (all of them without a share)
  const int64_t u0 = c->share_parts > 1 ? c->share_u0 : 0;
  const int64_t u1 = c->share_parts > 1 ? c->share_u1 : c->n_units;
  if (u1 <= u0) return AFD_OK;
  ForceArgs a;
  a.n_units = u1;
  a.u_base = u0;
  a.u_order = c->u_order_ok ? ptr<uint32_t>(c->u_order) : nullptr;
  a.n_items = c->u_order_ok ? ptr<uint32_t>(c->u_hist) + kOrderBuckets + 1 : nullptr;
  a.u_info = ptr<uint2>(c->u_info);
  a.g_first = ptr<uint32_t>(c->g_first);
  a.g_count = ptr<uint32_t>(c->g_count);
  a.g_self = ptr<uint32_t>(c->g_self);
  a.g_cell = ptr<uint32_t>(c->g_cell);
  a.jhi = a.ihi = ptr<float4>(c->jhi);
  a.jlo = a.ilo = ptr<float4>(c->jlo);
  a.shi = a.ohi = ptr<float4>(c->s_hi);
  a.slo = a.olo = ptr<float4>(c->s_lo);
  if (materialized) {  // j-data in list order, no index indirection
    a.jhi = ptr<float4>(c->m_ehi);
    a.jlo = ptr<float4>(c->m_elo);
    a.shi = ptr<float4>(c->m_shi);
    a.slo = ptr<float4>(c->m_slo);
  }
  a.sq0 = ptr<float4>(c->s_q0);
  a.sq1 = ptr<float4>(c->s_q1);
  const int far_p = c->cfg.multipole ? c->cfg.far_precision : 0;
  if (far_p) {
    // the cells' half records from the current moments (the groups' scales
    // came with the lists: the walk writes them)
    if (!c->fscale_ok) return AFD_ERR_NO_SAVED_LIST;
    if (reserve(c->s_h, sizeof(uint4) * (size_t)c->n_cells) != AFD_OK) return AFD_ERR_OOM;
    const unsigned nb_c = (unsigned)((c->n_cells + 255) / 256);
    if (far_p == 1)
      k_far_half<1><<<nb_c, 256, 0, c->stream>>>(c->n_cells, ptr<double>(c->c_quad),
                                                  ptr<double>(c->c_mass), ptr<float4>(c->node_f),
                                                  ptr<uint4>(c->s_h));
    else
      k_far_half<2><<<nb_c, 256, 0, c->stream>>>(c->n_cells, ptr<double>(c->c_quad),
                                                  ptr<double>(c->c_mass), ptr<float4>(c->node_f),
                                                  ptr<uint4>(c->s_h));
    c->launches++;
  }
  a.sh = ptr<uint4>(c->s_h);
  a.gscale = ptr<float>(c->g_fscale);
  a.off_e = ptr<uint64_t>(c->epj_off);
  a.off_s = ptr<uint64_t>(c->spj_off);
  a.epj = materialized ? nullptr : ptr<uint32_t>(c->epj);
  a.spj = materialized ? nullptr : ptr<uint32_t>(c->spj);
  a.perm = ptr<uint32_t>(c->perm);
  const float e = (float)c->cfg.eps;
  a.eps2 = e * e;
  a.out = reinterpret_cast<float4 *>(acc4);
  a.n = (uint64_t)c->n;
  a.n_cells = (uint64_t)c->n_cells;
  a.n_groups = (uint64_t)c->n_groups;
  a.n_epj = c->n_epj;
  a.n_spj = c->n_spj;
  a.queue = ptr<unsigned long long>(c->u64acc) + 2;
  const int warps = c->force_warps;
  unsigned nb = (unsigned)((u1 - u0 + warps - 1) / warps);
  if (AFD_FORCE_PERSISTENT) {
    if (cudaMemsetAsync(a.queue, 0, sizeof(unsigned long long), c->stream) != cudaSuccess)
      return AFD_ERR_CUDA;
    const unsigned cap = 152u * (65536u / (32u * AFD_FORCE_MAX_REGS)) / (unsigned)warps;  // resident warps per GPU
    if (nb > cap) nb = cap;
  }
  const bool guard = !(a.eps2 > 0.0f);
  // timing events only outside stream capture
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(c->stream, &cap);
  const bool timed = cap == cudaStreamCaptureStatusNone;
  if (timed) cudaEventRecord(c->ev0, c->stream);
  const int far = c->cfg.multipole ? c->cfg.far_precision : 0;
  const bool c64 = c->force_chunk == 64;
  int st = AFD_OK;
#define AFD_LAUNCH_FORCE(G, Q, F)                                                     \
  st = c64 ? launch_k_force<G, Q, F, 64>(a, nb, warps, c->stream)                     \
           : launch_k_force<G, Q, F, 32>(a, nb, warps, c->stream)
  if (!c->cfg.multipole) {
    if (guard) AFD_LAUNCH_FORCE(true, false, 0);
    else AFD_LAUNCH_FORCE(false, false, 0);
  } else if (far == 1) {
    if (guard) AFD_LAUNCH_FORCE(true, true, 1);
    else AFD_LAUNCH_FORCE(false, true, 1);
  } else if (far == 2) {
    if (guard) AFD_LAUNCH_FORCE(true, true, 2);
    else AFD_LAUNCH_FORCE(false, true, 2);
  } else {
    if (guard) AFD_LAUNCH_FORCE(true, true, 0);
    else AFD_LAUNCH_FORCE(false, true, 0);
  }
#undef AFD_LAUNCH_FORCE
  if (st != AFD_OK) return st;
  c->launches++;
  if (timed) {
    cudaEventRecord(c->ev1, c->stream);
    c->force_timed = true;
  }
  return cudaGetLastError() == cudaSuccess ? AFD_OK : AFD_ERR_CUDA;
}

}  // namespace afd
