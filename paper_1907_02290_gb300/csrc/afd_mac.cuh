// Learned opening criterion: the device arithmetic shared by the tree walk
// and the sampling / inference kernels. The criterion is not in the paper
// (which opens cells by the angle theta, Section 2); its definition:
//
//  features of a (group, cell) pair, eight FP32 numbers, no contraction,
//  in the order written in mac_features():
//    f0 = log2(s/d)   f1 = log2(M / (d^2 A_g))   f2 = log2(|Q|_F / (M s^2))
//    f3 = log2(e/d)   f4 = log2(n_c)   f5 = log2(eps/d)
//    f6 = u.Q.u / (|u|^2 |Q|_F)   f7 = log2(|u|/d)
//  with d the COM-to-box distance of the theta criterion, s the cell side,
//  M, Q the cell's monopole and traceless quadrupole (FP32), n_c its
//  particle count, A_g the smallest reference |a| of the group's particles,
//  u = box centre - COM, e = half the box diagonal; clamped to [-32, 32].
//  log2 here is mac_lg2(): the FP32 exponent plus t * p(t) on the mantissa
//  1 + t, p a least-squares quartic, Horner with fused multiply-adds.
//
//  network: 8-32-32-1, ReLU, every parameter an FP16 value; the inputs
//  x = RN16((f - mu) * isd) and the first-layer activations
//  h1 = RN16(min(max(b1 + W1 x, 0), 65504)) are FP16 (RN16: nearest FP16,
//  ties to even), h2 = max(b2 + W2 h1, 0) and y = b3 + w3 . h2 are FP32.
//  The two layers run on the tensor cores (mma.sync, FP16 operands, FP32
//  accumulation), sixteen (group, cell) pairs at a time, in whatever order
//  the tensor core sums; the output is summed over each lane's eight units
//  and then across the four lanes that share a row. A decision is fixed by
//  the network only when its output is further from tau than the bound on
//  two FP32 summation orders' difference that the definition states.
//
//  decision: open a cell holding the group's first particle; accept when
//  s^2 < theta_lo^2 d^2; open unless s^2 < theta_hi^2 d^2; otherwise accept
//  iff the network's output (a predicted log2 relative force error) < tau.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace afd {

constexpr int kMacNF = 8;
constexpr int kMacNH = 32;
// mu[8] isd[8] W1[32][8] b1[32] W2[32][32] b2[32] w3[32] b3[1]
constexpr int kMacNP = 2 * kMacNF + kMacNH * kMacNF + kMacNH + kMacNH * kMacNH + kMacNH + kMacNH + 1;
constexpr int kMacOffW1 = 2 * kMacNF;
constexpr int kMacOffB1 = kMacOffW1 + kMacNH * kMacNF;
constexpr int kMacOffW2 = kMacOffB1 + kMacNH;
constexpr int kMacOffB2 = kMacOffW2 + kMacNH * kMacNH;
constexpr int kMacOffW3 = kMacOffB2 + kMacNH;
constexpr int kMacOffB3 = kMacOffW3 + kMacNH;
constexpr int kMacTrain = kMacNP - kMacOffW1;  // trained parameters (mu, isd are data statistics)

__device__ __forceinline__ float mac_lg2(float x) {
  if (!(x >= __uint_as_float(0x00800000u))) return -127.0f;  // 0, negative, NaN, subnormal
  if (x > __uint_as_float(0x7f7fffffu)) return 128.0f;
  const uint32_t b = __float_as_uint(x);
  const int e = (int)((b >> 23) & 0xffu) - 127;
  const float t = __fsub_rn(__uint_as_float((b & 0x7fffffu) | 0x3f800000u), 1.0f);
  float p = 0.04526829347014427f;
  p = __fmaf_rn(p, t, -0.19351652264595032f);
  p = __fmaf_rn(p, t, 0.41524556279182434f);
  p = __fmaf_rn(p, t, -0.708865225315094f);
  p = __fmaf_rn(p, t, 1.4418798685073853f);
  return __fadd_rn(__int2float_rn(e), __fmul_rn(p, t));
}

__device__ __forceinline__ float mac_clamp(float v) {
  return v < -32.0f ? -32.0f : (v > 32.0f ? 32.0f : v);
}

__device__ __forceinline__ float mac_sep(float c, float lo, float hi) {
  float d = 0.0f;
  if (c < lo) d = __fsub_rn(lo, c);
  else if (c > hi) d = __fsub_rn(c, hi);
  return d;
}

__device__ __forceinline__ float mac_sq3(float a, float b, float c) {
  float s = __fmul_rn(a, a);
  s = __fadd_rn(s, __fmul_rn(b, b));
  return __fadd_rn(s, __fmul_rn(c, c));
}

// The features' terms that depend only on the group (and eps): log2 of the
// group's smallest reference |a|, of its box's half diagonal squared e^2,
// and of eps^2 -- a walk computes them once per group.
struct MacGroup {
  float lg_amin, lg_e2, lg_eps2;
};

__device__ __forceinline__ MacGroup mac_group(const float *bmin, const float *bmax, float amin,
                                              float eps2) {
  float w[3];
#pragma unroll
  for (int k = 0; k < 3; k++) w[k] = __fsub_rn(bmax[k], bmin[k]);
  const float e2 = __fmul_rn(mac_sq3(w[0], w[1], w[2]), 0.25f);
  MacGroup g;
  g.lg_amin = mac_lg2(amin);
  g.lg_e2 = mac_lg2(e2);
  g.lg_eps2 = mac_lg2(eps2);
  return g;
}

// q = (xx, yy, zz, xy), q1 = (xz, yz, -, -); d2 = mac_sq3 of the COM's
// separations from the box (mac_sep per axis), as the criterion has it.
__device__ __forceinline__ void mac_features_g(const float *bmin, const float *bmax, float cx,
                                               float cy, float cz, float s2, float M, float4 q,
                                               float2 q1, uint32_t count, float d2,
                                               const MacGroup &G, float *f) {
  const float com[3] = {cx, cy, cz};
  float u[3];
#pragma unroll
  for (int k = 0; k < 3; k++) u[k] = __fsub_rn(__fmul_rn(__fadd_rn(bmin[k], bmax[k]), 0.5f), com[k]);
  const float u2 = mac_sq3(u[0], u[1], u[2]);
  const float off = mac_sq3(q.w, q1.x, q1.y);
  const float q2 = __fadd_rn(mac_sq3(q.x, q.y, q.z), __fadd_rn(off, off));
  const float Qu0 = __fadd_rn(__fadd_rn(__fmul_rn(q.x, u[0]), __fmul_rn(q.w, u[1])), __fmul_rn(q1.x, u[2]));
  const float Qu1 = __fadd_rn(__fadd_rn(__fmul_rn(q.w, u[0]), __fmul_rn(q.y, u[1])), __fmul_rn(q1.y, u[2]));
  const float Qu2 = __fadd_rn(__fadd_rn(__fmul_rn(q1.x, u[0]), __fmul_rn(q1.y, u[1])), __fmul_rn(q.z, u[2]));
  const float uQu = __fadd_rn(__fadd_rn(__fmul_rn(u[0], Qu0), __fmul_rn(u[1], Qu1)), __fmul_rn(u[2], Qu2));
  const float ld = mac_lg2(d2), ls = mac_lg2(s2), lm = mac_lg2(M);
  f[0] = __fmul_rn(0.5f, __fsub_rn(ls, ld));
  f[1] = __fsub_rn(__fsub_rn(lm, ld), G.lg_amin);
  f[2] = __fsub_rn(__fsub_rn(__fmul_rn(0.5f, mac_lg2(q2)), lm), ls);
  f[3] = __fmul_rn(0.5f, __fsub_rn(G.lg_e2, ld));
  f[4] = mac_lg2(__uint2float_rn(count));
  f[5] = __fmul_rn(0.5f, __fsub_rn(G.lg_eps2, ld));
  f[6] = 0.0f;
  if (u2 > 0.0f && q2 > 0.0f) {
    const float den = __fmul_rn(u2, __fsqrt_rn(q2));
    if (den > 0.0f) f[6] = __fdiv_rn(uQu, den);
  }
  f[7] = __fmul_rn(0.5f, __fsub_rn(mac_lg2(u2), ld));
#pragma unroll
  for (int k = 0; k < kMacNF; k++) f[k] = mac_clamp(f[k]);
}

// The features of one pair from scratch (the group's terms included).
__device__ __forceinline__ void mac_features(const float *bmin, const float *bmax, float cx,
                                             float cy, float cz, float s2, float M, float4 q,
                                             float2 q1, uint32_t count, float eps2, float amin,
                                             float *f) {
  const float d2 = mac_sq3(mac_sep(cx, bmin[0], bmax[0]), mac_sep(cy, bmin[1], bmax[1]),
                           mac_sep(cz, bmin[2], bmax[2]));
  mac_features_g(bmin, bmax, cx, cy, cz, s2, M, q, q1, count, d2,
                 mac_group(bmin, bmax, amin, eps2), f);
}

// ---- the network on the tensor cores ----
// mma.sync m16n8k8 (layer 1, 8 inputs) and m16n8k16 (layer 2, 32 inputs),
// row.col, FP16 operands, FP32 accumulators: 16 rows (pairs) x 8 units per
// instruction. Fragment layout with g = lane / 4, t = lane % 4:
//   A (16 x k, rows = pairs): a0 = row g, cols 2t, 2t+1; a1 = row g + 8;
//     (k16) a2, a3 = the same rows, cols 8 + 2t, 8 + 2t + 1;
//   B (k x 8, col = unit): b0 = unit g, k 2t, 2t+1; (k16) b1 = k 8 + 2t, ..;
//   C, D: c0, c1 = row g, units 2t, 2t+1; c2, c3 = row g + 8.
// Layer 1's outputs of unit tiles 2s, 2s+1 are then exactly layer 2's A
// fragment of input slice s, so the hidden layer never leaves registers.
struct MacFrag {
  uint32_t w1[4][32];        // unit tile n: W1[8n + g][2t, 2t+1] (f16x2)
  uint32_t w2[2][4][2][32];  // slice s, unit tile n, reg r: W2[8n + g][16s + 8r + 2t, +1]
  float2 b1[4][32];          // unit tile n: (b1[8n + 2t], b1[8n + 2t + 1])
  float2 b2[4][32];
  float2 w3[4][32];
  float mu[kMacNF], isd[kMacNF];
  float b3;
};

__device__ __forceinline__ uint32_t mac_h2(float lo, float hi) {
  uint32_t r;
  asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
  return r;
}

// Fragments from the flat parameter vector (FP16 values held as FP32);
// threads tid of nt fill them (then a barrier is the caller's).
__device__ __forceinline__ void mac_frag_load(MacFrag &F, const float *w, int tid, int nt) {
  for (int i = tid; i < 4 * 32; i += nt) {
    const int n = i >> 5, l = i & 31, g = l >> 2, t = l & 3, u = 8 * n + g;
    F.w1[n][l] = mac_h2(w[kMacOffW1 + u * kMacNF + 2 * t], w[kMacOffW1 + u * kMacNF + 2 * t + 1]);
    const int v = 8 * n + 2 * t;
    F.b1[n][l] = make_float2(w[kMacOffB1 + v], w[kMacOffB1 + v + 1]);
    F.b2[n][l] = make_float2(w[kMacOffB2 + v], w[kMacOffB2 + v + 1]);
    F.w3[n][l] = make_float2(w[kMacOffW3 + v], w[kMacOffW3 + v + 1]);
  }
  for (int i = tid; i < 2 * 4 * 2 * 32; i += nt) {
    const int l = i & 31, r = (i >> 5) & 1, n = (i >> 6) & 3, sl = i >> 8;
    const int g = l >> 2, t = l & 3, u = 8 * n + g, k = 16 * sl + 8 * r + 2 * t;
    F.w2[sl][n][r][l] = mac_h2(w[kMacOffW2 + u * kMacNH + k], w[kMacOffW2 + u * kMacNH + k + 1]);
  }
  for (int i = tid; i < kMacNF; i += nt) {
    F.mu[i] = w[i];
    F.isd[i] = w[kMacNF + i];
  }
  if (tid == 0) F.b3 = w[kMacOffB3];
}

// One input row: RN16((f - mu) * isd) as four f16x2 words (inputs 0-1, 2-3, ..).
__device__ __forceinline__ uint4 mac_row16(const MacFrag &F, const float *f) {
  float x[kMacNF];
#pragma unroll
  for (int k = 0; k < kMacNF; k++) x[k] = __fmul_rn(__fsub_rn(f[k], F.mu[k]), F.isd[k]);
  return make_uint4(mac_h2(x[0], x[1]), mac_h2(x[2], x[3]), mac_h2(x[4], x[5]), mac_h2(x[6], x[7]));
}

__device__ __forceinline__ void mac_mma_k8(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t b0,
                                           float2 c) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.f16.f16.f32 {%0, %1, %2, %3}, {%4, %5}, {%6}, "
      "{%7, %8, %9, %10};"
      : "=f"(d[0]), "=f"(d[1]), "=f"(d[2]), "=f"(d[3])
      : "r"(a0), "r"(a1), "r"(b0), "f"(c.x), "f"(c.y), "f"(c.x), "f"(c.y));
}
__device__ __forceinline__ void mac_mma_k16(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2,
                                            uint32_t a3, uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, "
      "{%8, %9}, {%0, %1, %2, %3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

__device__ __forceinline__ float mac_h1(float v) { return fminf(fmaxf(v, 0.0f), 65504.0f); }

// The network on the 16 rows whose input words sit in x16 (row r: x16[r]);
// every lane of the warp calls it. Returns the outputs of rows g and g + 8
// (each lane of the row's quad holds them).
__device__ __forceinline__ float2 mac_mma_rows(const MacFrag &F, const uint4 *x16, int lane) {
  const int g = lane >> 2, t = lane & 3;
  const uint32_t *xw = reinterpret_cast<const uint32_t *>(x16);
  const uint32_t a0 = xw[g * 4 + t], a1 = xw[(g + 8) * 4 + t];
  // layer 1: four unit tiles, then ReLU, clamp and FP16 as layer 2's A fragments
  uint32_t hl[4], hh[4];
#pragma unroll
  for (int n = 0; n < 4; n++) {
    float d[4];
    mac_mma_k8(d, a0, a1, F.w1[n][lane], F.b1[n][lane]);
    hl[n] = mac_h2(mac_h1(d[0]), mac_h1(d[1]));
    hh[n] = mac_h2(mac_h1(d[2]), mac_h1(d[3]));
  }
  // layer 2: four unit tiles over two input slices; output dot products
  float ylo = 0.0f, yhi = 0.0f;
#pragma unroll
  for (int n = 0; n < 4; n++) {
    const float2 b = F.b2[n][lane];
    float d[4] = {b.x, b.y, b.x, b.y};
#pragma unroll
    for (int sl = 0; sl < 2; sl++)
      mac_mma_k16(d, hl[2 * sl], hh[2 * sl], hl[2 * sl + 1], hh[2 * sl + 1], F.w2[sl][n][0][lane],
                  F.w2[sl][n][1][lane]);
    const float2 w3 = F.w3[n][lane];
    ylo = __fmaf_rn(w3.x, fmaxf(d[0], 0.0f), ylo);
    ylo = __fmaf_rn(w3.y, fmaxf(d[1], 0.0f), ylo);
    yhi = __fmaf_rn(w3.x, fmaxf(d[2], 0.0f), yhi);
    yhi = __fmaf_rn(w3.y, fmaxf(d[3], 0.0f), yhi);
  }
#pragma unroll
  for (int o = 1; o < 4; o <<= 1) {
    ylo = __fadd_rn(ylo, __shfl_xor_sync(0xffffffffu, ylo, o));
    yhi = __fadd_rn(yhi, __shfl_xor_sync(0xffffffffu, yhi, o));
  }
  return make_float2(__fadd_rn(ylo, F.b3), __fadd_rn(yhi, F.b3));
}

}  // namespace afd
