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
//  network: 8-32-32-1, ReLU, inputs normalised as (f - mu) * isd, every
//  parameter an FP16 value held as FP32, each hidden unit its bias followed
//  by fused multiply-adds in input order. The output unit is b3 plus the 32
//  terms w3_j h2_j; this code sums the rounded products pairwise by halving
//  (j += j + 16, then 8, 4, 2, 1: a warp's xor butterfly, five shuffles
//  instead of a 32-step chain) and then adds b3. Any FP32 order of those
//  terms lies within 2 gamma_32 (|b3| + sum |w3_j h2_j|) of any other
//  (gamma_k = k 2^-24 / (1 - k 2^-24)), so a decision is fixed by the
//  network only when its output is further than that from tau.
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

// q = (xx, yy, zz, xy), q1 = (xz, yz, -, -)
__device__ __forceinline__ void mac_features(const float *bmin, const float *bmax, float cx,
                                             float cy, float cz, float s2, float M, float4 q,
                                             float2 q1, uint32_t count, float eps2, float amin,
                                             float *f) {
  const float com[3] = {cx, cy, cz};
  float d[3], u[3], w[3];
#pragma unroll
  for (int k = 0; k < 3; k++) {
    d[k] = mac_sep(com[k], bmin[k], bmax[k]);
    u[k] = __fsub_rn(__fmul_rn(__fadd_rn(bmin[k], bmax[k]), 0.5f), com[k]);
    w[k] = __fsub_rn(bmax[k], bmin[k]);
  }
  const float d2 = mac_sq3(d[0], d[1], d[2]);
  const float u2 = mac_sq3(u[0], u[1], u[2]);
  const float e2 = __fmul_rn(mac_sq3(w[0], w[1], w[2]), 0.25f);
  const float off = mac_sq3(q.w, q1.x, q1.y);
  const float q2 = __fadd_rn(mac_sq3(q.x, q.y, q.z), __fadd_rn(off, off));
  const float Qu0 = __fadd_rn(__fadd_rn(__fmul_rn(q.x, u[0]), __fmul_rn(q.w, u[1])), __fmul_rn(q1.x, u[2]));
  const float Qu1 = __fadd_rn(__fadd_rn(__fmul_rn(q.w, u[0]), __fmul_rn(q.y, u[1])), __fmul_rn(q1.y, u[2]));
  const float Qu2 = __fadd_rn(__fadd_rn(__fmul_rn(q1.x, u[0]), __fmul_rn(q1.y, u[1])), __fmul_rn(q.z, u[2]));
  const float uQu = __fadd_rn(__fadd_rn(__fmul_rn(u[0], Qu0), __fmul_rn(u[1], Qu1)), __fmul_rn(u[2], Qu2));
  const float ld = mac_lg2(d2), ls = mac_lg2(s2), lm = mac_lg2(M);
  f[0] = __fmul_rn(0.5f, __fsub_rn(ls, ld));
  f[1] = __fsub_rn(__fsub_rn(lm, ld), mac_lg2(amin));
  f[2] = __fsub_rn(__fsub_rn(__fmul_rn(0.5f, mac_lg2(q2)), lm), ls);
  f[3] = __fmul_rn(0.5f, __fsub_rn(mac_lg2(e2), ld));
  f[4] = mac_lg2(__uint2float_rn(count));
  f[5] = __fmul_rn(0.5f, __fsub_rn(mac_lg2(eps2), ld));
  f[6] = 0.0f;
  if (u2 > 0.0f && q2 > 0.0f) {
    const float den = __fmul_rn(u2, __fsqrt_rn(q2));
    if (den > 0.0f) f[6] = __fdiv_rn(uQu, den);
  }
  f[7] = __fmul_rn(0.5f, __fsub_rn(mac_lg2(u2), ld));
#pragma unroll
  for (int k = 0; k < kMacNF; k++) f[k] = mac_clamp(f[k]);
}

// ---- one lane evaluates the network, two units per instruction ----
// Shared-memory layout for mac_mlp_t (offsets as in the flat vector, the two
// weight matrices transposed to [input][unit]): mu, isd, W1T[8][32], b1,
// W2T[32][32], b2, w3, b3. Each unit accumulates its bias and then its
// inputs in index order with one rounding per fused multiply-add; the packed
// FMA (fma.rn.f32x2) rounds each half exactly like the scalar one.
__device__ __forceinline__ void mac_load_transposed(float *wt, const float *w, int tid, int nt) {
  for (int i = tid; i < kMacNP; i += nt) {
    float v;
    if (i >= kMacOffW1 && i < kMacOffB1) {  // W1T[k][j] = W1[j][k]
      const int k = (i - kMacOffW1) / kMacNH, j = (i - kMacOffW1) % kMacNH;
      v = w[kMacOffW1 + j * kMacNF + k];
    } else if (i >= kMacOffW2 && i < kMacOffB2) {  // W2T[k][j] = W2[j][k]
      const int k = (i - kMacOffW2) / kMacNH, j = (i - kMacOffW2) % kMacNH;
      v = w[kMacOffW2 + j * kMacNH + k];
    } else {
      v = w[i];
    }
    wt[i] = v;
  }
}

__device__ __forceinline__ unsigned long long mac_pk(float lo, float hi) {
  return ((unsigned long long)__float_as_uint(hi) << 32) | __float_as_uint(lo);
}
__device__ __forceinline__ float mac_lo(unsigned long long v) { return __uint_as_float((uint32_t)v); }
__device__ __forceinline__ float mac_hi(unsigned long long v) {
  return __uint_as_float((uint32_t)(v >> 32));
}
__device__ __forceinline__ unsigned long long mac_fma2(unsigned long long a, unsigned long long b,
                                                       unsigned long long c) {
  unsigned long long d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}

// wt: shared memory in the mac_load_transposed layout, 16-byte aligned.
__device__ __forceinline__ float mac_mlp_t(const float *wt, const float *f) {
  float x[kMacNF];
#pragma unroll
  for (int k = 0; k < kMacNF; k++) x[k] = __fmul_rn(__fsub_rn(f[k], wt[k]), wt[kMacNF + k]);
  unsigned long long acc[kMacNH / 2];
  const float4 *b1 = reinterpret_cast<const float4 *>(wt + kMacOffB1);
#pragma unroll
  for (int q = 0; q < kMacNH / 4; q++) {
    const float4 b = b1[q];
    acc[2 * q] = mac_pk(b.x, b.y);
    acc[2 * q + 1] = mac_pk(b.z, b.w);
  }
#pragma unroll
  for (int k = 0; k < kMacNF; k++) {
    const unsigned long long xk = mac_pk(x[k], x[k]);
    const float4 *row = reinterpret_cast<const float4 *>(wt + kMacOffW1 + k * kMacNH);
#pragma unroll
    for (int q = 0; q < kMacNH / 4; q++) {
      const float4 r = row[q];
      acc[2 * q] = mac_fma2(mac_pk(r.x, r.y), xk, acc[2 * q]);
      acc[2 * q + 1] = mac_fma2(mac_pk(r.z, r.w), xk, acc[2 * q + 1]);
    }
  }
  float h1[kMacNH];
#pragma unroll
  for (int q = 0; q < kMacNH / 2; q++) {
    const float a = mac_lo(acc[q]), b = mac_hi(acc[q]);
    h1[2 * q] = a > 0.0f ? a : 0.0f;
    h1[2 * q + 1] = b > 0.0f ? b : 0.0f;
  }
  const float4 *b2 = reinterpret_cast<const float4 *>(wt + kMacOffB2);
#pragma unroll
  for (int q = 0; q < kMacNH / 4; q++) {
    const float4 b = b2[q];
    acc[2 * q] = mac_pk(b.x, b.y);
    acc[2 * q + 1] = mac_pk(b.z, b.w);
  }
#pragma unroll
  for (int k = 0; k < kMacNH; k++) {
    const unsigned long long hk = mac_pk(h1[k], h1[k]);
    const float4 *row = reinterpret_cast<const float4 *>(wt + kMacOffW2 + k * kMacNH);
#pragma unroll
    for (int q = 0; q < kMacNH / 4; q++) {
      const float4 r = row[q];
      acc[2 * q] = mac_fma2(mac_pk(r.x, r.y), hk, acc[2 * q]);
      acc[2 * q + 1] = mac_fma2(mac_pk(r.z, r.w), hk, acc[2 * q + 1]);
    }
  }
  float p[kMacNH];
#pragma unroll
  for (int q = 0; q < kMacNH / 2; q++) {
    const float a = mac_lo(acc[q]), b = mac_hi(acc[q]);
    p[2 * q] = __fmul_rn(wt[kMacOffW3 + 2 * q], a > 0.0f ? a : 0.0f);
    p[2 * q + 1] = __fmul_rn(wt[kMacOffW3 + 2 * q + 1], b > 0.0f ? b : 0.0f);
  }
#pragma unroll
  for (int half = kMacNH / 2; half > 0; half /= 2)
#pragma unroll
    for (int k = 0; k < half; k++) p[k] = __fadd_rn(p[k], p[k + half]);
  return __fadd_rn(p[0], wt[kMacOffB3]);
}

}  // namespace afd
