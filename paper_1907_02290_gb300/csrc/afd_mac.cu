// Learned opening criterion (not in the paper): everything around the
// network that the walk evaluates (afd_mac.cuh).
//
//  * reference accelerations: |a| per particle (caller order) from the last
//    force evaluation or from the caller; the walk uses the smallest one of
//    each group (feature f1 scales a cell's force by it).
//  * training samples: the (group, cell) pairs whose decision the band
//    leaves to the network, found by a walk that accepts below theta_lo and
//    opens everything else; each gets its features and its target -- log2 of
//    the largest relative force error, over the group's particles, of
//    replacing the cell's particles by its superparticle, against the direct
//    sum over those particles (FP32 with compensated sums).
//  * the network's own training: forward and backward passes over tiles of
//    128 samples, block-partial gradients reduced in a fixed order, Adam.
//  * FP64 direct summation for sampled targets, the exact reference that
//    errors are judged against.
#include <cuda_fp16.h>

#include <cmath>
#include <vector>

#include "afd_internal.cuh"
#include "afd_mac.cuh"

namespace afd {
namespace {

inline int ck() { return cudaGetLastError() == cudaSuccess ? AFD_OK : AFD_ERR_CUDA; }

#define MAC_TRY(x)                 \
  do {                             \
    int _s = (x);                  \
    if (_s != AFD_OK) return _s;   \
  } while (0)

inline unsigned blocks_of(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

// ---------------------------------------------------------------------------
// Reference magnitudes
// ---------------------------------------------------------------------------
__global__ void k_amag(const float4 *__restrict__ acc, int64_t n, float *__restrict__ amag) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float4 a = acc[i];
  amag[i] = __fsqrt_rn(mac_sq3(a.x, a.y, a.z));
}

// Morton-order copy of the reference magnitudes and the smallest per group
// (one warp per group).
__global__ void k_group_amin(int64_t n_groups, const uint32_t *__restrict__ g_first,
                             const uint32_t *__restrict__ g_count, const uint32_t *__restrict__ perm,
                             const float *__restrict__ amag, float *__restrict__ amag_s,
                             float *__restrict__ g_amin) {
  const int64_t g = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (g >= n_groups) return;
  const uint32_t f = g_first[g], e = f + g_count[g];
  float lo = __uint_as_float(0x7f800000u);
  for (uint32_t k = f + lane; k < e; k += 32) {
    const float v = amag[perm[k]];
    amag_s[k] = v;
    lo = fminf(lo, v);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, o));
  if (lane == 0) g_amin[g] = lo;
}

// ---------------------------------------------------------------------------
// Band walk: the pairs left to the network
// ---------------------------------------------------------------------------
constexpr int kBandWarps = 4;
constexpr int kBandStack = 6144;  // cell ids per warp

struct BandArgs {
  int64_t n_groups;
  const float *boxf;
  const uint32_t *g_first, *g_root;
  const float4 *node_f;
  const uint2 *node_i;
  const uint32_t *child;
  float lo2, hi2;
  uint32_t keep_thr;
  bool keep_all;
  uint64_t seed;
  uint32_t *cnt;
  const uint64_t *off;
  uint32_t *pairs;
  uint64_t cap;
  int *status;
  uint32_t iter_cap;
};

__device__ __forceinline__ uint32_t pair_hash(uint64_t seed, uint32_t g, uint32_t c) {
  uint64_t z = seed + ((uint64_t)g << 32 | c) + 0x9e3779b97f4a7c15ull;  // splitmix64
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return (uint32_t)((z ^ (z >> 31)) >> 32);
}

template <bool FILL>
__global__ void __launch_bounds__(32 * kBandWarps) k_band(BandArgs a) {
  extern __shared__ uint32_t band_stack[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const unsigned lt = (1u << lane) - 1u;
  uint32_t *stk = band_stack + (size_t)wib * kBandStack;
  for (int64_t g = (int64_t)blockIdx.x * kBandWarps + wib; g < a.n_groups;
       g += (int64_t)gridDim.x * kBandWarps) {
    float bmin[3], bmax[3];
#pragma unroll
    for (int k = 0; k < 3; k++) {
      bmin[k] = a.boxf[g * 6 + k];
      bmax[k] = a.boxf[g * 6 + 3 + k];
    }
    const uint32_t gfirst = a.g_first[g];
    const uint64_t base = FILL ? a.off[g] : 0;
    uint32_t nout = 0;
    if (lane == 0) stk[0] = a.g_root[g];
    int sp = 1;
    uint32_t iters = 0;
    __syncwarp();
    while (sp > 0) {
      if (++iters > a.iter_cap) {
        if (lane == 0) atomicOr(a.status, kStWalkIter);
        break;
      }
      const int nv = sp < 32 ? sp : 32;
      const uint32_t c = lane < nv ? stk[sp - 1 - lane] : 0u;
      bool open = false, out = false;
      if (lane < nv) {
        const float4 nf = a.node_f[c];
        const uint2 ni = a.node_i[c];
        const bool leaf = (ni.y >> 31) != 0;
        const uint32_t first = ni.x, count = ni.y & 0x7fffffffu;
        if (gfirst >= first && gfirst - first < count) {
          open = !leaf;
        } else {
          const float dx = mac_sep(nf.x, bmin[0], bmax[0]);
          const float dy = mac_sep(nf.y, bmin[1], bmax[1]);
          const float dz = mac_sep(nf.z, bmin[2], bmax[2]);
          const float d2 = mac_sq3(dx, dy, dz);
          if (!(nf.w < __fmul_rn(a.lo2, d2))) {
            open = !leaf;
            if (nf.w < __fmul_rn(a.hi2, d2))
              out = a.keep_all || pair_hash(a.seed, (uint32_t)g, c) < a.keep_thr;
          }
        }
      }
      const unsigned om = __ballot_sync(0xffffffffu, out);
      if (FILL && out) {
        const uint64_t pos = base + nout + __popc(om & lt);
        if (pos < a.cap) {
          a.pairs[2 * pos] = (uint32_t)g;
          a.pairs[2 * pos + 1] = c;
        }
      }
      nout += __popc(om);
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
      if (spn + (int)K > kBandStack) {
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
    if (!FILL && lane == 0) a.cnt[g] = nout;
    __syncwarp();
  }
}

// Features of sampled pairs.
__global__ void k_pair_features(int64_t n, const uint32_t *__restrict__ pairs,
                                const float *__restrict__ boxf, const float4 *__restrict__ node_f,
                                const uint2 *__restrict__ node_i, const float4 *__restrict__ s_hi,
                                const float4 *__restrict__ s_q0, const float4 *__restrict__ s_q1,
                                const float *__restrict__ g_amin, float eps2,
                                float *__restrict__ feat) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint32_t g = pairs[2 * i], c = pairs[2 * i + 1];
  float bmin[3], bmax[3];
#pragma unroll
  for (int k = 0; k < 3; k++) {
    bmin[k] = boxf[(size_t)g * 6 + k];
    bmax[k] = boxf[(size_t)g * 6 + 3 + k];
  }
  const float4 nf = node_f[c];
  const float4 q1 = s_q1[c];
  float f[kMacNF];
  mac_features(bmin, bmax, nf.x, nf.y, nf.z, nf.w, s_hi[c].w, s_q0[c], make_float2(q1.x, q1.y),
               node_i[c].y & 0x7fffffffu, eps2, g_amin[g], f);
#pragma unroll
  for (int k = 0; k < kMacNF; k++) feat[i * kMacNF + k] = f[k];
}

// Targets of sampled pairs: one block per pair. Coordinates relative to the
// cell's COM in FP32; the exact sum over the cell's particles is compensated
// (Kahan) per component.
constexpr int kLabelThreads = 128;
constexpr int kLabelTile = 512;

struct LabelArgs {
  int64_t n;
  const uint32_t *pairs;
  const uint32_t *g_first, *g_count;
  const uint2 *node_i;
  const double *xs, *ys, *zs, *ms, *com, *mass;
  const float4 *s_q0, *s_q1;
  const float *amag_s;
  float eps2;
  int quad;
  float *label;
};

__device__ __forceinline__ void kahan(float &s, float &c, float v) {
  const float y = __fsub_rn(v, c);
  const float t = __fadd_rn(s, y);
  c = __fsub_rn(__fsub_rn(t, s), y);
  s = t;
}

__global__ void __launch_bounds__(kLabelThreads) k_pair_labels(LabelArgs a) {
  __shared__ float4 tile[kLabelTile];
  __shared__ float red[kLabelThreads / 32];
  for (int64_t p = blockIdx.x; p < a.n; p += gridDim.x) {
    const uint32_t g = a.pairs[2 * p], c = a.pairs[2 * p + 1];
    const uint32_t gf = a.g_first[g], gn = a.g_count[g];
    const uint2 ni = a.node_i[c];
    const uint32_t cf = ni.x, cn = ni.y & 0x7fffffffu;
    const double cx = a.com[3 * (size_t)c], cy = a.com[3 * (size_t)c + 1],
                 cz = a.com[3 * (size_t)c + 2];
    const float M = __double2float_rn(a.mass[c]);
    const float4 q0 = a.s_q0[c], q1 = a.s_q1[c];
    float worst = 0.0f;
    for (uint32_t i0 = 0; i0 < gn; i0 += kLabelThreads) {
      const uint32_t i = i0 + threadIdx.x;
      const bool on = i < gn;
      float xi = 0.0f, yi = 0.0f, zi = 0.0f;
      if (on) {
        xi = __double2float_rn(a.xs[gf + i] - cx);
        yi = __double2float_rn(a.ys[gf + i] - cy);
        zi = __double2float_rn(a.zs[gf + i] - cz);
      }
      float sx = 0.0f, sy = 0.0f, sz = 0.0f, kx = 0.0f, ky = 0.0f, kz = 0.0f;
      for (uint32_t j0 = 0; j0 < cn; j0 += kLabelTile) {
        const uint32_t nt = min((uint32_t)kLabelTile, cn - j0);
        __syncthreads();
        for (uint32_t t = threadIdx.x; t < nt; t += kLabelThreads) {
          const size_t j = (size_t)cf + j0 + t;
          tile[t] = make_float4(__double2float_rn(a.xs[j] - cx), __double2float_rn(a.ys[j] - cy),
                                __double2float_rn(a.zs[j] - cz), __double2float_rn(a.ms[j]));
        }
        __syncthreads();
        if (on) {
          for (uint32_t t = 0; t < nt; t++) {
            const float4 q = tile[t];
            const float dx = __fsub_rn(q.x, xi), dy = __fsub_rn(q.y, yi), dz = __fsub_rn(q.z, zi);
            const float r2 = __fadd_rn(mac_sq3(dx, dy, dz), a.eps2);
            if (r2 == 0.0f) continue;
            const float ri = __frsqrt_rn(r2);
            const float mr3 = __fmul_rn(__fmul_rn(q.w, ri), __fmul_rn(ri, ri));
            kahan(sx, kx, __fmul_rn(mr3, dx));
            kahan(sy, ky, __fmul_rn(mr3, dy));
            kahan(sz, kz, __fmul_rn(mr3, dz));
          }
        }
      }
      if (on) {
        // superparticle term at r = x_i - COM = (xi, yi, zi)
        const float r2 = __fadd_rn(mac_sq3(xi, yi, zi), a.eps2);
        float ax = 0.0f, ay = 0.0f, az = 0.0f;
        if (r2 > 0.0f) {
          const float ri = __frsqrt_rn(r2);
          const float ri2 = __fmul_rn(ri, ri);
          const float mr3 = __fmul_rn(__fmul_rn(M, ri), ri2);
          ax = -__fmul_rn(mr3, xi);
          ay = -__fmul_rn(mr3, yi);
          az = -__fmul_rn(mr3, zi);
          if (a.quad) {
            const float Qr0 = q0.x * xi + q0.w * yi + q1.x * zi;
            const float Qr1 = q0.w * xi + q0.y * yi + q1.y * zi;
            const float Qr2 = q1.x * xi + q1.y * yi + q0.z * zi;
            const float rQr = xi * Qr0 + yi * Qr1 + zi * Qr2;
            const float ri5 = ri2 * ri2 * ri, ri7 = ri5 * ri2;
            ax += Qr0 * ri5 - 2.5f * rQr * xi * ri7;
            ay += Qr1 * ri5 - 2.5f * rQr * yi * ri7;
            az += Qr2 * ri5 - 2.5f * rQr * zi * ri7;
          }
        }
        const float ex = ax - sx, ey = ay - sy, ez = az - sz;
        const float e = sqrtf(ex * ex + ey * ey + ez * ez) / a.amag_s[gf + i];
        worst = (e > worst || e != e) ? e : worst;
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float t = __shfl_xor_sync(0xffffffffu, worst, o);
      worst = (t > worst || t != t) ? t : worst;
    }
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = worst;
    __syncthreads();
    if (threadIdx.x == 0) {
      float w = red[0];
      for (int k = 1; k < kLabelThreads / 32; k++) w = (red[k] > w || red[k] != red[k]) ? red[k] : w;
      float lab = w > 0.0f ? log2f(w) : -40.0f;
      if (!(lab <= 8.0f)) lab = 8.0f;
      if (lab < -40.0f) lab = -40.0f;
      a.label[p] = lab;
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// The network: FP16 rounding, inference, feature statistics, training
// ---------------------------------------------------------------------------
__global__ void k_fp16_round(float *w, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) w[i] = __half2float(__float2half_rn(w[i]));
}

// Inference on the tensor cores, as the walk runs it: each warp takes
// sixteen rows at a time.
constexpr int kFwdWarps = 8;
__global__ void __launch_bounds__(32 * kFwdWarps) k_mlp_forward(const float *__restrict__ w,
                                                               const float *__restrict__ feat,
                                                               int64_t n, float *__restrict__ out) {
  __shared__ __align__(16) MacFrag mf;
  __shared__ __align__(16) uint4 x16_all[kFwdWarps][16];
  mac_frag_load(mf, w, threadIdx.x, blockDim.x);
  __syncthreads();
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  uint4 *x16 = x16_all[wib];
  const int64_t stride = (int64_t)gridDim.x * kFwdWarps * 16;
  for (int64_t base = ((int64_t)blockIdx.x * kFwdWarps + wib) * 16; base < n; base += stride) {
    if (lane < 16) {
      float f[kMacNF];
      const int64_t s = base + lane;
#pragma unroll
      for (int k = 0; k < kMacNF; k++) f[k] = s < n ? feat[s * kMacNF + k] : 0.0f;
      x16[lane] = mac_row16(mf, f);
    }
    __syncwarp();
    const float2 y = mac_mma_rows(mf, x16, lane);
    if ((lane & 3) == 0) {
      const int64_t r = base + (lane >> 2);
      if (r < n) out[r] = y.x;
      if (r + 8 < n) out[r + 8] = y.y;
    }
    __syncwarp();
  }
}

// Per-block FP64 sums of each feature, its square and the target.
constexpr int kStatThreads = 256;
constexpr int kStatBlocks = 304;
__global__ void __launch_bounds__(kStatThreads) k_feat_stats(const float *__restrict__ feat,
                                                             const float *__restrict__ label,
                                                             int64_t n, double *__restrict__ part) {
  __shared__ double red[kStatThreads];
  double acc[2 * kMacNF + 1];
#pragma unroll
  for (int k = 0; k < 2 * kMacNF + 1; k++) acc[k] = 0.0;
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < n;
       s += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
    for (int k = 0; k < kMacNF; k++) {
      const double v = feat[s * kMacNF + k];
      acc[k] += v;
      acc[kMacNF + k] += v * v;
    }
    acc[2 * kMacNF] += label[s];
  }
  for (int k = 0; k < 2 * kMacNF + 1; k++) {
    red[threadIdx.x] = acc[k];
    __syncthreads();
    for (int o = kStatThreads / 2; o > 0; o >>= 1) {
      if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
      __syncthreads();
    }
    if (threadIdx.x == 0) part[(size_t)blockIdx.x * (2 * kMacNF + 1) + k] = red[0];
    __syncthreads();
  }
}

// mu, isd (FP16 values) and the initial output bias (mean target).
__global__ void k_feat_stats_final(const double *__restrict__ part, int nblk, int64_t n,
                                   float *__restrict__ w) {
  const int k = threadIdx.x;
  if (k >= kMacNF + 1) return;
  if (k == kMacNF) {
    double s = 0.0;
    for (int b = 0; b < nblk; b++) s += part[(size_t)b * (2 * kMacNF + 1) + 2 * kMacNF];
    w[kMacOffB3] = (float)(s / (double)n);
    return;
  }
  double s = 0.0, s2 = 0.0;
  for (int b = 0; b < nblk; b++) {
    s += part[(size_t)b * (2 * kMacNF + 1) + k];
    s2 += part[(size_t)b * (2 * kMacNF + 1) + kMacNF + k];
  }
  const double mean = s / (double)n;
  const double var = fmax(s2 / (double)n - mean * mean, 0.0);
  const double sd = fmax(sqrt(var), 1e-2);
  w[k] = __half2float(__float2half_rn((float)mean));
  w[kMacNF + k] = __half2float(__float2half_rn((float)(1.0 / sd)));
}

// Forward + backward over a tile of 128 samples; writes the block's partial
// gradient of the trained parameters (W1 .. b3) and partial squared error.
constexpr int kTile = 128;
constexpr int kPad = kMacNH + 1;
constexpr size_t kGradSmem =
    sizeof(float) * ((size_t)kMacNP + kTile * kMacNF + 4 * (size_t)kTile * kPad + kTile);

struct GradArgs {
  const float *w;
  const float *feat, *label;
  int64_t n, start, count;
  uint64_t mul, add;  // sample of batch position b: (mul * (start + b) + add) mod n
  float scale;        // 2 / count
  float *part;        // [blocks][kMacTrain]
  float *loss_part;   // [blocks]
};

__global__ void __launch_bounds__(kTile) k_mlp_grad(GradArgs a) {
  extern __shared__ float sm[];
  float *wsm = sm;
  float *X = wsm + kMacNP;
  float *H1 = X + kTile * kMacNF;
  float *H2 = H1 + kTile * kPad;
  float *D1 = H2 + kTile * kPad;
  float *D2 = D1 + kTile * kPad;
  float *DY = D2 + kTile * kPad;
  __shared__ float red[kTile / 32];
  for (int i = threadIdx.x; i < kMacNP; i += kTile) wsm[i] = a.w[i];
  __syncthreads();
  const int t = threadIdx.x;
  const int64_t b = (int64_t)blockIdx.x * kTile + t;
  float r2 = 0.0f;
  float *x = X + t * kMacNF, *h1 = H1 + t * kPad, *h2 = H2 + t * kPad, *d1 = D1 + t * kPad,
        *d2 = D2 + t * kPad;
  if (b < a.count) {
    const uint64_t pos = (uint64_t)(a.start + b);
    const int64_t s = (int64_t)((a.mul * pos + a.add) % (uint64_t)a.n);
#pragma unroll
    for (int k = 0; k < kMacNF; k++)
      x[k] = (a.feat[s * kMacNF + k] - wsm[k]) * wsm[kMacNF + k];
    for (int j = 0; j < kMacNH; j++) {
      float acc = wsm[kMacOffB1 + j];
#pragma unroll
      for (int k = 0; k < kMacNF; k++) acc = fmaf(wsm[kMacOffW1 + j * kMacNF + k], x[k], acc);
      h1[j] = acc > 0.0f ? acc : 0.0f;
    }
    float y = wsm[kMacOffB3];
    for (int j = 0; j < kMacNH; j++) {
      float acc = wsm[kMacOffB2 + j];
      for (int k = 0; k < kMacNH; k++) acc = fmaf(wsm[kMacOffW2 + j * kMacNH + k], h1[k], acc);
      h2[j] = acc > 0.0f ? acc : 0.0f;
      y = fmaf(wsm[kMacOffW3 + j], h2[j], y);
    }
    const float r = y - a.label[s];
    r2 = r * r;
    const float dy = a.scale * r;
    DY[t] = dy;
    for (int j = 0; j < kMacNH; j++) d2[j] = h2[j] > 0.0f ? dy * wsm[kMacOffW3 + j] : 0.0f;
    for (int k = 0; k < kMacNH; k++) {
      float acc = 0.0f;
      for (int j = 0; j < kMacNH; j++) acc = fmaf(d2[j], wsm[kMacOffW2 + j * kMacNH + k], acc);
      d1[k] = h1[k] > 0.0f ? acc : 0.0f;
    }
  } else {
#pragma unroll
    for (int k = 0; k < kMacNF; k++) x[k] = 0.0f;
    for (int j = 0; j < kMacNH; j++) h1[j] = h2[j] = d1[j] = d2[j] = 0.0f;
    DY[t] = 0.0f;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) r2 += __shfl_xor_sync(0xffffffffu, r2, o);
  if ((t & 31) == 0) red[t >> 5] = r2;
  __syncthreads();
  if (t == 0) {
    float s = 0.0f;
    for (int k = 0; k < kTile / 32; k++) s += red[k];
    a.loss_part[blockIdx.x] = s;
  }
  // parameter gradients, summed over the tile in sample order
  float *out = a.part + (size_t)blockIdx.x * kMacTrain;
  for (int p = t; p < kMacTrain; p += kTile) {
    const int q = p + kMacOffW1;
    float acc = 0.0f;
    if (q < kMacOffB1) {
      const int j = (q - kMacOffW1) / kMacNF, k = (q - kMacOffW1) % kMacNF;
      for (int s = 0; s < kTile; s++) acc = fmaf(D1[s * kPad + j], X[s * kMacNF + k], acc);
    } else if (q < kMacOffW2) {
      const int j = q - kMacOffB1;
      for (int s = 0; s < kTile; s++) acc += D1[s * kPad + j];
    } else if (q < kMacOffB2) {
      const int j = (q - kMacOffW2) / kMacNH, k = (q - kMacOffW2) % kMacNH;
      for (int s = 0; s < kTile; s++) acc = fmaf(D2[s * kPad + j], H1[s * kPad + k], acc);
    } else if (q < kMacOffW3) {
      const int j = q - kMacOffB2;
      for (int s = 0; s < kTile; s++) acc += D2[s * kPad + j];
    } else if (q < kMacOffB3) {
      const int k = q - kMacOffW3;
      for (int s = 0; s < kTile; s++) acc = fmaf(DY[s], H2[s * kPad + k], acc);
    } else {
      for (int s = 0; s < kTile; s++) acc += DY[s];
    }
    out[p] = acc;
  }
}

// Fixed-order sum of the block partials: the full gradient and loss.
__global__ void k_grad_sum(const float *__restrict__ part, const float *__restrict__ loss_part,
                           int nblk, int64_t count, float *__restrict__ grad,
                           float *__restrict__ loss) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < kMacOffW1) grad[p] = 0.0f;
  if (p < kMacTrain) {
    float s = 0.0f;
    for (int b = 0; b < nblk; b++) s += part[(size_t)b * kMacTrain + p];
    grad[kMacOffW1 + p] = s;
  }
  if (p == 0) {
    double s = 0.0;
    for (int b = 0; b < nblk; b++) s += loss_part[b];
    *loss = (float)(s / (double)count);
  }
}

struct AdamArgs {
  float *w, *m, *v;
  const float *part, *loss_part;
  int nblk;
  int64_t count;
  float lr, b1, b2, eps, c1, c2;  // c1 = 1 - b1^t, c2 = 1 - b2^t
  float *loss_out;
};

__global__ void k_adam(AdamArgs a) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < kMacTrain) {
    float g = 0.0f;
    for (int b = 0; b < a.nblk; b++) g += a.part[(size_t)b * kMacTrain + p];
    const float m = a.b1 * a.m[p] + (1.0f - a.b1) * g;
    const float v = a.b2 * a.v[p] + (1.0f - a.b2) * g * g;
    a.m[p] = m;
    a.v[p] = v;
    a.w[kMacOffW1 + p] -= a.lr * (m / a.c1) / (sqrtf(v / a.c2) + a.eps);
  }
  if (p == 0) {
    double s = 0.0;
    for (int b = 0; b < a.nblk; b++) s += a.loss_part[b];
    *a.loss_out = (float)(s / (double)a.count);
  }
}

// ---------------------------------------------------------------------------
// FP64 direct summation for sampled targets
// ---------------------------------------------------------------------------
constexpr int kDirThreads = 256;
__global__ void __launch_bounds__(kDirThreads) k_direct(const double *__restrict__ x,
                                                        const double *__restrict__ y,
                                                        const double *__restrict__ z,
                                                        const double *__restrict__ m, int64_t n,
                                                        const uint32_t *__restrict__ tgt,
                                                        double eps2, double *__restrict__ out) {
  __shared__ double red[4][kDirThreads];
  const uint32_t i = tgt[blockIdx.x];
  if ((int64_t)i >= n) {
    if (threadIdx.x < 4) out[4 * (size_t)blockIdx.x + threadIdx.x] = __longlong_as_double(0x7ff8000000000000ll);
    return;
  }
  const double xi = x[i], yi = y[i], zi = z[i];
  double sx = 0.0, sy = 0.0, sz = 0.0, sp = 0.0;
  for (int64_t j = threadIdx.x; j < n; j += kDirThreads) {
    if (j == (int64_t)i) continue;
    const double dx = x[j] - xi, dy = y[j] - yi, dz = z[j] - zi;
    const double r2 = dx * dx + dy * dy + dz * dz + eps2;
    if (r2 == 0.0) continue;
    const double rinv = 1.0 / sqrt(r2);
    const double mr = m[j] * rinv;
    const double mr3 = mr * rinv * rinv;
    sx += mr3 * dx;
    sy += mr3 * dy;
    sz += mr3 * dz;
    sp -= mr;
  }
  red[0][threadIdx.x] = sx;
  red[1][threadIdx.x] = sy;
  red[2][threadIdx.x] = sz;
  red[3][threadIdx.x] = sp;
  __syncthreads();
  for (int o = kDirThreads / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o)
      for (int k = 0; k < 4; k++) red[k][threadIdx.x] += red[k][threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x < 4) out[4 * (size_t)blockIdx.x + threadIdx.x] = red[threadIdx.x][0];
}

// ---------------------------------------------------------------------------
// Host helpers
// ---------------------------------------------------------------------------
struct Scratch {  // device allocations of one context-free call
  std::vector<void *> ptrs;
  ~Scratch() {
    for (void *p : ptrs) cudaFree(p);
  }
  template <class T>
  int get(T **out, size_t count) {
    void *p = nullptr;
    if (cudaMalloc(&p, sizeof(T) * (count > 0 ? count : 1)) != cudaSuccess) {
      cudaGetLastError();
      return AFD_ERR_OOM;
    }
    ptrs.push_back(p);
    *out = static_cast<T *>(p);
    return AFD_OK;
  }
};

struct DevGuard {
  int prev = -1;
  bool ok = true;
  explicit DevGuard(cudaStream_t s) {
    // run on the device the stream belongs to (the current device for NULL)
    if (!s) return;
    int dev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess) {
      ok = false;
      return;
    }
#if CUDART_VERSION >= 12080
    if (cudaStreamGetDevice(s, &dev) == cudaSuccess && dev != prev)
      ok = cudaSetDevice(dev) == cudaSuccess;
#endif
  }
  ~DevGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

uint64_t splitmix(uint64_t &s) {
  uint64_t z = (s += 0x9e3779b97f4a7c15ull);
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

double normal(uint64_t &s) {  // Box-Muller on two 53-bit uniforms
  const double u1 = ((double)(splitmix(s) >> 11) + 1.0) * (1.0 / 9007199254740993.0);
  const double u2 = (double)(splitmix(s) >> 11) * (1.0 / 9007199254740992.0);
  return std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2);
}

uint64_t gcd_u64(uint64_t a, uint64_t b) {
  while (b) {
    const uint64_t t = a % b;
    a = b;
    b = t;
  }
  return a;
}

int upload_rounded(const float *params, float *w, cudaStream_t s) {
  if (cudaMemcpyAsync(w, params, sizeof(float) * kMacNP, cudaMemcpyHostToDevice, s) != cudaSuccess)
    return AFD_ERR_CUDA;
  k_fp16_round<<<blocks_of(kMacNP, 256), 256, 0, s>>>(w, kMacNP);
  return ck();
}

}  // namespace

bool mac_usable(const afd_ctx *c) {
  return c->cfg.mac && c->mac_ready && c->n > 0 && c->amag_n == c->n && c->q_current;
}

int launch_group_amin(afd_ctx *c) {
  MAC_TRY(reserve(c->amag_s, sizeof(float) * (size_t)c->n));
  MAC_TRY(reserve(c->g_amin, sizeof(float) * (size_t)c->n_groups));
  if (c->n_groups == 0) return AFD_OK;
  k_group_amin<<<blocks_of(c->n_groups * 32, 256), 256, 0, c->stream>>>(
      c->n_groups, ptr<uint32_t>(c->g_first), ptr<uint32_t>(c->g_count), ptr<uint32_t>(c->perm),
      ptr<float>(c->amag), ptr<float>(c->amag_s), ptr<float>(c->g_amin));
  c->launches++;
  return ck();
}

int launch_amag(afd_ctx *c, const float *acc4) {
  MAC_TRY(reserve(c->amag, sizeof(float) * (size_t)c->n));
  c->amag_n = c->n;
  if (c->n == 0) return AFD_OK;
  k_amag<<<blocks_of(c->n, 256), 256, 0, c->stream>>>(reinterpret_cast<const float4 *>(acc4),
                                                      c->n, ptr<float>(c->amag));
  c->launches++;
  return ck();
}

}  // namespace afd

using namespace afd;

namespace {

struct CtxDevice {
  int prev = -1;
  bool ok = true;
  explicit CtxDevice(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) {
      ok = false;
      prev = -1;
      return;
    }
    if (prev != dev) ok = cudaSetDevice(dev) == cudaSuccess;
  }
  ~CtxDevice() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

int sync_status(afd_ctx *c) {
  int *pin = static_cast<int *>(c->pinned);
  if (cudaMemcpyAsync(pin, c->status.p, sizeof(int), cudaMemcpyDeviceToHost, c->stream) !=
          cudaSuccess ||
      cudaStreamSynchronize(c->stream) != cudaSuccess)
    return AFD_ERR_CUDA;
  return pin[0] ? status_to_error(pin[0]) : AFD_OK;
}

}  // namespace

extern "C" {

int afd_mac_set(afd_ctx *c, const float *params, double theta_lo, double theta_hi, double tau) {
  if (!c) return AFD_ERR_ARG;
  if (!params) {
    c->mac_ready = false;
    return AFD_OK;
  }
  if (!c->cfg.mac || !std::isfinite(theta_lo) || !std::isfinite(theta_hi) ||
      !std::isfinite(tau) || theta_lo < 0.0 || theta_hi < theta_lo)
    return AFD_ERR_ARG;
  CtxDevice g(c->device);
  if (!g.ok) return AFD_ERR_CUDA;
  MAC_TRY(reserve(c->mac_w, sizeof(float) * kMacNP));
  MAC_TRY(upload_rounded(params, ptr<float>(c->mac_w), c->stream));
  c->launches++;
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) return AFD_ERR_CUDA;
  const float lo = (float)theta_lo, hi = (float)theta_hi;
  c->mac_lo2 = lo * lo;
  c->mac_hi2 = hi * hi;
  c->mac_tau = (float)tau;
  c->mac_ready = true;
  return AFD_OK;
}

int afd_mac_set_reference(afd_ctx *c, const float *amag, int64_t n) {
  if (!c || n < 0 || (n > 0 && !amag) || !c->cfg.mac) return AFD_ERR_ARG;
  CtxDevice g(c->device);
  if (!g.ok) return AFD_ERR_CUDA;
  MAC_TRY(reserve(c->amag, sizeof(float) * (size_t)n));
  if (n > 0 && cudaMemcpyAsync(c->amag.p, amag, sizeof(float) * (size_t)n,
                               cudaMemcpyDeviceToDevice, c->stream) != cudaSuccess)
    return AFD_ERR_CUDA;
  c->amag_n = n;
  return AFD_OK;
}

int afd_mac_samples(afd_ctx *c, double theta_lo, double theta_hi, double keep, uint64_t seed,
                    int64_t cap, float *feat, float *label, uint32_t *pair, int64_t *n_out) {
  if (!c || !n_out || cap < 0 || !(keep >= 0.0) || !std::isfinite(theta_lo) ||
      !std::isfinite(theta_hi) || theta_lo < 0.0 || theta_hi < theta_lo)
    return AFD_ERR_ARG;
  if (cap > 0 && (!feat || !label)) return AFD_ERR_ARG;
  if (!c->cfg.mac) return AFD_ERR_ARG;
  if (!c->have_tree) return AFD_ERR_NO_TREE;
  if (c->amag_n != c->n) return AFD_ERR_NO_REFERENCE;
  CtxDevice gd(c->device);
  if (!gd.ok) return AFD_ERR_CUDA;
  *n_out = 0;
  const int64_t ng = c->n_groups;
  if (ng == 0) return AFD_OK;
  if (!c->q_current) MAC_TRY(launch_moments(c, false, true));  // after reusing steps
  MAC_TRY(launch_group_amin(c));
  MAC_TRY(reserve(c->band_cnt, sizeof(uint32_t) * (size_t)ng));
  MAC_TRY(reserve(c->band_off, sizeof(uint64_t) * (size_t)(ng + 1)));
  BandArgs a;
  a.n_groups = ng;
  a.boxf = ptr<float>(c->g_boxf);
  a.g_first = ptr<uint32_t>(c->g_first);
  a.g_root = ptr<uint32_t>(c->g_root);
  a.node_f = ptr<float4>(c->node_f);
  a.node_i = ptr<uint2>(c->node_i);
  a.child = ptr<uint32_t>(c->c_child);
  const float lo = (float)theta_lo, hi = (float)theta_hi;
  a.lo2 = lo * lo;
  a.hi2 = hi * hi;
  a.keep_all = keep >= 1.0;
  a.keep_thr = a.keep_all ? 0xffffffffu : (uint32_t)(keep * 4294967296.0);
  a.seed = seed;
  a.cnt = ptr<uint32_t>(c->band_cnt);
  a.off = ptr<uint64_t>(c->band_off);
  a.pairs = nullptr;
  a.cap = 0;
  a.status = ptr<int>(c->status);
  a.iter_cap = (uint32_t)(c->n_cells + 64);
  const size_t smem = sizeof(uint32_t) * kBandWarps * kBandStack;
  if (cudaFuncSetAttribute(k_band<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
          cudaSuccess ||
      cudaFuncSetAttribute(k_band<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
          cudaSuccess)
    return AFD_ERR_CUDA;
  int64_t nb = (ng + kBandWarps - 1) / kBandWarps;
  if (nb > 152 * 8) nb = 152 * 8;
  k_band<false><<<(unsigned)nb, 32 * kBandWarps, smem, c->stream>>>(a);
  c->launches++;
  MAC_TRY(ck());
  MAC_TRY(scan_u32_to_u64(c, a.cnt, ptr<uint64_t>(c->band_off), ng));
  // pinned word 0 holds the status (sync_status), word 1 the total
  uint64_t *pin = static_cast<uint64_t *>(c->pinned) + 1;
  if (cudaMemcpyAsync(pin, ptr<uint64_t>(c->band_off) + ng, sizeof(uint64_t),
                      cudaMemcpyDeviceToHost, c->stream) != cudaSuccess)
    return AFD_ERR_CUDA;
  MAC_TRY(sync_status(c));
  const int64_t total = (int64_t)pin[0];
  *n_out = total;
  const int64_t m = total < cap ? total : cap;
  if (m == 0) return AFD_OK;
  uint32_t *pairs = pair;
  Scratch scratch;
  if (!pairs) MAC_TRY(scratch.get(&pairs, 2 * (size_t)m));
  a.pairs = pairs;
  a.cap = (uint64_t)m;
  k_band<true><<<(unsigned)nb, 32 * kBandWarps, smem, c->stream>>>(a);
  c->launches++;
  MAC_TRY(ck());
  const float e = (float)c->cfg.eps;
  k_pair_features<<<blocks_of(m, 256), 256, 0, c->stream>>>(
      m, pairs, ptr<float>(c->g_boxf), ptr<float4>(c->node_f), ptr<uint2>(c->node_i),
      ptr<float4>(c->s_hi), ptr<float4>(c->s_q0), ptr<float4>(c->s_q1), ptr<float>(c->g_amin),
      e * e, feat);
  c->launches++;
  MAC_TRY(ck());
  LabelArgs la;
  la.n = m;
  la.pairs = pairs;
  la.g_first = ptr<uint32_t>(c->g_first);
  la.g_count = ptr<uint32_t>(c->g_count);
  la.node_i = ptr<uint2>(c->node_i);
  la.xs = ptr<double>(c->xs);
  la.ys = ptr<double>(c->ys);
  la.zs = ptr<double>(c->zs);
  la.ms = ptr<double>(c->ms);
  la.com = ptr<double>(c->c_com);
  la.mass = ptr<double>(c->c_mass);
  la.s_q0 = ptr<float4>(c->s_q0);
  la.s_q1 = ptr<float4>(c->s_q1);
  la.amag_s = ptr<float>(c->amag_s);
  la.eps2 = e * e;
  la.quad = c->cfg.multipole;
  la.label = label;
  const int64_t lb = m < 152 * 16 ? m : 152 * 16;
  k_pair_labels<<<(unsigned)lb, kLabelThreads, 0, c->stream>>>(la);
  c->launches++;
  MAC_TRY(ck());
  return sync_status(c);
}

int afd_mac_info(afd_ctx *c, int64_t *out) {
  if (!c || !out) return AFD_ERR_ARG;
  out[0] = c->walk_learned ? 1 : 0;
  out[1] = out[2] = out[4] = 0;
  if (c->walk_learned && c->mac_cnt.p) {
    CtxDevice g(c->device);
    uint64_t *pin = static_cast<uint64_t *>(c->pinned);
    if (cudaMemcpyAsync(pin, c->mac_cnt.p, 3 * sizeof(uint64_t), cudaMemcpyDeviceToHost,
                        c->stream) != cudaSuccess ||
        cudaStreamSynchronize(c->stream) != cudaSuccess)
      return AFD_ERR_CUDA;
    out[1] = (int64_t)pin[0];
    out[2] = (int64_t)pin[1];
    out[4] = (int64_t)pin[2];
  }
  out[3] = (c->amag_n == c->n && c->n > 0) ? 1 : 0;
  return AFD_OK;
}

int afd_mlp_forward(const float *params, const float *feat, int64_t n, float *out, void *stream) {
  if (!params || n < 0 || (n > 0 && (!feat || !out))) return AFD_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  DevGuard g(s);
  if (!g.ok) return AFD_ERR_CUDA;
  Scratch scratch;
  float *w;
  MAC_TRY(scratch.get(&w, kMacNP));
  MAC_TRY(upload_rounded(params, w, s));
  if (n > 0) {
    const int64_t want = (n + 16 * kFwdWarps - 1) / (16 * kFwdWarps);
    k_mlp_forward<<<(unsigned)(want < 152 * 8 ? want : 152 * 8), 32 * kFwdWarps, 0, s>>>(w, feat, n,
                                                                                          out);
  }
  MAC_TRY(ck());
  return cudaStreamSynchronize(s) == cudaSuccess ? AFD_OK : AFD_ERR_CUDA;
}

int afd_mlp_loss_grad(const float *params, const float *feat, const float *label, int64_t n,
                      float *grad, float *loss, void *stream) {
  if (!params || !grad || !loss || n < 1 || n > (1 << 24) || !feat || !label) return AFD_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  DevGuard g(s);
  if (!g.ok) return AFD_ERR_CUDA;
  const int nblk = (int)((n + kTile - 1) / kTile);
  Scratch scratch;
  float *w, *part, *lpart, *gd, *ld;
  MAC_TRY(scratch.get(&w, kMacNP));
  MAC_TRY(scratch.get(&part, (size_t)nblk * kMacTrain));
  MAC_TRY(scratch.get(&lpart, (size_t)nblk));
  MAC_TRY(scratch.get(&gd, kMacNP));
  MAC_TRY(scratch.get(&ld, 1));
  if (cudaMemcpyAsync(w, params, sizeof(float) * kMacNP, cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)kGradSmem) != cudaSuccess)
    return AFD_ERR_CUDA;
  GradArgs a;
  a.w = w;
  a.feat = feat;
  a.label = label;
  a.n = n;
  a.start = 0;
  a.count = n;
  a.mul = 1;
  a.add = 0;
  a.scale = (float)(2.0 / (double)n);
  a.part = part;
  a.loss_part = lpart;
  k_mlp_grad<<<nblk, kTile, kGradSmem, s>>>(a);
  k_grad_sum<<<blocks_of(kMacNP, 256), 256, 0, s>>>(part, lpart, nblk, n, gd, ld);
  MAC_TRY(ck());
  if (cudaMemcpyAsync(grad, gd, sizeof(float) * kMacNP, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaMemcpyAsync(loss, ld, sizeof(float), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return AFD_ERR_CUDA;
  return AFD_OK;
}

int afd_mlp_train(const float *feat, const float *label, int64_t n, int epochs, int batch,
                  double lr, uint64_t seed, float *params, float *loss_hist, void *stream) {
  if (!feat || !label || !params || n < 1 || n > 0x7fffffff || epochs < 1 || batch < 1 ||
      batch > 65536 ||
      !(lr > 0.0) || !std::isfinite(lr))
    return AFD_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  DevGuard g(s);
  if (!g.ok) return AFD_ERR_CUDA;
  const int nblk = (batch + kTile - 1) / kTile;
  const int64_t steps_per_epoch = (n + batch - 1) / batch;
  const int64_t steps = steps_per_epoch * epochs;
  Scratch scratch;
  float *w, *m, *v, *part, *lpart, *lhist;
  double *stat;
  MAC_TRY(scratch.get(&w, kMacNP));
  MAC_TRY(scratch.get(&m, kMacTrain));
  MAC_TRY(scratch.get(&v, kMacTrain));
  MAC_TRY(scratch.get(&part, (size_t)nblk * kMacTrain));
  MAC_TRY(scratch.get(&lpart, (size_t)nblk));
  MAC_TRY(scratch.get(&lhist, (size_t)steps));
  MAC_TRY(scratch.get(&stat, (size_t)kStatBlocks * (2 * kMacNF + 1)));
  // initial weights: He-normal layers, zero biases (host, seeded)
  std::vector<float> w0(kMacNP, 0.0f);
  uint64_t rs = seed;
  for (int i = 0; i < kMacNH * kMacNF; i++)
    w0[kMacOffW1 + i] = (float)(normal(rs) * std::sqrt(2.0 / kMacNF));
  for (int i = 0; i < kMacNH * kMacNH; i++)
    w0[kMacOffW2 + i] = (float)(normal(rs) * std::sqrt(2.0 / kMacNH));
  for (int i = 0; i < kMacNH; i++) w0[kMacOffW3 + i] = (float)(normal(rs) * std::sqrt(1.0 / kMacNH));
  if (cudaMemcpyAsync(w, w0.data(), sizeof(float) * kMacNP, cudaMemcpyHostToDevice, s) !=
          cudaSuccess ||
      cudaMemsetAsync(m, 0, sizeof(float) * kMacTrain, s) != cudaSuccess ||
      cudaMemsetAsync(v, 0, sizeof(float) * kMacTrain, s) != cudaSuccess ||
      cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)kGradSmem) != cudaSuccess)
    return AFD_ERR_CUDA;
  // normalisation and initial output bias from the data
  k_feat_stats<<<kStatBlocks, kStatThreads, 0, s>>>(feat, label, n, stat);
  k_feat_stats_final<<<1, 32, 0, s>>>(stat, kStatBlocks, n, w);
  MAC_TRY(ck());
  const float b1 = 0.9f, b2 = 0.999f;
  double p1 = 1.0, p2 = 1.0;
  int64_t step = 0;
  for (int e = 0; e < epochs; e++) {
    // a fresh visiting order per epoch: k -> (mul k + add) mod n, gcd(mul, n) = 1
    uint64_t mul = 1, add = 0;
    if (n > 1) {
      do {
        mul = 1 + splitmix(rs) % (uint64_t)(n - 1);
      } while (gcd_u64(mul, (uint64_t)n) != 1);
      add = splitmix(rs) % (uint64_t)n;
    }
    const double lr_e = lr * (0.05 + 0.95 * 0.5 * (1.0 + std::cos(3.141592653589793 * e / epochs)));
    for (int64_t st = 0; st < n; st += batch, step++) {
      const int64_t cnt = (n - st) < batch ? (n - st) : batch;
      GradArgs a;
      a.w = w;
      a.feat = feat;
      a.label = label;
      a.n = n;
      a.start = st;
      a.count = cnt;
      a.mul = mul;
      a.add = add;
      a.scale = (float)(2.0 / (double)cnt);
      a.part = part;
      a.loss_part = lpart;
      const int nb = (int)((cnt + kTile - 1) / kTile);
      k_mlp_grad<<<nb, kTile, kGradSmem, s>>>(a);
      p1 *= b1;
      p2 *= b2;
      AdamArgs d;
      d.w = w;
      d.m = m;
      d.v = v;
      d.part = part;
      d.loss_part = lpart;
      d.nblk = nb;
      d.count = cnt;
      d.lr = (float)lr_e;
      d.b1 = b1;
      d.b2 = b2;
      d.eps = 1e-8f;
      d.c1 = (float)(1.0 - p1);
      d.c2 = (float)(1.0 - p2);
      d.loss_out = lhist + step;
      k_adam<<<blocks_of(kMacTrain, 256), 256, 0, s>>>(d);
    }
    MAC_TRY(ck());
  }
  std::vector<float> lh((size_t)steps);
  if (cudaMemcpyAsync(params, w, sizeof(float) * kMacNP, cudaMemcpyDeviceToHost, s) !=
          cudaSuccess ||
      cudaMemcpyAsync(lh.data(), lhist, sizeof(float) * (size_t)steps, cudaMemcpyDeviceToHost, s) !=
          cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return AFD_ERR_CUDA;
  if (loss_hist) {
    for (int e = 0; e < epochs; e++) {
      double acc = 0.0, wsum = 0.0;
      for (int64_t k = 0; k < steps_per_epoch; k++) {
        const int64_t st = k * batch;
        const double cnt = (double)((n - st) < batch ? (n - st) : batch);
        acc += lh[(size_t)(e * steps_per_epoch + k)] * cnt;
        wsum += cnt;
      }
      loss_hist[e] = (float)(acc / wsum);
    }
  }
  return AFD_OK;
}

int afd_direct_sum(const double *x, const double *y, const double *z, const double *m, int64_t n,
                   const uint32_t *targets, int64_t n_t, double eps, double *out, void *stream) {
  if (n < 0 || n_t < 0 || n_t > 0x7fffffff || !std::isfinite(eps) || eps < 0.0) return AFD_ERR_ARG;
  if (n_t == 0) return AFD_OK;
  if (!x || !y || !z || !m || !targets || !out) return AFD_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  DevGuard g(s);
  if (!g.ok) return AFD_ERR_CUDA;
  k_direct<<<(unsigned)n_t, kDirThreads, 0, s>>>(x, y, z, m, n, targets, eps * eps, out);
  return ck();
}

}  // extern "C"
