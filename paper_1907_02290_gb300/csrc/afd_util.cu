// Device buffers and device-wide exclusive scans (one launch: tiles taken in
// input order from a counter publish their totals and find their bases by
// decoupled look-back over the preceding tiles).
#include "afd_internal.cuh"

namespace afd {

int reserve(DevBuf &b, size_t bytes) {
  if (bytes == 0) bytes = 16;
  if (b.cap >= bytes) return AFD_OK;
  if (b.p) {
    cudaFree(b.p);
    b.p = nullptr;
    b.cap = 0;
  }
  size_t want = bytes + bytes / 8;  // headroom against small growth
  if (cudaMalloc(&b.p, want) != cudaSuccess) {
    cudaGetLastError();
    b.p = nullptr;
    return AFD_ERR_OOM;
  }
  b.cap = want;
  return AFD_OK;
}

void release(DevBuf &b) {
  if (b.p) cudaFree(b.p);
  b.p = nullptr;
  b.cap = 0;
}

int status_to_error(int bits) {
  if (bits & kStNonFinite) return AFD_ERR_NONFINITE;
  if (bits & kStWalkStack) return AFD_ERR_WALK_STACK;
  if (bits & (kStWalkIter | kStSpin | kStClimb)) return AFD_ERR_TIMEOUT;
  if (bits & kStOverflow) return AFD_ERR_LIST_OVERFLOW;
  if (bits & kStBadRadius) return AFD_ERR_BAD_RADIUS;
  return AFD_OK;
}

namespace {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 16;
constexpr int kScanTile = kScanThreads * kScanItems;

// Exclusive scan of one value per thread across the block; the block total
// is returned through *total. NT <= 1024.
template <class T, int NT>
__device__ T block_exclusive(T v, T *total) {
  __shared__ T warp_sums[NT / 32];
  __shared__ T block_total;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  T inc = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T t = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += t;
  }
  if (lane == 31) warp_sums[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    T w = lane < NT / 32 ? warp_sums[lane] : T(0);
    T winc = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      T t = __shfl_up_sync(0xffffffffu, winc, o);
      if (lane >= o) winc += t;
    }
    if (lane < NT / 32) warp_sums[lane] = winc - w;
    if (lane == NT / 32 - 1) block_total = winc;
  }
  __syncthreads();
  T res = warp_sums[warp] + inc - v;
  *total = block_total;
  __syncthreads();
  return res;
}

// Look-back words: the tile total (or inclusive prefix) in bits 0-61, the
// state in bits 62-63 (0: not yet published).
constexpr unsigned long long kScanAgg = 1ull << 62, kScanPrefix = 2ull << 62;
constexpr unsigned long long kScanValue = (1ull << 62) - 1ull;
constexpr uint32_t kScanSpinLimit = 1u << 22;  // polls of one predecessor's word

// look[t] are the tiles' look-back words and look[nb] the tile counter, all
// zero at launch; out[n] receives the total.
template <class Tin, class Tout>
__global__ void __launch_bounds__(kScanThreads) k_scan(const Tin *__restrict__ in, int64_t n,
                                                       Tout *__restrict__ out,
                                                       unsigned long long *look, int64_t nb,
                                                       int *status) {
  __shared__ unsigned long long s_tile, s_base;
  if (threadIdx.x == 0) s_tile = atomicAdd(&look[nb], 1ull);
  __syncthreads();
  const int64_t tile = (int64_t)s_tile;
  const int64_t base = tile * kScanTile + (int64_t)threadIdx.x * kScanItems;
  Tout v[kScanItems];
  Tout s = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; k++) {
    const int64_t i = base + k;
    v[k] = i < n ? (Tout)in[i] : Tout(0);
    s += v[k];
  }
  Tout total;
  Tout ex = block_exclusive<Tout, kScanThreads>(s, &total);
  if (threadIdx.x == 0) {
    volatile unsigned long long *vl = look;
    unsigned long long excl = 0;
    if (tile == 0) {
      vl[0] = kScanPrefix | ((unsigned long long)total & kScanValue);
    } else {
      vl[tile] = kScanAgg | ((unsigned long long)total & kScanValue);
      for (int64_t t = tile - 1; t >= 0; t--) {
        unsigned long long w = vl[t];
        for (uint32_t k = 0; (w & ~kScanValue) == 0ull; k++) {
          if (k == kScanSpinLimit) {  // give up: the result is wrong, the call fails
            atomicOr(status, kStSpin);
            w = kScanPrefix;
            break;
          }
          __nanosleep(32);
          w = vl[t];
        }
        excl += w & kScanValue;
        if ((w & ~kScanValue) == kScanPrefix) break;
      }
      vl[tile] = kScanPrefix | ((excl + (unsigned long long)total) & kScanValue);
    }
    s_base = excl;
    if (tile == nb - 1) out[n] = (Tout)(excl + (unsigned long long)total);
  }
  __syncthreads();
  ex += (Tout)s_base;
#pragma unroll
  for (int k = 0; k < kScanItems; k++) {
    const int64_t i = base + k;
    if (i < n) out[i] = ex;
    ex += v[k];
  }
}

template <class Tin, class Tout>
int scan_impl(afd_ctx *c, const Tin *in, Tout *out, int64_t n) {
  const int64_t nb = (n + kScanTile - 1) / kScanTile;
  if (nb == 0) {
    if (cudaMemsetAsync(out, 0, sizeof(Tout), c->stream) != cudaSuccess) return AFD_ERR_CUDA;
    return AFD_OK;
  }
  int st = reserve(c->scan_tmp, sizeof(unsigned long long) * (size_t)(nb + 1));
  if (st) return st;
  unsigned long long *look = ptr<unsigned long long>(c->scan_tmp);
  if (cudaMemsetAsync(look, 0, sizeof(unsigned long long) * (size_t)(nb + 1), c->stream) !=
      cudaSuccess)
    return AFD_ERR_CUDA;
  k_scan<Tin, Tout><<<(unsigned)nb, kScanThreads, 0, c->stream>>>(in, n, out, look, nb,
                                                                  ptr<int>(c->status));
  c->launches++;
  return cudaGetLastError() == cudaSuccess ? AFD_OK : AFD_ERR_CUDA;
}

}  // namespace

int scan_u32(afd_ctx *c, const uint32_t *in, uint32_t *out, int64_t n) {
  return scan_impl<uint32_t, uint32_t>(c, in, out, n);
}

int scan_u32_to_u64(afd_ctx *c, const uint32_t *in, uint64_t *out, int64_t n) {
  return scan_impl<uint32_t, uint64_t>(c, in, out, n);
}

}  // namespace afd
