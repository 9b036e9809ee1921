// Device buffers and device-wide exclusive scans (three phases: per-tile
// totals, one-block scan of the totals, per-tile scan with its base).
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
  if (bits & kStWalkIter) return AFD_ERR_TIMEOUT;
  if (bits & kStOverflow) return AFD_ERR_LIST_OVERFLOW;
  if (bits & kStBadRadius) return AFD_ERR_BAD_RADIUS;
  return AFD_OK;
}

namespace {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 16;
constexpr int kScanTile = kScanThreads * kScanItems;
constexpr int kScanOneBlock = 1024;

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

template <class Tin, class Tout>
__global__ void k_scan_reduce(const Tin *__restrict__ in, int64_t n, Tout *__restrict__ part) {
  const int64_t base = (int64_t)blockIdx.x * kScanTile;
  Tout s = 0;
  for (int k = threadIdx.x; k < kScanTile; k += kScanThreads) {
    const int64_t i = base + k;
    if (i < n) s += (Tout)in[i];
  }
  Tout total;
  block_exclusive<Tout, kScanThreads>(s, &total);
  if (threadIdx.x == 0) part[blockIdx.x] = total;
}

template <class Tout>
__global__ void k_scan_single(Tout *__restrict__ part, int64_t nb, Tout *__restrict__ out_total) {
  const int64_t per = (nb + kScanOneBlock - 1) / kScanOneBlock;
  const int64_t b0 = (int64_t)threadIdx.x * per;
  Tout s = 0;
  for (int64_t k = 0; k < per; k++)
    if (b0 + k < nb) s += part[b0 + k];
  Tout total;
  Tout ex = block_exclusive<Tout, kScanOneBlock>(s, &total);
  for (int64_t k = 0; k < per; k++)
    if (b0 + k < nb) {
      Tout v = part[b0 + k];
      part[b0 + k] = ex;
      ex += v;
    }
  if (threadIdx.x == 0) *out_total = total;
}

template <class Tin, class Tout>
__global__ void k_scan_down(const Tin *__restrict__ in, int64_t n, const Tout *__restrict__ part,
                            Tout *__restrict__ out) {
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  Tout v[kScanItems];
  Tout s = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; k++) {
    const int64_t i = base + k;
    v[k] = i < n ? (Tout)in[i] : Tout(0);
    s += v[k];
  }
  Tout total;
  Tout ex = block_exclusive<Tout, kScanThreads>(s, &total) + part[blockIdx.x];
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
  int st = reserve(c->scan_tmp, sizeof(Tout) * (size_t)(nb + 1));
  if (st) return st;
  Tout *part = ptr<Tout>(c->scan_tmp);
  k_scan_reduce<Tin, Tout><<<(unsigned)nb, kScanThreads, 0, c->stream>>>(in, n, part);
  c->launches++;
  k_scan_single<Tout><<<1, kScanOneBlock, 0, c->stream>>>(part, nb, out + n);
  c->launches++;
  k_scan_down<Tin, Tout><<<(unsigned)nb, kScanThreads, 0, c->stream>>>(in, n, part, out);
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
