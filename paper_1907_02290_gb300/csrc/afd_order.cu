// Counting sort of work items by their work, largest first (the protocol is
// in afd_order.cuh).
#include "afd_internal.cuh"
#include "afd_order.cuh"

namespace afd {
namespace {

__device__ __forceinline__ int order_bucket(uint32_t w, uint32_t wmax) {
  const int b = (int)(((uint64_t)(w & ~kOrderFlag) * kOrderBuckets) / ((uint64_t)wmax + 1u));
  return kOrderBuckets - 1 - b;
}

__global__ void k_order_hist(int64_t n, const uint32_t *__restrict__ work,
                             uint32_t *__restrict__ hist) {
  __shared__ uint32_t h[kOrderBuckets];
  for (int b = threadIdx.x; b < kOrderBuckets; b += blockDim.x) h[b] = 0u;
  __syncthreads();
  const uint32_t wmax = hist[kOrderBuckets];
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x)
    if (work[k] != kNoItem) atomicAdd(&h[order_bucket(work[k], wmax)], 1u);
  __syncthreads();
  for (int b = threadIdx.x; b < kOrderBuckets; b += blockDim.x)
    if (h[b]) atomicAdd(&hist[b], h[b]);
}

// one block of kOrderBuckets threads: bucket counts -> first position of
// each bucket (exclusive scan), in place
__global__ void k_order_scan(uint32_t *__restrict__ hist) {
  __shared__ uint32_t v[kOrderBuckets];
  const int t = threadIdx.x;
  v[t] = hist[t];
  __syncthreads();
  for (int o = 1; o < kOrderBuckets; o <<= 1) {
    const uint32_t add = t >= o ? v[t - o] : 0u;
    __syncthreads();
    v[t] += add;
    __syncthreads();
  }
  hist[t] = t > 0 ? v[t - 1] : 0u;
}

__global__ void k_order_scatter(int64_t n, int64_t base, const uint32_t *__restrict__ work,
                                uint32_t *__restrict__ hist, uint32_t *__restrict__ order) {
  const uint32_t wmax = hist[kOrderBuckets];
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t w = work[k];
    if (w == kNoItem) continue;
    const uint32_t pos = atomicAdd(&hist[order_bucket(w, wmax)], 1u);
    if (AFD_IN(pos, (uint64_t)n, "order position"))
      order[pos] = (uint32_t)(base + k) | (w & kOrderFlag);
  }
}

}  // namespace

cudaError_t order_by_work(cudaStream_t s, int64_t n, int64_t base, const uint32_t *work,
                          uint32_t *hist, uint32_t *order, int64_t *launches) {
  if (n <= 0) return cudaSuccess;
  constexpr int kT = 256;
  const int64_t want = (n + kT - 1) / kT;
  const unsigned nb = (unsigned)(want < 152 * 8 ? want : 152 * 8);
  k_order_hist<<<nb, kT, 0, s>>>(n, work, hist);
  k_order_scan<<<1, kOrderBuckets, 0, s>>>(hist);
  k_order_scatter<<<nb, kT, 0, s>>>(n, base, work, hist, order);
  *launches += 3;
  return cudaGetLastError();
}

}  // namespace afd
