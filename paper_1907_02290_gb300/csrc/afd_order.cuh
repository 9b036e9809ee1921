// Launch order of a kernel's work items by their work, largest first.
//
// A block's warp slots are freed only when its slowest warp ends, and blocks
// are dispatched in index order: items sorted by work put equal work in each
// block, and largest first the launch also ends without a few long items
// running alone. The order only schedules: a kernel launched through it must
// give the same results in any order.
//
// Protocol: the caller zeroes hist (kOrderBuckets + 2 words), runs its own
// kernel that writes work[k] for its n items (kNoItem: no item; bit 31 is a
// flag carried into the order; the work is the low 31 bits), raises
// hist[kOrderBuckets] to the largest work (atomicMax) and adds the number of
// items to hist[kOrderBuckets + 1]; then order_by_work writes
// order[0 .. items) = base + k (| the flag), largest work first: a counting
// sort over kOrderBuckets buckets of work.
#pragma once

#include <cstdint>

#include <cuda_runtime.h>

namespace afd {

constexpr int kOrderBuckets = 256;
constexpr uint32_t kNoItem = 0xffffffffu;
constexpr uint32_t kOrderFlag = 0x80000000u;
constexpr uint32_t kOrderWorkMax = 0x7ffffffeu;

// Adds a warp's largest work and item count into hist (every lane calls it).
__device__ __forceinline__ void order_reduce(uint32_t *hist, uint32_t wmax, uint32_t items) {
  for (int o = 16; o > 0; o >>= 1) {
    wmax = max(wmax, __shfl_xor_sync(0xffffffffu, wmax, o));
    items += __shfl_xor_sync(0xffffffffu, items, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMax(&hist[kOrderBuckets], wmax);
    if (items) atomicAdd(&hist[kOrderBuckets + 1], items);
  }
}

// hist, work, order: device; n items; launches three kernels on s and adds
// their count to *launches. Returns cudaGetLastError().
cudaError_t order_by_work(cudaStream_t s, int64_t n, int64_t base, const uint32_t *work,
                          uint32_t *hist, uint32_t *order, int64_t *launches);

}  // namespace afd
