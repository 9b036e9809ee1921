// Root-cell reduction that allocates nothing (afd_root_cell_static).
//
// Some callers cannot allocate device memory: their device memory is owned
// by another allocator (a framework's memory pool holding the whole GPU), or
// they run where no allocation may happen after start-up (cudaMalloc and
// cudaFree can synchronise the device and stall a latency-critical loop).
// afd_create allocates, so such callers cannot use a context. This variant
// of the root-cell kernel keeps its per-block partials, block counter and
// non-finite flag in a file-scope static device array instead: every GPU
// that loads the library holds that array (kScratchBytes) until the process
// exits, and every call on a device shares it.
#include <cfloat>
#include <mutex>

#include "afd_internal.cuh"

namespace {

constexpr int kThreads = 256;
constexpr int kBlocks = 608;  // grid cap: one partial slot per block
constexpr size_t kPartBytes = sizeof(unsigned long long) * 6 * kBlocks;  // 29184
constexpr size_t kCounterOffset = (kPartBytes + 255) / 256 * 256;    // 29184 (256-aligned)
constexpr size_t kScratchBytes = kCounterOffset + 256;               // 29440
constexpr int64_t kMaxParticles = ((int64_t)1 << 31) - 1;
constexpr int kMaxDevices = 64;

// Shared by every call on a device. Host code must not pass this symbol to
// a kernel: in host code it names a host-side stand-in, not device memory.
static __device__ __align__(256) unsigned char g_root_scratch[kScratchBytes];

struct DeviceScratch {
  unsigned char *ptr = nullptr;  // device address of g_root_scratch
};
DeviceScratch g_scratch[kMaxDevices];
std::mutex g_scratch_mu;

// Same reduction and root rule as the context path (the order-preserving
// integer keys of the doubles, so that -0 and +0 come out as afd_tree_build
// gives them, and the side from root_side): centre (min+max)/2 per axis,
// side = smallest power of two >= 1.000001 * largest extent (1 when the
// extent is 0, and the root (0, 0, 0, 1) when n = 0).
__global__ void __launch_bounds__(kThreads) k_root_static(
    const double *__restrict__ x, const double *__restrict__ y, const double *__restrict__ z,
    const double *__restrict__ m, int64_t n, unsigned char *scratch, double *__restrict__ root,
    int *__restrict__ nonfinite) {
  unsigned long long *part = reinterpret_cast<unsigned long long *>(scratch);
  unsigned *counter = reinterpret_cast<unsigned *>(scratch + kCounterOffset);
  unsigned *flag = counter + 1;
  unsigned long long klo[3] = {~0ull, ~0ull, ~0ull}, khi[3] = {0ull, 0ull, 0ull};
  int bad = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double v[3] = {x[i], y[i], z[i]};
    bad |= !isfinite(m[i]);
#pragma unroll
    for (int d = 0; d < 3; d++) {
      bad |= !isfinite(v[d]);
      afd::box_keys(v[d], klo[d], khi[d]);
    }
  }
  __shared__ unsigned long long sh[kThreads / 32][6];
  __shared__ bool last;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int d = 0; d < 3; d++) {
    klo[d] = afd::warp_min_key(klo[d]);
    khi[d] = afd::warp_max_key(khi[d]);
  }
  if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(flag, 1u);
  if (lane == 0)
    for (int d = 0; d < 3; d++) {
      sh[warp][d] = klo[d];
      sh[warp][3 + d] = khi[d];
    }
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long b[6];
    for (int d = 0; d < 6; d++) b[d] = sh[0][d];
    for (int w = 1; w < kThreads / 32; w++)
      for (int d = 0; d < 3; d++) {
        b[d] = min(b[d], sh[w][d]);
        b[3 + d] = max(b[3 + d], sh[w][3 + d]);
      }
    for (int d = 0; d < 6; d++) part[blockIdx.x * 6 + d] = b[d];
    __threadfence();
    last = atomicAdd(counter, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last || threadIdx.x != 0) return;
  __threadfence();
  if (n == 0) {
    root[0] = root[1] = root[2] = 0.0;
    root[3] = 1.0;
    *nonfinite = 0;
    return;
  }
  unsigned long long b[6];
  for (int d = 0; d < 6; d++) b[d] = __ldcg(&part[d]);
  for (unsigned k = 1; k < gridDim.x; k++)
    for (int d = 0; d < 3; d++) {
      b[d] = min(b[d], __ldcg(&part[k * 6 + d]));
      b[3 + d] = max(b[3 + d], __ldcg(&part[k * 6 + 3 + d]));
    }
  const bool side_ok = afd::root_from_keys(b, b + 3, root);
  *nonfinite = (__ldcg(flag) || !side_ok) ? 1 : 0;
}

// Device address of the static array on the current device, looked up once
// per device (not stream-ordered; see the header).
int scratch_for_current_device(unsigned char **out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return AFD_ERR_CUDA;
  }
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch[dev].ptr) {
    void *p = nullptr;
    const cudaError_t rc = cudaGetSymbolAddress(&p, g_root_scratch);
    if (rc != cudaSuccess || p == nullptr) {
      cudaGetLastError();
      return AFD_ERR_CUDA;
    }
    g_scratch[dev].ptr = static_cast<unsigned char *>(p);
  }
  *out = g_scratch[dev].ptr;
  return AFD_OK;
}

}  // namespace

extern "C" int afd_root_cell_static(const double *x, const double *y, const double *z,
                                    const double *m, int64_t n, double *root_out,
                                    int *nonfinite_out, void *stream) {
  if (n < 0 || !root_out || !nonfinite_out) return AFD_ERR_ARG;
  if (n > kMaxParticles) return AFD_ERR_TOO_LARGE;
  if (n > 0 && (!x || !y || !z || !m)) return AFD_ERR_ARG;
  unsigned char *scratch = nullptr;
  int st = scratch_for_current_device(&scratch);
  if (st != AFD_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // The block counter and the non-finite flag must start at zero; the
  // partials are fully overwritten by each call.
  if (cudaMemsetAsync(scratch + kCounterOffset, 0, 2 * sizeof(unsigned), s) != cudaSuccess) {
    cudaGetLastError();
    return AFD_ERR_CUDA;
  }
  int64_t nb = (n + kThreads * 4 - 1) / (kThreads * 4);
  if (nb > kBlocks) nb = kBlocks;
  if (nb < 1) nb = 1;
  k_root_static<<<(unsigned)nb, kThreads, 0, s>>>(x, y, z, m, n, scratch, root_out,
                                                 nonfinite_out);
  if (cudaGetLastError() != cudaSuccess) return AFD_ERR_CUDA;
  return AFD_OK;
}
