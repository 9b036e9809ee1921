// Measured FP32 rate of the GPU (the F_GPU of the kernel model in Appendix
// A): every thread runs eight independent chains of packed f32x2 FMAs; the
// rate is lane-FMAs x 2 flops / CUDA-event time. afd_pipe_rates measures the
// other instruction streams the kernels rely on the same way: scalar FP32
// FMA, the MUFU reciprocal square root and packed half-precision FMA.
#include <cuda_fp16.h>

#include "afd_internal.cuh"

namespace {

constexpr int kProbeIter = 4096;
constexpr int kProbeThreads = 256;

__global__ void __launch_bounds__(kProbeThreads) k_fma_probe(float *sink, float a, float b) {
  unsigned long long x[8], A, B;
  asm("mov.b64 %0, {%1, %1};" : "=l"(A) : "f"(a));
  asm("mov.b64 %0, {%1, %1};" : "=l"(B) : "f"(b));
#pragma unroll
  for (int k = 0; k < 8; k++) {
    const float v = threadIdx.x * 1e-3f + k;
    asm("mov.b64 %0, {%1, %2};" : "=l"(x[k]) : "f"(v), "f"(0.5f * k));
  }
  for (int i = 0; i < kProbeIter; i++) {
#pragma unroll
    for (int k = 0; k < 8; k++)
      asm volatile("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(x[k]) : "l"(A), "l"(B));
  }
  unsigned long long s = 0;
#pragma unroll
  for (int k = 0; k < 8; k++) s ^= x[k];
  if (s == 0x123456789abcdefull) sink[0] = 1.0f;  // keeps the chains live
}

// kind 1: scalar fma.rn.f32; 2: rsqrt.approx.ftz.f32; 3: fma.rn.f16x2.
template <int KIND>
__global__ void __launch_bounds__(kProbeThreads) k_pipe_probe(float *sink, float a, float b) {
  float x[8];
  __half2 h[8];
  const __half2 ha = __floats2half2_rn(a, a), hb = __floats2half2_rn(b, b);
#pragma unroll
  for (int k = 0; k < 8; k++) {
    x[k] = threadIdx.x * 1e-3f + k + 1.0f;
    h[k] = __floats2half2_rn(x[k] * 1e-3f, 0.5f * k);
  }
  for (int i = 0; i < kProbeIter; i++) {
#pragma unroll
    for (int k = 0; k < 8; k++) {
      if (KIND == 1) x[k] = fmaf(x[k], a, b);
      if (KIND == 2) asm volatile("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(x[k]) : "f"(x[k] + b));
      if (KIND == 3) h[k] = __hfma2(h[k], ha, hb);
    }
  }
  float s = 0.0f;
#pragma unroll
  for (int k = 0; k < 8; k++) s += x[k] + __low2float(h[k]) + __high2float(h[k]);
  if (s == 1234.5f) sink[0] = s;  // keeps the chains live
}

template <class F>
int time_best(F launch, cudaStream_t s, cudaEvent_t e0, cudaEvent_t e1, float *best) {
  *best = 1e30f;
  for (int rep = 0; rep < 3; rep++) {  // the first launch also ramps the clocks
    cudaEventRecord(e0, s);
    launch();
    cudaEventRecord(e1, s);
    float ms = 0.0f;
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
      return AFD_ERR_CUDA;
    if (ms < *best) *best = ms;
  }
  return AFD_OK;
}

}  // namespace

extern "C" int afd_pipe_rates(int device, void *stream, double *out) {
  if (!out) return AFD_ERR_ARG;
  int prev = -1;
  cudaGetDevice(&prev);
  if (cudaSetDevice(device) != cudaSuccess) return AFD_ERR_CUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int sms = 0;
  float *sink = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int st = AFD_OK;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
      cudaMalloc(&sink, sizeof(float)) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
      cudaEventCreate(&e1) != cudaSuccess) {
    st = AFD_ERR_CUDA;
  } else {
    const unsigned grid = (unsigned)sms * 8u;
    const double lanes = 8.0 * kProbeIter * (double)grid * kProbeThreads;  // per lane-op kind
    float ms[4];
    st = time_best([&] { k_fma_probe<<<grid, kProbeThreads, 0, s>>>(sink, 0.999f, 1e-3f); }, s, e0,
                   e1, &ms[0]);
    if (st == AFD_OK)
      st = time_best([&] { k_pipe_probe<1><<<grid, kProbeThreads, 0, s>>>(sink, 0.999f, 1e-3f); },
                     s, e0, e1, &ms[1]);
    if (st == AFD_OK)
      st = time_best([&] { k_pipe_probe<2><<<grid, kProbeThreads, 0, s>>>(sink, 0.999f, 0.5f); },
                     s, e0, e1, &ms[2]);
    if (st == AFD_OK)
      st = time_best([&] { k_pipe_probe<3><<<grid, kProbeThreads, 0, s>>>(sink, 0.999f, 1e-3f); },
                     s, e0, e1, &ms[3]);
    if (st == AFD_OK) {
      out[0] = 2.0 * 2.0 * lanes / (ms[0] * 1e-3) / 1e12;  // packed: 2 lanes x 2 flops
      out[1] = 2.0 * lanes / (ms[1] * 1e-3) / 1e12;
      out[2] = lanes / (ms[2] * 1e-3) / 1e12;
      out[3] = 2.0 * 2.0 * lanes / (ms[3] * 1e-3) / 1e12;
    }
  }
  cudaGetLastError();
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (sink) cudaFree(sink);
  if (prev >= 0) cudaSetDevice(prev);
  return st;
}

extern "C" int afd_fp32_peak(int device, void *stream, double *tflops_out) {
  if (!tflops_out) return AFD_ERR_ARG;
  int prev = -1;
  cudaGetDevice(&prev);
  if (cudaSetDevice(device) != cudaSuccess) return AFD_ERR_CUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int sms = 0;
  float *sink = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int st = AFD_OK;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
      cudaMalloc(&sink, sizeof(float)) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
      cudaEventCreate(&e1) != cudaSuccess) {
    st = AFD_ERR_CUDA;
  } else {
    const unsigned grid = (unsigned)sms * 8u;
    float best = 1e30f;
    for (int rep = 0; rep < 3; rep++) {  // the first launch also ramps the clocks
      cudaEventRecord(e0, s);
      k_fma_probe<<<grid, kProbeThreads, 0, s>>>(sink, 0.999f, 1e-3f);
      cudaEventRecord(e1, s);
      float ms = 0.0f;
      if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
        st = AFD_ERR_CUDA;
        break;
      }
      if (ms < best) best = ms;
    }
    if (st == AFD_OK) {
      const double flops = 2.0 * 2.0 * 8.0 * kProbeIter * (double)grid * kProbeThreads;
      *tflops_out = flops / (best * 1e-3) / 1e12;
    }
  }
  cudaGetLastError();
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (sink) cudaFree(sink);
  if (prev >= 0) cudaSetDevice(prev);
  return st;
}
