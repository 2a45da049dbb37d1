// Roofline denominators measured on the device the library runs on: the FP64 and
// FP32 fused multiply-add rates of the CUDA cores and the device-to-device copy
// bandwidth of HBM.  The assembly, operator-product and orthogonalisation kernels of
// this library are bound by the FP64 pipe or by HBM, so their roofline fractions are
// taken against these numbers, measured in the same process as the kernels.
//
// FP64/FP32: every thread runs ILP independent multiply-add chains a <- a*b + c for
// `iters` steps (b just below 1, so the values stay bounded), on a grid that fills
// every SM with 8 blocks of 256 threads; flops = 2 x threads x ILP x iters.  The sum
// of the chains is stored so that the compiler keeps them.  Copy: one pass of 16-byte
// loads and stores over a buffer pair; bytes = read + write.  Each figure is the best
// of several timed launches (CUDA events) after a warm-up launch.
#include <cuda_runtime.h>

#include "iga_internal.h"

namespace {

template <typename T, int ILP>
__global__ void __launch_bounds__(256) k_fma_chains(T *__restrict__ out, int iters, T b, T c) {
  T a[ILP];
#pragma unroll
  for (int k = 0; k < ILP; k++) a[k] = (T)(threadIdx.x + k);
  for (int it = 0; it < iters; it++) {
#pragma unroll
    for (int k = 0; k < ILP; k++) a[k] = fma(a[k], b, c);
  }
  T s = 0;
#pragma unroll
  for (int k = 0; k < ILP; k++) s += a[k];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(256) k_copy16(const float4 *__restrict__ src, float4 *__restrict__ dst, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = src[i];
}

template <typename F>
static cudaError_t best_ms(cudaStream_t s, int reps, F launch, float *best) {
  cudaEvent_t a, b;
  cudaError_t ce = cudaEventCreate(&a);
  if (ce) return ce;
  ce = cudaEventCreate(&b);
  if (ce) {
    cudaEventDestroy(a);
    return ce;
  }
  launch();  // warm-up
  *best = 1e30f;
  for (int r = 0; r < reps && ce == cudaSuccess; r++) {
    cudaEventRecord(a, s);
    launch();
    cudaEventRecord(b, s);
    ce = cudaEventSynchronize(b);
    float ms = 0.f;
    if (ce == cudaSuccess) ce = cudaEventElapsedTime(&ms, a, b);
    if (ce == cudaSuccess && ms < *best) *best = ms;
  }
  if (ce == cudaSuccess) ce = cudaGetLastError();
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return ce;
}

}  // namespace

extern "C" iga_status iga_measure_peaks(void *stream, iga_peaks *out) {
  if (!out) return IGA_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return IGA_ECUDA;
  const int blocks = sms * 8, threads = 256;
  const int64_t nthr = (int64_t)blocks * threads;
  void *sink = nullptr;
  if (cudaMalloc(&sink, nthr * sizeof(double)) != cudaSuccess) return IGA_ENOMEM;
  constexpr int ILP64 = 8, ILP32 = 16;
  const int it64 = 2048, it32 = 8192;
  float ms64 = 0.f, ms32 = 0.f, msc = 0.f;
  cudaError_t ce = best_ms(s, 5, [&] {
    k_fma_chains<double, ILP64><<<blocks, threads, 0, s>>>((double *)sink, it64, 0.9999999, 1e-7);
  }, &ms64);
  if (ce == cudaSuccess)
    ce = best_ms(s, 5, [&] {
      k_fma_chains<float, ILP32><<<blocks, threads, 0, s>>>((float *)sink, it32, 0.9999f, 1e-4f);
    }, &ms32);
  cudaFree(sink);
  if (ce != cudaSuccess) return IGA_ECUDA;
  // copy: 2 x 512 MiB, several times the 126 MB L2
  const size_t bytes = (size_t)512 << 20;
  void *src = nullptr, *dst = nullptr;
  if (cudaMalloc(&src, bytes) != cudaSuccess) return IGA_ENOMEM;
  if (cudaMalloc(&dst, bytes) != cudaSuccess) {
    cudaFree(src);
    return IGA_ENOMEM;
  }
  ce = cudaMemsetAsync(src, 0, bytes, s);
  const int64_t n16 = (int64_t)(bytes / 16);
  if (ce == cudaSuccess)
    ce = best_ms(s, 10, [&] { k_copy16<<<sms * 8, 256, 0, s>>>((const float4 *)src, (float4 *)dst, n16); }, &msc);
  cudaFree(src);
  cudaFree(dst);
  if (ce != cudaSuccess) return IGA_ECUDA;
  out->fp64_tflops = 2.0 * nthr * ILP64 * (double)it64 / (ms64 * 1e-3) / 1e12;
  out->fp32_tflops = 2.0 * nthr * ILP32 * (double)it32 / (ms32 * 1e-3) / 1e12;
  out->copy_gbs = 2.0 * (double)bytes / (msc * 1e-3) / 1e9;
  out->sms = sms;
  return IGA_OK;
}
