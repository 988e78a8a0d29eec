// Fused multiply-add throughput probe (fsmc_probe_fma_peaks in include/fsmc.h).
//
// Every thread runs eight independent multiply-add chains acc = acc * b + c for a fixed number
// of iterations, with eight blocks of 256 threads per SM (2048 threads), so each
// scheduler always has an independent multiply-add to issue.  The chains' sum is compared with a
// value it cannot take, which keeps the arithmetic live without a store per thread.  The rate is
// the launch's multiply-adds x 2 over its CUDA-event time, after one untimed launch.
#include <cuda_runtime.h>

#include "engine_internal.h"

namespace {

constexpr int kChains = 8;

template <typename T>
__global__ void __launch_bounds__(256) fma_probe_kernel(int iters, T b, T c, T* sink) {
  T acc[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) acc[i] = T(1) + T(i) * T(1e-3) + T(threadIdx.x) * T(1e-6);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < kChains; ++i) acc[i] = fma(acc[i], b, c);
  }
  T s = T(0);
#pragma unroll
  for (int i = 0; i < kChains; ++i) s += acc[i];
  if (s == T(-1234.5)) sink[0] = s;  // never true: the chains stay live
}

template <typename T>
cudaError_t time_probe(int sms, int iters, T* sink, cudaStream_t st, double* tflops) {
  const int threads = 256, blocks = sms * 8;
  const T b = T(0.9999999), c = T(1e-7);
  fma_probe_kernel<T><<<blocks, threads, 0, st>>>(iters, b, c, sink);  // untimed
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess) e = cudaEventRecord(e0, st);
  if (e == cudaSuccess) {
    fma_probe_kernel<T><<<blocks, threads, 0, st>>>(iters, b, c, sink);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(e1, st);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (e == cudaSuccess)
    *tflops = 2.0 * kChains * (double)iters * (double)blocks * threads / (ms * 1e-3) / 1e12;
  return e;
}

}  // namespace

extern "C" fsmc_status fsmc_probe_fma_peaks(int device, double* fp32_tflops, double* fp64_tflops) {
  if (!fp32_tflops || !fp64_tflops) return fsmc_fail(FSMC_EINVAL, "fsmc_probe_fma_peaks: NULL output");
  int prev = 0;
  cudaError_t e = cudaGetDevice(&prev);
  if (e != cudaSuccess) return fsmc_cuda_fail(e, "cudaGetDevice");
  if ((e = cudaSetDevice(device)) != cudaSuccess) return fsmc_cuda_fail(e, "cudaSetDevice");
  int sms = 0;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  double* sink = nullptr;
  cudaStream_t st = nullptr;
  if (e == cudaSuccess) e = cudaMalloc((void**)&sink, sizeof(double));
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  // about 0.13 s of single-precision and 0.2 s of double-precision work at the nominal rates
  // (77 and 1.25 TFLOP/s on a B300)
  if (e == cudaSuccess) e = time_probe<float>(sms, 2048, (float*)sink, st, fp32_tflops);
  if (e == cudaSuccess) e = time_probe<double>(sms, 48, sink, st, fp64_tflops);
  if (st) cudaStreamDestroy(st);
  if (sink) cudaFree(sink);
  cudaSetDevice(prev);
  if (e != cudaSuccess) return fsmc_cuda_fail(e, "fsmc_probe_fma_peaks");
  return FSMC_OK;
}
