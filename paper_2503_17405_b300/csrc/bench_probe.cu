// Throughput probe for the benchmark's roofline denominators (libfsmc_probe.so, loaded by
// bench.py; not part of libfsmc.so or its C ABI).  The paper has no counterpart: it measures, on
// the device the benchmark runs on and at whatever clocks it runs, the peak rates of the units
// the sampler kernels are bound by -- single- and double-precision multiply-add, and the
// multi-function unit's base-2 exponential and logarithm (ex2.approx, lg2.approx).
//
// Every thread runs eight independent chains of one operation for a fixed number of iterations,
// with eight blocks of 256 threads per SM (2048 threads), so each scheduler always has an
// independent instruction of that kind to issue.  The chains' sum is compared with a value it
// cannot take, which keeps the work live without a store per thread.  A rate is the launch's
// operations over its CUDA-event time, after one untimed launch.
#include <cuda_runtime.h>

namespace {

constexpr int kChains = 8;
enum Op { FMA = 0, EX2 = 1, LG2 = 2 };

template <typename T, int OP>
__global__ void __launch_bounds__(256) probe_kernel(int iters, T b, T c, T* sink) {
  T acc[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) acc[i] = T(1) + T(i) * T(1e-3) + T(threadIdx.x) * T(1e-6);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < kChains; ++i) {
      if constexpr (OP == FMA) {
        acc[i] = fma(acc[i], b, c);
      } else if constexpr (OP == EX2) {
        float y;  // 2^x iterated runs off to +inf; the unit's rate does not depend on the value
        asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"((float)acc[i]));
        acc[i] = y;
      } else {
        float y;  // log2 iterated from ~1 reaches 0, then -inf, then NaN: same rate throughout
        asm volatile("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"((float)acc[i]));
        acc[i] = y;
      }
    }
  }
  T s = T(0);
#pragma unroll
  for (int i = 0; i < kChains; ++i) s += acc[i];
  if (s == T(-1234.5)) sink[0] = s;  // never true: the chains stay live
}

// ops per element of work: 2 flops per multiply-add, 1 per exponential or logarithm
template <typename T, int OP>
cudaError_t time_probe(int sms, int iters, T* sink, cudaStream_t st, double* rate_t) {
  const int threads = 256, blocks = sms * 8;
  const T b = T(0.9999999), c = T(1e-7);
  probe_kernel<T, OP><<<blocks, threads, 0, st>>>(iters, b, c, sink);  // untimed
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess) e = cudaEventRecord(e0, st);
  if (e == cudaSuccess) {
    probe_kernel<T, OP><<<blocks, threads, 0, st>>>(iters, b, c, sink);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(e1, st);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  const double per = OP == FMA ? 2.0 : 1.0;
  if (e == cudaSuccess)
    *rate_t = per * kChains * (double)iters * (double)blocks * threads / (ms * 1e-3) / 1e12;
  return e;
}

}  // namespace

// Rates in units of 1e12 per second: FP32 and FP64 multiply-add TFLOP/s (two flops each),
// ex2.approx and lg2.approx tera-operations/s.  Returns 0, -1 for a NULL output, or the CUDA
// error code.  Allocates one 8-byte device buffer and one stream, frees both, and leaves the
// caller's current device as it was.  About 0.4 s of device time on a B300.
extern "C" int fsmc_bench_probe(int device, double* fp32_tflops, double* fp64_tflops, double* ex2_tops,
                                double* lg2_tops) {
  if (!fp32_tflops || !fp64_tflops || !ex2_tops || !lg2_tops) return -1;
  int prev = 0;
  cudaError_t e = cudaGetDevice(&prev);
  if (e != cudaSuccess) return (int)e;
  if ((e = cudaSetDevice(device)) != cudaSuccess) return (int)e;
  int sms = 0;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  double* sink = nullptr;
  cudaStream_t st = nullptr;
  if (e == cudaSuccess) e = cudaMalloc((void**)&sink, sizeof(double));
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  // about 0.13 s of single-precision, 0.2 s of double-precision multiply-adds and 0.05 s of each
  // multi-function operation at the nominal rates of a B300
  if (e == cudaSuccess) e = time_probe<float, FMA>(sms, 2048, (float*)sink, st, fp32_tflops);
  if (e == cudaSuccess) e = time_probe<double, FMA>(sms, 48, sink, st, fp64_tflops);
  if (e == cudaSuccess) e = time_probe<float, EX2>(sms, 512, (float*)sink, st, ex2_tops);
  if (e == cudaSuccess) e = time_probe<float, LG2>(sms, 512, (float*)sink, st, lg2_tops);
  if (st) cudaStreamDestroy(st);
  if (sink) cudaFree(sink);
  cudaSetDevice(prev);
  return e == cudaSuccess ? 0 : (int)e;
}
