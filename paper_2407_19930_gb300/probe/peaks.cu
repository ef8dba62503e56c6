// FP64 peak probes for the roofline of the FP64 kernels: the DFMA pipe (SIMT fused multiply-add
// on registers) and the FP64 tensor path (mma.sync m8n8k4 .f64, the instruction the FP64 GEMM of
// the chi0 contraction issues).  Each probe keeps independent accumulator chains in registers,
// touches no memory in its loop, and is timed with CUDA events around one launch that fills
// every SM.  Not part of the library's C ABI: the benchmark loads it to measure the peaks live,
// on the GPU and clocks of the run.
#include <cuda_runtime.h>

#include <cstdio>

namespace {

constexpr int kChains = 8;

__global__ void __launch_bounds__(256) k_dfma(int iters, double seed, double *sink) {
  double a[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) a[c] = seed + threadIdx.x * 1e-9 + c * 1e-7;
  const double x = 1.0 - 1e-12, y = 1e-13;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = fma(a[c], x, y);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += a[c];
  if (s == 12345.678) sink[blockIdx.x] = s;   // never true for these inputs; keeps the loop live
}

__global__ void __launch_bounds__(256) k_dmma(int iters, double seed, double *sink) {
  double c0[kChains], c1[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) c0[c] = c1[c] = 0.0;
  const double a = seed + (threadIdx.x & 31) * 1e-9, b = 1.0 - 1e-12;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c)
      asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
                   : "+d"(c0[c]), "+d"(c1[c])
                   : "d"(a), "d"(b));
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += c0[c] + c1[c];
  if (s == 12345.678) sink[blockIdx.x] = s;
}

}  // namespace

// kind 0: DFMA (2 flops per lane and instruction), kind 1: DMMA m8n8k4 (512 flops per warp and
// instruction).  Launches ctas_per_sm x SMs CTAs of 256 threads, iters loop trips, once to warm
// up and once timed.  Returns 0 and writes TFLOP/s and the timed launch's milliseconds, or the
// CUDA error code.
extern "C" int librpa_probe_fp64(int kind, int iters, int ctas_per_sm, double *tflops, double *ms) {
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return (int)e;
  const int grid = sms * ctas_per_sm;
  double *sink = nullptr;
  if ((e = cudaMalloc(&sink, grid * sizeof(double))) != cudaSuccess) return (int)e;
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  for (int rep = 0; rep < 2; ++rep) {
    cudaEventRecord(a);
    if (kind == 0)
      k_dfma<<<grid, 256>>>(iters, 0.5, sink);
    else
      k_dmma<<<grid, 256>>>(iters, 0.5, sink);
    cudaEventRecord(b);
  }
  e = cudaEventSynchronize(b);
  if (e == cudaSuccess) e = cudaGetLastError();
  float t = 0.f;
  cudaEventElapsedTime(&t, a, b);
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  cudaFree(sink);
  if (e != cudaSuccess) return (int)e;
  const double per = kind == 0 ? 2.0 * kChains * 256.0 : 512.0 * kChains * 8.0;   // flops per CTA and trip
  *ms = t;
  *tflops = per * (double)grid * iters / (t * 1e-3) / 1e12;
  return 0;
}
