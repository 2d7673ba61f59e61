// Throughput probes for the roofline denominators that the measured-peaks file
// does not hold: FP64 and FP32 fused multiply-add rates of the SIMT pipes.  Each
// thread runs eight independent FMA chains so that latency is hidden; the
// result is 2 * FMAs / elapsed time (CUDA events on the given stream).
#include <cuda_runtime.h>

#include <cstdint>

namespace {

template <typename T>
__global__ void fma_chains(T* out, int iters, T a, T b) {
  T x0 = threadIdx.x, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3, x4 = x0 + 4, x5 = x0 + 5, x6 = x0 + 6, x7 = x0 + 7;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
      x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
    }
  }
  T s = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
  if (s == (T)12345.678) out[0] = s;  // keeps the chains alive
}

template <typename T>
int run(double* gflops, int reps, cudaStream_t stream) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 1;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 1;
  T* out = nullptr;
  if (cudaMallocAsync(&out, 64, stream) != cudaSuccess) return 1;
  const int blocks = sms * 8, threads = 256;
  const int iters = sizeof(T) == 8 ? 2048 : 16384;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  double best = 0.0;
  for (int r = 0; r < reps + 1; ++r) {
    cudaEventRecord(e0, stream);
    fma_chains<T><<<blocks, threads, 0, stream>>>(out, iters, (T)1.0000001, (T)1e-9);
    cudaEventRecord(e1, stream);
    if (cudaEventSynchronize(e1) != cudaSuccess) return 1;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    double fl = 2.0 * 64.0 * (double)iters * blocks * threads;
    if (r > 0 && fl / (ms * 1e6) > best) best = fl / (ms * 1e6);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFreeAsync(out, stream);
  *gflops = best;
  return cudaStreamSynchronize(stream) == cudaSuccess ? 0 : 1;
}

}  // namespace

extern "C" {
// Best-of-reps GFLOP/s of the FP64 FMA pipe; returns 0 on success.
int pngf_peak_fp64_gflops(double* gflops, int reps, void* stream) {
  return run<double>(gflops, reps, static_cast<cudaStream_t>(stream));
}
// Best-of-reps GFLOP/s of the FP32 FMA pipe; returns 0 on success.
int pngf_peak_fp32_gflops(double* gflops, int reps, void* stream) {
  return run<float>(gflops, reps, static_cast<cudaStream_t>(stream));
}
}
