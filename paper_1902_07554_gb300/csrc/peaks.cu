// peaks.cu -- measured FMA throughput of the FP32 and FP64 pipes.
//
// The engine's predicates run an FP32 stage, then an FP64 filter: the
// arithmetic roofs of its kernels are these two pipes' rates on this GPU.
// The kernel keeps CHAINS independent fused multiply-add chains per thread
// (enough to cover the pipe latency) on 8 blocks of 256 threads per SM, and
// is timed with CUDA events; the rate counts 2 flops per FMA.
#include <cuda_runtime.h>

#include <algorithm>

#include "../../include/dt.h"

namespace {

constexpr int CHAINS = 8;

template <typename T>
__global__ void __launch_bounds__(256) k_fma_chains(T x, T y, int iters, T* sink) {
  T a[CHAINS];
#pragma unroll
  for (int c = 0; c < CHAINS; c++) a[c] = (T)(threadIdx.x + c) * (T)1e-3;
#pragma unroll 4
  for (int it = 0; it < iters; it++) {
#pragma unroll
    for (int c = 0; c < CHAINS; c++) a[c] = fma(a[c], x, y);
  }
  T s = 0;
#pragma unroll
  for (int c = 0; c < CHAINS; c++) s += a[c];
  // never true for the arguments passed below; keeps the chains live
  if (s == (T)-12345.0) sink[blockIdx.x] = s;
}

template <typename T>
int measure(int device, int reps, double* tflops) {
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess || sms < 1) {
    cudaGetLastError();
    return DT_E_CUDA;
  }
  const unsigned grid = (unsigned)sms * 8, block = 256;
  // about 10-40 ms per launch on either pipe
  const int iters = sizeof(T) == 4 ? (1 << 18) : (1 << 13);
  T* sink = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaStream_t s = nullptr;
  int rc = DT_OK;
  if (cudaMalloc(&sink, sizeof(T) * grid) != cudaSuccess || cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) ||
      cudaEventCreate(&e0) || cudaEventCreate(&e1)) {
    cudaGetLastError();
    rc = DT_E_CUDA;
  }
  double best = 0.0;
  // x slightly below 1 and y small: the chains stay finite for any iteration count
  const T x = (T)0.999999, y = (T)1e-7;
  for (int r = -1; rc == DT_OK && r < reps; r++) {   // r = -1: untimed warm-up
    cudaEventRecord(e0, s);
    k_fma_chains<T><<<grid, block, 0, s>>>(x, y, iters, sink);
    cudaEventRecord(e1, s);
    if (cudaEventSynchronize(e1) != cudaSuccess) { cudaGetLastError(); rc = DT_E_CUDA; break; }
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    if (r >= 0 && ms > 0) {
      const double flops = 2.0 * CHAINS * (double)iters * grid * block;
      best = std::max(best, flops / (ms * 1e-3) / 1e12);
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (s) cudaStreamDestroy(s);
  if (sink) cudaFree(sink);
  if (rc == DT_OK) *tflops = best;
  return rc;
}

}  // namespace

extern "C" int dt_measure_fma_rate(int device, int precision, int reps, double* tflops) {
  if (!tflops || (precision != 32 && precision != 64) || reps < 1 || reps > 1000) return DT_E_ARG;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return DT_E_ARG;
  }
  int prev = -1;
  if (cudaGetDevice(&prev) != cudaSuccess) { cudaGetLastError(); prev = -1; }
  if (cudaSetDevice(device) != cudaSuccess) { cudaGetLastError(); return DT_E_CUDA; }
  const int rc = precision == 32 ? measure<float>(device, reps, tflops) : measure<double>(device, reps, tflops);
  if (prev >= 0) cudaSetDevice(prev);
  return rc;
}
