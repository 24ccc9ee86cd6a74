// bbox.cuh -- per-instance axis-aligned bounding boxes of point sets, kept as
// order-preserving 64-bit keys so that they can be combined with atomicMin /
// atomicMax.  Points of one instance are contiguous in every caller, so a warp
// whose lanes share an instance reduces in registers first and issues one
// atomic per coordinate (a warp straddling two instances falls back to one
// atomic per lane).
#pragma once
#include "common.cuh"
#include "predicates.cuh"

namespace gdt {

// Order-preserving map of doubles to unsigned integers, and back.
__device__ __forceinline__ unsigned long long box_key(double x) {
  unsigned long long b = (unsigned long long)__double_as_longlong(x + 0.0);
  return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}
__device__ __forceinline__ double box_unkey(unsigned long long u) {
  unsigned long long b = (u >> 63) ? (u & 0x7fffffffffffffffull) : ~u;
  return __longlong_as_double((long long)b);
}

// ub: per instance lo[3], hi[3] keys.
static __global__ void k_box_init(unsigned long long* ub, int ninst) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < 6 * ninst) ub[i] = (i % 6) < 3 ? ~0ull : 0ull;
}

template <int D>
static __global__ void k_box_reduce(const typename PT<D>::T* P, const int* pinst, int64_t n, unsigned long long* ub) {
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < n;
       base += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = base + lane;
    const bool v = p < n;
    const int inst = v ? (pinst ? pinst[p] : 0) : -1;
    unsigned long long lo[3] = {~0ull, ~0ull, ~0ull}, hi[3] = {0, 0, 0};
    if (v)
      for (int c = 0; c < D; c++) lo[c] = hi[c] = box_key(comp(P[p], c));
    const int i0 = __shfl_sync(FULL, inst, 0);
    if (__all_sync(FULL, inst == i0 || inst < 0)) {
      for (int off = 16; off; off >>= 1)
        for (int c = 0; c < D; c++) {
          const unsigned long long a = __shfl_xor_sync(FULL, lo[c], off), b = __shfl_xor_sync(FULL, hi[c], off);
          lo[c] = a < lo[c] ? a : lo[c];
          hi[c] = b > hi[c] ? b : hi[c];
        }
      if (lane == 0)
        for (int c = 0; c < D; c++) {
          atomicMin(&ub[6 * i0 + c], lo[c]);
          atomicMax(&ub[6 * i0 + 3 + c], hi[c]);
        }
    } else if (v) {
      for (int c = 0; c < D; c++) {
        atomicMin(&ub[6 * inst + c], lo[c]);
        atomicMax(&ub[6 * inst + 3 + c], hi[c]);
      }
    }
  }
}

// Keys -> doubles (lo[3], hi[3] per instance; unused coordinates 0).
static __global__ void k_box_to_double(const unsigned long long* ub, int ninst, int dim, double* box) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 6 * ninst) return;
  box[i] = (i % 3) < dim ? box_unkey(ub[i]) : 0.0;
}

// Grid size of the reduction: enough blocks to fill the GPU, at most one pass.
__host__ inline unsigned box_grid(int64_t n) {
  int64_t b = (n + 255) / 256;
  return (unsigned)(b < 1 ? 1 : (b > 152 * 8 ? 152 * 8 : b));
}

}  // namespace gdt
