// common.cuh -- shared definitions for the GB300 Delaunay kernels.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/dt.h"

namespace gdt {

// Vertex code of the infinite vertex inside a simplex; a dead simplex has
// DEAD in slot 0 and, in its neighbour slot 0, a redirect to a live simplex
// created by the same insertion.
constexpr int INF_V = -1;
constexpr int DEAD = -2;
// Neighbour links are packed as (simplex << 2) | facet.
__host__ __device__ __forceinline__ int pack_nb(int s, int f) { return (s << 2) | f; }
__host__ __device__ __forceinline__ int nb_simplex(int p) { return p >> 2; }
__host__ __device__ __forceinline__ int nb_face(int p) { return p & 3; }

// Device-side status word.  Kernels never trap: they record the first error
// code here and return.
struct DevStatus {
  int error;          // first DT_E_* code seen (0 = ok)
  int detail;         // kernel-specific detail (which check)
  int overflow_cav;   // a candidate's cavity exceeded its scratch capacity
  int pad;
  unsigned long long exact_calls;   // exact-arithmetic fallbacks taken
  int dbg[16];        // diagnostics of the first internal error
};

__device__ __forceinline__ void set_error(DevStatus* st, int code, int detail) {
  if (atomicCAS(&st->error, 0, code) == 0) st->detail = detail;
}

// murmur3 fmix32: a bijection on 32-bit words, used to give every point a
// distinct pseudo-random insertion priority.
__host__ __device__ __forceinline__ uint32_t fmix32(uint32_t h) {
  h ^= h >> 16; h *= 0x85ebca6bu;
  h ^= h >> 13; h *= 0xc2b2ae35u;
  h ^= h >> 16;
  return h;
}

// SplitMix64 step (advance by the golden-ratio increment, then finalise).
__host__ __device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

template <typename T>
__host__ __device__ __forceinline__ T ceil_div(T a, T b) { return (a + b - 1) / b; }

}  // namespace gdt

#define CUDA_OK(expr)                                                     \
  do {                                                                    \
    cudaError_t _e = (expr);                                              \
    if (_e != cudaSuccess) return gdt_cuda_fail(_e, #expr, __FILE__, __LINE__); \
  } while (0)

int gdt_cuda_fail(cudaError_t e, const char* what, const char* file, int line);
