// noalloc.cu -- sample selection (Alg. 2 (sampling)) without any allocation.
//
// Some callers cannot call cudaMalloc at all: code running under a memory
// pool it does not own, inside an allocator callback, in a process whose
// allocations are capped or audited, or in a real-time path where an
// allocation (and its implicit synchronisation) is not allowed.  For them,
// dt_select_sample_noalloc runs the same radix selection as dt_triangulate's
// divide step, but keeps all of its scratch in one file-scope device array of
// fixed size instead of pool buffers, and needs no context.
//
// The scratch array (struct NoAllocScratch, 9240 bytes) lives in every GPU
// that loads this library until the process exits.  All calls share it, and
// it keeps the contents of the last call: every call clears what must start
// at zero.  Two calls whose kernels overlap on the GPU (different streams, or
// different host threads on one device) race on it; callers must order them.
//
// Set-up: the first call on a device, with that device current, looks up the
// device address of the array with cudaGetSymbolAddress and caches it; make
// that first call before any stream capture.
#include <mutex>

#include "common.cuh"

namespace gdt {

constexpr int NA_BLOCKS = 1024;     // chunks of the index range (per-chunk counts)
constexpr int NA_THREADS = 256;

struct NoAllocScratch {
  unsigned long long prefix, mask;  // radix-select state
  long long rank;
  int hist[256];
  int counts[NA_BLOCKS];
  int offs[NA_BLOCKS];
};

static __device__ __align__(256) NoAllocScratch g_noalloc_scratch;

__device__ __forceinline__ unsigned long long na_key(unsigned long long s, long long i) {
  return splitmix64(s ^ (unsigned long long)i);
}

__global__ void k_na_reset(NoAllocScratch* S, long long eta) {
  int t = threadIdx.x;
  if (t == 0) { S->prefix = 0; S->mask = 0; S->rank = eta - 1; }
  for (int i = t; i < 256; i += blockDim.x) S->hist[i] = 0;
  for (int i = t; i < NA_BLOCKS; i += blockDim.x) { S->counts[i] = 0; S->offs[i] = 0; }
}

__global__ void k_na_hist(long long n, unsigned long long s, NoAllocScratch* S, int shift) {
  __shared__ int h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  unsigned long long pre = S->prefix, msk = S->mask;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    unsigned long long k = na_key(s, i);
    if ((k & msk) == pre) atomicAdd(&h[(k >> shift) & 255], 1);
  }
  __syncthreads();
  if (h[threadIdx.x]) atomicAdd(&S->hist[threadIdx.x], h[threadIdx.x]);
}

__global__ void k_na_pick(NoAllocScratch* S, int shift) {
  long long r = S->rank, cum = 0;
  int b = 0;
  for (; b < 256; b++) {
    if (cum + S->hist[b] > r) break;
    cum += S->hist[b];
  }
  if (b > 255) b = 255;
  S->prefix |= (unsigned long long)b << shift;
  S->mask |= 255ull << shift;
  S->rank = r - cum;
  for (int i = 0; i < 256; i++) S->hist[i] = 0;
}

// Block b owns the contiguous index chunk [b*chunk, (b+1)*chunk).
__global__ void k_na_count(long long n, long long chunk, unsigned long long s, NoAllocScratch* S) {
  __shared__ int tot;
  if (threadIdx.x == 0) tot = 0;
  __syncthreads();
  long long lo = blockIdx.x * chunk, hi = min(n, lo + chunk);
  int c = 0;
  unsigned long long K = S->prefix;
  for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) c += na_key(s, i) <= K;
  atomicAdd(&tot, c);
  __syncthreads();
  if (threadIdx.x == 0) S->counts[blockIdx.x] = tot;
}

__global__ void k_na_scan(NoAllocScratch* S) {
  if (threadIdx.x == 0) {
    int run = 0;
    for (int b = 0; b < NA_BLOCKS; b++) { S->offs[b] = run; run += S->counts[b]; }
  }
}

// Ordered write of each chunk's selected indices (tile by tile, block scan).
__global__ void k_na_write(long long n, long long chunk, unsigned long long s, const NoAllocScratch* S, int* out) {
  __shared__ int sh[NA_THREADS];
  long long lo = blockIdx.x * chunk, hi = min(n, lo + chunk);
  int base = S->offs[blockIdx.x];
  unsigned long long K = S->prefix;
  for (long long t0 = lo; t0 < hi; t0 += NA_THREADS) {
    long long i = t0 + threadIdx.x;
    int f = (i < hi && na_key(s, i) <= K) ? 1 : 0;
    sh[threadIdx.x] = f;
    __syncthreads();
    for (int off = 1; off < NA_THREADS; off <<= 1) {
      int v = threadIdx.x >= off ? sh[threadIdx.x - off] : 0;
      __syncthreads();
      sh[threadIdx.x] += v;
      __syncthreads();
    }
    if (f) out[base + sh[threadIdx.x] - 1] = (int)i;
    int total = sh[NA_THREADS - 1];
    __syncthreads();
    base += total;
  }
}

static std::mutex g_na_mu;
static void* g_na_addr[64];
static int g_na_sms[64];

// Restores the caller's current device on every return path: the call has
// no context of its own, so it must not leave `device` current behind it.
struct DeviceGuard {
  int prev = -1;
  DeviceGuard() { if (cudaGetDevice(&prev) != cudaSuccess) { cudaGetLastError(); prev = -1; } }
  ~DeviceGuard() { if (prev >= 0) cudaSetDevice(prev); }
};

}  // namespace gdt

using namespace gdt;

extern "C" int dt_select_sample_noalloc(int device, void* cuda_stream, int64_t n, int64_t eta, uint64_t seed,
                                        int32_t* out_ids) {
  if (device < 0 || device >= 64 || !out_ids) return DT_E_ARG;
  if (n < 1 || n > 0x7fffffffLL || eta < 1 || eta > n) return DT_E_ARG;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device >= ndev) { cudaGetLastError(); return DT_E_ARG; }
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, out_ids) != cudaSuccess) { cudaGetLastError(); return DT_E_ARG; }
  if (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged) return DT_E_ARG;   // needs device memory
  if (a.type == cudaMemoryTypeDevice && a.device != device) return DT_E_ARG;                 // of this device
  DeviceGuard guard;
  if (cudaSetDevice(device) != cudaSuccess) { cudaGetLastError(); return DT_E_CUDA; }
  NoAllocScratch* S = nullptr;
  int sms = 0;
  {
    std::lock_guard<std::mutex> lk(g_na_mu);
    if (!g_na_addr[device]) {
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
        cudaGetLastError();
        return DT_E_CUDA;
      }
      int m = 0;
      if (cudaDeviceGetAttribute(&m, cudaDevAttrMultiProcessorCount, device) != cudaSuccess || m < 1) {
        cudaGetLastError();
        return DT_E_CUDA;
      }
      g_na_sms[device] = m;
      g_na_addr[device] = p;
    }
    S = (NoAllocScratch*)g_na_addr[device];
    sms = g_na_sms[device];
  }
  cudaStream_t s = (cudaStream_t)cuda_stream;
  unsigned long long sm = splitmix64(seed);
  k_na_reset<<<1, 256, 0, s>>>(S, (long long)eta);
  // histogram passes: at most 8 blocks of 256 threads per SM (grid-stride loop)
  unsigned g = (unsigned)std::min<long long>((n + 255) / 256, (long long)sms * 8);
  for (int shift = 56; shift >= 0; shift -= 8) {
    k_na_hist<<<g, 256, 0, s>>>((long long)n, sm, S, shift);
    k_na_pick<<<1, 1, 0, s>>>(S, shift);
  }
  long long chunk = (n + NA_BLOCKS - 1) / NA_BLOCKS;
  k_na_count<<<NA_BLOCKS, NA_THREADS, 0, s>>>((long long)n, chunk, sm, S);
  k_na_scan<<<1, 32, 0, s>>>(S);
  k_na_write<<<NA_BLOCKS, NA_THREADS, 0, s>>>((long long)n, chunk, sm, S, out_ids);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return DT_E_CUDA;
  e = cudaStreamSynchronize(s);
  return e == cudaSuccess ? DT_OK : DT_E_CUDA;
}
