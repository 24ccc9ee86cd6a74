// util.cu -- buffer pool, error reporting, device-wide exclusive scan.
#include <cstdio>
#include <string>

#include "ctx.cuh"

static thread_local std::string g_fail_msg;

int gdt_cuda_fail(cudaError_t e, const char* what, const char* file, int line) {
  char buf[512];
  snprintf(buf, sizeof(buf), "CUDA error %d (%s) in %s at %s:%d", (int)e, cudaGetErrorString(e), what, file,
           line);
  g_fail_msg = buf;
  cudaGetLastError();   // clear sticky-free errors so the context stays usable
  return DT_E_CUDA;
}

namespace gdt {

const char* last_cuda_fail() { return g_fail_msg.c_str(); }

void* pool_get(dt_ctx* c, const std::string& name, size_t bytes) {
  if (bytes == 0) bytes = 16;
  auto& b = c->pool[name];
  if (b.cap >= bytes) return b.p;
  if (b.p) cudaFree(b.p);
  b.p = nullptr;
  b.cap = 0;
  size_t want = bytes + bytes / 8 + 256;
  if (cudaMalloc(&b.p, want) != cudaSuccess) {
    cudaGetLastError();
    b.p = nullptr;
    return nullptr;
  }
  b.cap = want;
  return b.p;
}

void pool_free_all(dt_ctx* c) {
  for (auto& kv : c->pool)
    if (kv.second.p) cudaFree(kv.second.p);
  c->pool.clear();
}

int set_err(dt_ctx* c, int code, const std::string& msg) {
  c->err = msg;
  if (code == DT_E_CUDA && !g_fail_msg.empty()) c->err += std::string(": ") + g_fail_msg;
  return code;
}

int check_status(dt_ctx* c, const char* where) {
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return set_err(c, gdt_cuda_fail(e, where, __FILE__, __LINE__), where);
  e = cudaMemcpy(c->status_host, c->status, sizeof(DevStatus), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return set_err(c, gdt_cuda_fail(e, where, __FILE__, __LINE__), where);
  int code = c->status_host->error;
  if (code) {
    char buf[256];
    const int* d = c->status_host->dbg;
    snprintf(buf, sizeof(buf), "%s: device error %d (check %d) [%d %d %d %d %d %d %d %d %d %d %d %d]", where, code,
             c->status_host->detail, d[0], d[1], d[2], d[3], d[4], d[5], d[6], d[7], d[8], d[9], d[10], d[11]);
    return set_err(c, code, buf);
  }
  return 0;
}

// ---------------------------------------------------------------- scan
constexpr int SCAN_T = 512, SCAN_IPT = 4, SCAN_TILE = SCAN_T * SCAN_IPT;

template <typename T>
__global__ void k_scan_tiles(const T* in, T* out, T* sums, int64_t n) {
  __shared__ T sh[SCAN_T];
  int64_t base = (int64_t)blockIdx.x * SCAN_TILE + threadIdx.x * SCAN_IPT;
  T v[SCAN_IPT];
  T run = 0;
#pragma unroll
  for (int k = 0; k < SCAN_IPT; k++) {
    v[k] = (base + k < n) ? in[base + k] : T(0);
    T x = v[k];
    v[k] = run;
    run += x;
  }
  sh[threadIdx.x] = run;
  __syncthreads();
  for (int off = 1; off < SCAN_T; off <<= 1) {
    T add = threadIdx.x >= off ? sh[threadIdx.x - off] : T(0);
    __syncthreads();
    sh[threadIdx.x] += add;
    __syncthreads();
  }
  T excl = threadIdx.x ? sh[threadIdx.x - 1] : T(0);
#pragma unroll
  for (int k = 0; k < SCAN_IPT; k++)
    if (base + k < n) out[base + k] = v[k] + excl;
  if (threadIdx.x == SCAN_T - 1 && sums) sums[blockIdx.x] = sh[SCAN_T - 1];
}

template <typename T>
__global__ void k_scan_add(T* out, const T* offs, int64_t n) {
  int64_t i = (int64_t)blockIdx.x * SCAN_TILE + threadIdx.x;
  T o = offs[blockIdx.x];
  for (int k = 0; k < SCAN_IPT; k++, i += SCAN_T)
    if (i < n) out[i] += o;
}

template <typename T>
static int scan_rec(dt_ctx* c, const T* in, T* out, int64_t n, int depth) {
  int64_t nb = ceil_div<int64_t>(n, SCAN_TILE);
  if (nb == 1) {
    k_scan_tiles<T><<<1, SCAN_T, (++c->launches, 0), c->stream>>>(in, out, (T*)nullptr, n);
    return 0;
  }
  T* sums = (T*)pool_get(c, "scan.s" + std::to_string(depth), sizeof(T) * nb);
  T* soff = (T*)pool_get(c, "scan.o" + std::to_string(depth), sizeof(T) * nb);
  if (!sums || !soff) return set_err(c, DT_E_NOMEM, "scan");
  k_scan_tiles<T><<<(unsigned)nb, SCAN_T, (++c->launches, 0), c->stream>>>(in, out, sums, n);
  int rc = scan_rec<T>(c, sums, soff, nb, depth + 1);
  if (rc) return rc;
  k_scan_add<T><<<(unsigned)nb, SCAN_T, (++c->launches, 0), c->stream>>>(out, soff, n);
  return 0;
}

// Exclusive scan; if total_host is non-null, the total is returned there
// (synchronising the stream).
int exclusive_scan_i32(dt_ctx* c, const int* in, int* out, int64_t n, int* total_host) {
  if (n <= 0) { if (total_host) *total_host = 0; return 0; }
  int rc = scan_rec<int>(c, in, out, n, 0);
  if (rc) return rc;
  if (total_host) {
    int last_in = 0, last_out = 0;
    CUDA_OK(cudaMemcpyAsync(&last_in, in + n - 1, 4, cudaMemcpyDeviceToHost, c->stream));
    CUDA_OK(cudaMemcpyAsync(&last_out, out + n - 1, 4, cudaMemcpyDeviceToHost, c->stream));
    CUDA_OK(cudaStreamSynchronize(c->stream));
    *total_host = last_in + last_out;
  }
  return 0;
}

int exclusive_scan_i64(dt_ctx* c, const long long* in, long long* out, int64_t n) {
  if (n <= 0) return 0;
  return scan_rec<long long>(c, in, out, n, 100);
}

}  // namespace gdt
