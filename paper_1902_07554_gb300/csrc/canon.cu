// canon.cu -- canonical output form: sorted global-index tuples, rows in
// lexicographic order.  Rows are bucketed by their smallest vertex (a
// counting sort over n buckets: one histogram, one scan, one scatter), then
// each bucket -- a handful of rows -- is sorted by one thread.
#include "ctx.cuh"

namespace gdt {

__device__ __forceinline__ void sort4(int& a, int& b, int& c, int& d) {
#define CSWAP(x, y) { if (x > y) { int t_ = x; x = y; y = t_; } }
  CSWAP(a, b) CSWAP(c, d) CSWAP(a, c) CSWAP(b, d) CSWAP(b, c)
#undef CSWAP
}
__device__ __forceinline__ void sort3(int& a, int& b, int& c) {
#define CSWAP(x, y) { if (x > y) { int t_ = x; x = y; y = t_; } }
  CSWAP(a, b) CSWAP(b, c) CSWAP(a, b)
#undef CSWAP
}

// Instance of an arena slot (binary search over the instance offsets).
__device__ __forceinline__ int inst_of_slot(const int* toff, int ninst, int s) {
  int lo = 0, hi = ninst - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (toff[mid] <= s) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Every live finite simplex in the used part of each instance's arena,
// mapped to global indices and sorted; keep (optional, per slot) filters.
// src (optional) receives, per row, the slot it came from plus src_base.
template <int D>
__global__ void k_collect_finite(const int4* tv, const int* toff, const int* tcount, int ninst, int nslots,
                                 const int* gid, const unsigned char* flag, int mode, int4* rows, int* nrows,
                                 int* src, int src_base) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  bool take = false;
  int4 r = make_int4(0, 0, 0, 0);
  if (s < nslots) {
    int i = inst_of_slot(toff, ninst, s);
    bool sel = mode == 0 || (mode == 1 && !flag[s]) || (mode == 2 && flag[s]);
    if (s < tcount[i] && sel) {
      int4 v = tv[s];
      bool fin = v.x >= 0 && v.y >= 0 && v.z >= 0 && (D == 2 || v.w >= 0);
      if (fin) {
        take = true;
        int a = gid[v.x], b = gid[v.y], c = gid[v.z], d = D == 3 ? gid[v.w] : 0x7fffffff;
        if (D == 3) sort4(a, b, c, d); else sort3(a, b, c);
        r = make_int4(a, b, c, d);
      }
    }
  }
  unsigned mask = __ballot_sync(0xffffffffu, take);
  if (!mask) return;
  int lane = threadIdx.x & 31, leader = __ffs(mask) - 1, base = 0;
  if (lane == leader) base = atomicAdd(nrows, __popc(mask));
  base = __shfl_sync(0xffffffffu, base, leader);
  if (take) {
    int pos = base + __popc(mask & ((1u << lane) - 1));
    rows[pos] = r;
    if (src) src[pos] = s + src_base;
  }
}

__global__ void k_bucket_count(const int4* rows, int64_t nrows, int* bucket_count) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < nrows) atomicAdd(&bucket_count[rows[i].x], 1);
}

// Scatter into buckets; the payload (optional) travels with its row.
__global__ void k_bucket_scatter(const int4* rows, const int* pay, int64_t nrows, const int* bstart, int* bfill,
                                 int4* out, int* pay_out) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= nrows) return;
  int4 r = rows[i];
  int pos = bstart[r.x] + atomicAdd(&bfill[r.x], 1);
  out[pos] = r;
  if (pay) pay_out[pos] = pay[i];
}

__device__ __forceinline__ bool row_less(const int4& a, const int4& b) {
  if (a.y != b.y) return a.y < b.y;
  if (a.z != b.z) return a.z < b.z;
  return a.w < b.w;
}

template <int D>
__global__ void k_bucket_sort(int4* rows, int* pay, const int* bstart, const int* bcount, int64_t nb, int32_t* out) {
  int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (b >= nb) return;
  int s = bstart[b], m = bcount[b];
  for (int i = 1; i < m; i++) {
    int4 x = rows[s + i];
    int px = pay ? pay[s + i] : 0;
    int j = i - 1;
    while (j >= 0 && row_less(x, rows[s + j])) {
      rows[s + j + 1] = rows[s + j];
      if (pay) pay[s + j + 1] = pay[s + j];
      j--;
    }
    rows[s + j + 1] = x;
    if (pay) pay[s + j + 1] = px;
  }
  for (int i = 0; i < m; i++) {
    int4 x = rows[s + i];
    int32_t* o = out + (int64_t)(s + i) * (D + 1);
    o[0] = x.x; o[1] = x.y; o[2] = x.z;
    if (D == 3) o[3] = x.w;
  }
}

// rows: unsorted canonical tuples (sorted within each row); nbuckets > every
// vertex id.  Writes *out (device, pool-owned) with nrows*(dim+1) int32.
// src (optional): a payload per input row; *src_out then receives the
// payload of each output row, in output order (pool-owned).
int canonicalize_rows(dt_ctx* c, int dim, const int4* rows, int64_t nrows, int64_t nbuckets, int32_t** out,
                      int64_t* nout, const std::string& tag, const int* src, int** src_out) {
  cudaStream_t s = c->stream;
  *nout = nrows;
  int32_t* o = (int32_t*)pool_get(c, tag + ".out", sizeof(int32_t) * (dim + 1) * std::max<int64_t>(nrows, 1));
  int* bc = (int*)pool_get(c, "canon.bc", 4 * nbuckets);
  int* bs = (int*)pool_get(c, "canon.bs", 4 * nbuckets);
  int* bf = (int*)pool_get(c, "canon.bf", 4 * nbuckets);
  int4* tmp = (int4*)pool_get(c, "canon.tmp", 16 * std::max<int64_t>(nrows, 1));
  int* pay = src ? (int*)pool_get(c, tag + ".src", 4 * std::max<int64_t>(nrows, 1)) : nullptr;
  if (!o || !bc || !bs || !bf || !tmp || (src && !pay)) return set_err(c, DT_E_NOMEM, "canonicalise buffers");
  *out = o;
  if (src_out) *src_out = pay;
  if (nrows == 0) return 0;
  CUDA_OK(cudaMemsetAsync(bc, 0, 4 * nbuckets, s));
  CUDA_OK(cudaMemsetAsync(bf, 0, 4 * nbuckets, s));
  unsigned g = (unsigned)ceil_div<int64_t>(nrows, 256);
  k_bucket_count<<<g, 256, (++c->launches, 0), s>>>(rows, nrows, bc);
  int rc = exclusive_scan_i32(c, bc, bs, nbuckets, nullptr);
  if (rc) return rc;
  k_bucket_scatter<<<g, 256, (++c->launches, 0), s>>>(rows, src, nrows, bs, bf, tmp, pay);
  unsigned gb = (unsigned)ceil_div<int64_t>(nbuckets, 128);
  if (dim == 2) k_bucket_sort<2><<<gb, 128, (++c->launches, 0), s>>>(tmp, pay, bs, bc, nbuckets, o);
  else k_bucket_sort<3><<<gb, 128, (++c->launches, 0), s>>>(tmp, pay, bs, bc, nbuckets, o);
  return 0;
}

// Collect the finite live simplices of an engine run as canonical rows in
// *rows (pool-owned), count in *nrows.  mode 0: all; 1: slots not flagged;
// 2: flagged slots only.
// src (optional) receives the pool-owned per-row source slot (+ src_base).
int collect_finite(dt_ctx* c, const EngineRun& run, const int* gid, const unsigned char* flag, int mode,
                   int4** rows, int64_t* nrows, const std::string& tag, int** src, int src_base) {
  cudaStream_t s = c->stream;
  int64_t ns = run.total_slots;
  int4* r = (int4*)pool_get(c, tag + ".rows", 16 * std::max<int64_t>(ns / 4, 16));
  int* cnt = (int*)pool_get(c, "collect.cnt", 16);
  if (!r || !cnt) return set_err(c, DT_E_NOMEM, "collect buffers");
  CUDA_OK(cudaMemsetAsync(cnt, 0, 4, s));
  // the rows buffer must hold every live finite simplex: at most the used slots
  int64_t used = 0;
  for (int i = 0; i < run.ninst; i++) used += run.h_tcount[i] - run.h_toff[i];
  r = (int4*)pool_get(c, tag + ".rows", 16 * std::max<int64_t>(used, 16));
  int* sr = src ? (int*)pool_get(c, tag + ".slot", 4 * std::max<int64_t>(used, 16)) : nullptr;
  if (!r || (src && !sr)) return set_err(c, DT_E_NOMEM, "collect rows");
  if (src) *src = sr;
  unsigned g = (unsigned)ceil_div<int64_t>(ns, 256);
  if (mode && !flag) mode = 0;
  if (run.dim == 2)
    k_collect_finite<2><<<g, 256, (++c->launches, 0), s>>>((const int4*)run.tv, run.toff, run.tcount, run.ninst, (int)ns, gid,
                                          flag, mode, r, cnt, sr, src_base);
  else
    k_collect_finite<3><<<g, 256, (++c->launches, 0), s>>>((const int4*)run.tv, run.toff, run.tcount, run.ninst, (int)ns, gid,
                                          flag, mode, r, cnt, sr, src_base);
  int h = 0;
  CUDA_OK(cudaMemcpyAsync(&h, cnt, 4, cudaMemcpyDeviceToHost, s));
  CUDA_OK(cudaStreamSynchronize(s));
  *rows = r;
  *nrows = h;
  return 0;
}

}  // namespace gdt
