// sort.cu -- stable LSD radix sort of (key, value) pairs and stable ranks
// within groups.  8-bit digits; a tile of 1024 elements is processed as four
// stable sub-tiles of 256 (one element per thread), ranks inside a warp come
// from __match_any_sync, across warps from per-warp digit counts in shared
// memory.  Tile histograms are laid out digit-major so one exclusive scan
// yields every (digit, tile) output offset.
#include "ctx.cuh"
#include "sort.cuh"

namespace gdt {

constexpr int RS_T = 256, RS_IPT = 4, RS_TILE = RS_T * RS_IPT;

template <typename K>
__global__ void k_rs_hist(const K* keys, int64_t n, int shift, int* hist, int ntiles) {
  __shared__ int h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  int64_t base = (int64_t)blockIdx.x * RS_TILE;
  for (int it = 0; it < RS_IPT; it++) {
    int64_t i = base + it * RS_T + threadIdx.x;
    if (i < n) atomicAdd(&h[(int)((keys[i] >> shift) & 255)], 1);
  }
  __syncthreads();
  hist[(int64_t)threadIdx.x * ntiles + blockIdx.x] = h[threadIdx.x];
}

// Group histogram: g[i] in [0, ngroups) or negative (ignored), ngroups <= 256.
__global__ void k_grp_hist(const int* g, int64_t n, int* hist, int ntiles) {
  __shared__ int h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  int64_t base = (int64_t)blockIdx.x * RS_TILE;
  for (int it = 0; it < RS_IPT; it++) {
    int64_t i = base + it * RS_T + threadIdx.x;
    if (i < n) {
      int d = g[i];
      if (d >= 0 && d < 256) atomicAdd(&h[d], 1);
    }
  }
  __syncthreads();
  hist[(int64_t)threadIdx.x * ntiles + blockIdx.x] = h[threadIdx.x];
}

// Shared part: given digit d (256 = none) of this thread's element in the
// current sub-tile, returns its stable position among equal digits of the
// tile so far (base[d] + rank) and advances base[].
__device__ __forceinline__ int tile_rank(int d, int* base, int (*wcnt)[256]) {
  int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int j = threadIdx.x; j < 8 * 256; j += RS_T) wcnt[j >> 8][j & 255] = 0;
  __syncthreads();
  unsigned peers = __match_any_sync(0xffffffffu, d);
  int lrank = __popc(peers & ((1u << lane) - 1));
  if (d < 256 && lrank == 0) wcnt[warp][d] = __popc(peers);
  __syncthreads();
  int pos = -1;
  if (d < 256) {
    int r = base[d] + lrank;
    for (int w = 0; w < warp; w++) r += wcnt[w][d];
    pos = r;
  }
  __syncthreads();
  int add = 0;
  for (int w = 0; w < 8; w++) add += wcnt[w][threadIdx.x];
  base[threadIdx.x] += add;
  __syncthreads();
  return pos;
}

template <typename K, typename V>
__global__ void k_rs_scatter(const K* kin, const V* vin, K* kout, V* vout, int64_t n, int shift, const int* offs,
                             int ntiles) {
  __shared__ int base[256];
  __shared__ int wcnt[8][256];
  base[threadIdx.x] = offs[(int64_t)threadIdx.x * ntiles + blockIdx.x];
  __syncthreads();
  int64_t tb = (int64_t)blockIdx.x * RS_TILE;
  for (int it = 0; it < RS_IPT; it++) {
    int64_t i = tb + it * RS_T + threadIdx.x;
    K k = 0;
    V v = 0;
    int d = 256;
    if (i < n) { k = kin[i]; v = vin[i]; d = (int)((k >> shift) & 255); }
    int pos = tile_rank(d, base, wcnt);
    if (pos >= 0) { kout[pos] = k; vout[pos] = v; }
  }
}

__global__ void k_grp_rank(const int* g, int64_t n, const int* offs, int ntiles, int* rank) {
  __shared__ int base[256];
  __shared__ int wcnt[8][256];
  // rank relative to the group's start: subtract the offset of tile 0
  base[threadIdx.x] = offs[(int64_t)threadIdx.x * ntiles + blockIdx.x] - offs[(int64_t)threadIdx.x * ntiles];
  __syncthreads();
  int64_t tb = (int64_t)blockIdx.x * RS_TILE;
  for (int it = 0; it < RS_IPT; it++) {
    int64_t i = tb + it * RS_T + threadIdx.x;
    int d = 256;
    if (i < n) { int x = g[i]; if (x >= 0 && x < 256) d = x; }
    int pos = tile_rank(d, base, wcnt);
    if (i < n) rank[i] = pos;
  }
}

template <typename K, typename V>
int radix_sort_pairs(dt_ctx* c, K* keys, V* vals, int64_t n, int bits, const std::string& tag) {
  if (n <= 1) return 0;
  cudaStream_t s = c->stream;
  int ntiles = (int)ceil_div<int64_t>(n, RS_TILE);
  K* kt = (K*)pool_get(c, tag + ".rsk", sizeof(K) * n);
  V* vt = (V*)pool_get(c, tag + ".rsv", sizeof(V) * n);
  int* hist = (int*)pool_get(c, "rs.hist", 4 * (size_t)256 * ntiles);
  int* offs = (int*)pool_get(c, "rs.offs", 4 * (size_t)256 * ntiles);
  if (!kt || !vt || !hist || !offs) return set_err(c, DT_E_NOMEM, "radix sort buffers");
  K* ka = keys; V* va = vals; K* kb = kt; V* vb = vt;
  int passes = (bits + 7) / 8;
  for (int p = 0; p < passes; p++) {
    int shift = p * 8;
    k_rs_hist<K><<<ntiles, RS_T, (++c->launches, 0), s>>>(ka, n, shift, hist, ntiles);
    int rc = exclusive_scan_i32(c, hist, offs, (int64_t)256 * ntiles, nullptr);
    if (rc) return rc;
    k_rs_scatter<K, V><<<ntiles, RS_T, (++c->launches, 0), s>>>(ka, va, kb, vb, n, shift, offs, ntiles);
    std::swap(ka, kb);
    std::swap(va, vb);
  }
  if (ka != keys) {
    CUDA_OK(cudaMemcpyAsync(keys, ka, sizeof(K) * n, cudaMemcpyDeviceToDevice, s));
    CUDA_OK(cudaMemcpyAsync(vals, va, sizeof(V) * n, cudaMemcpyDeviceToDevice, s));
  }
  return 0;
}

template int radix_sort_pairs<uint32_t, int>(dt_ctx*, uint32_t*, int*, int64_t, int, const std::string&);
template int radix_sort_pairs<unsigned long long, int>(dt_ctx*, unsigned long long*, int*, int64_t, int,
                                                       const std::string&);

// Stable rank of each element within its group (groups 0..255, negative =
// none -> rank -1), plus group sizes (device, ngroups ints) when sizes != 0.
int group_rank(dt_ctx* c, const int* g, int64_t n, int* rank, int* sizes, int ngroups) {
  if (n <= 0) return 0;
  cudaStream_t s = c->stream;
  int ntiles = (int)ceil_div<int64_t>(n, RS_TILE);
  int* hist = (int*)pool_get(c, "gr.hist", 4 * (size_t)256 * ntiles + 4);
  int* offs = (int*)pool_get(c, "gr.offs", 4 * (size_t)256 * ntiles + 4);
  if (!hist || !offs) return set_err(c, DT_E_NOMEM, "group rank buffers");
  k_grp_hist<<<ntiles, RS_T, (++c->launches, 0), s>>>(g, n, hist, ntiles);
  int rc = exclusive_scan_i32(c, hist, offs, (int64_t)256 * ntiles, nullptr);
  if (rc) return rc;
  k_grp_rank<<<ntiles, RS_T, (++c->launches, 0), s>>>(g, n, offs, ntiles, rank);
  if (sizes) {
    // size of group d = offs[(d+1)*ntiles] - offs[d*ntiles]; the last needs the total
    rc = group_sizes_from_offsets(c, hist, offs, ntiles, sizes, ngroups);
    if (rc) return rc;
  }
  return 0;
}

__global__ void k_grp_sizes(const int* hist, int ntiles, int* sizes, int ngroups) {
  int d = blockIdx.x * blockDim.x + threadIdx.x;
  if (d >= ngroups) return;
  int s = 0;
  for (int t = 0; t < ntiles; t++) s += hist[(int64_t)d * ntiles + t];
  sizes[d] = s;
}

int group_sizes_from_offsets(dt_ctx* c, const int* hist, const int* offs, int ntiles, int* sizes, int ngroups) {
  (void)offs;
  k_grp_sizes<<<ceil_div(ngroups, 128), 128, (++c->launches, 0), c->stream>>>(hist, ntiles, sizes, ngroups);
  return 0;
}

}  // namespace gdt
