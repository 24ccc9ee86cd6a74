// merge.cu -- the merge of Alg. 1: T = (U T_i) \ B, plus every
// simplex s_b of T_B = DT(vertices(B)) whose vertices lie in more than one
// partition, or which equals a border simplex.  The equality test is a
// lookup in a lock-free open-addressing hash table in HBM that stores indices
// of the border simplices (keys: their sorted global-index tuples; slots are
// claimed with atomicCAS, keys compared against the stored rows).
#include "merge.cuh"

namespace gdt {

__device__ __forceinline__ unsigned long long row_hash(const int4& r) {
  unsigned long long h = splitmix64((unsigned long long)(unsigned)r.x);
  h = splitmix64(h ^ (unsigned)r.y);
  h = splitmix64(h ^ (unsigned)r.z);
  return splitmix64(h ^ (unsigned)r.w);
}
__device__ __forceinline__ bool row_eq(const int4& a, const int4& b) {
  return a.x == b.x && a.y == b.y && a.z == b.z && a.w == b.w;
}

__global__ void k_hash_insert(const int4* rows, int64_t n, int* table, unsigned mask, int* fail) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  unsigned slot = (unsigned)row_hash(rows[i]) & mask;
  for (unsigned probe = 0; probe <= mask; probe++) {
    if (atomicCAS(&table[slot], -1, (int)i) == -1) return;
    slot = (slot + 1) & mask;
  }
  atomicExch(fail, 1);
}

__device__ __forceinline__ bool hash_find(const int4* rows, const int* table, unsigned mask, const int4& key) {
  unsigned slot = (unsigned)row_hash(key) & mask;
  for (unsigned probe = 0; probe <= mask; probe++) {
    int j = table[slot];
    if (j < 0) return false;
    if (row_eq(rows[j], key)) return true;
    slot = (slot + 1) & mask;
  }
  return false;
}

// Select the simplices of T_B that enter T; append them to out.
// tbsrc/out_src (optional): the source slot of each row travels with it.
template <int D>
__global__ void k_merge_select(const int4* tb, const int* tbsrc, int64_t ntb, const int* label_by_gid,
                               const int4* brows, const int* table, unsigned mask, int4* out, int* out_src,
                               int* nout) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  bool keep = false;
  int4 r = make_int4(0, 0, 0, 0);
  if (i < ntb) {
    r = tb[i];
    int l0 = label_by_gid[r.x];
    bool mixed = label_by_gid[r.y] != l0 || label_by_gid[r.z] != l0 || (D == 3 && label_by_gid[r.w] != l0);
    keep = mixed || hash_find(brows, table, mask, r);
  }
  unsigned m = __ballot_sync(0xffffffffu, keep);
  if (!m) return;
  int lane = threadIdx.x & 31, leader = __ffs(m) - 1, base = 0;
  if (lane == leader) base = atomicAdd(nout, __popc(m));
  base = __shfl_sync(0xffffffffu, base, leader);
  if (keep) {
    int pos = base + __popc(m & ((1u << lane) - 1));
    out[pos] = r;
    if (out_src) out_src[pos] = tbsrc[i];
  }
}

int merge(dt_ctx* c, int dim, const EngineRun& parts, const int* gid_sorted, const unsigned char* bflag,
          const EngineRun& border, const int* gid_border, const int* label_by_gid, int4** rows_out,
          int64_t* nrows_out, MergeStats* ms, int** src_out) {
  cudaStream_t s = c->stream;
  int4 *brows, *tbrows, *trows;
  int *tbsrc = nullptr, *tsrc = nullptr;
  int64_t nb, ntb, nt;
  const bool want_src = src_out != nullptr;
  int rc = collect_finite(c, parts, gid_sorted, bflag, 2, &brows, &nb, "m.B");
  if (rc) return rc;
  rc = collect_finite(c, border, gid_border, nullptr, 0, &tbrows, &ntb, "m.TB", want_src ? &tbsrc : nullptr,
                      (int)parts.total_slots);
  if (rc) return rc;
  rc = collect_finite(c, parts, gid_sorted, bflag, 1, &trows, &nt, "m.T", want_src ? &tsrc : nullptr, 0);
  if (rc) return rc;
  unsigned tsize = 64;
  while (tsize < 2 * nb + 2) tsize <<= 1;
  int* table = (int*)pool_get(c, "m.table", 4 * (size_t)tsize);
  int* cnt = (int*)pool_get(c, "m.cnt", 16);
  int4* all = (int4*)pool_get(c, "m.all", 16 * (size_t)(nt + ntb + 1));
  int* allsrc = want_src ? (int*)pool_get(c, "m.allsrc", 4 * (size_t)(nt + ntb + 1)) : nullptr;
  if (!table || !cnt || !all || (want_src && !allsrc)) return set_err(c, DT_E_NOMEM, "merge buffers");
  CUDA_OK(cudaMemsetAsync(table, 0xff, 4 * (size_t)tsize, s));
  CUDA_OK(cudaMemsetAsync(cnt, 0, 16, s));
  if (nb) k_hash_insert<<<(unsigned)ceil_div<int64_t>(nb, 256), 256, (++c->launches, 0), s>>>(brows, nb, table, tsize - 1, cnt + 1);
  if (nt) CUDA_OK(cudaMemcpyAsync(all, trows, 16 * (size_t)nt, cudaMemcpyDeviceToDevice, s));
  if (nt && want_src) CUDA_OK(cudaMemcpyAsync(allsrc, tsrc, 4 * (size_t)nt, cudaMemcpyDeviceToDevice, s));
  if (ntb) {
    unsigned g = (unsigned)ceil_div<int64_t>(ntb, 256);
    int* osrc = want_src ? allsrc + nt : nullptr;
    if (dim == 2)
      k_merge_select<2><<<g, 256, (++c->launches, 0), s>>>(tbrows, tbsrc, ntb, label_by_gid, brows, table, tsize - 1,
                                                           all + nt, osrc, cnt);
    else
      k_merge_select<3><<<g, 256, (++c->launches, 0), s>>>(tbrows, tbsrc, ntb, label_by_gid, brows, table, tsize - 1,
                                                           all + nt, osrc, cnt);
  }
  int h[2];
  CUDA_OK(cudaMemcpyAsync(h, cnt, 8, cudaMemcpyDeviceToHost, s));
  CUDA_OK(cudaStreamSynchronize(s));
  if (h[1]) return set_err(c, DT_E_OVERFLOW, "border hash table full");
  *rows_out = all;
  if (want_src) *src_out = allsrc;
  *nrows_out = nt + h[0];
  ms->n_border_simplices = nb;
  ms->n_tb = ntb;
  ms->n_kept = h[0];
  ms->n_partial_kept = nt;
  return 0;
}

}  // namespace gdt
