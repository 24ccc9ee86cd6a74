// sort.cuh -- stable radix sort and group ranks (sort.cu).
#pragma once
#include <string>

#include "ctx.cuh"

namespace gdt {
// Sorts (keys, vals) in place by the low `bits` bits of the keys, stably.
template <typename K, typename V>
int radix_sort_pairs(dt_ctx* c, K* keys, V* vals, int64_t n, int bits, const std::string& tag);
// rank[i] = number of j < i with g[j] == g[i] (g in [0,256) or negative: rank -1);
// sizes (optional) receives the count of each group 0..ngroups-1.
int group_rank(dt_ctx* c, const int* g, int64_t n, int* rank, int* sizes, int ngroups);
int group_sizes_from_offsets(dt_ctx* c, const int* hist, const int* offs, int ntiles, int* sizes, int ngroups);
}  // namespace gdt
