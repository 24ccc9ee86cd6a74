// merge.cuh -- hash-table merge of the partial and border triangulations (merge.cu).
#pragma once
#include "ctx.cuh"

namespace gdt {
struct MergeStats {
  int64_t n_border_simplices = 0, n_tb = 0, n_kept = 0, n_partial_kept = 0;
};
// Rows (canonical tuples, unsorted order) of the merged triangulation.
// src_out (optional) receives each row's source: a slot of the partial
// arena, or parts.total_slots + a slot of the border arena.
int merge(dt_ctx* c, int dim, const EngineRun& parts, const int* gid_sorted, const unsigned char* bflag,
          const EngineRun& border, const int* gid_border, const int* label_by_gid, int4** rows_out,
          int64_t* nrows_out, MergeStats* ms, int** src_out = nullptr);
}  // namespace gdt
