// divide.cuh -- divide step (divide.cu).
#pragma once
#include <vector>

#include "ctx.cuh"

namespace gdt {

// Weighted sample graph: unique edges E (u < v, sorted), integer weights w,
// symmetric CSR (rowptr, col, cw) and the sample bounding box (lo[3], hi[3]).
struct SampleGraph {
  int64_t eta = 0, m = 0;
  int2* E = nullptr;
  long long* w = nullptr;
  int* rowptr = nullptr;
  int* col = nullptr;
  long long* cw = nullptr;
  double* box = nullptr;
};

int64_t sample_size(int64_t n, double frac, int D);
int select_sample(dt_ctx* c, int64_t n, int64_t eta, uint64_t seed, int* ids);
int gather_points(dt_ctx* c, int dim, const void* P, const int* ids, int64_t m, void* out);
int sample_graph(dt_ctx* c, const EngineRun& run, const void* PS, int dim, int kind, SampleGraph& G);
int build_csr(dt_ctx* c, SampleGraph& G);
int graph_bbox(dt_ctx* c, int dim, const void* PS, int64_t eta, double* box);
void partition_bounds(int64_t eta, int k, double eps, int* lmin, int* lmax);
int partition_graph(dt_ctx* c, const void* PS, int dim, SampleGraph& G, int k, double eps, int rounds, int init,
                    int* block);
int partition_multilevel(dt_ctx* c, const SampleGraph& G, int k, double eps, int rounds, int* block);
int cut_weight(dt_ctx* c, const SampleGraph& G, const int* block, long long* out);
int label_points(dt_ctx* c, int dim, const void* P, int64_t n, const void* S, const int* srank, const SampleGraph& G,
                 const int* block, int* label, int* nearest);
int map_labels(dt_ctx* c, const int* nearest, const int* block, int64_t n, int* label);
int kd_divide(dt_ctx* c, int dim, const void* P, int64_t n, int k, int* label, const char* tag = "kd");
int scatter_by_label(dt_ctx* c, int dim, const void* P, const int* label, int64_t n, int k, void* Ps, int* gid,
                     int* pinst, std::vector<int64_t>& poff, std::vector<int64_t>& sizes_out);
__global__ void k_fill_int(int* a, int64_t n, int v);

}  // namespace gdt
