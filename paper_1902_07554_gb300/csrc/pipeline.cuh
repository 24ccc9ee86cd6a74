// pipeline.cuh -- orchestration of Alg. 1 (divide, partial DTs, border,
// border DT, merge) on the context's stream.
#pragma once
#include "ctx.cuh"

namespace gdt {
int run_pipeline(dt_ctx* c, const double* points, int64_t n, int dim, int k, double frac);
int stage_points(dt_ctx* c, const double* points, int64_t n, int dim, void** P_out, const char* tag,
                 const int* inst = nullptr);
int run_batch(dt_ctx* c, const double* points, const int64_t* offsets, int count, int dim);
int ensure_neighbors(dt_ctx* c);
void* stage_in(dt_ctx* c, const void* src, size_t bytes, const std::string& name, int* rc);
int copy_out(dt_ctx* c, void* dst, const void* src, size_t bytes);
bool is_device_ptr(const void* p);
__global__ void k_iota(int* a, int64_t n, int start);
// Base case of Alg. 1: one triangulation of all points (pipeline.cu).
int run_direct(dt_ctx* c, const void* P, int64_t n, int dim);
// Recursive bisection (recursive.cu).
int run_recursive(dt_ctx* c, const void* P, int64_t n, int dim, int k, double frac);
// Indices i with flag[i] set, ascending; *m receives the count.
int compact_flags(dt_ctx* c, const unsigned char* flag, int64_t n, int* out, int64_t* m, const char* tag);
__global__ void k_gather_i32(const int* src, const int* idx, int64_t m, int* out);
__global__ void k_flag_by_gid(const unsigned char* vflag, const int* gid, int64_t n, unsigned char* fg);
}  // namespace gdt
