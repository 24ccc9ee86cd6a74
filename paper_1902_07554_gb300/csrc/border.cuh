// border.cuh -- border detection (border.cu).
#pragma once
#include <vector>

#include "ctx.cuh"

namespace gdt {
// Flags border simplices of the partial triangulations (bflag, per slot) and
// their vertices (vflag, per partition-sorted point); *nborder receives the
// number of finite border simplices.  others (optional, host, one mask per
// instance): the partitions whose points each instance is tested against
// (default: every other partition; 0: none).
int border_detect(dt_ctx* c, int dim, const EngineRun& parts, const void* Ps, const int* pinst, int k, double cell,
                  int prim, unsigned char** bflag, unsigned char** vflag, int64_t* nborder,
                  const std::vector<unsigned long long>* others = nullptr);
}  // namespace gdt
