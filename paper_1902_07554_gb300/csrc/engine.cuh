// engine.cuh -- batched parallel Delaunay insertion on the GPU.
//
// Triangulates many independent point sets ("instances": the k partitions of
// Alg. 1, the sample of Alg. 2, the border vertex set, or a batch of separate
// problems) in the same kernel launches.  Each instance is built by
// Bowyer-Watson insertion with an explicit infinite vertex; points are
// inserted in rounds:
//   pick    -- every simplex holding uninserted points nominates the one with
//              the highest priority (one atomicMax per point);
//   cavity  -- each nominee grows its conflict region (simplices whose
//              perturbed circumsphere contains it) and claims it, plus the ring
//              of simplices across the region's boundary, with 64-bit
//              (round, priority) keys;
//   insert  -- a nominee whose region and ring are not touched by a stronger
//              nominee's region (and whose region is not inside a stronger
//              nominee's ring) replaces its region by the star of new simplices
//              over the boundary facets.  Such insertions commute, so the
//              round's result equals inserting the winners one at a time;
//   relocate-- points whose conflict simplex was destroyed walk (visibility
//              walk with exact orientation) to a simplex in conflict with them.
// The strongest nominee of an instance always wins, so every round inserts at
// least one point per unfinished instance.
#pragma once
#include <vector>

#include "common.cuh"
#include "predicates.cuh"

namespace gdt {

// Device views of one engine run.
template <int D>
struct TriView {
  using P = typename PT<D>::T;
  const P* pts;             // points (all instances, concatenated)
  const float4* xs;         // FP32 copies relative to the instance origin; w = error bound eta
  const int* gid;           // global index of each point (perturbation rank)
  const int* pinst;         // instance of each point
  int4* tv;                 // simplex vertex tuples (D+1 used)
  int4* tn;                 // packed neighbour links
  unsigned long long* claimA;   // strongest key having the simplex in region or ring
  unsigned long long* claimC;   // strongest key having the simplex in its region
  int* tcount;              // per instance: next free simplex slot (absolute)
  const int* tend;          // per instance: end of its simplex arena (absolute)
  int* loc;                 // per point: a simplex in conflict with it (or -1)
  unsigned char* state;     // per point: 0 uninserted, 1 inserted
  DevStatus* st;
  int nslots;               // total simplex slots (bounds for every link)
  int npts;                 // total points (bounds for every vertex)
  unsigned long long* prof; // profile counters (null unless profiling):
                            // [0] bytes touched by k_cavity, [1] its conflict tests
  // per-instance hint grids: a recently created simplex per cell, used as the
  // start of the walk when a dormant point is activated
  int* hint;                // cells of all instances, -1 = none
  int* hint2;               // coarse cells (4 x 4 x 4 fine cells each), -1 = none
  const double* glo;        // per instance: grid origin (3) and inverse cell edge (3)
  const int* gdim;          // per instance: cells per axis (3), first fine cell, first coarse cell
  const int* toff;          // per instance: first simplex slot
  int ninst;
  unsigned long long* dbg;  // walk statistics (debug runs only; null otherwise)
  int rings;                // neighbour rings a nominee must hold the strongest pick in (1 or 2)
  int* inst_kept;           // per instance: points still active after the round (continuous batching; else null)
  int walk_limit;           // steps of one location walk before DT_E_TIMEOUT
};

struct CandScratch {
  int* cand;      // candidate point per slot
  int4* meta;     // (cavity size, boundary size, status, 0)
  int* cav;       // capC entries per slot
  int* bnd;       // capB entries per slot (packed simplex, facet)
  int* outer;     // capB entries per slot
  int* count;     // slots taken this round
  int cap, capC, capB;
  // regions too large for the lists above (grown again by k_cavity_big)
  int* bigcav;    // capCbig entries per large region
  int* bigbnd;    // capBbig entries per large region
  int* bigout;    // capBbig entries per large region
  int* biglist;   // slot of each large region
  int* nbig;      // large regions this round
  int capCbig, capBbig;
};

// Host-side engine run: owns the buffers of one triangulation batch.
struct EngineRun {
  int dim = 0;
  int ninst = 0;
  int64_t npts = 0;
  int64_t total_slots = 0;
  std::vector<int64_t> h_poff;   // instance point offsets (host)
  std::vector<int64_t> h_toff;   // instance simplex arena offsets (host)
  std::vector<int> h_status;     // per instance: 0 ok, 1 degenerate, 2 too small
  std::vector<int> h_tcount;     // per instance: slots used (absolute end)
  int rounds = 0;
  // device buffers (owned by the context's allocator)
  void* tv = nullptr;
  void* tn = nullptr;
  int* tcount = nullptr;
  int* toff = nullptr;
  int* tend = nullptr;
  int* inst_status = nullptr;
};

// Where each output row came from: a slot of the first arena (partial or
// direct triangulation), or base1 + a slot of the second (border) arena.
struct LinkSources {
  const int4* tv0 = nullptr;
  const int4* tn0 = nullptr;
  const int* gid0 = nullptr;
  int64_t base1 = 0;
  const int4* tv1 = nullptr;
  const int4* tn1 = nullptr;
  const int* gid1 = nullptr;
  int64_t total = 0;            // base1 + slots of the second arena
  const int* origin = nullptr;  // per output row
};

}  // namespace gdt
