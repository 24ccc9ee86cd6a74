// engine_core.cuh -- batched parallel Bowyer-Watson insertion (see engine.cuh).
//
// Included by engine.cu (the 2D instantiation and the functions shared by both
// dimensions, GDT_ENGINE_SHARED) and by engine3.cu (the 3D instantiation), so
// that the two dimensions compile as separate translation units in parallel.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>

#include "ctx.cuh"
#include "bbox.cuh"
#include "pipeline.cuh"
#include "sort.cuh"
#include "stream.cuh"

namespace gdt {

constexpr int TAGBIT = (int)0x80000000;

// Candidate key of point p in a round: the round in the high word (older
// claims compare smaller), a per-round pseudo-random priority in the low word
// (p -> p ^ c and fmix32 are bijections, so keys are unique within a round).
// Round key of point p: (round, hash of p and round, pass bit).  The pass bit
// is set when a large region is grown a second time (k_cavity_big): the
// nominee then outranks its own first-pass claims but no other nominee.
static __device__ __forceinline__ unsigned long long mkkey(unsigned round, int p) {
  return ((unsigned long long)round << 33) |
         ((unsigned long long)fmix32((uint32_t)p ^ (round * 0x9E3779B9u)) << 1);
}
static __device__ __forceinline__ int get4(const int4& v, int i) {
  return i == 0 ? v.x : (i == 1 ? v.y : (i == 2 ? v.z : v.w));
}
static __device__ __forceinline__ void set4(int4& v, int i, int x) {
  if (i == 0) v.x = x; else if (i == 1) v.y = x; else if (i == 2) v.z = x; else v.w = x;
}
static __device__ __forceinline__ int* comp_ptr(int4* a, int s, int i) { return reinterpret_cast<int*>(a + s) + i; }

// Appends `val` to list/counter for the lanes with pred set; every lane of
// the warp must call this.
static __device__ __forceinline__ void warp_append(int* list, int* counter, bool pred, int val) {
  unsigned mask = __ballot_sync(0xffffffffu, pred);
  if (!mask) return;
  int lane = threadIdx.x & 31;
  int leader = __ffs(mask) - 1;
  int base = 0;
  if (lane == leader) base = atomicAdd(counter, __popc(mask));
  base = __shfl_sync(0xffffffffu, base, leader);
  if (pred) list[base + __popc(mask & ((1u << lane) - 1))] = val;
}

static __device__ __forceinline__ bool collinear3(double4_32a a, double4_32a b, double4_32a c) {
  double2 pa, pb, pc;
  pa = make_double2(a.x, a.y); pb = make_double2(b.x, b.y); pc = make_double2(c.x, c.y);
  if (orient2(pa, pb, pc) != 0) return false;
  pa = make_double2(a.y, a.z); pb = make_double2(b.y, b.z); pc = make_double2(c.y, c.z);
  if (orient2(pa, pb, pc) != 0) return false;
  pa = make_double2(a.x, a.z); pb = make_double2(b.x, b.z); pc = make_double2(c.x, c.z);
  return orient2(pa, pb, pc) == 0;
}

// Bounds guards: a corrupted link or vertex records an error instead of
// touching memory outside the arena.
template <int D>
__device__ __forceinline__ bool slot_ok(const TriView<D>& T, int s) { return (unsigned)s < (unsigned)T.nslots; }
template <int D>
__device__ __forceinline__ bool verts_ok(const TriView<D>& T, const int4& v) {
  bool ok = true;
  for (int i = 0; i <= D; i++) {
    int x = get4(v, i);
    ok &= (x == INF_V) || ((unsigned)x < (unsigned)T.npts);
  }
  return ok;
}

// Hint cells of point p: the fine grid (about n_i / 4 cells) and a coarse
// one (4 x 4 x 4 fine cells per cell), both per instance.
template <int D>
__device__ __forceinline__ void hint_cells(const TriView<D>& T, int p, int& fine, int& coarse) {
  int i = T.pinst[p];
  const double* g = T.glo + 6 * i;
  const int* d = T.gdim + 5 * i;
  typename PT<D>::T q = T.pts[p];
  int id = 0, id2 = 0;
  for (int c = D - 1; c >= 0; c--) {
    double f = (comp(q, c) - g[c]) * g[3 + c];
    int x = f < 0 ? 0 : (f >= d[c] ? d[c] - 1 : (int)f);
    id = id * d[c] + x;
    id2 = id2 * ((d[c] + 3) >> 2) + (x >> 2);
  }
  fine = d[3] + id;
  coarse = d[4] + id2;
}

template <int D>
__device__ __forceinline__ int orient_tuple(const TriView<D>& T, const int4& v) {
  int t[4] = {v.x, v.y, v.z, v.w};
  return orient_px(T.pts, T.xs, t);
}

// ---------------------------------------------------------------- init
// One thread per instance: the first D+1 affinely independent points (in
// index order) form a positively oriented simplex, surrounded by D+1 ghost
// simplices (infinite vertex + one hull facet each).
constexpr int NLEV = 96;   // activation levels (BRIO batches)
constexpr int BIGCAP = 256;      // large regions grown per round
constexpr int BIG_C = 16384, BIG_B = 32768;   // their list capacities

// Round state of the device-driven insertion loop (a CUDA graph whose
// conditional WHILE node repeats one round: begin, activate, nominate,
// cavity, insert, relocate, end).  The kernels take their round, active lists
// and activation range from here when the pointer is non-null, and from their
// parameters when the host drives the rounds (profile and debug runs).
struct EngCtl {
  unsigned round;      // current round
  int* ain;            // active points of this round
  int* aout;           // active points of the next round
  int next_level;      // next activation level (-1: none left)
  int last_batch;      // active count right after the last activation
  int act_lo, act_n;   // this round's activation range in the level list
  int last_nact;       // active count after the previous round
  int stalled;         // consecutive rounds without an insertion
  int activated;       // points activated this round
  int done;            // 0 running; 1 finished; 2 device error; 3 stalled; 4 round limit
  int drain;           // the next batch is activated when the active set is last_batch / drain
  int small;           // 1: the next rounds are small enough for k_small_rounds (one CTA)
  int small_max;       // active points up to which a round counts as small
  float ratio;         // > 0: continuous activation (active set kept near ratio x points inserted)
  int min_active;      // continuous activation: the active set's floor
  long long activated_total;   // points activated so far (continuous activation)
  int round_limit;     // rounds before the run stops with DT_E_TIMEOUT
};

// Programmatic dependent launch inside the round graph: each round kernel
// first waits for the kernel before it to complete (griddepcontrol.wait: its
// memory is then visible), then lets the next one start launching, so that
// the next launch overlaps this kernel's run.  Both are no-ops in a launch
// without the programmatic attribute.
static __device__ __forceinline__ void pdl_enter() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;");
}

template <int D>
__global__ void k_init(TriView<D> T, int ninst, const long long* poff, const int* toff, int* inst_status) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= ninst) return;
  long long a = poff[i], b = poff[i + 1];
  int base = toff[i];
  T.tcount[i] = base;
  if (b - a < D + 1) { inst_status[i] = 2; return; }
  int pick[4];
  int np = 0;
  pick[np++] = (int)a;
  for (long long q = a + 1; q < b && np < D + 1; q++) {
    bool ok;
    if (np == 1) {
      ok = true;
    } else if (D == 3 && np == 2) {
      ok = !collinear3(reinterpret_cast<const double4_32a*>(T.pts)[pick[0]],
                       reinterpret_cast<const double4_32a*>(T.pts)[pick[1]],
                       reinterpret_cast<const double4_32a*>(T.pts)[q]);
    } else {
      int t[4] = {pick[0], pick[1], pick[2], pick[3]};
      t[np] = (int)q;
      ok = orient_p(T.pts, t) != 0;
    }
    if (ok) pick[np++] = (int)q;
  }
  if (np < D + 1) { inst_status[i] = 1; return; }
  int4 v0 = make_int4(pick[0], pick[1], pick[2], D == 3 ? pick[3] : -3);
  if (orient_tuple(T, v0) < 0) { int t = v0.x; v0.x = v0.y; v0.y = t; }
  int s0 = base;
  T.tv[s0] = v0;
  int4 g[4];
  for (int k = 0; k <= D; k++) {
    int4 gv = v0;
    set4(gv, k, INF_V);
    int x = (k + 1) % (D + 1), y = (k + 2) % (D + 1);
    int tx = get4(gv, x), ty = get4(gv, y);
    set4(gv, x, ty); set4(gv, y, tx);
    g[k] = gv;
    T.tv[s0 + 1 + k] = gv;
  }
  int4 n0 = make_int4(0, 0, 0, 0);
  for (int k = 0; k <= D; k++) set4(n0, k, pack_nb(s0 + 1 + k, k));
  T.tn[s0] = n0;
  for (int k = 0; k <= D; k++) {
    int4 nk = make_int4(0, 0, 0, 0);
    for (int j = 0; j <= D; j++) {
      int w = get4(g[k], j);
      if (w == INF_V) { set4(nk, j, pack_nb(s0, k)); continue; }
      int m = -1;
      for (int l = 0; l <= D; l++) if (get4(v0, l) == w) m = l;
      // in ghost m, the facet opposite the vertex ghost k lacks (v0[k])
      int vk = get4(v0, k), f = -1;
      for (int l = 0; l <= D; l++) if (get4(g[m], l) == vk) f = l;
      set4(nk, j, pack_nb(s0 + 1 + m, f));
    }
    T.tn[s0 + 1 + k] = nk;
  }
  for (int k = 0; k <= D; k++) { T.state[pick[k]] = 1; T.loc[pick[k]] = s0; }
  T.tcount[i] = base + D + 2;
  inst_status[i] = 0;
}

// Initial conflict simplex of every other point: a ghost whose hull facet it
// lies strictly beyond, else the initial simplex (it lies in it, closed).
// Activation level of a point: the number of leading zeros of a hash of its
// global index (P(level >= L) = 2^-L).  Points are activated in batches of
// decreasing level, so the set of points taking part doubles batch by batch
// (a randomized insertion order with a growing prefix, as in biased randomized
// insertion orders).  -1: not to be inserted (initial simplex / bad instance).
template <int D>
__global__ void k_levels(TriView<D> T, int64_t npts, const int* inst_status, int* level, float inv_log2_growth) {
  int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= npts) return;
  int l = -1;
  if (inst_status[T.pinst[p]] == 0 && T.state[p] == 0) {
    // P(level >= l) = growth^-l: activating the levels from the top, each
    // batch is about (growth - 1) times the points activated before it
    const uint32_t h = fmix32((uint32_t)T.gid[p] * 0x9E3779B1u + 0x7F4A7C15u);
    const float u = ((float)(h >> 8) + 0.5f) * (1.0f / 16777216.0f);
    l = min(NLEV - 1, (int)(-__log2f(u) * inv_log2_growth));
  }
  level[p] = l;
}

template <int D>
__global__ void k_locate_init(TriView<D> T, int64_t npts, const int* toff, const int* inst_status,
                              const int* level, int min_level, int* act, int* nact) {
  int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  bool active = false;
  if (p < npts) {
    int i = T.pinst[p];
    if (inst_status[i] == 0 && T.state[p] == 0) {
      T.loc[p] = toff[i];                  // dormant points wait on the initial simplex
    }
    if (inst_status[i] == 0 && T.state[p] == 0 && level[p] >= min_level) {
      active = true;
      int s0 = toff[i];
      int4 vv = T.tv[s0];
      int loc = s0;
      for (int j = 0; j <= D; j++) {
        int4 t = vv;
        set4(t, j, (int)p);
        if (orient_tuple(T, t) < 0) { loc = nb_simplex(get4(T.tn[s0], j)); break; }
      }
      T.loc[p] = loc;
    }
  }
  warp_append(act, nact, active, (int)p);
}

// ---------------------------------------------------------------- rounds
template <int D>
__global__ void k_pick(TriView<D> T, const int* act, int nact, unsigned round) {
  int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= nact) return;
  int p = act[idx];
  atomicMax(&T.claimC[T.loc[p]], mkkey(round, p));
}

enum { CAND_OK = 0, CAND_LOST = 1, CAND_OVER = 2 };

// Nominees of a round: the point holding the strongest key of its simplex
// (left in claimC by the pick), unless a neighbour of that simplex holds a
// stronger key -- every neighbour lies in the nominee's region or ring, and a
// stronger key there belongs to a nominee whose region contains it, so the
// weaker one would lose anyway.  Nominees go to a dense list.
// Nominees go to NBUCKET lists by the top bits of their key, strongest
// first: the cavity kernel takes them in that order, so the regions of strong
// nominees are claimed early and weaker ones stop at their first contact.
constexpr int NBUCKET = 8;
static __device__ __forceinline__ int key_bucket(unsigned long long key) {
  return NBUCKET - 1 - (int)((key >> 30) & 7);   // the top 3 bits of the hash
}

// Slot -> nominee: slots enumerate the buckets in order (bcnt: bucket sizes,
// of which the first seg entries are stored; seg: the capacity of one list).
// The caller keeps slot below the number stored, which k_nominate counts.
static __device__ __forceinline__ int nominee_at(const int* nom, const int* bcnt, int seg, int slot) {
  int q = 0, base = 0;
#pragma unroll
  for (int b = 0; b < NBUCKET - 1; b++) {
    const int c = min(bcnt[b], seg);
    if (slot >= base + c) { base += c; q = b + 1; }
    else break;
  }
  return nom[(int64_t)q * seg + (slot - base)];
}

// Is a key stronger than `key` picked in a simplex of the second ring of t0
// (the neighbours of t0's neighbours)?
template <int D>
__device__ __forceinline__ bool stronger_in_ring2(const TriView<D>& T, int t0, const int4& nn0,
                                                  unsigned long long key) {
  for (int i = 0; i <= D; i++) {
    const int u = nb_simplex(get4(nn0, i));
    if (!slot_ok(T, u)) continue;
    const int4 nu = T.tn[u];
    for (int j = 0; j <= D; j++) {
      const int w = nb_simplex(get4(nu, j));
      if (w != t0 && slot_ok(T, w) && *((volatile unsigned long long*)&T.claimC[w]) > key) return true;
    }
  }
  return false;
}

template <int D>
__global__ void __launch_bounds__(256) k_nominate(TriView<D> T, const int* act, const int* nact_p, unsigned round,
                                                  int* nom, int* nnom, int* bcnt, int seg, const EngCtl* ctl) {
  pdl_enter();
  __shared__ int s_cnt[NBUCKET], s_base[NBUCKET];
  if (ctl) {
    if (ctl->small || ctl->done) return;
    act = ctl->ain; round = ctl->round;
  }
  const int nact = *nact_p;
  for (int64_t blk = (int64_t)blockIdx.x * blockDim.x; blk < nact; blk += (int64_t)gridDim.x * blockDim.x) {
  __syncthreads();
  if (threadIdx.x < NBUCKET) s_cnt[threadIdx.x] = 0;
  __syncthreads();
  const int64_t idx = blk + threadIdx.x;
  bool take = false;
  int p = -1, bucket = -1;
  if (idx < nact) {
    p = act[idx];
    unsigned long long key = mkkey(round, p);
    int t0 = T.loc[p];
    if (*((volatile unsigned long long*)&T.claimC[t0]) == key) {
      take = true;
      int4 nn0 = T.tn[t0];
      for (int i = 0; i <= D; i++) {
        int u = nb_simplex(get4(nn0, i));
        if (slot_ok(T, u) && *((volatile unsigned long long*)&T.claimC[u]) > key) take = false;
      }
      // a stronger pick two rings away would most likely claim part of this region too
      if (take && T.rings > 1 && stronger_in_ring2(T, t0, nn0, key)) take = false;
    }
    if (take) bucket = key_bucket(key);
  }
  // offsets within the block per bucket (lanes grouped by bucket), then one
  // global atomic per bucket and block
  const int lane = threadIdx.x & 31;
  const unsigned grp = __match_any_sync(0xffffffffu, bucket);
  const int leader = __ffs(grp) - 1;
  int wbase = 0;
  if (take && lane == leader) wbase = atomicAdd(&s_cnt[bucket], __popc(grp));
  wbase = __shfl_sync(0xffffffffu, wbase, leader);
  const int local = wbase + __popc(grp & ((1u << lane) - 1));
  __syncthreads();
  if (threadIdx.x < NBUCKET) {
    const int cnt = s_cnt[threadIdx.x];
    int gb = 0;
    if (cnt) {
      gb = atomicAdd(&bcnt[threadIdx.x], cnt);
      const int stored = max(0, min(cnt, seg - gb));   // a full list drops the rest this round
      if (stored) atomicAdd(nnom, stored);
    }
    s_base[threadIdx.x] = gb;
  }
  __syncthreads();
  if (take) {
    const int at = s_base[bucket] + local;
    if (at < seg) nom[(int64_t)bucket * seg + at] = p;
  }
  }
}

// One warp per nominee grows its conflict region: each lane inspects one
// (region simplex, facet) pair per step, up to 32/(D+1) region simplices per
// step.  Conflicting neighbours join the region (claimC/claimA atomicMax; the
// returned old value also deduplicates lanes that reach the same simplex),
// the others become boundary facets (ring claim in claimA).
// A group of G lanes (G = 32: a whole warp) grows nominee p's conflict region
// into C (region simplices; NB: optional copies of their links) and B
// (boundary facets), claiming as it goes; each step inspects G/(D+1) region
// simplices x (D+1) facets.  Groups of one warp run side by side (warp-wide
// ballots, each group reading its own bits).  has = false: an idle group.
// status: CAND_OK, CAND_LOST (met a stronger claim) or CAND_OVER (lists full).
template <int D, int G>
__device__ __forceinline__ void grow_region(const TriView<D>& T, bool has, int p, unsigned long long key, int* C,
                                            int4* NB, int* B, int capC, int capB, int& nc_out, int& nbd_out,
                                            int& status_out, unsigned long long& pbytes, unsigned long long& ptests) {
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int gl = lane % G, gbase = lane - gl;
  const unsigned gmask = G == 32 ? FULL : (((1u << G) - 1u) << gbase);
  const unsigned below = gmask & ((1u << lane) - 1u);
  constexpr int PER = G / (D + 1);
  int status = has ? CAND_OK : CAND_LOST;
  int t0 = has ? T.loc[p] : 0;
  if (has && gl == 0) {
    if (NB) NB[0] = T.tn[t0];
    // the located simplex carries p's pick (= key) already, except on a second
    // pass (key has its pass bit): claim it in both words so that no lane adds
    // it to the region a second time
    unsigned long long oc = atomicMax(&T.claimC[t0], key);
    unsigned long long o = atomicMax(&T.claimA[t0], key);
    if (o > key || oc > key) status = CAND_LOST;
    C[0] = t0;
    pbytes += sizeof(typename PT<D>::T) + 4 + 8 + 16 * (D + 1) + 16 + 4;
  }
  status = __shfl_sync(FULL, status, gbase);
  int nc = 1, nbd = 0, h = 0, nsteps = 0;
  __syncwarp();
  for (;;) {
    const bool act = status == CAND_OK && h < nc;
    if (!__any_sync(FULL, act)) break;
    nsteps += act;
    const int nc0 = nc;                                // region simplices known at this step
    int j = h + gl / (D + 1), i = gl % (D + 1);
    bool valid = act && gl < PER * (D + 1) && j < nc0;
    bool addC = false, addB = false, lost = false, bad = false;
    int t = -1, u = -1;
    int4 links = make_int4(0, 0, 0, 0);
    if (valid) {
      t = C[j];
      u = nb_simplex(NB ? get4(NB[j], i) : *comp_ptr(T.tn, t, i));
      if (!slot_ok(T, u)) {
        bad = true;
      } else {
        const int4 vv = T.tv[u];                       // loaded beside the claim, not after it
        unsigned long long cC = *((volatile unsigned long long*)&T.claimC[u]);
        pbytes += 16;
        if (cC > key) {
          lost = true;                                 // inside a stronger region
        } else if (cC != key) {
          pbytes += 16 + (D + 1) * sizeof(typename PT<D>::T);
          ptests++;
          if (!verts_ok(T, vv)) {
            bad = true;
          } else {
            int vt[4] = {vv.x, vv.y, vv.z, vv.w};
            if (in_conflict_x(T.pts, T.xs, T.gid, vt, p, D)) {
              // both claims at once; the region claim decides, the ring claim
              // can only raise claimA to a key that is no stronger than needed
              if (NB) links = T.tn[u];                   // in flight beside the two claims
              unsigned long long o = atomicMax(&T.claimC[u], key);
              unsigned long long o2 = atomicMax(&T.claimA[u], key);
              if (o > key || o2 > key) {
                lost = true;
              } else if (o < key) {                    // first lane to claim it
                addC = true;
                pbytes += 16 + 16 + 4;
              }
            } else {
              atomicMax(&T.claimA[u], key);
              addB = true;
              pbytes += 8 + 4;
            }
          }
        }
      }
    }
    if (bad) set_error(T.st, DT_E_INTERNAL, 10);
    const unsigned mL = __ballot_sync(FULL, lost || bad) & gmask;
    const unsigned mC = __ballot_sync(FULL, addC) & gmask, mB = __ballot_sync(FULL, addB) & gmask;
    if (act) {
      const int nC = __popc(mC), nB = __popc(mB);
      if (mL) {
        status = CAND_LOST;
      } else if (nc + nC > capC || nbd + nB > capB) {
        status = CAND_OVER;
      } else {
        if (addC) {
          C[nc + __popc(mC & below)] = u;
          if (NB) NB[nc + __popc(mC & below)] = links;
        }
        if (addB) B[nbd + __popc(mB & below)] = pack_nb(t, i);
        nc += nC;
        nbd += nB;
        h = min(h + PER, nc0);                         // simplices appended now come next
      }
    }
    __syncwarp();
  }
  if (T.dbg && has && gl == 0) atomicAdd(&T.dbg[7], (unsigned long long)nsteps);   // [7] growth steps
  nc_out = nc;
  nbd_out = nbd;
  status_out = status;
}

// Profile and debug counters of a group's region (group leader).
template <int D, int G>
__device__ __forceinline__ void region_stats(const TriView<D>& T, bool has, int status, int nc,
                                             unsigned long long pbytes, unsigned long long ptests) {
  const unsigned FULL = 0xffffffffu;
  if (T.prof) {
    for (int off = 16; off; off >>= 1) {
      pbytes += __shfl_down_sync(FULL, pbytes, off);
      ptests += __shfl_down_sync(FULL, ptests, off);
    }
    if ((threadIdx.x & 31) == 0) { atomicAdd(&T.prof[0], pbytes); atomicAdd(&T.prof[1], ptests); }
  }
  if (T.dbg && has && (threadIdx.x & 31) % G == 0) {
    // [4] complete regions, [5] region simplices grown by all nominees
    if (status == CAND_OK) atomicAdd(&T.dbg[4], 1ull);
    atomicAdd(&T.dbg[5], (unsigned long long)nc);
  }
}

// Nominees in groups of G lanes (32 / G per warp), strongest list first.  A
// region that outgrows the regular lists is queued for k_cavity_big (up to
// BIGCAP per round).  G = 16 puts two nominees in one warp: four region
// simplices per step each, twice the nominees in flight per warp.
template <int D, int MINB, int G>
__global__ void __launch_bounds__(128, MINB) k_cavity_w(TriView<D> T, const int* nom, const int* nnom_p, unsigned round,
                                                  CandScratch S, const int* bcnt, const EngCtl* ctl) {
  pdl_enter();
  if (ctl) {
    if (ctl->small || ctl->done) return;
    round = ctl->round;
  }
  constexpr int GPW = 32 / G;                          // groups per warp
  const int lane = threadIdx.x & 31, grp = lane / G, gl = lane % G;
  const int wid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarp = (gridDim.x * blockDim.x) >> 5;
  const int nnom = min(*nnom_p, S.cap);
  // the region list lives in shared memory while it fits (copied out at the end)
  // together with the neighbour links of each region simplex (loaded when the
  // simplex joins, beside its claims, instead of one step later)
  constexpr int SHC = 128;
  __shared__ int s_region[4 * GPW][SHC];
  __shared__ int4 s_links[4 * GPW][SHC];
  const bool in_shared = S.capC <= SHC && blockDim.x <= 128;
  const int sg = (threadIdx.x >> 5) * GPW + grp;
  for (int first = wid * GPW; first < nnom; first += nwarp * GPW) {
    const int slot = first + grp;
    const bool has = slot < nnom;
    const int p = has ? nominee_at(nom, bcnt, S.cap, slot) : 0;
    const unsigned long long key = mkkey(round, p);
    int* Cg = S.cav + (int64_t)(has ? slot : 0) * S.capC;
    int* C = in_shared ? s_region[sg] : Cg;
    int4* NB = in_shared ? s_links[sg] : nullptr;
    int* B = S.bnd + (int64_t)(has ? slot : 0) * S.capB;
    if (has && gl == 0) S.cand[slot] = p;
    unsigned long long pbytes = 0, ptests = 0;
    int nc, nbd, status;
    grow_region<D, G>(T, has, p, key, C, NB, B, S.capC, S.capB, nc, nbd, status, pbytes, ptests);
    if (has && in_shared && status == CAND_OK)
      for (int q = gl; q < nc; q += G) Cg[q] = C[q];
    region_stats<D, G>(T, has, status, nc, pbytes, ptests);
    if (has && gl == 0) {
      if (status == CAND_OVER) {
        if (T.dbg) atomicAdd(&T.dbg[6], 1ull);
        const int q = atomicAdd(S.nbig, 1);
        if (q < BIGCAP) S.biglist[q] = slot;
        else atomicExch(&T.st->overflow_cav, 1);
      }
      S.meta[slot] = make_int4(nc, nbd, status, 0);
    }
    __syncwarp();
  }
}

// The region-growth kernel compiled for 8, 12 or 16 resident blocks per SM
// (register caps 64, 40, 32 per thread): more resident warps hide more of the
// load latency the growth waits on, fewer registers spill more.  group = 16:
// two nominees per warp (8 blocks per SM).
template <int D>
static decltype(&k_cavity_w<D, 8, 32>) cavity_kernel(int occupancy, int group) {
  if (group == 16) return &k_cavity_w<D, 8, 16>;
  if (occupancy >= 16) return &k_cavity_w<D, 16, 32>;
  if (occupancy >= 12) return &k_cavity_w<D, 12, 32>;
  return &k_cavity_w<D, 8, 32>;
}

// Region growth by a whole thread block of NT threads (NT / (D+1) region
// simplices x (D+1) facets per step), for the large regions: their
// breadth-first front is wide, so a step of one block does the work of NT/32
// warp steps at about the latency of one.  The rules are those of
// grow_region: the same claims, the same boundary facets, the same statuses;
// the per-step additions are placed by a scan over the block's warps.
template <int D, int NT>
__device__ __forceinline__ void grow_region_cta(const TriView<D>& T, int p, unsigned long long key, int* C, int* B,
                                                int capC, int capB, int& nc_out, int& nbd_out, int& status_out,
                                                unsigned long long& pbytes, unsigned long long& ptests) {
  const unsigned FULL = 0xffffffffu;
  constexpr int NW = NT / 32, PER = NT / (D + 1);
  __shared__ int s_add[NW][3];                         // per warp: region, boundary, lost
  __shared__ int s_first;                              // status after the located simplex
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const unsigned below = (1u << lane) - 1u;
  if (tid == 0) {
    const int t0 = T.loc[p];
    unsigned long long oc = atomicMax(&T.claimC[t0], key);
    unsigned long long o = atomicMax(&T.claimA[t0], key);
    s_first = (o > key || oc > key) ? CAND_LOST : CAND_OK;
    C[0] = t0;
    pbytes += sizeof(typename PT<D>::T) + 4 + 8 + 16 * (D + 1) + 16 + 4;
  }
  __syncthreads();
  int status = s_first, nc = 1, nbd = 0, h = 0, nsteps = 0;
  while (status == CAND_OK && h < nc) {                // block-uniform
    const int nc0 = nc;
    const int j = h + tid / (D + 1), i = tid % (D + 1);
    const bool valid = tid < PER * (D + 1) && j < nc0;
    bool addC = false, addB = false, lost = false, bad = false;
    int t = -1, u = -1;
    if (valid) {
      t = C[j];
      u = nb_simplex(*comp_ptr(T.tn, t, i));
      if (!slot_ok(T, u)) {
        bad = true;
      } else {
        const int4 vv = T.tv[u];
        unsigned long long cC = *((volatile unsigned long long*)&T.claimC[u]);
        pbytes += 16;
        if (cC > key) {
          lost = true;
        } else if (cC != key) {
          pbytes += 16 + (D + 1) * sizeof(typename PT<D>::T);
          ptests++;
          if (!verts_ok(T, vv)) {
            bad = true;
          } else {
            int vt[4] = {vv.x, vv.y, vv.z, vv.w};
            if (in_conflict_x(T.pts, T.xs, T.gid, vt, p, D)) {
              unsigned long long o = atomicMax(&T.claimC[u], key);
              unsigned long long o2 = atomicMax(&T.claimA[u], key);
              if (o > key || o2 > key) {
                lost = true;
              } else if (o < key) {
                addC = true;
                pbytes += 16 + 4;
              }
            } else {
              atomicMax(&T.claimA[u], key);
              addB = true;
              pbytes += 8 + 4;
            }
          }
        }
      }
    }
    if (bad) set_error(T.st, DT_E_INTERNAL, 10);
    const unsigned mL = __ballot_sync(FULL, lost || bad), mC = __ballot_sync(FULL, addC),
                   mB = __ballot_sync(FULL, addB);
    if (lane == 0) { s_add[w][0] = __popc(mC); s_add[w][1] = __popc(mB); s_add[w][2] = mL != 0u; }
    __syncthreads();
    int offC = 0, offB = 0, nC = 0, nB = 0, anyL = 0;
#pragma unroll
    for (int q = 0; q < NW; q++) {
      if (q < w) { offC += s_add[q][0]; offB += s_add[q][1]; }
      nC += s_add[q][0]; nB += s_add[q][1]; anyL |= s_add[q][2];
    }
    if (anyL) {
      status = CAND_LOST;
    } else if (nc + nC > capC || nbd + nB > capB) {
      status = CAND_OVER;
    } else {
      if (addC) C[nc + offC + __popc(mC & below)] = u;
      if (addB) B[nbd + offB + __popc(mB & below)] = pack_nb(t, i);
      nc += nC;
      nbd += nB;
      h = min(h + PER, nc0);
    }
    __syncthreads();                                   // list entries visible, s_add free again
    nsteps++;
  }
  if (T.dbg && tid == 0) atomicAdd(&T.dbg[7], (unsigned long long)nsteps);
  nc_out = nc;
  nbd_out = nbd;
  status_out = status;
}

// Threads per block of the large-region kernel (one block per region).
constexpr int BIG_NT = 256;

// Second growth of large region q (one block of NT threads, all of which call).
template <int D, int NT>
__device__ __forceinline__ void big_region(const TriView<D>& T, unsigned round, const CandScratch& S, int q) {
  const int slot = S.biglist[q];
  const int p = S.cand[slot];
  const unsigned long long key = mkkey(round, p) | 1ull;   // second pass: see mkkey
  int* C = S.bigcav + (int64_t)q * S.capCbig;
  int* B = S.bigbnd + (int64_t)q * S.capBbig;
  unsigned long long pbytes = 0, ptests = 0;
  int nc, nbd, status;
  grow_region_cta<D, NT>(T, p, key, C, B, S.capCbig, S.capBbig, nc, nbd, status, pbytes, ptests);
  // counters: every warp adds its own lanes' bytes and tests, the first thread the region's
  if (T.prof) {
    for (int off = 16; off; off >>= 1) {
      pbytes += __shfl_down_sync(0xffffffffu, pbytes, off);
      ptests += __shfl_down_sync(0xffffffffu, ptests, off);
    }
    if ((threadIdx.x & 31) == 0) { atomicAdd(&T.prof[0], pbytes); atomicAdd(&T.prof[1], ptests); }
  }
  if (threadIdx.x == 0) {
    if (T.dbg) {
      if (status == CAND_OK) atomicAdd(&T.dbg[4], 1ull);
      atomicAdd(&T.dbg[5], (unsigned long long)nc);
    }
    if (status == CAND_OVER) atomicExch(&T.st->overflow_cav, 1);
    S.meta[slot] = make_int4(nc, nbd, status, q + 1);
  }
  __syncthreads();
}

// Large regions: the nominees whose region outgrew the regular lists grow it
// again into lists of capCbig / capBbig entries (their claims so far stand;
// atomicMax makes the repeated claims harmless), one block per region.
template <int D>
__global__ void __launch_bounds__(BIG_NT) k_cavity_big(TriView<D> T, unsigned round, CandScratch S, const EngCtl* ctl) {
  pdl_enter();
  if (ctl) {
    if (ctl->small || ctl->done) return;
    round = ctl->round;
  }
  const int nbig = min(*S.nbig, BIGCAP);
  for (int q = blockIdx.x; q < nbig; q += gridDim.x) big_region<D, BIG_NT>(T, round, S, q);
}

// Blocks of the large-region kernel: at most one per region, at most one per SM.
static inline unsigned big_grid(int sms) { return (unsigned)std::min(BIGCAP, std::max(sms, 1)); }

// One warp per nominee: a nominee wins if no stronger nominee claimed any of
// its region (claimA) or has any of its ring in its own region (claimC).
// Winners replace their region by the star of new simplices in fresh slots.
// Insertion of the candidate in `slot` if it won (one warp): verify the
// claims, build the star over the boundary, retire the region.
template <int D>
__device__ __forceinline__ void insert_winner(const TriView<D>& T, unsigned round, const CandScratch& S, int slot,
                                              int* nwin) {
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;

  int4 m = S.meta[slot];
  if (m.z != CAND_OK) return;
  int p = S.cand[slot];
  const bool big = m.w > 0;
  const unsigned long long key = mkkey(round, p) | (big ? 1ull : 0ull);
  const int* C = big ? S.bigcav + (int64_t)(m.w - 1) * S.capCbig : S.cav + (int64_t)slot * S.capC;
  const int* B = big ? S.bigbnd + (int64_t)(m.w - 1) * S.capBbig : S.bnd + (int64_t)slot * S.capB;
  int* OUT = big ? S.bigout + (int64_t)(m.w - 1) * S.capBbig : S.outer + (int64_t)slot * S.capB;
  int nc = m.x, nbd = m.y;
  bool ok = true;
  for (int j = lane; j < nc; j += 32)
    if (*((volatile unsigned long long*)&T.claimA[C[j]]) != key) ok = false;
  // a region shared with a stronger winner may already carry its tags: stop here
  if (!__all_sync(FULL, ok)) return;
  for (int b = lane; b < nbd; b += 32) {
    int t = nb_simplex(B[b]), i = nb_face(B[b]);
    int u = nb_simplex(*comp_ptr(T.tn, t, i));
    if (!slot_ok(T, u)) { set_error(T.st, DT_E_INTERNAL, 12); ok = false; }
    else if (*((volatile unsigned long long*)&T.claimC[u]) > key) ok = false;
  }
  if (!__all_sync(FULL, ok)) return;
  int inst = T.pinst[p];
  int base = 0;
  if (lane == 0) base = atomicAdd(&T.tcount[inst], nbd);
  base = __shfl_sync(FULL, base, 0);
  if (base + nbd > T.tend[inst]) {
    if (lane == 0) set_error(T.st, DT_E_OVERFLOW, 1);
    return;
  }
  // phase 1: remember the outside links, tag boundary facets with their new simplex
  for (int b = lane; b < nbd; b += 32) {
    int t = nb_simplex(B[b]), i = nb_face(B[b]);
    int* cp = comp_ptr(T.tn, t, i);
    OUT[b] = *cp;
    *cp = TAGBIT | (base + b);
  }
  __syncwarp();
  // phase 2: build the star of p over the boundary
  for (int b = lane; b < nbd; b += 32) {
    int t = nb_simplex(B[b]), i = nb_face(B[b]);
    int4 vv = T.tv[t];
    set4(vv, i, p);
    int4 nn = make_int4(0, 0, 0, 0);
    int out = OUT[b];
    set4(nn, i, out);
    if (slot_ok(T, nb_simplex(out))) *comp_ptr(T.tn, nb_simplex(out), nb_face(out)) = pack_nb(base + b, i);
    else set_error(T.st, DT_E_INTERNAL, 13);
    for (int j = 0; j <= D; j++) {
      if (j == i) continue;
      // rotate around the ridge (t minus slots i and j) inside the region
      int cur = t, as = j, bs = i;
      int link = -1;
      for (int it = 0; it <= nc + 1; it++) {
        int nx = *comp_ptr(T.tn, cur, as);
        if (nx < 0) { link = pack_nb(nx & ~TAGBIT, bs); break; }
        int nxt = nb_simplex(nx);
        if (!slot_ok(T, nxt)) break;
        int bvtx = get4(T.tv[cur], bs);
        int4 nv = T.tv[nxt];
        int nas = -1;
        for (int l = 0; l <= D; l++) if (get4(nv, l) == bvtx) nas = l;
        bs = nb_face(nx);
        as = nas;
        cur = nxt;
        if (as < 0) break;
      }
      if (link < 0) {
        if (atomicCAS(&T.st->error, 0, DT_E_INTERNAL) == 0) {
          T.st->detail = 2;
          int* d = T.st->dbg;
          d[0] = (int)round; d[1] = p; d[2] = nc; d[3] = nbd; d[4] = b; d[5] = j; d[6] = t; d[7] = i;
          d[8] = cur; d[9] = as; d[10] = bs; d[11] = slot;
        }
        link = 0;
      }
      set4(nn, j, link);
    }
    T.tv[base + b] = vv;
    T.tn[base + b] = nn;
  }
  __syncwarp();
  // phase 3: retire the region.  A dead slot redirects to a new simplex
  // near the points it held: the one over one of its own boundary facets,
  // else the one a neighbouring region simplex redirects to, else the
  // first one.  (Until now every link of a region simplex is an old slot,
  // below every base of this round, so a link into [base, base + nbd) is
  // a redirect already written.)
  for (int h = lane; h < nc; h += 32) *comp_ptr(T.tv, C[h], 0) = DEAD;
  for (int b = lane; b < nbd; b += 32) *comp_ptr(T.tn, nb_simplex(B[b]), 0) = pack_nb(base + b, 0);
  __syncwarp();
  for (int h = lane; h < nc; h += 32) {
    const int t = C[h];
    const int4 nt = T.tn[t];
    auto fresh = [&](int link) { const int q = nb_simplex(link); return link >= 0 && q >= base && q < base + nbd; };
    if (fresh(nt.x)) continue;
    int red = pack_nb(base, 0);
    for (int k = 0; k <= D; k++) {
      const int u = nb_simplex(get4(nt, k));
      if (!slot_ok(T, u)) continue;
      const int r = *comp_ptr(T.tn, u, 0);
      if (fresh(r)) { red = r; break; }
    }
    *comp_ptr(T.tn, t, 0) = red;
  }
  if (lane == 0) {
    T.state[p] = 1;
    T.loc[p] = base;
    atomicAdd(nwin, 1);
    if (T.hint) {
      int f, g;
      hint_cells(T, p, f, g);
      T.hint[f] = base;
      T.hint2[g] = base;
    }
  }
  __syncwarp();

}

template <int D>
__global__ void __launch_bounds__(128) k_insert_w(TriView<D> T, unsigned round, CandScratch S, const int* nnom_p,
                                                  int* nwin, const EngCtl* ctl) {
  pdl_enter();
  if (ctl) {
    if (ctl->small || ctl->done) return;
    round = ctl->round;
  }
  const int nwarp = (gridDim.x * blockDim.x) >> 5;
  const int total = min(*nnom_p, S.cap);
  for (int slot = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; slot < total; slot += nwarp)
    insert_winner<D>(T, round, S, slot, nwin);
}

// Visibility walk to a simplex in conflict with point p: a finite simplex
// containing p (closed), or a ghost entered through its hull facet.
template <int D>
__device__ int walk_to(const TriView<D>& T, int s, int p, int limit, int* steps_out = nullptr) {
  if (!slot_ok(T, s)) return -1;
  int4 vv = T.tv[s];
  for (int i = 0; i <= D; i++)
    if (get4(vv, i) == INF_V) {
      s = nb_simplex(get4(T.tn[s], i));
      if (!slot_ok(T, s)) return -1;
      vv = T.tv[s];
      break;
    }
  int skip = -1;
  for (int it = 0; it < limit; it++) {
    bool ghost = false;
    for (int i = 0; i <= D; i++) ghost |= (get4(vv, i) == INF_V);
    if (ghost) return s;
    if (!verts_ok(T, vv)) return -1;
    int next = -1, nf = -1;
    for (int i = 0; i <= D; i++) {
      if (i == skip) continue;
      int4 t = vv;
      set4(t, i, p);
      if (orient_tuple(T, t) < 0) {
        int nx = get4(T.tn[s], i);
        next = nb_simplex(nx);
        nf = nb_face(nx);
        break;
      }
    }
    if (steps_out) (*steps_out)++;
    if (next < 0) return s;
    if (!slot_ok(T, next)) return -1;
    s = next;
    skip = nf;
    vv = T.tv[s];
  }
  return -1;
}

// Keeps uninserted points for the next round; points whose simplex died go
// to the walker list, the others make the next round's pick right away.
// Relocation check of the 32 active points from `base` (one warp): points
// still uninserted stay active; those whose simplex died go to the walk list,
// the others pick their simplex for the next round.
template <int D>
__device__ __forceinline__ void reloc_check_warp(const TriView<D>& T, const int* act, int nact, int* act_out,
                                                 int* nact_out, int* walk, int* nwalk, unsigned next_round,
                                                 int64_t base) {
  const int64_t idx = base + (threadIdx.x & 31);
  bool keep = false, walker = false;
  int p = -1;
  if (idx < nact) {
    p = act[idx];
    if (T.state[p] == 0) {
      keep = true;
      int s = T.loc[p];
      if (*comp_ptr(T.tv, s, 0) == DEAD) walker = true;
      else atomicMax(&T.claimC[s], mkkey(next_round, p));
    }
  }
  warp_append(act_out, nact_out, keep, p);
  warp_append(walk, nwalk, walker, p);
  if (T.inst_kept && keep) atomicAdd(&T.inst_kept[T.pinst[p]], 1);
  if (T.prof) {
    // act 4, state 1, loc 4, slot word 4, pick 8, output 4
    unsigned long long b = idx < nact ? 25 : 0;
    for (int off = 16; off; off >>= 1) b += __shfl_down_sync(0xffffffffu, b, off);
    if ((threadIdx.x & 31) == 0) atomicAdd(&T.prof[3], b);
  }
}

template <int D>
__global__ void k_reloc_check(TriView<D> T, const int* act, const int* nact_p, int* act_out, int* nact_out,
                              int* walk, int* nwalk, unsigned next_round, const EngCtl* ctl) {
  pdl_enter();
  if (ctl) {
    if (ctl->small || ctl->done) return;
    act = ctl->ain; act_out = ctl->aout; next_round = ctl->round + 1;
  }
  const int nact = *nact_p;
  // warp-uniform grid-stride loop (warp_append needs every lane)
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < nact;
       base += (int64_t)gridDim.x * blockDim.x)
    reloc_check_warp<D>(T, act, nact, act_out, nact_out, walk, nwalk, next_round, base);
}

// Activates a batch of dormant points: from the simplex each was parked on,
// follow the redirects of dead simplices to a live one, walk to a simplex in
// conflict with the point, make its pick for the next round, and append it
// to the active list.
// Activation of the 32 dormant points from `base` of list (one warp):
// locate each from its hint cell (or its parked simplex) and pick.
// Is simplex slot h inside instance i's arena?
template <int D>
__device__ __forceinline__ bool in_instance(const TriView<D>& T, int h, int i) {
  return slot_ok(T, h) && h >= T.toff[i] && h < T.tend[i];
}

// Locates dormant point p from its hint cell (or its parked simplex) and
// makes its pick for next_round; false when the walk gave up.
template <int D>
__device__ __forceinline__ bool activate_point(const TriView<D>& T, int p, unsigned next_round) {
  int s = T.loc[p];
  if (T.hint) {
    int f, g;
    hint_cells(T, p, f, g);
    const int i = T.pinst[p];
    int h = T.hint[f];
    if (!in_instance(T, h, i)) h = T.hint2[g];
    if (in_instance(T, h, i)) s = h;
  }
  for (int hop = 0; hop < T.walk_limit && slot_ok(T, s) && *comp_ptr(T.tv, s, 0) == DEAD; hop++)
    s = nb_simplex(*comp_ptr(T.tn, s, 0));
  int steps = 0;
  int r = walk_to(T, s, p, T.walk_limit, &steps);
  if (T.dbg) { atomicAdd(&T.dbg[2], (unsigned long long)steps); atomicMax(&T.dbg[3], (unsigned long long)steps); }
  if (r < 0) {
    set_error(T.st, DT_E_TIMEOUT, 4);
    return false;
  }
  T.loc[p] = r;
  atomicMax(&T.claimC[r], mkkey(next_round, p));
  return true;
}

template <int D>
__device__ __forceinline__ void activate_warp(const TriView<D>& T, const int* list, int m, int* act, int* nact,
                                              unsigned next_round, int64_t base) {
  const int64_t idx = base + (threadIdx.x & 31);
  bool ok = false;
  int p = -1;
  if (idx < m) {
    p = list[idx];
    ok = activate_point(T, p, next_round);
  }
  warp_append(act, nact, ok, p);
}

template <int D>
__global__ void __launch_bounds__(128, 8) k_activate(TriView<D> T, const int* list, int m, int* act, int* nact,
                                                  unsigned next_round, const EngCtl* ctl) {
  pdl_enter();
  if (ctl) {
    if (ctl->small || ctl->done) return;
    list += ctl->act_lo; m = ctl->act_n; act = ctl->ain; next_round = ctl->round;
  }
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < m;
       base += (int64_t)gridDim.x * blockDim.x)
    activate_warp<D>(T, list, m, act, nact, next_round, base);
}

// Opt-in self-check of the mesh (GDT_CHECK): every live simplex's links are
// symmetric and neighbours share the facet's vertices.
template <int D>
__global__ void k_check_mesh(TriView<D> T, const int* toff, const int* tcount, int ninst, unsigned round) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= T.nslots) return;
  int lo = 0, hi = ninst - 1;
  while (lo < hi) { int mid = (lo + hi + 1) >> 1; if (toff[mid] <= s) lo = mid; else hi = mid - 1; }
  if (s >= tcount[lo]) return;
  int4 v = T.tv[s];
  if (v.x == DEAD) return;
  int4 n = T.tn[s];
  for (int i = 0; i <= D; i++) {
    int x = get4(n, i);
    int u = nb_simplex(x), f = nb_face(x);
    bool bad = !slot_ok(T, u);
    if (!bad) {
      int4 w = T.tv[u];
      bad = w.x == DEAD || get4(T.tn[u], f) != pack_nb(s, i);
      if (!bad) {
        for (int a = 0; a <= D; a++) {
          if (a == i) continue;
          bool found = false;
          for (int b = 0; b <= D; b++) if (b != f && get4(w, b) == get4(v, a)) found = true;
          bad |= !found;
        }
      }
    }
    if (bad && atomicCAS(&T.st->error, 0, DT_E_INTERNAL) == 0) {
      T.st->detail = 30;
      int* d = T.st->dbg;
      d[0] = (int)round; d[1] = s; d[2] = i; d[3] = x; d[4] = v.x; d[5] = v.y; d[6] = v.z; d[7] = v.w;
    }
  }
}

// Relocation walk of point p whose simplex died.
template <int D>
__device__ __forceinline__ void reloc_walk_one(const TriView<D>& T, int p, unsigned next_round) {
  int s = nb_simplex(*comp_ptr(T.tn, T.loc[p], 0));
  int steps = 0;
  int r = walk_to(T, s, p, T.walk_limit, &steps);
  if (r < 0) { set_error(T.st, DT_E_TIMEOUT, 3); return; }
  T.loc[p] = r;
  atomicMax(&T.claimC[r], mkkey(next_round, p));
  // per step: vertex tuple 16, links 16, D+1 points; per point: 4 + 4 + 8
  if (T.prof) atomicAdd(&T.prof[2], (unsigned long long)steps * (32 + (D + 1) * sizeof(typename PT<D>::T)) + 16);
  if (T.dbg) { atomicAdd(&T.dbg[0], (unsigned long long)steps); atomicMax(&T.dbg[1], (unsigned long long)steps); }
}

template <int D>
__global__ void __launch_bounds__(128, 8) k_reloc_walk(TriView<D> T, const int* walk, const int* nwalk_p,
                                                    unsigned next_round, const EngCtl* ctl) {
  pdl_enter();
  if (ctl) {
    if (ctl->small || ctl->done) return;
    next_round = ctl->round + 1;
  }
  const int nwalk = *nwalk_p;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < nwalk;
       idx += (int64_t)gridDim.x * blockDim.x)
    reloc_walk_one<D>(T, walk[idx], next_round);
}

static __device__ __forceinline__ unsigned long long ord_key(double x) {
  unsigned long long b = (unsigned long long)__double_as_longlong(x + 0.0);
  return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}
// FP32 copies for the first predicate stage: X = fl32(x - o_i), w = eta_i
// (xo: per instance the origin (3) and eta (1)).
template <int D>
__global__ void k_make_x32(const typename PT<D>::T* pts, const int* pinst, int64_t npts, const double* xo, float4* xs) {
  int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= npts) return;
  const double* o = xo + 4 * (pinst ? pinst[p] : 0);
  const typename PT<D>::T q = pts[p];
  xs[p] = make_float4((float)(cx(q) - o[0]), (float)(cy(q) - o[1]), D == 3 ? (float)(cz(q) - o[2]) : 0.0f,
                      (float)o[3]);
}

static __global__ void k_scatter_levels(const int* level, const int* rank, const int* loff, int64_t n, int* list) {
  int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p < n && level[p] >= 0) list[loff[level[p]] + rank[p]] = (int)p;
}

static __global__ void k_move_count(int* dst, int* src) {
  *dst = *src;
  *src = 0;
}

// Start of a device-driven round: activate the next level(s) when the active
// set has drained to a quarter of the last batch (the rule of the host
// loop), advance the round, clear the round's counters.
static __device__ void round_begin(EngCtl& C, int* cnt, const int* loffd) {
  int nact = cnt[0];
  int lo = -1, hi = -1;
  // drain rule: the next level(s) once the active set has drained to
  // last_batch / drain; continuous rule: levels while the active set is
  // below ratio x the points inserted so far (activated - still active)
  auto wants = [&]() {
    if (C.ratio <= 0.0f) return nact <= C.last_batch / C.drain;
    const long long inserted = C.activated_total - nact;
    return (long long)nact < max((long long)C.min_active, (long long)(C.ratio * (float)inserted));
  };
  while (C.next_level >= 0 && wants()) {
    const int l = C.next_level;
    const int m = loffd[l + 1] - loffd[l];
    if (m > 0) {
      if (hi < 0) hi = loffd[l + 1];
      lo = loffd[l];
      nact += m;
      C.activated_total += m;
      C.last_batch = nact;
    }
    C.next_level--;
  }
  C.act_lo = lo < 0 ? 0 : lo;
  C.act_n = lo < 0 ? 0 : hi - lo;
  C.activated = C.act_n;
  C.small = nact <= C.small_max ? 1 : 0;
  if (nact > 0) C.round++;
  if (C.round > (unsigned)C.round_limit && C.done == 0) C.done = 4;
  cnt[1] = cnt[2] = cnt[3] = cnt[4] = cnt[5] = 0;
  for (int b = 0; b < NBUCKET; b++) cnt[8 + b] = 0;
}

// The first round's start (before the loop).  One thread.
static __global__ void k_round_begin(EngCtl* ctl, int* cnt, const int* loffd) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  round_begin(*ctl, cnt, loffd);
}

// End of a device-driven round and start of the next: the next active list
// becomes current; the loop ends when nothing is left, on a device error,
// after 4 rounds in a row without an insertion (a cavity overflowed its
// scratch: the host grows it), or at the round limit.  One thread.
static __device__ void round_end_begin(EngCtl& C, int* cnt, const int* loffd, const DevStatus* st) {
  const int had = cnt[0];
  const int nnew = cnt[1];
  cnt[0] = nnew;
  cnt[1] = 0;
  int* t = C.ain;
  C.ain = C.aout;
  C.aout = t;
  if (C.done == 0) {
    if (st->error) C.done = 2;
    else if (nnew == 0 && C.next_level < 0) C.done = 1;
    else if (had > 0 && cnt[3] == 0 && ++C.stalled >= 4) C.done = 3;
    else if (cnt[3] > 0) C.stalled = 0;
  }
  C.last_nact = nnew;
  if (C.done == 0) round_begin(C, cnt, loffd);
}

static __global__ void k_round_step(EngCtl* ctl, int* cnt, const int* loffd, const DevStatus* st,
                             cudaGraphConditionalHandle handle) {
  pdl_enter();
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  EngCtl& C = *ctl;
  // small rounds were run and closed by k_small_rounds
  if (!C.small) round_end_begin(C, cnt, loffd, st);
  cudaGraphSetConditional(handle, C.done == 0 ? 1u : 0u);
}

// Nomination of the 32 active points from `base` into one list (small rounds).
template <int D>
__device__ __forceinline__ void nominate_warp(const TriView<D>& T, const int* act, int nact, unsigned round,
                                              int* nom, int* nnom, int64_t base) {
  const int64_t idx = base + (threadIdx.x & 31);
  bool take = false;
  int p = -1;
  if (idx < nact) {
    p = act[idx];
    const unsigned long long key = mkkey(round, p);
    const int t0 = T.loc[p];
    if (*((volatile unsigned long long*)&T.claimC[t0]) == key) {
      take = true;
      const int4 nn0 = T.tn[t0];
      for (int i = 0; i <= D; i++) {
        const int u = nb_simplex(get4(nn0, i));
        if (slot_ok(T, u) && *((volatile unsigned long long*)&T.claimC[u]) > key) take = false;
      }
      if (take && T.rings > 1 && stronger_in_ring2(T, t0, nn0, key)) take = false;
    }
  }
  warp_append(nom, nnom, take, p);
}

// Region growth of the nominee in `slot` with its lists in global memory (one warp).
template <int D>
__device__ __forceinline__ void cavity_slot(const TriView<D>& T, unsigned round, const CandScratch& S, const int* nom,
                                            const int* bcnt, int slot) {
  const int lane = threadIdx.x & 31;
  const int p = nominee_at(nom, bcnt, S.cap, slot);
  const unsigned long long key = mkkey(round, p);
  int* C = S.cav + (int64_t)slot * S.capC;
  int* B = S.bnd + (int64_t)slot * S.capB;
  if (lane == 0) S.cand[slot] = p;
  unsigned long long pbytes = 0, ptests = 0;
  int nc, nbd, status;
  grow_region<D, 32>(T, true, p, key, C, nullptr, B, S.capC, S.capB, nc, nbd, status, pbytes, ptests);
  region_stats<D, 32>(T, true, status, nc, pbytes, ptests);
  if (lane == 0) {
    if (status == CAND_OVER) {
      const int q = atomicAdd(S.nbig, 1);
      if (q < BIGCAP) S.biglist[q] = slot;
      else atomicExch(&T.st->overflow_cav, 1);
    }
    S.meta[slot] = make_int4(nc, nbd, status, 0);
  }
  __syncwarp();
}

// Small rounds in one CTA: while the active set is at most small_max points
// (the sample triangulation, the first and the last rounds of every run),
// every phase of a round runs here between __syncthreads barriers instead of
// as separate launches.  Up to SMALL_ITERS rounds per launch; the round state
// is the same control block, so the regular kernels take over (or resume)
// whenever a round is not small.
constexpr int SMALL_ITERS = 256;

template <int D>
__global__ void __launch_bounds__(1024) k_small_rounds(TriView<D> T, EngCtl* ctl, int* cnt, const int* loffd,
                                                       const int* llist, int* nom, int* walk, CandScratch S) {
  __shared__ int s_go;
  const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int it = 0; it < SMALL_ITERS; it++) {
    if (threadIdx.x == 0) s_go = (ctl->done == 0 && ctl->small) ? 1 : 0;
    __syncthreads();
    if (!s_go) return;
    volatile int* vc = cnt;
    const unsigned round = ctl->round;
    int* ain = ctl->ain;
    int* aout = ctl->aout;
    const int m = ctl->act_n;
    const int* list = llist + ctl->act_lo;
    for (int64_t base = warp * 32; base < m; base += nw * 32) activate_warp<D>(T, list, m, ain, cnt + 0, round, base);
    __syncthreads();
    const int nact = vc[0];
    for (int64_t base = warp * 32; base < nact; base += nw * 32)
      nominate_warp<D>(T, ain, nact, round, nom, cnt + 2, base);
    __syncthreads();
    if (threadIdx.x < NBUCKET) vc[8 + threadIdx.x] = threadIdx.x == 0 ? vc[2] : 0;
    __syncthreads();
    const int nn = min(vc[2], S.cap);
    for (int slot = warp; slot < nn; slot += nw) cavity_slot<D>(T, round, S, nom, cnt + 8, slot);
    __syncthreads();
    const int nbig = min(vc[5], BIGCAP);
    for (int q = 0; q < nbig; q++) big_region<D, 1024>(T, round, S, q);   // the whole block, region by region
    __syncthreads();
    for (int slot = warp; slot < nn; slot += nw) insert_winner<D>(T, round, S, slot, cnt + 3);
    __syncthreads();
    for (int64_t base = warp * 32; base < nact; base += nw * 32)
      reloc_check_warp<D>(T, ain, nact, aout, cnt + 1, walk, cnt + 4, round + 1, base);
    __syncthreads();
    const int nwk = vc[4];
    for (int i = threadIdx.x; i < nwk; i += blockDim.x) reloc_walk_one<D>(T, walk[i], round + 1);
    __syncthreads();
    if (threadIdx.x == 0) round_end_begin(*ctl, cnt, loffd, T.st);
    __syncthreads();
  }
}

// ---------------------------------------------------------------- host
static __global__ void k_read_pred_counters(unsigned long long* calls, int* range, int reset) {
  *calls = g_exact_calls;
  *range = g_range_error;
  if (reset) g_exact_calls = 0;
}

static double host_from_orderable(unsigned long long u) {
  unsigned long long b = (u >> 63) ? (u & 0x7fffffffffffffffull) : ~u;
  double x;
  memcpy(&x, &b, 8);
  return x;
}

// Profile mode: events recorded between the engine's launches without any
// synchronisation; the times are read once, after the last round.
static cudaEvent_t prof_event(dt_ctx* c, size_t i) {
  while (c->evpool.size() <= i) {
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) { cudaGetLastError(); return nullptr; }
    c->evpool.push_back(e);
  }
  return c->evpool[i];
}

#ifdef GDT_ENGINE_SHARED
void prof_add(dt_ctx* c, const char* name, double ms, double bytes, double flops) {
  for (auto& k : c->kprof)
    if (!strcmp(k.name, name)) {
      if (ms > 0) { k.ms += ms; k.launches++; }
      k.bytes += bytes;
      k.flops += flops;
      return;
    }
  c->kprof.push_back({name, ms > 0 ? 1 : 0, ms, bytes, flops});
}

#endif

// Exact-stage counters of this translation unit's predicates (each unit
// holds its own copy of the device counters).
static int pred_counters_local(dt_ctx* c, unsigned long long* calls, int* range, bool reset) {
  void* buf = pool_get(c, "predctr_eng", 64);
  if (!buf) return set_err(c, DT_E_NOMEM, "predicate counters");
  k_read_pred_counters<<<1, 1, (++c->launches, 0), c->stream>>>((unsigned long long*)buf, (int*)((char*)buf + 8), reset);
  unsigned long long h[2];
  CUDA_OK(cudaMemcpyAsync(h, buf, 16, cudaMemcpyDeviceToHost, c->stream));
  CUDA_OK(cudaStreamSynchronize(c->stream));
  *calls = h[0];
  *range = (int)(h[1] & 0xffffffff);
  return 0;
}

#ifdef GDT_ENGINE_SHARED
// FP32 copies of the points for the first predicate stage (see
// predicates.cuh): per instance (pinst, or one instance when null) the
// bounding box gives the origin o (its centre) and eta = 2 (u32 + 2 u64) R
// rounded up, R the largest |x_c - o_c|.  *hu_out receives the boxes as
// orderable keys (lo[3], hi[3] per instance).
int fp32_points(dt_ctx* c, int dim, const void* pts, const int* pinst, int64_t npts, int ninst, const std::string& tag,
                float4** xs_out, std::vector<unsigned long long>* hu_out, const double** xo_out) {
  cudaStream_t s = c->stream;
  float4* xs = (float4*)pool_get(c, tag, 16 * (size_t)std::max<int64_t>(npts, 1));
  double* xo = (double*)pool_get(c, tag + ".o", 8 * 4 * (size_t)ninst);
  unsigned long long* ub = (unsigned long long*)pool_get(c, tag + ".box", 8 * 6 * (size_t)ninst);
  if (!xs || !xo || !ub) return set_err(c, DT_E_NOMEM, "fp32 points");
  *xs_out = xs;
  if (xo_out) *xo_out = xo;
  std::vector<unsigned long long>& hu = *hu_out;
  hu.assign(6 * (size_t)ninst, 0);
  if (npts == 0) return 0;
  unsigned g = (unsigned)ceil_div<int64_t>(npts, 256);
  k_box_init<<<ceil_div(6 * ninst, 128), 128, (++c->launches, 0), s>>>(ub, ninst);
  if (dim == 2) k_box_reduce<2><<<box_grid(npts), 256, (++c->launches, 0), s>>>((const double2*)pts, pinst, npts, ub);
  else k_box_reduce<3><<<box_grid(npts), 256, (++c->launches, 0), s>>>((const double4_32a*)pts, pinst, npts, ub);
  CUDA_OK(cudaMemcpyAsync(hu.data(), ub, 8 * 6 * (size_t)ninst, cudaMemcpyDeviceToHost, s));
  CUDA_OK(cudaStreamSynchronize(s));
  std::vector<double> hxo(4 * (size_t)ninst, 0.0);
  for (int i = 0; i < ninst; i++) {
    if (hu[6 * i] == ~0ull) continue;   // no points
    double R = 0.0;
    for (int cc = 0; cc < dim; cc++) {
      double lo = host_from_orderable(hu[6 * i + cc]), hi = host_from_orderable(hu[6 * i + 3 + cc]);
      double o = 0.5 * lo + 0.5 * hi;
      hxo[4 * i + cc] = o;
      R = std::max(R, std::max(hi - o, o - lo));
    }
    // eta >= 2 (u32 + 2 u64) R, with slack for the roundings of this line
    double eta = 2.02 * (std::ldexp(1.0, -24) + std::ldexp(1.0, -52)) * R * (1.0 + 1e-9);
    float ef = (float)eta;
    if (!((double)ef >= eta)) ef = std::nextafter(ef, INFINITY);
    hxo[4 * i + 3] = (double)ef;
  }
  CUDA_OK(cudaMemcpyAsync(xo, hxo.data(), 8 * 4 * (size_t)ninst, cudaMemcpyHostToDevice, s));
  if (dim == 2) k_make_x32<2><<<g, 256, (++c->launches, 0), s>>>((const double2*)pts, pinst, npts, xo, xs);
  else k_make_x32<3><<<g, 256, (++c->launches, 0), s>>>((const double4_32a*)pts, pinst, npts, xo, xs);
  CUDA_OK(cudaStreamSynchronize(s));   // hxo goes out of scope
  return 0;
}

#endif

// Scratch of the large regions (shared by every round; counter cnt[5]).
static int big_scratch(dt_ctx* c, CandScratch& S, int* cnt) {
  S.capCbig = BIG_C;
  S.capBbig = BIG_B;
  S.bigcav = (int*)pool_get(c, "eng.bigcav", 4 * (size_t)BIGCAP * BIG_C);
  S.bigbnd = (int*)pool_get(c, "eng.bigbnd", 4 * (size_t)BIGCAP * BIG_B);
  S.bigout = (int*)pool_get(c, "eng.bigout", 4 * (size_t)BIGCAP * BIG_B);
  S.biglist = (int*)pool_get(c, "eng.biglist", 4 * (size_t)BIGCAP);
  S.nbig = cnt + 5;
  if (!S.bigcav || !S.bigbnd || !S.bigout || !S.biglist) return set_err(c, DT_E_NOMEM, "large-region scratch");
  return 0;
}

// Capture stream of the context (created on first use).
static cudaStream_t capture_stream(dt_ctx* c) {
  if (!c->cap_stream && cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    c->cap_stream = nullptr;
  }
  return c->cap_stream;
}

// Every insertion round on the device: a graph whose conditional WHILE node
// repeats begin / activate / nominate / cavity / insert / relocate / end
// until k_round_end clears the condition.  Grids are fixed (the kernels loop
// over their items); the candidate scratch is sized for the largest round.
// A round loop that stalls on cavity-scratch overflow is relaunched with
// twice the scratch; the state lives on the device, so it resumes.
template <int D>
static int graph_rounds(dt_ctx* c, TriView<D>& T, EngineRun& run, int64_t npts, int* cnt, const int* loffd,
                        const std::vector<int64_t>& loff, const int* llist, int* nom, int* walk, int* act0, int* act1,
                        int nact, int last_batch, int next_level, int capC, int capB, int min_active,
                        unsigned* round_out, bool* failed) {
  cudaStream_t s = c->stream;
  cudaStream_t cs = capture_stream(c);
  EngCtl* ctl = (EngCtl*)pool_get(c, "eng.ctl", sizeof(EngCtl));
  if (!cs || !ctl) return set_err(c, DT_E_NOMEM, "round graph");
  EngCtl h0;
  memset(&h0, 0, sizeof(h0));
  h0.ain = act0;
  h0.aout = act1;
  h0.next_level = next_level;
  h0.last_batch = last_batch;
  h0.last_nact = nact;
  h0.small_max = c->cfg.small_rounds > 0 ? c->cfg.small_rounds : -1;
  h0.drain = c->cfg.brio_drain > 1 ? c->cfg.brio_drain : 8;
  h0.ratio = c->cfg.active_ratio > 0 ? (float)c->cfg.active_ratio / 100.0f : 0.0f;
  h0.min_active = min_active;
  h0.activated_total = nact;
  h0.round_limit = c->cfg.round_limit > 0 ? c->cfg.round_limit : 400000;
  CUDA_OK(cudaMemcpyAsync(ctl, &h0, sizeof(EngCtl), cudaMemcpyHostToDevice, s));
  const int capCand = (int)std::max<int64_t>(1, std::min<int64_t>(npts, int64_t(1) << 22));
  int64_t max_level = 1;
  for (size_t l = 0; l + 1 < loff.size(); l++) max_level = std::max<int64_t>(max_level, loff[l + 1] - loff[l]);
  const int64_t sms = c->sms, cb = c->cfg.cavity_blocks > 0 ? c->cfg.cavity_blocks : 16;
  const unsigned gn = (unsigned)std::min<int64_t>(ceil_div<int64_t>(npts, 256), sms * 8);
  const unsigned gr = (unsigned)std::min<int64_t>(ceil_div<int64_t>(npts, 128), sms * 16);
  const unsigned ga = (unsigned)std::min<int64_t>(ceil_div<int64_t>(max_level, 128), sms * 16);
  const unsigned gw = (unsigned)std::min<int64_t>(ceil_div<int64_t>((int64_t)capCand * 32, 128), sms * cb);
  EngCtl h1;
  memset(&h1, 0, sizeof(h1));
  for (int grow = 0;; grow++) {
    CandScratch S;
    memset(&S, 0, sizeof(S));
    S.cap = capCand;
    S.capC = capC << grow;
    S.capB = capB << grow;
    S.cand = (int*)pool_get(c, "eng.cand", 4 * (size_t)capCand);
    S.meta = (int4*)pool_get(c, "eng.meta", 16 * (size_t)capCand);
    S.cav = (int*)pool_get(c, "eng.cav", 4 * (size_t)capCand * S.capC);
    S.bnd = (int*)pool_get(c, "eng.bnd", 4 * (size_t)capCand * S.capB);
    S.outer = (int*)pool_get(c, "eng.outer", 4 * (size_t)capCand * S.capB);
    S.count = cnt + 2;
    if (!S.cand || !S.meta || !S.cav || !S.bnd || !S.outer) return set_err(c, DT_E_NOMEM, "candidate scratch");
    { int rcb = big_scratch(c, S, cnt); if (rcb) return rcb; }
    // every parameter baked into the graph: an equal key means an equal graph
    std::string key;
    auto put = [&](const void* p, size_t nb) { key.append((const char*)p, nb); };
    const int dimk = D, pdlk = c->pdl_ok ? 1 : 0, smallk = c->cfg.small_rounds > 0 ? 1 : 0;
    const void* ptrs[9] = {ctl, cnt, loffd, llist, nom, walk, c->status, cs,
                           (const void*)cavity_kernel<D>(c->cfg.cavity_occupancy, c->cfg.cavity_group)};
    const unsigned grids[4] = {gn, gr, ga, gw};
    put(&dimk, 4); put(&pdlk, 4); put(&smallk, 4); put(&T, sizeof(T)); put(&S, sizeof(S)); put(ptrs, sizeof(ptrs));
    put(grids, sizeof(grids)); put(&capCand, 4);
    cudaGraph_t g = nullptr;
    cudaGraphExec_t gx = nullptr;
    size_t cached = c->round_graphs.size();
    for (size_t q = 0; q < c->round_graphs.size(); q++)
      if (c->round_graphs[q].key == key) cached = q;
    cudaError_t e = cudaSuccess;
    if (cached < c->round_graphs.size()) {
      gx = c->round_graphs[cached].gx;
      c->graphs_reused++;
      k_round_begin<<<1, 32, 0, s>>>(ctl, cnt, loffd);
      e = cudaGraphLaunch(gx, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) return set_err(c, gdt_cuda_fail(e, "round graph", __FILE__, __LINE__), "round graph");
      gx = nullptr;
    } else {
    e = cudaGraphCreate(&g, 0);
    cudaGraphConditionalHandle hc = 0;
    if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&hc, g, 1, cudaGraphCondAssignDefault);
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = hc;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t node;
    if (e == cudaSuccess) e = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &cp);
    cudaGraph_t body = e == cudaSuccess ? cp.conditional.phGraph_out[0] : nullptr;
    if (e == cudaSuccess) e = cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      // body: one round; programmatic edges let each launch overlap the kernel before it
      const bool pdl = c->pdl_ok;
      cudaLaunchAttribute at[1];
      at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
      at[0].val.programmaticStreamSerializationAllowed = 1;
      auto cfg = [&](unsigned grid, unsigned block) {
        cudaLaunchConfig_t lc = {};
        lc.gridDim = dim3(grid);
        lc.blockDim = dim3(block);
        lc.stream = cs;
        lc.attrs = pdl ? at : nullptr;
        lc.numAttrs = pdl ? 1 : 0;
        return lc;
      };
      cudaLaunchConfig_t l0 = cfg(1, 1024), l1 = cfg(ga, 128), l2 = cfg(gn, 256), l3 = cfg(gw, 128), l4 = cfg(gw, 128),
                         l5 = cfg(gn, 256), l6 = cfg(gr, 128), l7 = cfg(1, 32), l8 = cfg(big_grid(c->sms), BIG_NT);
      // the body's first node has no kernel before it inside the body; the
      // single-block rounds are a node only when they are enabled
      if (c->cfg.small_rounds > 0) {
        l0.numAttrs = 0;
        cudaLaunchKernelEx(&l0, k_small_rounds<D>, T, ctl, cnt, loffd, (const int*)llist, nom, walk, S);
      } else {
        l1.numAttrs = 0;
      }
      cudaLaunchKernelEx(&l1, k_activate<D>, T, (const int*)llist, 0, (int*)nullptr, cnt + 0, 0u, (const EngCtl*)ctl);
      cudaLaunchKernelEx(&l2, k_nominate<D>, T, (const int*)nullptr, (const int*)(cnt + 0), 0u, nom, cnt + 2, cnt + 8,
                         capCand, (const EngCtl*)ctl);
      cudaLaunchKernelEx(&l3, cavity_kernel<D>(c->cfg.cavity_occupancy, c->cfg.cavity_group), T, (const int*)nom, (const int*)(cnt + 2), 0u, S,
                         (const int*)(cnt + 8),
                         (const EngCtl*)ctl);
      cudaLaunchKernelEx(&l8, k_cavity_big<D>, T, 0u, S, (const EngCtl*)ctl);
      cudaLaunchKernelEx(&l4, k_insert_w<D>, T, 0u, S, (const int*)(cnt + 2), cnt + 3, (const EngCtl*)ctl);
      cudaLaunchKernelEx(&l5, k_reloc_check<D>, T, (const int*)nullptr, (const int*)(cnt + 0), (int*)nullptr, cnt + 1,
                         walk, cnt + 4, 0u, (const EngCtl*)ctl);
      cudaLaunchKernelEx(&l6, k_reloc_walk<D>, T, (const int*)walk, (const int*)(cnt + 4), 0u, (const EngCtl*)ctl);
      cudaLaunchKernelEx(&l7, k_round_step, ctl, cnt, loffd, (const DevStatus*)c->status, hc);
      cudaGraph_t captured = nullptr;
      e = cudaStreamEndCapture(cs, &captured);
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&gx, g, 0);
    if (e != cudaSuccess && c->pdl_ok) {
      // programmatic edges refused inside the loop body: capture again without them
      cudaGetLastError();
      if (gx) cudaGraphExecDestroy(gx);
      if (g) cudaGraphDestroy(g);
      c->pdl_ok = false;
      grow--;
      continue;
    }
    if (e == cudaSuccess) k_round_begin<<<1, 32, 0, s>>>(ctl, cnt, loffd);
    if (e == cudaSuccess) e = cudaGraphLaunch(gx, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) {
      // keep it for later runs with the same parameters (at most 16, oldest out)
      if (c->round_graphs.size() >= 16) {
        cudaGraphExecDestroy(c->round_graphs.front().gx);
        cudaGraphDestroy(c->round_graphs.front().g);
        c->round_graphs.erase(c->round_graphs.begin());
      }
      c->round_graphs.push_back({key, g, gx});
      c->graphs_built++;
      g = nullptr;
      gx = nullptr;
    }
    if (gx) cudaGraphExecDestroy(gx);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess) return set_err(c, gdt_cuda_fail(e, "round graph", __FILE__, __LINE__), "round graph");
    }
    const unsigned r0 = h1.round;
    CUDA_OK(cudaMemcpyAsync(&h1, ctl, sizeof(EngCtl), cudaMemcpyDeviceToHost, s));
    CUDA_OK(cudaMemcpyAsync(c->status_host, c->status, sizeof(DevStatus), cudaMemcpyDeviceToHost, s));
    CUDA_OK(cudaStreamSynchronize(s));
    c->launches += 1 + (c->cfg.small_rounds > 0 ? 9 : 8) * (int64_t)(h1.round - r0 + 1);   // body nodes per round
    if (h1.done == 3 && c->status_host->overflow_cav && grow < 8) {
      // cavities outgrew their scratch: twice the room, same state
      CUDA_OK(cudaMemsetAsync(&c->status->overflow_cav, 0, 4, s));
      EngCtl h2 = h1;
      h2.done = 0;
      h2.stalled = 0;
      CUDA_OK(cudaMemcpyAsync(ctl, &h2, sizeof(EngCtl), cudaMemcpyHostToDevice, s));
      CUDA_OK(cudaStreamSynchronize(s));
      continue;
    }
    break;
  }
  *round_out = h1.round;
  if (h1.done == 1) return 0;
  if (h1.done == 2) {
    if (c->status_host->error == DT_E_OVERFLOW && c->status_host->detail == 1) { *failed = true; return 0; }
    return check_status(c, "insertion round");
  }
  if (h1.done == 4) return set_err(c, DT_E_TIMEOUT, "insertion rounds exceeded");
  return set_err(c, DT_E_INTERNAL, "insertion rounds made no progress");
}

template <int D>
static int engine_run_t(dt_ctx* c, EngineRun& run, const void* pts, const int* gid, const int* pinst,
                        int64_t npts, const std::vector<int64_t>& poff, const std::string& tag) {
  using P = typename PT<D>::T;
  cudaStream_t s = c->stream;
  int ninst = (int)poff.size() - 1;
  run.dim = D;
  run.ninst = ninst;
  run.npts = npts;
  run.h_poff = poff;
  run.rounds = 0;
  // arena: per instance mult * n_i + pad slots
  const int64_t mult = c->cfg.arena_factor > 0 ? c->cfg.arena_factor : (D == 2 ? 8 : 36), pad = 32;
  int64_t grow = 1;
  for (int attempt = 0; attempt < 4; attempt++) {
    run.h_toff.assign(ninst + 1, 0);
    for (int i = 0; i < ninst; i++)
      run.h_toff[i + 1] = run.h_toff[i] + grow * (mult * (poff[i + 1] - poff[i]) + pad);
    int64_t total = run.h_toff[ninst];
    if (total >= (int64_t(1) << 29)) return set_err(c, DT_E_NOMEM, "simplex arena exceeds 2^29 slots");
    run.total_slots = total;
    unsigned long long calls0; int range0;
    { int rc0 = pred_counters_local(c, &calls0, &range0, false); if (rc0) return rc0; }
    run.tv = pool_get(c, tag + ".tv", sizeof(int4) * total);
    run.tn = pool_get(c, tag + ".tn", sizeof(int4) * total);
    auto* claimA = (unsigned long long*)pool_get(c, tag + ".cA", 8 * total);
    auto* claimC = (unsigned long long*)pool_get(c, tag + ".cC", 8 * total);
    run.tcount = (int*)pool_get(c, tag + ".tcount", 4 * (ninst + 1));
    run.toff = (int*)pool_get(c, tag + ".toff", 4 * (ninst + 1));
    run.tend = (int*)pool_get(c, tag + ".tend", 4 * (ninst + 1));
    run.inst_status = (int*)pool_get(c, tag + ".ist", 4 * (ninst + 1));
    long long* dpoff = (long long*)pool_get(c, tag + ".poff", 8 * (ninst + 1));
    int* loc = (int*)pool_get(c, tag + ".loc", 4 * std::max<int64_t>(npts, 1));
    unsigned char* state = (unsigned char*)pool_get(c, tag + ".state", std::max<int64_t>(npts, 1));
    int* act0 = (int*)pool_get(c, "eng.act0", 4 * std::max<int64_t>(npts, 1));
    int* act1 = (int*)pool_get(c, "eng.act1", 4 * std::max<int64_t>(npts, 1));
    int* cnt = (int*)pool_get(c, "eng.cnt", 64);
    if (!run.tv || !run.tn || !claimA || !claimC || !run.tcount || !run.toff || !run.tend ||
        !run.inst_status || !dpoff || !loc || !state || !act0 || !act1 || !cnt)
      return set_err(c, DT_E_NOMEM, "engine buffers");
    std::vector<int> h_toff32(ninst + 1), h_tend(ninst + 1);
    for (int i = 0; i <= ninst; i++) h_toff32[i] = (int)run.h_toff[i];
    for (int i = 0; i < ninst; i++) h_tend[i] = (int)run.h_toff[i + 1];
    std::vector<long long> h_poff(poff.begin(), poff.end());
    CUDA_OK(cudaMemcpyAsync(run.toff, h_toff32.data(), 4 * (ninst + 1), cudaMemcpyHostToDevice, s));
    CUDA_OK(cudaMemcpyAsync(run.tend, h_tend.data(), 4 * (ninst + 1), cudaMemcpyHostToDevice, s));
    CUDA_OK(cudaMemcpyAsync(dpoff, h_poff.data(), 8 * (ninst + 1), cudaMemcpyHostToDevice, s));
    CUDA_OK(cudaMemsetAsync(claimA, 0, 8 * total, s));
    CUDA_OK(cudaMemsetAsync(claimC, 0, 8 * total, s));
    CUDA_OK(cudaMemsetAsync(state, 0, std::max<int64_t>(npts, 1), s));
    CUDA_OK(cudaMemsetAsync(cnt, 0, 64, s));
    CUDA_OK(cudaMemsetAsync(c->status, 0, sizeof(DevStatus), s));

    TriView<D> T;
    memset(&T, 0, sizeof(T));   // padding too: the round-graph cache compares the bytes
    T.pts = (const P*)pts;
    T.gid = gid;
    T.pinst = pinst;
    T.tv = (int4*)run.tv;
    T.tn = (int4*)run.tn;
    T.claimA = claimA;
    T.claimC = claimC;
    T.tcount = run.tcount;
    T.tend = run.tend;
    T.loc = loc;
    T.state = state;
    T.st = c->status;
    T.nslots = (int)total;
    T.npts = (int)npts;
    T.prof = nullptr;
    T.dbg = nullptr;
    T.rings = c->cfg.nominate_rings > 1 ? 2 : 1;
    T.walk_limit = c->cfg.walk_limit > 0 ? c->cfg.walk_limit : (1 << 16);
    if (getenv("GDT_DEBUG")) {
      T.dbg = (unsigned long long*)pool_get(c, "eng.dbg", 64);
      if (!T.dbg) return set_err(c, DT_E_NOMEM, "debug counters");
      CUDA_OK(cudaMemsetAsync(T.dbg, 0, 64, s));
    }
    unsigned long long* profc = nullptr;
    if (c->cfg.profile) {
      profc = (unsigned long long*)pool_get(c, "eng.prof", 64);
      if (!profc) return set_err(c, DT_E_NOMEM, "profile counters");
      CUDA_OK(cudaMemsetAsync(profc, 0, 64, s));
      T.prof = profc;
    }

    // per-instance bounding boxes: origins and error bounds of the FP32
    // predicate stage, and the hint grids
    std::vector<unsigned long long> hu;
    float4* xs = nullptr;
    { int rc0 = fp32_points(c, D, pts, pinst, npts, ninst, "eng.xs", &xs, &hu); if (rc0) return rc0; }
    T.xs = xs;
    k_init<D><<<ceil_div(ninst, 64), 64, (++c->launches, 0), s>>>(T, ninst, dpoff, run.toff, run.inst_status);
    T.toff = run.toff;
    T.ninst = ninst;
    T.hint = nullptr;
    if (npts > 0 && !getenv("GDT_NOHINT")) {
      // grids of about n_i / 4 cells
      double* glo = (double*)pool_get(c, tag + ".glo", 8 * 6 * (size_t)ninst);
      int* gdim = (int*)pool_get(c, tag + ".gdim", 4 * 5 * (size_t)ninst);
      if (!glo || !gdim) return set_err(c, DT_E_NOMEM, "hint grids");
      std::vector<double> hg(6 * (size_t)ninst, 0.0);
      std::vector<int> hd(5 * (size_t)ninst, 1);
      int64_t cells = 0, cells2 = 0;
      for (int i = 0; i < ninst; i++) {
        int64_t ni = poff[i + 1] - poff[i];
        double lo[3], ext[3], vol = 1.0;
        int nd = 0;
        for (int cc = 0; cc < D; cc++) {
          lo[cc] = host_from_orderable(hu[6 * i + cc]);
          double hi = host_from_orderable(hu[6 * i + 3 + cc]);
          ext[cc] = (ni > 0 && hi > lo[cc]) ? hi - lo[cc] : 0.0;
          if (ext[cc] > 0) { vol *= ext[cc]; nd++; }
        }
        double target = std::max<double>(1.0, (double)ni / 4.0);
        double side = nd ? std::pow(vol / target, 1.0 / nd) : 1.0;
        int64_t ci = 1, ci2 = 1;
        for (int cc = 0; cc < 3; cc++) {
          int d = 1;
          if (cc < D && ext[cc] > 0 && side > 0) d = (int)std::min(1024.0, std::max(1.0, std::ceil(ext[cc] / side)));
          hd[5 * i + cc] = d;
          hg[6 * i + cc] = cc < D && ni > 0 ? lo[cc] : 0.0;
          hg[6 * i + 3 + cc] = (cc < D && ext[cc] > 0) ? d / ext[cc] : 0.0;
          ci *= d;
          ci2 *= (d + 3) >> 2;
        }
        hd[5 * i + 3] = (int)cells;
        hd[5 * i + 4] = (int)cells2;
        cells += ci;
        cells2 += ci2;
      }
      int* hint = (int*)pool_get(c, tag + ".hint", 4 * std::max<int64_t>(cells, 1));
      int* hint2 = (int*)pool_get(c, tag + ".hint2", 4 * std::max<int64_t>(cells2, 1));
      if (!hint || !hint2) return set_err(c, DT_E_NOMEM, "hint cells");
      CUDA_OK(cudaMemsetAsync(hint, 0xff, 4 * std::max<int64_t>(cells, 1), s));
      CUDA_OK(cudaMemsetAsync(hint2, 0xff, 4 * std::max<int64_t>(cells2, 1), s));
      CUDA_OK(cudaMemcpyAsync(glo, hg.data(), 8 * 6 * (size_t)ninst, cudaMemcpyHostToDevice, s));
      CUDA_OK(cudaMemcpyAsync(gdim, hd.data(), 4 * 5 * (size_t)ninst, cudaMemcpyHostToDevice, s));
      CUDA_OK(cudaStreamSynchronize(s));   // host vectors go out of scope
      T.hint = hint;
      T.hint2 = hint2;
      T.glo = glo;
      T.gdim = gdim;
    }
    // activation levels and the per-level lists of dormant points
    int* level = (int*)pool_get(c, tag + ".level", 4 * std::max<int64_t>(npts, 1));
    int* lrank = (int*)pool_get(c, "eng.lrank", 4 * std::max<int64_t>(npts, 1));
    int* lsize = (int*)pool_get(c, "eng.lsize", 4 * (NLEV + 1));
    int* llist = (int*)pool_get(c, tag + ".llist", 4 * std::max<int64_t>(npts, 1));
    int* loffd = (int*)pool_get(c, "eng.loff", 4 * (NLEV + 1));
    if (!level || !lrank || !lsize || !llist || !loffd) return set_err(c, DT_E_NOMEM, "activation levels");
    std::vector<int64_t> loff(NLEV + 1, 0);
    int first_level = 0;
    if (npts > 0) {
      unsigned gpp = (unsigned)ceil_div<int64_t>(npts, 256);
      const double growth = c->cfg.brio_growth > 100 ? c->cfg.brio_growth / 100.0 : 1.5;
      k_levels<D><<<gpp, 256, (++c->launches, 0), s>>>(T, npts, run.inst_status, level,
                                                       (float)(1.0 / std::log2(growth)));
      int rc = group_rank(c, level, npts, lrank, lsize, NLEV);
      if (rc) return rc;
      int hs[NLEV];
      CUDA_OK(cudaMemcpyAsync(hs, lsize, 4 * NLEV, cudaMemcpyDeviceToHost, s));
      CUDA_OK(cudaStreamSynchronize(s));
      for (int l = 0; l < NLEV; l++) loff[l + 1] = loff[l] + hs[l];
      std::vector<int> lo32(NLEV + 1);
      for (int l = 0; l <= NLEV; l++) lo32[l] = (int)loff[l];
      CUDA_OK(cudaMemcpyAsync(loffd, lo32.data(), 4 * (NLEV + 1), cudaMemcpyHostToDevice, s));
      k_scatter_levels<<<gpp, 256, (++c->launches, 0), s>>>(level, lrank, loffd, npts, llist);
      // the first batch: about first_batch points per instance
      const int fb = c->cfg.first_batch > 0 ? c->cfg.first_batch : 32;
      int64_t want = (int64_t)fb * ninst;
      first_level = NLEV - 1;
      while (first_level > 0 && loff[NLEV] - loff[first_level] < want) first_level--;
      if (getenv("GDT_NOBRIO")) first_level = 0;
      k_locate_init<D><<<gpp, 256, (++c->launches, 0), s>>>(T, npts, run.toff, run.inst_status, level, first_level,
                                                            act0, cnt);
    }
    int next_level = first_level - 1;    // next batch to activate (levels below are later)
    // continuous activation keeps at least about first_batch points per instance active
    const int min_active = (c->cfg.first_batch > 0 ? c->cfg.first_batch : 32) * std::max(ninst, 1);
    const int round_limit = c->cfg.round_limit > 0 ? c->cfg.round_limit : 400000;
    int* h = c->counters_host;
    CUDA_OK(cudaMemcpyAsync(h, cnt, 4, cudaMemcpyDeviceToHost, s));
    CUDA_OK(cudaStreamSynchronize(s));
    int nact = h[0];            // an upper bound between synchronisations
    int last_batch = nact;
    // candidate scratch
    int capC = D == 2 ? 32 : 96, capB = D == 2 ? 48 : 192;
    if (c->cfg.cavity_cap > 0) {
      capC = c->cfg.cavity_cap;
      capB = D == 2 ? c->cfg.cavity_cap * 3 / 2 : c->cfg.cavity_cap * 2;
    }
    int* nom = (int*)pool_get(c, "eng.nom", 4 * (size_t)NBUCKET * std::max<int64_t>(std::min<int64_t>(npts, int64_t(1) << 22), 1));
    int* walk = (int*)pool_get(c, "eng.walk", 4 * std::max<int64_t>(npts, 1));
    if (!nom || !walk) return set_err(c, DT_E_NOMEM, "nominee lists");
    // device counters: [0] active, [1] next active, [2] nominees, [3] winners, [4] walkers
    int overflow_grow = 0;
    bool failed = false;
    int* ain = act0;
    int* aout = act1;
    unsigned round = 0;
    int last_sync_nact = nact;
    const bool prof = c->cfg.profile != 0;
    const int SYNC_EVERY = 4;
    // profile records: (start event, end event, kernel)
    struct ProfRec { int a, b, k; unsigned r; };
    std::vector<ProfRec> recs;
    size_t nev = 0;
    auto mark = [&]() -> int {
      if (!prof) return -1;
      cudaEvent_t e = prof_event(c, nev);
      if (!e) return -1;
      cudaEventRecord(e, s);
      return (int)nev++;
    };
    static const char* const knames[2][7] = {
        {"k_nominate<2>", "k_cavity_w<2>", "k_insert_w<2>", "k_reloc_check<2>", "k_reloc_walk<2>", "k_activate<2>",
         "k_cavity_big<2>"},
        {"k_nominate<3>", "k_cavity_w<3>", "k_insert_w<3>", "k_reloc_check<3>", "k_reloc_walk<3>", "k_activate<3>",
         "k_cavity_big<3>"}};
    // Profile and debug runs drive the rounds from the host (events and
    // checks between launches); otherwise one CUDA graph runs every round.
    const bool host_loop = prof || getenv("GDT_DEBUG") || getenv("GDT_CHECK");
    const int drain = c->cfg.brio_drain > 1 ? c->cfg.brio_drain : 8;
    if (nact > 0)
      k_pick<D><<<(unsigned)ceil_div(nact, 256), 256, (++c->launches, 0), s>>>(T, ain, nact, 1);
    if (!host_loop && (nact > 0 || next_level >= 0)) {
      int rc = graph_rounds<D>(c, T, run, npts, cnt, loffd, loff, llist, nom, walk, act0, act1, nact, last_batch,
                               next_level, capC, capB, min_active, &round, &failed);
      if (rc) return rc;
      nact = 0;
      next_level = -1;
    }
    // the activation rules of the device loop (round_begin); with continuous
    // activation the host reads the active count after every round
    const float ratio = c->cfg.active_ratio > 0 ? (float)c->cfg.active_ratio / 100.0f : 0.0f;
    long long activated = nact;
    auto wants = [&]() {
      if (ratio <= 0.0f) return nact <= last_batch / drain;
      const long long inserted = activated - nact;
      return (long long)nact < std::max<long long>(min_active, (long long)(ratio * (float)inserted));
    };
    while (nact > 0 || next_level >= 0) {
      while (next_level >= 0 && wants()) {
        int m = (int)(loff[next_level + 1] - loff[next_level]);
        if (m > 0) {
          const int a0 = mark();
          k_activate<D><<<(unsigned)ceil_div(m, 128), 128, (++c->launches, 0), s>>>(
              T, llist + loff[next_level], m, ain, cnt + 0, round + 1, nullptr);
          const int a1 = mark();
          if (a0 >= 0 && a1 >= 0) recs.push_back({a0, a1, 5, round + 1});
          nact += m;
          activated += m;
          last_batch = nact;
          last_sync_nact = -1;         // activation changes the count: skip one progress check
        }
        next_level--;
      }
      if (nact <= 0) break;
      round++;
      if (round > (unsigned)round_limit) return set_err(c, DT_E_TIMEOUT, "insertion rounds exceeded");
      int capCand = (int)std::min<int64_t>(nact, int64_t(1) << 22);
      CandScratch S;
      S.cap = capCand;
      S.capC = capC << overflow_grow;
      S.capB = capB << overflow_grow;
      S.cand = (int*)pool_get(c, "eng.cand", 4 * (size_t)capCand);
      S.meta = (int4*)pool_get(c, "eng.meta", 16 * (size_t)capCand);
      S.cav = (int*)pool_get(c, "eng.cav", 4 * (size_t)capCand * S.capC);
      S.bnd = (int*)pool_get(c, "eng.bnd", 4 * (size_t)capCand * S.capB);
      S.outer = (int*)pool_get(c, "eng.outer", 4 * (size_t)capCand * S.capB);
      S.count = cnt + 2;
      if (!S.cand || !S.meta || !S.cav || !S.bnd || !S.outer) return set_err(c, DT_E_NOMEM, "candidate scratch");
      { int rcb = big_scratch(c, S, cnt); if (rcb) return rcb; }
      CUDA_OK(cudaMemsetAsync(cnt + 1, 0, 20, s));
      CUDA_OK(cudaMemsetAsync(cnt + 8, 0, 4 * NBUCKET, s));
      unsigned gp = (unsigned)ceil_div(nact, 256);
      unsigned gw = (unsigned)std::min<int64_t>(ceil_div<int64_t>((int64_t)capCand * 32, 128),
                                                (int64_t)c->sms * (c->cfg.cavity_blocks > 0 ? c->cfg.cavity_blocks : 16));
      int ev[6];
      ev[0] = mark();
      k_nominate<D><<<gp, 256, (++c->launches, 0), s>>>(T, ain, cnt + 0, round, nom, cnt + 2, cnt + 8, capCand,
                                                        nullptr);
      ev[1] = mark();
      cavity_kernel<D>(c->cfg.cavity_occupancy, c->cfg.cavity_group)<<<gw, 128, (++c->launches, 0), s>>>(T, nom, cnt + 2, round, S, cnt + 8,
                                                                                   nullptr);
      const int evb = mark();
      k_cavity_big<D><<<big_grid(c->sms), BIG_NT, (++c->launches, 0), s>>>(T, round, S, nullptr);
      ev[2] = mark();
      k_insert_w<D><<<gw, 128, (++c->launches, 0), s>>>(T, round, S, cnt + 2, cnt + 3, nullptr);
      ev[3] = mark();
      k_reloc_check<D><<<gp, 256, (++c->launches, 0), s>>>(T, ain, cnt + 0, aout, cnt + 1, walk, cnt + 4, round + 1,
                                                           nullptr);
      ev[4] = mark();
      k_reloc_walk<D><<<(unsigned)ceil_div(nact, 128), 128, (++c->launches, 0), s>>>(T, walk, cnt + 4, round + 1,
                                                                                      nullptr);
      ev[5] = mark();
      for (int q = 0; q < 5; q++)
        if (ev[q] >= 0 && ev[q + 1] >= 0) {
          if (q == 1 && evb >= 0) {                    // region growth, then the large regions
            recs.push_back({ev[1], evb, 1, round});
            recs.push_back({evb, ev[2], 6, round});
          } else {
            recs.push_back({ev[q], ev[q + 1], q, round});
          }
        }
      if (getenv("GDT_DEBUG")) {
        int hc[5];
        unsigned long long hd[8];
        cudaMemcpyAsync(hc, cnt, 20, cudaMemcpyDeviceToHost, s);
        cudaMemcpyAsync(hd, T.dbg, 64, cudaMemcpyDeviceToHost, s);
        cudaMemsetAsync(T.dbg, 0, 64, s);
        cudaStreamSynchronize(s);
        fprintf(stderr,
                "round %u nact %d cand %d win %d walk %d steps %llu max %llu act_steps %llu act_max %llu "
                "complete %llu grown %llu large %llu grow_steps %llu\n",
                round, hc[0], hc[2], hc[3], hc[4], hd[0], hd[1], hd[2], hd[3], hd[4], hd[5], hd[6], hd[7]);
      }
      k_move_count<<<1, 1, (++c->launches, 0), s>>>(cnt + 0, cnt + 1);
      std::swap(ain, aout);
      const bool check = getenv("GDT_CHECK") != nullptr;
      if (check)
        k_check_mesh<D><<<(unsigned)ceil_div<int64_t>(total, 256), 256, (++c->launches, 0), s>>>(
            T, run.toff, run.tcount, ninst, round);
      if (round % SYNC_EVERY != 0 && nact > 4096 && !check && ratio <= 0.0f) continue;
      CUDA_OK(cudaMemcpyAsync(h, cnt + 0, 4, cudaMemcpyDeviceToHost, s));
      CUDA_OK(cudaMemcpyAsync(c->status_host, c->status, sizeof(DevStatus), cudaMemcpyDeviceToHost, s));
      CUDA_OK(cudaStreamSynchronize(s));
      if (c->status_host->error == DT_E_OVERFLOW && c->status_host->detail == 1) { failed = true; break; }
      if (c->status_host->error) return check_status(c, "insertion round");
      int nnew = h[0];
      if (nnew == last_sync_nact && nnew > 0) {
        // no insertion since the last check: only possible when nominees overflowed their scratch
        if (c->status_host->overflow_cav && overflow_grow < 8) {
          overflow_grow++;
          CUDA_OK(cudaMemsetAsync(&c->status->overflow_cav, 0, 4, s));
        } else {
          return set_err(c, DT_E_INTERNAL, "insertion rounds made no progress");
        }
      }
      nact = nnew;
      last_sync_nact = nnew;
    }
    if (c->status_host->error == 0) {
      CUDA_OK(cudaMemcpyAsync(c->status_host, c->status, sizeof(DevStatus), cudaMemcpyDeviceToHost, s));
      CUDA_OK(cudaStreamSynchronize(s));
      if (c->status_host->error) return check_status(c, "activation");
    }
    run.rounds = (int)round;
    if (failed) { grow *= 2; continue; }
    if (prof && !recs.empty()) {
      CUDA_OK(cudaStreamSynchronize(s));
      const bool roundlog = getenv("GDT_ROUNDLOG") != nullptr;   // per-round kernel times on stderr
      for (const ProfRec& r : recs) {
        float ms = 0;
        cudaEventElapsedTime(&ms, c->evpool[r.a], c->evpool[r.b]);
        prof_add(c, knames[D - 2][r.k], ms, 0, 0);
        if (roundlog) fprintf(stderr, "rt %s %u %d %.4f\n", tag.c_str(), r.r, r.k, ms);
      }
    }
    if (profc) {
      unsigned long long hp[2];
      CUDA_OK(cudaMemcpyAsync(hp, profc, 16, cudaMemcpyDeviceToHost, s));
      CUDA_OK(cudaStreamSynchronize(s));
      // FP32 insphere stage: about 220 operations in 3D (determinant and both permanents), 70 in 2D
      prof_add(c, D == 2 ? "k_cavity_w<2>" : "k_cavity_w<3>", 0, (double)hp[0], (double)hp[1] * (D == 2 ? 70 : 220));
      unsigned long long hr[2] = {0, 0};
      CUDA_OK(cudaMemcpyAsync(hr, profc + 2, 16, cudaMemcpyDeviceToHost, s));
      CUDA_OK(cudaStreamSynchronize(s));
      prof_add(c, D == 2 ? "k_reloc_walk<2>" : "k_reloc_walk<3>", 0, (double)hr[0], 0);
      prof_add(c, D == 2 ? "k_reloc_check<2>" : "k_reloc_check<3>", 0, (double)hr[1], 0);
    }
    run.h_status.assign(ninst, 0);
    run.h_tcount.assign(ninst, 0);
    CUDA_OK(cudaMemcpyAsync(run.h_status.data(), run.inst_status, 4 * ninst, cudaMemcpyDeviceToHost, s));
    CUDA_OK(cudaMemcpyAsync(run.h_tcount.data(), run.tcount, 4 * ninst, cudaMemcpyDeviceToHost, s));
    CUDA_OK(cudaStreamSynchronize(s));
    unsigned long long calls; int range;
    int rc = pred_counters_local(c, &calls, &range, false);
    if (rc) return rc;
    if (range != range0) return set_err(c, DT_E_RANGE, "coordinate range too wide for the exact fallback");
    return 0;
  }
  return set_err(c, DT_E_OVERFLOW, "simplex arena overflow after retries");
}


// ---------------------------------------------------------------- continuous batching
// The stream engine (stream.cuh): the same round kernels over the resident
// instances, with an activation schedule per instance and a round loop that
// yields to the host when an instance has finished or jobs are waiting.

// Activation plan of the next round, one thread per instance (the whole CTA
// calls it): every running instance activates its next level(s) once its
// active set has drained to last_batch / drain; seg[0..J) receives each
// instance's range start in llist, seg[J..2J] the exclusive prefix of the
// range lengths.
static __device__ void stream_plan(EngCtl& C, SlotState* ss, int J, int* seg, int* cnt, int drain) {
  __shared__ int s_len[STREAM_MAX_JOBS];
  for (int t = threadIdx.x; t < J; t += blockDim.x) {
    SlotState& q = ss[t];
    int len = 0, lo = -1, hi = -1;
    if (q.status == 1) {
      int nact = q.nact;
      while (q.next_level >= 0 && nact <= q.last_batch / drain) {
        const int l = q.next_level;
        const int m = q.loff[l + 1] - q.loff[l];
        if (m > 0) {
          if (hi < 0) hi = q.loff[l + 1];
          lo = q.loff[l];
          nact += m;
          q.last_batch = nact;
        }
        q.next_level--;
      }
      q.nact = nact;
      if (lo >= 0) len = hi - lo;
    }
    seg[t] = lo;
    s_len[t] = len;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int run = 0;
    for (int t = 0; t < J; t++) { seg[J + t] = run; run += s_len[t]; }
    seg[2 * J] = run;
    C.act_lo = 0;
    C.act_n = run;
    C.activated = run;
    if (cnt[0] + run > 0) C.round++;
    cnt[1] = cnt[2] = cnt[3] = cnt[4] = cnt[5] = 0;
    for (int b = 0; b < NBUCKET; b++) cnt[8 + b] = 0;
  }
  __syncthreads();
}

static __global__ void k_stream_begin(EngCtl* ctl, SlotState* ss, int J, int* seg, int* cnt, int drain) {
  stream_plan(*ctl, ss, J, seg, cnt, drain);
}

// End of a round: per-instance survivors, finished instances, the yield
// decision, then the plan of the next round.
static __global__ void k_stream_step(EngCtl* ctl, SlotState* ss, int J, int* seg, int* cnt, int* kept,
                                     const DevStatus* st, const volatile int* admit, int drain,
                                     cudaGraphConditionalHandle handle) {
  pdl_enter();
  __shared__ int s_fin, s_live;
  EngCtl& C = *ctl;
  if (threadIdx.x == 0) {
    s_fin = 0;
    s_live = 0;
    const int had = cnt[0];
    const int nnew = cnt[1];
    cnt[0] = nnew;
    cnt[1] = 0;
    int* t = C.ain;
    C.ain = C.aout;
    C.aout = t;
    if (C.done == 0) {
      if (st->error) C.done = 2;
      else if (had > 0 && cnt[3] == 0 && ++C.stalled >= 4) C.done = 3;
      else if (cnt[3] > 0) C.stalled = 0;
    }
    C.last_nact = nnew;
  }
  __syncthreads();
  for (int t = threadIdx.x; t < J; t += blockDim.x) {
    SlotState& q = ss[t];
    if (q.status == 1) {
      q.nact = kept[t];
      if (q.nact == 0 && q.next_level < 0) {
        q.status = 2;
        atomicAdd(&s_fin, 1);
      } else {
        atomicAdd(&s_live, 1);
      }
    }
    kept[t] = 0;
  }
  __syncthreads();
  if (threadIdx.x == 0 && C.done == 0) {
    if (s_fin > 0 || *admit) C.done = 5;        // yield: extract / admit at this round boundary
    else if (s_live == 0) C.done = 1;
  }
  __syncthreads();
  if (C.done == 0) stream_plan(C, ss, J, seg, cnt, drain);
  if (threadIdx.x == 0) cudaGraphSetConditional(handle, C.done == 0 ? 1u : 0u);
}

// Activation over the per-instance ranges of the plan.
template <int D>
__global__ void __launch_bounds__(128, 8) k_stream_activate(TriView<D> T, const int* llist, const int* seg, int J,
                                                         int* nact, const EngCtl* ctl) {
  pdl_enter();
  if (ctl->done) return;
  const int m = ctl->act_n;
  int* act = ctl->ain;
  const unsigned next_round = ctl->round;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < m;
       base += (int64_t)gridDim.x * blockDim.x) {
    const int64_t idx = base + (threadIdx.x & 31);
    bool ok = false;
    int p = -1;
    if (idx < m) {
      int lo = 0, hi = J - 1;                   // the last instance whose range starts at or before idx
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (seg[J + mid] <= idx) lo = mid; else hi = mid - 1;
      }
      p = llist[seg[lo] + (int)(idx - seg[J + lo])];
      ok = activate_point(T, p, next_round);
    }
    warp_append(act, nact, ok, p);
  }
}

// Points of a newly admitted instance: every point waits on the initial
// simplex; those of the first levels are located in it, pick for
// next_round and join the active list.
template <int D>
__global__ void k_stream_locate(TriView<D> T, int slot, int64_t p0, int64_t n, const int* level, int first_level,
                                int* act, int* nact, SlotState* ss, unsigned next_round) {
  const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  bool active = false;
  const int p = (int)(p0 + q);
  if (q < n && T.state[p] == 0) {
    const int s0 = T.toff[slot];
    T.loc[p] = s0;
    if (level[p] >= first_level) {
      const int4 vv = T.tv[s0];
      int loc = s0;
      for (int j = 0; j <= D; j++) {
        int4 t = vv;
        set4(t, j, p);
        if (orient_tuple(T, t) < 0) { loc = nb_simplex(get4(T.tn[s0], j)); break; }
      }
      T.loc[p] = loc;
      atomicMax(&T.claimC[loc], mkkey(next_round, p));
      active = true;
      atomicAdd(&ss[slot].nact, 1);
      atomicAdd(&ss[slot].last_batch, 1);
    }
  }
  warp_append(act, nact, active, p);
}

// The level lists of an admitted instance: point p0 + q goes to its level's
// range at its rank there.
static __global__ void k_stream_scatter_levels(const int* level, const int* rank, const SlotState* ss, int slot, int64_t p0,
                                        int64_t n, int* llist) {
  const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (q >= n) return;
  const int l = level[p0 + q];
  if (l >= 0) llist[ss[slot].loff[l] + rank[p0 + q]] = (int)(p0 + q);
}

static __global__ void k_stream_fill(int* a, int64_t n, int v) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) a[i] = v;
}

static __global__ void k_stream_iota(int* a, int64_t n) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) a[i] = (int)i;
}

static __device__ __forceinline__ void cswap(int& a, int& b) {
  if (b < a) { const int t = a; a = b; b = t; }
}

// Finite live simplices of one instance's arena range as rows of local
// indices, each sorted.
template <int D>
__global__ void k_stream_rows(const int4* tv, int a, int b, const int* gid, int4* rows, int* nrows) {
  const int s = a + blockIdx.x * blockDim.x + threadIdx.x;
  bool take = false;
  int4 r = make_int4(0, 0, 0, 0);
  if (s < b) {
    const int4 v = tv[s];
    if (v.x >= 0 && v.y >= 0 && v.z >= 0 && (D == 2 || v.w >= 0)) {
      take = true;
      int x = gid[v.x], y = gid[v.y], z = gid[v.z], w = D == 3 ? gid[v.w] : 0x7fffffff;
      cswap(x, y); cswap(z, w); cswap(x, z); cswap(y, w); cswap(y, z);   // a sorting network (w = max for 2D)
      r = make_int4(x, y, z, w);
    }
  }
  const unsigned mask = __ballot_sync(0xffffffffu, take);
  if (!mask) return;
  const int lane = threadIdx.x & 31, leader = __ffs(mask) - 1;
  int base = 0;
  if (lane == leader) base = atomicAdd(nrows, __popc(mask));
  base = __shfl_sync(0xffffffffu, base, leader);
  if (take) rows[base + __popc(mask & ((1u << lane) - 1))] = r;
}

template <int D>
static TriView<D> stream_view(dt_ctx* c, StreamState& st) {
  TriView<D> T;
  memset(&T, 0, sizeof(T));
  T.pts = (const typename PT<D>::T*)st.pts;
  T.xs = st.xs;
  T.gid = st.gid;
  T.pinst = st.pinst;
  T.tv = st.tv;
  T.tn = st.tn;
  T.claimA = st.claimA;
  T.claimC = st.claimC;
  T.tcount = st.tcount;
  T.tend = st.tend;
  T.loc = st.loc;
  T.state = st.state;
  T.st = c->status;
  T.nslots = (int)(st.arena_factor * st.cap + 64);
  T.npts = (int)st.cap;
  T.hint = st.hint;
  T.hint2 = st.hint2;
  T.glo = st.glo;
  T.gdim = st.gdim;
  T.toff = st.toff;
  T.ninst = st.max_jobs;
  T.rings = c->cfg.nominate_rings > 1 ? 2 : 1;
  T.walk_limit = c->cfg.walk_limit > 0 ? c->cfg.walk_limit : (1 << 16);
  T.inst_kept = st.kept;
  return T;
}

// Allocates the stream's device buffers for st.cap points and st.max_jobs
// instances (held until the stream closes) and resets its round state.
template <int D>
static int stream_setup_t(dt_ctx* c, StreamState& st) {
  cudaStream_t s = c->stream;
  const int64_t cap = st.cap, J = st.max_jobs, A = st.arena_factor * cap + 64;
  bool ok = true;
  auto get = [&](size_t bytes) -> void* {
    void* p = nullptr;
    if (!ok || cudaMalloc(&p, std::max<size_t>(bytes, 16)) != cudaSuccess) { cudaGetLastError(); ok = false; return nullptr; }
    st.owned.push_back(p);
    st.bytes += std::max<size_t>(bytes, 16);
    return p;
  };
  if (!st.pts) {                       // first call: allocate; later calls only reset
  st.pts = get(sizeof(typename PT<D>::T) * cap);
  st.gid = (int*)get(4 * cap); st.pinst = (int*)get(4 * cap); st.loc = (int*)get(4 * cap);
  st.level = (int*)get(4 * cap); st.lrank = (int*)get(4 * cap); st.lsize = (int*)get(4 * (STREAM_NLEV + 1));
  st.state = (unsigned char*)get(cap); st.xs = (float4*)get(16 * cap);
  st.llist = (int*)get(4 * cap); st.act0 = (int*)get(4 * cap); st.act1 = (int*)get(4 * cap); st.walk = (int*)get(4 * cap);
  st.nom = (int*)get(4 * (size_t)NBUCKET * st.cap_cand);
  st.tv = (int4*)get(16 * A); st.tn = (int4*)get(16 * A);
  st.claimA = (unsigned long long*)get(8 * A); st.claimC = (unsigned long long*)get(8 * A);
  st.toff = (int*)get(4 * J); st.tend = (int*)get(4 * J); st.tcount = (int*)get(4 * J); st.inst_status = (int*)get(4 * J);
  st.xo = (double*)get(8 * 4 * J); st.glo = (double*)get(8 * 6 * J); st.gdim = (int*)get(4 * 5 * J);
  st.hint = (int*)get(4 * cap); st.hint2 = (int*)get(4 * cap);
  st.ss = (SlotState*)get(sizeof(SlotState) * J); st.seg = (int*)get(4 * (2 * J + 1)); st.kept = (int*)get(4 * J);
  st.cnt = (int*)get(64); st.ctl = get(sizeof(EngCtl));
  CandScratch& S = st.S;
  memset(&S, 0, sizeof(S));
  S.cap = (int)st.cap_cand;
  S.capC = st.capC;
  S.capB = st.capB;
  S.cand = (int*)get(4 * st.cap_cand); S.meta = (int4*)get(16 * st.cap_cand);
  S.cav = (int*)get(4 * st.cap_cand * st.capC); S.bnd = (int*)get(4 * st.cap_cand * st.capB);
  S.outer = (int*)get(4 * st.cap_cand * st.capB);
  S.count = st.cnt + 2;
  S.capCbig = BIG_C; S.capBbig = BIG_B;
  S.bigcav = (int*)get(4 * (size_t)BIGCAP * BIG_C); S.bigbnd = (int*)get(4 * (size_t)BIGCAP * BIG_B);
  S.bigout = (int*)get(4 * (size_t)BIGCAP * BIG_B); S.biglist = (int*)get(4 * (size_t)BIGCAP);
  S.nbig = st.cnt + 5;
  if (!ok) return set_err(c, DT_E_NOMEM, "stream buffers");
  }
  CUDA_OK(cudaMemsetAsync(st.toff, 0, 4 * J, s));
  CUDA_OK(cudaMemsetAsync(st.tend, 0, 4 * J, s));
  CUDA_OK(cudaMemsetAsync(st.claimA, 0, 8 * (size_t)A, s));
  CUDA_OK(cudaMemsetAsync(st.claimC, 0, 8 * (size_t)A, s));
  CUDA_OK(cudaMemsetAsync(st.ss, 0, sizeof(SlotState) * st.max_jobs, s));
  CUDA_OK(cudaMemsetAsync(st.kept, 0, 4 * st.max_jobs, s));
  CUDA_OK(cudaMemsetAsync(st.cnt, 0, 64, s));
  CUDA_OK(cudaMemsetAsync(c->status, 0, sizeof(DevStatus), s));
  EngCtl h0;
  memset(&h0, 0, sizeof(h0));
  h0.ain = st.act0;
  h0.aout = st.act1;
  h0.next_level = -1;
  h0.small_max = -1;
  h0.drain = c->cfg.brio_drain > 1 ? c->cfg.brio_drain : 8;
  h0.round_limit = 0x7fffffff;
  CUDA_OK(cudaMemcpyAsync(st.ctl, &h0, sizeof(EngCtl), cudaMemcpyHostToDevice, s));
  CUDA_OK(cudaStreamSynchronize(s));
  st.round = 0;
  return 0;
}

// Sets up job j in its range [p0, p0 + n) and instance slot: points (already
// in the engine's layout at P, staged and checked), FP32 copies, hint grid,
// initial simplex, level lists, first batch.
template <int D>
static int stream_admit_t(dt_ctx* c, StreamState& st, StreamJob& j, const void* P) {
  using PTT = typename PT<D>::T;
  cudaStream_t s = c->stream;
  const int slot = j.slot;
  const int64_t p0 = j.p0, n = j.n;
  const unsigned g = (unsigned)ceil_div<int64_t>(std::max<int64_t>(n, 1), 256);
  PTT* pts = (PTT*)st.pts + p0;
  CUDA_OK(cudaMemcpyAsync(pts, P, sizeof(PTT) * n, cudaMemcpyDeviceToDevice, s));
  k_stream_iota<<<g, 256, (++c->launches, 0), s>>>(st.gid + p0, n);
  k_stream_fill<<<g, 256, (++c->launches, 0), s>>>(st.pinst + p0, n, slot);
  CUDA_OK(cudaMemsetAsync(st.state + p0, 0, (size_t)n, s));
  // bounding box: FP32 origin and error bound, hint grid of about n / 4 cells
  unsigned long long* ub = (unsigned long long*)pool_get(c, "stream.box", 8 * 6);
  if (!ub) return set_err(c, DT_E_NOMEM, "stream box");
  k_box_init<<<1, 32, (++c->launches, 0), s>>>(ub, 1);
  k_box_reduce<D><<<box_grid(n), 256, (++c->launches, 0), s>>>(pts, nullptr, n, ub);
  unsigned long long hu[6];
  CUDA_OK(cudaMemcpyAsync(hu, ub, 48, cudaMemcpyDeviceToHost, s));
  CUDA_OK(cudaStreamSynchronize(s));
  double xo[4] = {0, 0, 0, 0}, glo[6] = {0, 0, 0, 0, 0, 0};
  int gd[5] = {1, 1, 1, (int)p0, (int)p0};
  double R = 0.0, lo[3] = {0, 0, 0}, ext[3] = {0, 0, 0}, vol = 1.0;
  int nd = 0;
  for (int cc = 0; cc < D; cc++) {
    lo[cc] = host_from_orderable(hu[cc]);
    const double hi = host_from_orderable(hu[3 + cc]);
    const double o = 0.5 * lo[cc] + 0.5 * hi;
    xo[cc] = o;
    R = std::max(R, std::max(hi - o, o - lo[cc]));
    ext[cc] = hi > lo[cc] ? hi - lo[cc] : 0.0;
    if (ext[cc] > 0) { vol *= ext[cc]; nd++; }
  }
  const double eta = 2.02 * (std::ldexp(1.0, -24) + std::ldexp(1.0, -52)) * R * (1.0 + 1e-9);
  float ef = (float)eta;
  if (!((double)ef >= eta)) ef = std::nextafter(ef, INFINITY);
  xo[3] = (double)ef;
  // fine cells: at most n (the job's share of the cell arrays), about n / 4
  double side = nd ? std::pow(vol / std::max(1.0, (double)n / 4.0), 1.0 / nd) : 1.0;
  int64_t cells = 1;
  for (int tries = 0; tries < 200; tries++) {
    cells = 1;
    for (int cc = 0; cc < 3; cc++) {
      int d = 1;
      if (cc < D && ext[cc] > 0 && side > 0) d = (int)std::min(1024.0, std::max(1.0, std::ceil(ext[cc] / side)));
      gd[cc] = d;
      cells *= d;
    }
    if (cells <= std::max<int64_t>(n, 1)) break;
    side *= 1.1;
  }
  for (int cc = 0; cc < 3; cc++) {
    glo[cc] = cc < D ? lo[cc] : 0.0;
    glo[3 + cc] = (cc < D && ext[cc] > 0) ? gd[cc] / ext[cc] : 0.0;
  }
  int64_t cells2 = 1;
  for (int cc = 0; cc < 3; cc++) cells2 *= (gd[cc] + 3) >> 2;
  CUDA_OK(cudaMemcpyAsync(st.xo + 4 * slot, xo, 32, cudaMemcpyHostToDevice, s));
  CUDA_OK(cudaMemcpyAsync(st.glo + 6 * slot, glo, 48, cudaMemcpyHostToDevice, s));
  CUDA_OK(cudaMemcpyAsync(st.gdim + 5 * slot, gd, 20, cudaMemcpyHostToDevice, s));
  CUDA_OK(cudaMemsetAsync(st.hint + p0, 0xff, 4 * (size_t)cells, s));
  CUDA_OK(cudaMemsetAsync(st.hint2 + p0, 0xff, 4 * (size_t)cells2, s));
  k_make_x32<D><<<g, 256, (++c->launches, 0), s>>>(pts, st.pinst + p0, n, st.xo, st.xs + p0);
  // arena and initial simplex (k_init on a view whose instance 0 is this slot)
  const int a0 = (int)(st.arena_factor * p0);
  const int a1 = (int)(st.arena_factor * (p0 + n) + 32);
  const int bounds[2] = {a0, a1};
  CUDA_OK(cudaMemcpyAsync(st.toff + slot, &bounds[0], 4, cudaMemcpyHostToDevice, s));
  CUDA_OK(cudaMemcpyAsync(st.tend + slot, &bounds[1], 4, cudaMemcpyHostToDevice, s));
  long long* dpoff = (long long*)pool_get(c, "stream.poff", 16);
  if (!dpoff) return set_err(c, DT_E_NOMEM, "stream offsets");
  const long long hpoff[2] = {(long long)p0, (long long)(p0 + n)};
  CUDA_OK(cudaMemcpyAsync(dpoff, hpoff, 16, cudaMemcpyHostToDevice, s));
  TriView<D> T = stream_view<D>(c, st);
  TriView<D> Ti = T;
  Ti.tcount = st.tcount + slot;
  k_init<D><<<1, 32, (++c->launches, 0), s>>>(Ti, 1, dpoff, st.toff + slot, st.inst_status + slot);
  int istat = 0;
  CUDA_OK(cudaMemcpyAsync(&istat, st.inst_status + slot, 4, cudaMemcpyDeviceToHost, s));
  CUDA_OK(cudaStreamSynchronize(s));
  if (istat != 0) {
    j.status = istat == 1 ? DT_E_DEGENERATE : DT_E_ARG;
    return 0;
  }
  // activation levels and the instance's level lists
  const double growth = c->cfg.brio_growth > 100 ? c->cfg.brio_growth / 100.0 : 1.5;
  TriView<D> Tl = T;
  Tl.pinst = st.pinst + p0;
  Tl.state = st.state + p0;
  Tl.gid = st.gid + p0;
  k_levels<D><<<g, 256, (++c->launches, 0), s>>>(Tl, n, st.inst_status, st.level + p0,
                                                 (float)(1.0 / std::log2(growth)));
  int rc = group_rank(c, st.level + p0, n, st.lrank + p0, st.lsize, STREAM_NLEV);
  if (rc) return rc;
  int hs[STREAM_NLEV];
  CUDA_OK(cudaMemcpyAsync(hs, st.lsize, 4 * STREAM_NLEV, cudaMemcpyDeviceToHost, s));
  CUDA_OK(cudaStreamSynchronize(s));
  SlotState q;
  memset(&q, 0, sizeof(q));
  q.loff[0] = (int)p0;
  for (int l = 0; l < STREAM_NLEV; l++) q.loff[l + 1] = q.loff[l] + hs[l];
  const int fb = c->cfg.first_batch > 0 ? c->cfg.first_batch : 32;
  int first_level = STREAM_NLEV - 1;
  while (first_level > 0 && q.loff[STREAM_NLEV] - q.loff[first_level] < fb) first_level--;
  q.status = 1;
  q.next_level = first_level - 1;
  CUDA_OK(cudaMemcpyAsync(st.ss + slot, &q, sizeof(SlotState), cudaMemcpyHostToDevice, s));
  k_stream_scatter_levels<<<g, 256, (++c->launches, 0), s>>>(st.level, st.lrank, st.ss, slot, p0, n, st.llist);
  EngCtl h;
  CUDA_OK(cudaMemcpyAsync(&h, st.ctl, sizeof(EngCtl), cudaMemcpyDeviceToHost, s));
  CUDA_OK(cudaStreamSynchronize(s));
  k_stream_locate<D><<<g, 256, (++c->launches, 0), s>>>(T, slot, p0, n, st.level, first_level, h.ain, st.cnt + 0,
                                                        st.ss, h.round + 1);
  j.status = 1;
  return 0;
}

// Builds the round graph of the stream: the same body as the engine's
// graph, with the per-instance activation and round end.
template <int D>
static int stream_graph(dt_ctx* c, StreamState& st, cudaGraphConditionalHandle* hc_out) {
  cudaStream_t cs = capture_stream(c);
  if (!cs) return set_err(c, DT_E_NOMEM, "capture stream");
  stream_release_graph(st);
  TriView<D> T = stream_view<D>(c, st);
  const int capCand = (int)st.cap_cand;
  const int J = st.max_jobs;
  const int64_t sms = c->sms, cb = c->cfg.cavity_blocks > 0 ? c->cfg.cavity_blocks : 16;
  const unsigned gn = (unsigned)std::min<int64_t>(ceil_div<int64_t>(st.cap, 256), sms * 8);
  const unsigned gr = (unsigned)std::min<int64_t>(ceil_div<int64_t>(st.cap, 128), sms * 16);
  const unsigned gw = (unsigned)std::min<int64_t>(ceil_div<int64_t>((int64_t)capCand * 32, 128), sms * cb);
  const int drain = c->cfg.brio_drain > 1 ? c->cfg.brio_drain : 8;
  const unsigned tb = (unsigned)std::min(1024, std::max(32, ((J + 31) / 32) * 32));
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaGraphCreate(&g, 0);
  cudaGraphConditionalHandle hc = 0;
  if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&hc, g, 1, cudaGraphCondAssignDefault);
  cudaGraphNodeParams cp = {};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = hc;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t node;
  if (e == cudaSuccess) e = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &cp);
  cudaGraph_t body = e == cudaSuccess ? cp.conditional.phGraph_out[0] : nullptr;
  if (e == cudaSuccess) e = cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    const bool pdl = st.graph_pdl;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    auto cfg = [&](unsigned grid, unsigned block) {
      cudaLaunchConfig_t lc = {};
      lc.gridDim = dim3(grid);
      lc.blockDim = dim3(block);
      lc.stream = cs;
      lc.attrs = pdl ? at : nullptr;
      lc.numAttrs = pdl ? 1 : 0;
      return lc;
    };
    EngCtl* ctl = (EngCtl*)st.ctl;
    int* cnt = st.cnt;
    cudaLaunchConfig_t l1 = cfg(gr, 128), l2 = cfg(gn, 256), l3 = cfg(gw, 128), l4 = cfg(gw, 128), l5 = cfg(gn, 256),
                       l6 = cfg(gr, 128), l7 = cfg(1, tb), l8 = cfg(big_grid(c->sms), BIG_NT);
    l1.numAttrs = 0;
    cudaLaunchKernelEx(&l1, k_stream_activate<D>, T, (const int*)st.llist, (const int*)st.seg, J, cnt + 0,
                       (const EngCtl*)ctl);
    cudaLaunchKernelEx(&l2, k_nominate<D>, T, (const int*)nullptr, (const int*)(cnt + 0), 0u, st.nom, cnt + 2, cnt + 8,
                       capCand, (const EngCtl*)ctl);
    cudaLaunchKernelEx(&l3, cavity_kernel<D>(c->cfg.cavity_occupancy, c->cfg.cavity_group), T, (const int*)st.nom, (const int*)(cnt + 2), 0u,
                       st.S,
                       (const int*)(cnt + 8), (const EngCtl*)ctl);
    cudaLaunchKernelEx(&l8, k_cavity_big<D>, T, 0u, st.S, (const EngCtl*)ctl);
    cudaLaunchKernelEx(&l4, k_insert_w<D>, T, 0u, st.S, (const int*)(cnt + 2), cnt + 3, (const EngCtl*)ctl);
    cudaLaunchKernelEx(&l5, k_reloc_check<D>, T, (const int*)nullptr, (const int*)(cnt + 0), (int*)nullptr, cnt + 1,
                       st.walk, cnt + 4, 0u, (const EngCtl*)ctl);
    cudaLaunchKernelEx(&l6, k_reloc_walk<D>, T, (const int*)st.walk, (const int*)(cnt + 4), 0u, (const EngCtl*)ctl);
    cudaLaunchKernelEx(&l7, k_stream_step, ctl, st.ss, J, st.seg, cnt, st.kept, (const DevStatus*)c->status,
                       (const volatile int*)st.admit_dev, drain, hc);
    cudaGraph_t captured = nullptr;
    e = cudaStreamEndCapture(cs, &captured);
  }
  cudaGraphExec_t gx = nullptr;
  if (e == cudaSuccess) e = cudaGraphInstantiate(&gx, g, 0);
  if (e != cudaSuccess) {
    cudaGetLastError();
    if (gx) cudaGraphExecDestroy(gx);
    if (g) cudaGraphDestroy(g);
    if (st.graph_pdl) {   // programmatic edges refused: without them
      st.graph_pdl = false;
      return stream_graph<D>(c, st, hc_out);
    }
    return set_err(c, gdt_cuda_fail(e, "stream graph", __FILE__, __LINE__), "stream graph");
  }
  st.g = g;
  st.gx = gx;
  *hc_out = hc;
  return 0;
}

// One quantum: plan, then rounds until an instance finishes, jobs wait, the
// active set empties, or an error.  *yield: the loop's end code.
template <int D>
static int stream_quantum_t(dt_ctx* c, StreamState& st, int* yield) {
  cudaStream_t s = c->stream;
  for (int grow = 0;; grow++) {
    // the graph bakes configuration values in (walk limit, rings, tiles): rebuild it
    // when the context's configuration changed since it was built
    if (st.gx && memcmp(&st.graph_cfg, &c->cfg, sizeof(dt_config)) != 0) stream_release_graph(st);
    if (!st.gx) {
      cudaGraphConditionalHandle hc;
      int rc = stream_graph<D>(c, st, &hc);
      if (rc) return rc;
      st.graph_cfg = c->cfg;
    }
    const int drain = c->cfg.brio_drain > 1 ? c->cfg.brio_drain : 8;
    const unsigned tb = (unsigned)std::min(1024, std::max(32, ((st.max_jobs + 31) / 32) * 32));
    // the graph's first round: clear the end code, plan
    EngCtl h;
    CUDA_OK(cudaMemcpyAsync(&h, st.ctl, sizeof(EngCtl), cudaMemcpyDeviceToHost, s));
    CUDA_OK(cudaStreamSynchronize(s));
    const unsigned r0 = h.round;
    h.done = 0;
    h.stalled = 0;
    CUDA_OK(cudaMemcpyAsync(st.ctl, &h, sizeof(EngCtl), cudaMemcpyHostToDevice, s));
    k_stream_begin<<<1, tb, 0, s>>>((EngCtl*)st.ctl, st.ss, st.max_jobs, st.seg, st.cnt, drain);
    cudaError_t e = cudaGraphLaunch(st.gx, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return set_err(c, gdt_cuda_fail(e, "stream rounds", __FILE__, __LINE__), "stream rounds");
    CUDA_OK(cudaMemcpyAsync(&h, st.ctl, sizeof(EngCtl), cudaMemcpyDeviceToHost, s));
    CUDA_OK(cudaMemcpyAsync(c->status_host, c->status, sizeof(DevStatus), cudaMemcpyDeviceToHost, s));
    CUDA_OK(cudaStreamSynchronize(s));
    st.quanta++;
    st.rounds_run += h.round - r0;
    c->launches += 2 + 8 * (int64_t)(h.round - r0 + 1);
    st.round = h.round;
    if (h.done == 3 && c->status_host->overflow_cav && grow < 6) {
      // cavities outgrew their scratch: twice the room, a new graph, same state
      CUDA_OK(cudaMemsetAsync(&c->status->overflow_cav, 0, 4, s));
      st.capC *= 2;
      st.capB *= 2;
      st.S.capC = st.capC;
      st.S.capB = st.capB;
      st.S.cav = (int*)pool_get(c, "stream.cav", 4 * (size_t)st.cap_cand * st.capC);
      st.S.bnd = (int*)pool_get(c, "stream.bnd", 4 * (size_t)st.cap_cand * st.capB);
      st.S.outer = (int*)pool_get(c, "stream.outer", 4 * (size_t)st.cap_cand * st.capB);   // pool-owned from now on
      if (!st.S.cav || !st.S.bnd || !st.S.outer) return set_err(c, DT_E_NOMEM, "stream cavity scratch");
      stream_release_graph(st);
      continue;
    }
    *yield = h.done;
    if (h.done == 2) return check_status(c, "stream round");
    if (h.done == 3) return set_err(c, DT_E_INTERNAL, "stream rounds made no progress");
    return 0;
  }
}

template <int D>
static int stream_extract_t(dt_ctx* c, StreamState& st, StreamJob& j) {
  cudaStream_t s = c->stream;
  int ab[2] = {0, 0};
  CUDA_OK(cudaMemcpyAsync(&ab[0], st.toff + j.slot, 4, cudaMemcpyDeviceToHost, s));
  CUDA_OK(cudaMemcpyAsync(&ab[1], st.tcount + j.slot, 4, cudaMemcpyDeviceToHost, s));
  CUDA_OK(cudaStreamSynchronize(s));
  const int64_t used = std::max(0, ab[1] - ab[0]);
  int4* rows = (int4*)pool_get(c, "stream.rows", 16 * std::max<int64_t>(used, 16));
  int* cnt = (int*)pool_get(c, "stream.rowcnt", 16);
  if (!rows || !cnt) return set_err(c, DT_E_NOMEM, "stream rows");
  CUDA_OK(cudaMemsetAsync(cnt, 0, 4, s));
  if (used > 0)
    k_stream_rows<D><<<(unsigned)ceil_div<int64_t>(used, 256), 256, (++c->launches, 0), s>>>(st.tv, ab[0], ab[1], st.gid,
                                                                                             rows, cnt);
  int nrows = 0;
  CUDA_OK(cudaMemcpyAsync(&nrows, cnt, 4, cudaMemcpyDeviceToHost, s));
  CUDA_OK(cudaStreamSynchronize(s));
  int32_t* out = nullptr;
  int64_t nout = 0;
  int rc = canonicalize_rows(c, D, rows, nrows, std::max<int64_t>(j.n, 1), &out, &nout, "stream.canon");
  if (rc) return rc;
  j.rows.resize((size_t)nout * (D + 1));
  if (nout) CUDA_OK(cudaMemcpyAsync(j.rows.data(), out, 4 * (size_t)nout * (D + 1), cudaMemcpyDeviceToHost, s));
  CUDA_OK(cudaStreamSynchronize(s));
  return 0;
}

}  // namespace gdt
