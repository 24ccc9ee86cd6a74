// border.cu -- border detection (Alg. 1, lines 6-18) and vertices(B).
//
// Every live simplex of every partial triangulation T_i is tested (one
// parallel sweep; a superset of what a breadth-first search from the hull
// reaches).  A finite simplex is a border simplex when its circumsphere,
// inflated by a bound on the floating-point error of the circumcentre, meets
// a region occupied by another partition.  A ghost simplex (infinite vertex +
// hull facet f) stands for the open halfspace beyond f; it is a border
// simplex when that halfspace (with slack) meets another partition.
// Regions (Sec. 3.2):
//   grid -- cells of a uniform grid with a bit mask of the partitions whose
//           points they contain, plus a pyramid of coarser levels (each cell
//           the OR of its 2^d children) playing the role of the AABB tree;
//   bbox -- one axis-aligned bounding box per partition.
// A partition that could not be triangulated (too few or flat points)
// contributes all its points to vertices(B).
#include <cmath>

#include "border.cuh"
#include "pipeline.cuh"

namespace gdt {

constexpr int MAXLEV = 16;

// Order-preserving map of doubles to unsigned integers (for atomic min/max).
__device__ __forceinline__ unsigned long long orderable_key(double x) {
  unsigned long long b = (unsigned long long)__double_as_longlong(x + 0.0);
  return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}
__device__ __forceinline__ double from_orderable_key(unsigned long long u) {
  unsigned long long b = (u >> 63) ? (u & 0x7fffffffffffffffull) : ~u;
  return __longlong_as_double((long long)b);
}
__global__ void k_init_ubox(unsigned long long* ubox, int k) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < 6 * k) ubox[i] = (i % 6) < 3 ? ~0ull : 0ull;
}

struct GridView {
  double lo[3], h[MAXLEV];       // origin, cell edge per level
  int dims[MAXLEV][3];
  long long off[MAXLEV];         // start of each level's masks
  int levels;
  const unsigned long long* mask;
};

template <int D>
__device__ __forceinline__ long long cell_index(const GridView& G, int lev, const int* x) {
  long long id = 0;
  for (int c = D - 1; c >= 0; c--) id = id * G.dims[lev][c] + x[c];
  return G.off[lev] + id;
}

template <int D>
__global__ void k_occupy(const typename PT<D>::T* P, const int* label, int64_t n, GridView G,
                         unsigned long long* mask) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  int x[3] = {0, 0, 0};
  for (int c = 0; c < D; c++) {
    double f = (comp(P[i], c) - G.lo[c]) / G.h[0];
    int v = f < 0 ? 0 : (int)f;
    x[c] = min(v, G.dims[0][c] - 1);
  }
  atomicOr(&mask[cell_index<D>(G, 0, x)], 1ull << label[i]);
}

template <int D>
__global__ void k_pyramid(GridView G, int lev, unsigned long long* mask) {
  long long ncell = (long long)G.dims[lev][0] * G.dims[lev][1] * (D == 3 ? G.dims[lev][2] : 1);
  long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (id >= ncell) return;
  int x[3] = {0, 0, 0};
  long long r = id;
  for (int c = 0; c < D; c++) { x[c] = (int)(r % G.dims[lev][c]); r /= G.dims[lev][c]; }
  unsigned long long m = 0;
  for (int k = 0; k < (1 << D); k++) {
    int y[3];
    bool ok = true;
    for (int c = 0; c < D; c++) {
      y[c] = 2 * x[c] + ((k >> c) & 1);
      ok &= y[c] < G.dims[lev - 1][c];
    }
    if (ok) m |= mask[cell_index<D>(G, lev - 1, y)];
  }
  mask[G.off[lev] + id] = m;
}

// ---------------------------------------------------------------- shapes
// A closed ball (center, radius) or a closed halfspace {x : n.(x - a) >= -slack}.
struct Shape {
  double c[3];
  double r;
  double n[3], pn[3];   // halfspace normal and the permanent bounding its rounding error
  double slack;
  bool half;
};

template <int D>
__device__ __forceinline__ bool box_hits(const Shape& S, const double* blo, const double* bhi) {
  if (!S.half) {
    double d2 = 0;
    for (int c = 0; c < D; c++) {
      double v = S.c[c] < blo[c] ? blo[c] - S.c[c] : (S.c[c] > bhi[c] ? S.c[c] - bhi[c] : 0.0);
      d2 += v * v;
    }
    return d2 <= S.r * S.r;
  }
  // the corner maximising n.x; slack covers the rounding of n (through its
  // permanent), of the differences and of the sum, with a factor > 1000
  double v = 0, mag = 0;
  for (int c = 0; c < D; c++) {
    double x = S.n[c] > 0 ? bhi[c] : blo[c];
    v += S.n[c] * (x - S.c[c]);
    mag += (fabs(S.n[c]) + S.pn[c]) * (fabs(x) + fabs(S.c[c]));
  }
  return v >= -(S.slack + 1e-12 * mag);
}

// Is there a cell, occupied by a partition in `others`, that the shape meets?
template <int D>
__device__ bool grid_query(const GridView& G, const Shape& S, unsigned long long others) {
  // start level: the finest level where the shape's bounding range spans at most 3 cells
  int lev = G.levels - 1;
  int lo_[3], hi_[3];
  if (!S.half) {
    for (int l = 0; l < G.levels; l++) {
      bool small = true;
      for (int c = 0; c < D; c++) {
        double a = floor((S.c[c] - S.r - G.lo[c]) / G.h[l]);
        double b = floor((S.c[c] + S.r - G.lo[c]) / G.h[l]);
        small &= (b - a) <= 2.0;
      }
      if (small) { lev = l; break; }
    }
    for (int c = 0; c < D; c++) {
      double fa = floor((S.c[c] - S.r - G.lo[c]) / G.h[lev]);
      double fb = floor((S.c[c] + S.r - G.lo[c]) / G.h[lev]);
      lo_[c] = (int)fmax(0.0, fmin(fa, (double)G.dims[lev][c] - 1));
      hi_[c] = (int)fmax(0.0, fmin(fb, (double)G.dims[lev][c] - 1));
      if (fb < 0 || fa > G.dims[lev][c] - 1) return false;   // ball outside the grid
    }
  } else {
    for (int c = 0; c < D; c++) { lo_[c] = 0; hi_[c] = G.dims[lev][c] - 1; }
  }
  // depth-first search; stack entries (level, cell coords)
  int stk[192][4];
  int sp = 0;
  for (int z = (D == 3 ? lo_[2] : 0); z <= (D == 3 ? hi_[2] : 0); z++)
    for (int y = lo_[1]; y <= hi_[1]; y++)
      for (int x = lo_[0]; x <= hi_[0]; x++) {
        if (sp >= 192) return true;   // stack exhausted: conservative answer
        stk[sp][0] = lev; stk[sp][1] = x; stk[sp][2] = y; stk[sp][3] = z;
        sp++;
      }
  while (sp > 0) {
    sp--;
    int l = stk[sp][0];
    int x[3] = {stk[sp][1], stk[sp][2], stk[sp][3]};
    unsigned long long m = G.mask[cell_index<D>(G, l, x)];
    if (!(m & others)) continue;
    double blo[3], bhi[3];
    for (int c = 0; c < D; c++) {
      blo[c] = G.lo[c] + x[c] * G.h[l];
      bhi[c] = G.lo[c] + (x[c] + 1) * G.h[l];
      // slack for the rounding of the box corners
      double e = 1e-12 * (fabs(blo[c]) + fabs(bhi[c]) + G.h[l]);
      blo[c] -= e; bhi[c] += e;
    }
    if (!box_hits<D>(S, blo, bhi)) continue;
    if (l == 0) return true;
    for (int k = 0; k < (1 << D); k++) {
      int y[3] = {0, 0, 0};
      bool ok = true;
      for (int c = 0; c < D; c++) {
        y[c] = 2 * x[c] + ((k >> c) & 1);
        ok &= y[c] < G.dims[l - 1][c];
      }
      if (!ok) continue;
      if (sp >= 192) return true;
      stk[sp][0] = l - 1; stk[sp][1] = y[0]; stk[sp][2] = y[1]; stk[sp][3] = y[2];
      sp++;
    }
  }
  return false;
}

// Is the shape meeting the bounding box of a partition in `others`?
template <int D>
__device__ bool bbox_query(const double* boxes, int k, const Shape& S, unsigned long long others, int self) {
  for (int j = 0; j < k; j++) {
    if (j == self) continue;
    if (k <= 64 && !((others >> j) & 1ull)) continue;
    const double* b = boxes + 6 * j;
    if (!(b[0] <= b[3])) continue;   // empty partition
    double blo[3], bhi[3];
    for (int c = 0; c < D; c++) {
      double e = 1e-12 * (fabs(b[c]) + fabs(b[3 + c]));
      blo[c] = b[c] - e; bhi[c] = b[3 + c] + e;
    }
    if (box_hits<D>(S, blo, bhi)) return true;
  }
  return false;
}

// Conservative circumball of a finite simplex: centre and a radius that
// covers the exact circumsphere.  The centre relative to vertex a is
// N / (2 det); |err(N_j)| and |err(det)| are bounded by 1e-14 times the
// permanents of their expressions (more than ten times the rounding bound),
// and the centre error follows from the quotient.  Returns false when the
// determinant is too small to bound (the caller then treats the simplex as a
// border simplex).
template <int D>
__device__ bool circumball(const typename PT<D>::T* P, const int4& v, Shape& S) {
  using Pt = typename PT<D>::T;
  Pt a = P[v.x];
  double N[3] = {0, 0, 0}, pN[3] = {0, 0, 0}, det, pdet;
  if (D == 2) {
    Pt b = P[v.y], c = P[v.z];
    double bx = comp(b, 0) - comp(a, 0), by = comp(b, 1) - comp(a, 1);
    double cxx = comp(c, 0) - comp(a, 0), cyy = comp(c, 1) - comp(a, 1);
    double lb = bx * bx + by * by, lc = cxx * cxx + cyy * cyy;
    det = bx * cyy - by * cxx;
    pdet = fabs(bx * cyy) + fabs(by * cxx);
    N[0] = lb * cyy - lc * by;
    N[1] = lc * bx - lb * cxx;
    pN[0] = lb * fabs(cyy) + lc * fabs(by);
    pN[1] = lc * fabs(bx) + lb * fabs(cxx);
  } else {
    Pt b = P[v.y], c = P[v.z], d = P[v.w];
    double b0 = comp(b, 0) - comp(a, 0), b1 = comp(b, 1) - comp(a, 1), b2 = comp(b, 2) - comp(a, 2);
    double c0 = comp(c, 0) - comp(a, 0), c1 = comp(c, 1) - comp(a, 1), c2 = comp(c, 2) - comp(a, 2);
    double d0 = comp(d, 0) - comp(a, 0), d1 = comp(d, 1) - comp(a, 1), d2 = comp(d, 2) - comp(a, 2);
    double lb = b0 * b0 + b1 * b1 + b2 * b2, lc = c0 * c0 + c1 * c1 + c2 * c2, ld = d0 * d0 + d1 * d1 + d2 * d2;
    // cross products and their absolute counterparts
    double cd[3] = {c1 * d2 - c2 * d1, c2 * d0 - c0 * d2, c0 * d1 - c1 * d0};
    double db[3] = {d1 * b2 - d2 * b1, d2 * b0 - d0 * b2, d0 * b1 - d1 * b0};
    double bc[3] = {b1 * c2 - b2 * c1, b2 * c0 - b0 * c2, b0 * c1 - b1 * c0};
    double pcd[3] = {fabs(c1 * d2) + fabs(c2 * d1), fabs(c2 * d0) + fabs(c0 * d2), fabs(c0 * d1) + fabs(c1 * d0)};
    double pdb[3] = {fabs(d1 * b2) + fabs(d2 * b1), fabs(d2 * b0) + fabs(d0 * b2), fabs(d0 * b1) + fabs(d1 * b0)};
    double pbc[3] = {fabs(b1 * c2) + fabs(b2 * c1), fabs(b2 * c0) + fabs(b0 * c2), fabs(b0 * c1) + fabs(b1 * c0)};
    det = b0 * cd[0] + b1 * cd[1] + b2 * cd[2];
    pdet = fabs(b0) * pcd[0] + fabs(b1) * pcd[1] + fabs(b2) * pcd[2];
    for (int j = 0; j < 3; j++) {
      N[j] = lb * cd[j] + lc * db[j] + ld * bc[j];
      pN[j] = lb * pcd[j] + lc * pdb[j] + ld * pbc[j];
    }
  }
  double edet = 1e-14 * pdet;
  if (!(fabs(det) > 4.0 * edet) || !(pdet > 1e-250) || !isfinite(det)) return false;
  double inv = 0.5 / det;
  double cc[3] = {0, 0, 0}, err2 = 0, r2 = 0;
  for (int j = 0; j < D; j++) {
    cc[j] = N[j] * inv;
    double eN = 1e-14 * pN[j];
    // |N/det - N'/det'| <= (|N| edet + |det| eN) / (|det| (|det| - edet)), halved
    double e = 0.5 * (fabs(N[j]) * edet + fabs(det) * eN) / (fabs(det) * (fabs(det) - edet));
    e += 1e-15 * fabs(cc[j]);
    err2 += e * e;
    r2 += cc[j] * cc[j];
  }
  double r = sqrt(r2), err = sqrt(err2);
  if (!isfinite(r) || !isfinite(err)) return false;
  double amag = 0;
  for (int j = 0; j < D; j++) {
    S.c[j] = comp(a, j) + cc[j];
    amag = fmax(amag, fabs(comp(a, j)) + fabs(cc[j]));
  }
  for (int j = D; j < 3; j++) S.c[j] = 0;
  // the centre may be off by err, the radius by err plus rounding of sqrt
  S.r = (r + 2.0 * err) * (1.0 + 1e-12) + 1e-12 * amag + 1e-300;
  S.half = false;
  S.n[0] = S.n[1] = S.n[2] = 0;
  S.pn[0] = S.pn[1] = S.pn[2] = 0;
  return true;
}

// Halfspace beyond a ghost's hull facet: orient(ghost with the infinite
// vertex replaced by x) >= 0, written as n.(x - a) >= -slack.
template <int D>
__device__ void ghost_halfspace(const typename PT<D>::T* P, const int4& v, int g, Shape& S) {
  using Pt = typename PT<D>::T;
  int t[4] = {v.x, v.y, v.z, v.w};
  // orient(t with t[g] = x) is affine in x: coefficient of x = cofactor vector
  int f[3], k = 0;
  for (int i = 0; i <= D; i++) if (i != g) f[k++] = i;
  Pt a = P[t[f[0]]];
  double n[3] = {0, 0, 0};
  if (D == 2) {
    // orient2(p0,p1,p2) with x at slot g; rows relative to the first finite vertex a
    Pt b = P[t[f[1]]];
    double ex = comp(b, 0) - comp(a, 0), ey = comp(b, 1) - comp(a, 1);
    // orient(x, a, b) = det[a - x, b - x] = (a-x) x (b-x) = cross(b - a, x - a) with sign by slot
    double nx = -ey, ny = ex;          // orient(a, b, x) = ex*(x.y-a.y) - ey*(x.x-a.x)
    S.pn[0] = fabs(ey); S.pn[1] = fabs(ex); S.pn[2] = 0;
    // slot permutation sign: the tuple (t with x at g) vs (a, b, x)
    int perm[3] = {f[0], f[1], g};
    int sgn = 1;
    for (int i = 0; i < 3; i++) for (int j = i + 1; j < 3; j++) if (perm[i] > perm[j]) sgn = -sgn;
    n[0] = sgn * nx; n[1] = sgn * ny;
  } else {
    Pt b = P[t[f[1]]], c = P[t[f[2]]];
    double e1[3] = {comp(b, 0) - comp(a, 0), comp(b, 1) - comp(a, 1), comp(b, 2) - comp(a, 2)};
    double e2[3] = {comp(c, 0) - comp(a, 0), comp(c, 1) - comp(a, 1), comp(c, 2) - comp(a, 2)};
    // orient(a, b, c, x) = det[b - a, c - a, x - a] = (e1 x e2) . (x - a)
    double cr[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
    S.pn[0] = fabs(e1[1] * e2[2]) + fabs(e1[2] * e2[1]);
    S.pn[1] = fabs(e1[2] * e2[0]) + fabs(e1[0] * e2[2]);
    S.pn[2] = fabs(e1[0] * e2[1]) + fabs(e1[1] * e2[0]);
    int perm[4] = {f[0], f[1], f[2], g};
    int sgn = 1;
    for (int i = 0; i < 4; i++) for (int j = i + 1; j < 4; j++) if (perm[i] > perm[j]) sgn = -sgn;
    for (int j = 0; j < 3; j++) n[j] = sgn * cr[j];
  }
  double mag = 0;
  for (int j = 0; j < D; j++) { S.n[j] = n[j]; S.c[j] = comp(a, j); mag += fabs(n[j]); }
  for (int j = D; j < 3; j++) { S.n[j] = 0; S.c[j] = 0; S.pn[j] = 0; }
  S.slack = 1e-300;
  S.half = true;
  (void)mag;
}

struct BorderArgs {
  const int4* tv;
  const int* toff;
  const int* tcount;
  const int* inst_status;
  int ninst, nslots, k;
  int prim;
  GridView G;
  const double* boxes;     // 6 per partition (bbox primitive)
  unsigned char* bflag;    // per slot
  unsigned char* vflag;    // per (partition-sorted) point
  int* nborder;            // finite border simplices counter
};

template <int D>
__global__ void k_border(const typename PT<D>::T* P, BorderArgs A) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= A.nslots) return;
  int lo = 0, hi = A.ninst - 1;
  while (lo < hi) { int mid = (lo + hi + 1) >> 1; if (A.toff[mid] <= s) lo = mid; else hi = mid - 1; }
  int i = lo;
  A.bflag[s] = 0;
  if (s >= A.tcount[i] || A.inst_status[i] != 0) return;
  int4 v = A.tv[s];
  if (v.x == DEAD) return;
  int t[4] = {v.x, v.y, v.z, v.w};
  int g = -1;
  for (int j = 0; j <= D; j++) if (t[j] == INF_V) g = j;
  Shape S;
  bool hit;
  unsigned long long others = A.k >= 64 ? ~(1ull << i) : (((1ull << A.k) - 1) & ~(1ull << i));
  if (g >= 0) {
    ghost_halfspace<D>(P, v, g, S);
    hit = A.prim == DT_PRIM_GRID ? grid_query<D>(A.G, S, others) : bbox_query<D>(A.boxes, A.k, S, others, i);
  } else if (!circumball<D>(P, v, S)) {
    hit = true;
  } else {
    hit = A.prim == DT_PRIM_GRID ? grid_query<D>(A.G, S, others) : bbox_query<D>(A.boxes, A.k, S, others, i);
  }
  if (!hit) return;
  A.bflag[s] = 1;
  if (g < 0) atomicAdd(A.nborder, 1);
  for (int j = 0; j <= D; j++) if (t[j] >= 0) A.vflag[t[j]] = 1;
}

// points of partitions that could not be triangulated are border vertices
__global__ void k_flag_bad_partitions(const int* pinst, const int* inst_status, int64_t n, unsigned char* vflag) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n && inst_status[pinst[i]] != 0) vflag[i] = 1;
}

template <int D>
__global__ void k_part_boxes(const typename PT<D>::T* P, const int* pinst, int64_t n, unsigned long long* ubox) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  int l = pinst[i];
  for (int c = 0; c < D; c++) {
    unsigned long long key = orderable_key(comp(P[i], c));
    atomicMin(&ubox[6 * l + c], key);
    atomicMax(&ubox[6 * l + 3 + c], key);
  }
}

__global__ void k_boxes_to_double(const unsigned long long* ubox, int k, double* box) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < 6 * k) {
    unsigned long long u = ubox[i];
    if (u == ~0ull || u == 0ull) { box[i] = (i % 6) < 3 ? INFINITY : -INFINITY; return; }
    box[i] = from_orderable_key(u);
  }
}

int border_detect(dt_ctx* c, int dim, const EngineRun& parts, const void* Ps, const int* pinst, int k, double cell,
                  int prim, unsigned char** bflag_out, unsigned char** vflag_out, int64_t* nborder) {
  cudaStream_t s = c->stream;
  int64_t n = parts.npts;
  unsigned char* bflag = (unsigned char*)pool_get(c, "b.bflag", std::max<int64_t>(parts.total_slots, 1));
  unsigned char* vflag = (unsigned char*)pool_get(c, "b.vflag", std::max<int64_t>(n, 1));
  int* cnt = (int*)pool_get(c, "b.cnt", 16);
  double* box = (double*)pool_get(c, "b.box", 48);
  double* boxes = (double*)pool_get(c, "b.boxes", 8 * 6 * (size_t)k);
  unsigned long long* ubox = (unsigned long long*)pool_get(c, "b.ubox", 8 * 6 * (size_t)k);
  if (!bflag || !vflag || !cnt || !box || !boxes || !ubox) return set_err(c, DT_E_NOMEM, "border buffers");
  CUDA_OK(cudaMemsetAsync(vflag, 0, std::max<int64_t>(n, 1), s));
  CUDA_OK(cudaMemsetAsync(cnt, 0, 16, s));
  unsigned g = (unsigned)ceil_div<int64_t>(n, 256);
  k_flag_bad_partitions<<<g, 256, (++c->launches, 0), s>>>(pinst, parts.inst_status, n, vflag);
  BorderArgs A;
  A.tv = (const int4*)parts.tv;
  A.toff = parts.toff;
  A.tcount = parts.tcount;
  A.inst_status = parts.inst_status;
  A.ninst = parts.ninst;
  A.nslots = (int)parts.total_slots;
  A.k = k;
  A.prim = prim;
  A.boxes = boxes;
  A.bflag = bflag;
  A.vflag = vflag;
  A.nborder = cnt;
  memset(&A.G, 0, sizeof(A.G));
  // per-partition boxes (bbox primitive and the grid's extent)
  CUDA_OK(cudaMemsetAsync(ubox, 0, 8 * 6 * (size_t)k, s));
  k_init_ubox<<<ceil_div(6 * k, 128), 128, (++c->launches, 0), s>>>(ubox, k);
  if (dim == 2) k_part_boxes<2><<<g, 256, (++c->launches, 0), s>>>((const double2*)Ps, pinst, n, ubox);
  else k_part_boxes<3><<<g, 256, (++c->launches, 0), s>>>((const double4_32a*)Ps, pinst, n, ubox);
  k_boxes_to_double<<<ceil_div(6 * k, 128), 128, (++c->launches, 0), s>>>(ubox, k, boxes);
  if (prim == DT_PRIM_GRID) {
    if (k > 64) return set_err(c, DT_E_ARG, "the grid primitive supports k <= 64");
    std::vector<double> hb(6 * (size_t)k);
    CUDA_OK(cudaMemcpyAsync(hb.data(), boxes, 8 * 6 * (size_t)k, cudaMemcpyDeviceToHost, s));
    CUDA_OK(cudaStreamSynchronize(s));
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int j = 0; j < k; j++)
      for (int cc = 0; cc < dim; cc++) {
        if (hb[6 * j + cc] <= hb[6 * j + 3 + cc]) {
          lo[cc] = std::min(lo[cc], hb[6 * j + cc]);
          hi[cc] = std::max(hi[cc], hb[6 * j + 3 + cc]);
        }
      }
    double vol = 1.0, maxext = 0;
    int nd = 0;
    for (int cc = 0; cc < dim; cc++) {
      double e = hi[cc] - lo[cc];
      maxext = std::max(maxext, e);
      if (e > 0) { vol *= e; nd++; }
    }
    // c_G times the mean point spacing (vol / n)^(1/d), with at most ~2^24 cells
    double h0 = nd ? cell * std::pow(vol / (double)n, 1.0 / nd) : 1.0;
    if (!(h0 > 0)) h0 = maxext > 0 ? maxext : 1.0;
    for (;;) {
      double cells = 1;
      for (int cc = 0; cc < dim; cc++) cells *= std::max(1.0, std::ceil((hi[cc] - lo[cc]) / h0 + 1));
      if (cells <= double(1 << 24)) break;
      h0 *= 1.25;
    }
    GridView& G = A.G;
    long long total = 0;
    int lev = 0;
    for (; lev < MAXLEV; lev++) {
      G.h[lev] = h0 * std::ldexp(1.0, lev);
      long long cells = 1;
      int maxd = 1;
      for (int cc = 0; cc < 3; cc++) {
        int d = 1;
        if (cc < dim) d = (int)std::max(1.0, std::floor((hi[cc] - lo[cc]) / G.h[lev]) + 1);
        G.dims[lev][cc] = d;
        cells *= d;
        maxd = std::max(maxd, d);
      }
      G.off[lev] = total;
      total += cells;
      if (maxd <= 2) { lev++; break; }
    }
    G.levels = lev;
    for (int cc = 0; cc < 3; cc++) G.lo[cc] = cc < dim ? lo[cc] : 0.0;
    unsigned long long* mask = (unsigned long long*)pool_get(c, "b.mask", 8 * (size_t)total);
    if (!mask) return set_err(c, DT_E_NOMEM, "grid masks");
    CUDA_OK(cudaMemsetAsync(mask, 0, 8 * (size_t)total, s));
    G.mask = mask;
    if (dim == 2) k_occupy<2><<<g, 256, (++c->launches, 0), s>>>((const double2*)Ps, pinst, n, G, mask);
    else k_occupy<3><<<g, 256, (++c->launches, 0), s>>>((const double4_32a*)Ps, pinst, n, G, mask);
    for (int l = 1; l < G.levels; l++) {
      long long cells = (long long)G.dims[l][0] * G.dims[l][1] * G.dims[l][2];
      unsigned gl = (unsigned)ceil_div<long long>(cells, 256);
      if (dim == 2) k_pyramid<2><<<gl, 256, (++c->launches, 0), s>>>(G, l, mask);
      else k_pyramid<3><<<gl, 256, (++c->launches, 0), s>>>(G, l, mask);
    }
  }
  unsigned gs = (unsigned)ceil_div<int64_t>(parts.total_slots, 128);
  if (dim == 2) k_border<2><<<gs, 128, (++c->launches, 0), s>>>((const double2*)Ps, A);
  else k_border<3><<<gs, 128, (++c->launches, 0), s>>>((const double4_32a*)Ps, A);
  int h = 0;
  CUDA_OK(cudaMemcpyAsync(&h, cnt, 4, cudaMemcpyDeviceToHost, s));
  CUDA_OK(cudaStreamSynchronize(s));
  *nborder = h;
  *bflag_out = bflag;
  *vflag_out = vflag;
  return 0;
}

}  // namespace gdt
