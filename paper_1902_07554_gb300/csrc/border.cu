// border.cu -- border detection (the border step of Alg. 1) and vertices(B).
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

#include "bbox.cuh"
#include "border.cuh"
#include "pipeline.cuh"

namespace gdt {

constexpr int MAXLEV = 16;
// Point primitive: points of other partitions one simplex may test before the
// query answers "hit" (always safe: the border may only grow).
constexpr int POINT_BUDGET = 1024;

// Order-preserving map of doubles to unsigned integers (for atomic min/max).
__device__ __forceinline__ unsigned long long orderable_key(double x) {
  unsigned long long b = (unsigned long long)__double_as_longlong(x + 0.0);
  return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}
__device__ __forceinline__ double from_orderable_key(unsigned long long u) {
  unsigned long long b = (u >> 63) ? (u & 0x7fffffffffffffffull) : ~u;
  return __longlong_as_double((long long)b);
}

struct GridView {
  double lo[3], h[MAXLEV];       // origin, cell edge per level
  double inv_h0;                 // 1 / h[0]
  int dims[MAXLEV][3];
  long long off[MAXLEV];         // start of each level's masks
  int levels;
  const unsigned long long* mask;
  const unsigned long long* dil; // per cell: OR of the masks of its 3^d block (same layout)
  // point primitive: the points of each level-0 cell (cell_start[ncell0 + 1], cell_pts[n])
  const int* cell_start;
  const int* cell_pts;
  const void* pts;               // partition-sorted points
  const int* label;              // partition of each point
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

// OR of the masks of the 3^d block of cells around each cell of one level.
template <int D>
__global__ void k_dilate_mask(GridView G, int lev, const unsigned long long* mask, unsigned long long* dil) {
  long long ncell = (long long)G.dims[lev][0] * G.dims[lev][1] * (D == 3 ? G.dims[lev][2] : 1);
  long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (id >= ncell) return;
  int x[3] = {0, 0, 0};
  long long r = id;
  for (int c = 0; c < D; c++) { x[c] = (int)(r % G.dims[lev][c]); r /= G.dims[lev][c]; }
  unsigned long long m = 0;
  for (int dz = (D == 3 ? -1 : 0); dz <= (D == 3 ? 1 : 0); dz++)
    for (int dy = -1; dy <= 1; dy++)
      for (int dx = -1; dx <= 1; dx++) {
        int y[3] = {x[0] + dx, x[1] + dy, x[2] + dz};
        bool ok = true;
        for (int c = 0; c < D; c++) ok &= y[c] >= 0 && y[c] < G.dims[lev][c];
        if (ok) m |= mask[cell_index<D>(G, lev, y)];
      }
  dil[G.off[lev] + id] = m;
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
// Balls are handled in grid units (u = (x - lo) / h0) and FP32, with a
// margin of 2^-8 cell + 2^-20 |u| on the radius that covers the rounding of
// u and of the box tests many times over.  The
// cell of level l holding u is floor(u / 2^l), an exact scaling.  First, at
// the finest level whose cell edge is at least the radius, the ball lies in
// the 3^d block around its centre's cell: one load of that block's OR-ed
// mask settles most simplices.  Otherwise a depth-first search descends the
// pyramid (one frame per level).  Halfspaces (ghost simplices) are tested in
// world coordinates; their search answers "hit" after 64 cells (a
// conservative answer: the border may only grow).
template <int D>
__device__ __forceinline__ bool unit_box_hits(const float* u, float ru2, const int* x, float w) {
  float d2 = 0;
  for (int c = 0; c < D; c++) {
    const float lo = x[c] * w, hi = lo + w;
    const float v = u[c] < lo ? lo - u[c] : (u[c] > hi ? u[c] - hi : 0.0f);
    d2 = fmaf(v, v, d2);
  }
  return d2 <= ru2;
}

// Is the whole cell x of edge w inside the ball (its farthest corner within ru)?
template <int D>
__device__ __forceinline__ bool unit_box_inside(const float* u, float ru2, const int* x, float w) {
  float d2 = 0;
  for (int c = 0; c < D; c++) {
    const float lo = x[c] * w, hi = lo + w;
    const float v = fmaxf(u[c] - lo, hi - u[c]);
    d2 = fmaf(v, v, d2);
  }
  return d2 <= ru2;
}

// 2^-l as a float, exactly (no division).
__device__ __forceinline__ float pow2f_neg(int l) { return __int_as_float((127 - l) << 23); }

// Point primitive: does a point of a partition in `others`, held by level-0
// cell x, lie in the closed shape?  The ball and the halfspace already cover
// the exact circumsphere / hull side with slack; the tests below add a
// relative margin for their own rounding.
template <int D>
__device__ bool cell_points_hit(const GridView& G, const Shape& S, unsigned long long others, const int* x,
                                int& budget) {
  using Pt = typename PT<D>::T;
  const Pt* P = (const Pt*)G.pts;
  long long id = 0;
  for (int c = D - 1; c >= 0; c--) id = id * G.dims[0][c] + x[c];
  const int b = G.cell_start[id], e = G.cell_start[id + 1];
  budget -= e - b;
  if (budget < 0) return true;   // too many points near the shape: answer "hit"
  for (int k = b; k < e; k++) {
    const int q = G.cell_pts[k];
    const int l = G.label[q];
    if (l >= 64 || !((others >> l) & 1ull)) continue;
    const Pt pq = P[q];
    if (!S.half) {
      double d2 = 0;
      for (int c = 0; c < D; c++) { const double d = comp(pq, c) - S.c[c]; d2 += d * d; }
      if (d2 <= S.r * S.r * (1.0 + 1e-12)) return true;
    } else {
      double v = 0, mag = 0;
      for (int c = 0; c < D; c++) {
        v += S.n[c] * (comp(pq, c) - S.c[c]);
        mag += (fabs(S.n[c]) + S.pn[c]) * (fabs(comp(pq, c)) + fabs(S.c[c]));
      }
      if (v >= -(S.slack + 1e-12 * mag)) return true;
    }
  }
  return false;
}

template <int D>
__device__ bool grid_query(const GridView& G, const Shape& S, unsigned long long others, bool points = false) {
  int lev = G.levels - 1;
  int lo_[3] = {0, 0, 0}, hi_[3] = {0, 0, 0};
  float u[3] = {0, 0, 0}, ru = 0, ru2 = 0;
  if (!S.half) {
    float umax = 0;
    for (int c = 0; c < D; c++) {
      u[c] = (float)((S.c[c] - G.lo[c]) * G.inv_h0);
      umax = fmaxf(umax, fabsf(u[c]));
    }
    if (!(umax < 3e7f)) return true;
    // margin: 2^-8 cell, plus 2^-20 |u| for the FP32 rounding of u and of the box tests
    ru = (float)(S.r * G.inv_h0) * 1.0001f + 0.00390625f + umax * 9.5367431640625e-07f;
    ru2 = ru * ru * 1.0001f;
    if (!(ru2 < 1e12f)) return true;
    for (int l = 0; l < G.levels; l++) {
      if (ru > (float)(1 << l)) continue;
      int x[3] = {0, 0, 0};
      bool inside = true;
      for (int c = 0; c < D; c++) {
        const float f = floorf(u[c] * pow2f_neg(l));
        inside &= f >= 0 && f < G.dims[l][c];
        x[c] = inside ? (int)f : 0;
      }
      if (inside && !(G.dil[cell_index<D>(G, l, x)] & others)) return false;
      break;
    }
    // the finest level where the ball's range spans at most 3 cells per axis
    for (int l = 0; l < G.levels; l++) {
      const float sc = pow2f_neg(l);
      bool small = true;
      for (int c = 0; c < D; c++) small &= floorf((u[c] + ru) * sc) - floorf((u[c] - ru) * sc) <= 2.0f;
      if (small) { lev = l; break; }
    }
    const float sc = pow2f_neg(lev);
    for (int c = 0; c < D; c++) {
      const float fa = floorf((u[c] - ru) * sc), fb = floorf((u[c] + ru) * sc);
      if (fb < 0 || fa > G.dims[lev][c] - 1) return false;   // ball outside the grid
      lo_[c] = (int)fmaxf(0.0f, fa);
      hi_[c] = (int)fminf(fb, (float)(G.dims[lev][c] - 1));
    }
  } else {
    for (int c = 0; c < D; c++) { lo_[c] = 0; hi_[c] = G.dims[lev][c] - 1; }
  }
  struct Frame { int x[3]; int child; };
  Frame st[MAXLEV + 1];
  int visits = 0, budget = POINT_BUDGET;
  for (int z = (D == 3 ? lo_[2] : 0); z <= (D == 3 ? hi_[2] : 0); z++)
    for (int y = lo_[1]; y <= hi_[1]; y++)
      for (int x = lo_[0]; x <= hi_[0]; x++) {
        int depth = 0;
        st[0].x[0] = x; st[0].x[1] = y; st[0].x[2] = z; st[0].child = -1;
        while (depth >= 0) {
          Frame& f = st[depth];
          const int l = lev - depth;
          if (f.child < 0) {
            const unsigned long long m = G.mask[cell_index<D>(G, l, f.x)];
            bool hit = (m & others) != 0;
            if (hit) {
              if (!S.half) {
                hit = unit_box_hits<D>(u, ru2, f.x, (float)(1 << l));
                // a cell inside the ball holding a point of another partition settles it
                if (hit && unit_box_inside<D>(u, ru2, f.x, (float)(1 << l))) return true;
              } else {
                if (++visits > 64) return true;
                double blo[3], bhi[3];
                for (int c = 0; c < D; c++) {
                  blo[c] = G.lo[c] + f.x[c] * G.h[l];
                  bhi[c] = G.lo[c] + (f.x[c] + 1) * G.h[l];
                  const double e = 1e-12 * (fabs(blo[c]) + fabs(bhi[c]) + G.h[l]);
                  blo[c] -= e; bhi[c] += e;
                }
                hit = box_hits<D>(S, blo, bhi);
              }
            }
            if (hit && l == 0 && points) hit = cell_points_hit<D>(G, S, others, f.x, budget);
            if (!hit) { depth--; continue; }
            if (l == 0) return true;
            f.child = 0;
          }
          if (f.child >= (1 << D)) { depth--; continue; }
          const int k = f.child++;
          Frame& nf = st[depth + 1];
          bool ok = true;
          for (int c = 0; c < 3; c++) {
            nf.x[c] = c < D ? 2 * f.x[c] + ((k >> c) & 1) : 0;
            if (c < D) ok &= nf.x[c] < G.dims[l - 1][c];
          }
          if (!ok) continue;
          nf.child = -1;
          depth++;
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

// The same ball from the FP32 copies of the points (X = fl32(x - o), X.w = eta;
// see predicates.cuh): every FP32 difference d is within e(d) = eta + u32 |d|
// / (1 - u32) of the exact one, so with D = |d| + e(d) the determinant and the
// numerators N_j are off by at most P(D) - P(|d|) + 1e-5 P(D) (P: their
// permanents).  The centre offset N / (2 det) then follows as in the FP64 ball,
// the vertex a itself is off by at most eta / 2 per coordinate, and the
// radius covers both, plus a relative 1e-8 so that the ball also contains the
// FP64 ball (the FP32 ball is only used to rule a simplex out).  Returns false
// when the bound cannot be established.
template <int D>
__device__ bool circumball_f32(const float4* X, const double* o, const int4& v, Shape& S) {
  const float4 a = X[v.x];
  const float eta = a.w;
  float N[3] = {0, 0, 0}, EN[3] = {0, 0, 0}, det, Edet, pdd;
  if (D == 2) {
    const float4 b = X[v.y], c = X[v.z];
    const float bx = b.x - a.x, by = b.y - a.y, cx_ = c.x - a.x, cy_ = c.y - a.y;
    const float Bx = f32_up(bx, eta), By = f32_up(by, eta), Cx = f32_up(cx_, eta), Cy = f32_up(cy_, eta);
    const float lb = bx * bx + by * by, lc = cx_ * cx_ + cy_ * cy_;
    const float LB = Bx * Bx + By * By, LC = Cx * Cx + Cy * Cy;
    det = bx * cy_ - by * cx_;
    const float p0d = fabsf(bx * cy_) + fabsf(by * cx_);
    pdd = Bx * Cy + By * Cx;
    Edet = (pdd - p0d) + 1e-5f * pdd;
    N[0] = lb * cy_ - lc * by;
    N[1] = lc * bx - lb * cx_;
    const float p00 = lb * fabsf(cy_) + lc * fabsf(by), p01 = lc * fabsf(bx) + lb * fabsf(cx_);
    const float pd0 = LB * Cy + LC * By, pd1 = LC * Bx + LB * Cx;
    EN[0] = (pd0 - p00) + 1e-5f * pd0;
    EN[1] = (pd1 - p01) + 1e-5f * pd1;
  } else {
    const float4 b = X[v.y], c = X[v.z], d = X[v.w];
    const float b0 = b.x - a.x, b1 = b.y - a.y, b2 = b.z - a.z;
    const float c0 = c.x - a.x, c1 = c.y - a.y, c2 = c.z - a.z;
    const float d0 = d.x - a.x, d1 = d.y - a.y, d2 = d.z - a.z;
    const float B0 = f32_up(b0, eta), B1 = f32_up(b1, eta), B2 = f32_up(b2, eta);
    const float C0 = f32_up(c0, eta), C1 = f32_up(c1, eta), C2 = f32_up(c2, eta);
    const float D0 = f32_up(d0, eta), D1 = f32_up(d1, eta), D2 = f32_up(d2, eta);
    const float lb = b0 * b0 + b1 * b1 + b2 * b2, lc = c0 * c0 + c1 * c1 + c2 * c2, ld = d0 * d0 + d1 * d1 + d2 * d2;
    const float LB = B0 * B0 + B1 * B1 + B2 * B2, LC = C0 * C0 + C1 * C1 + C2 * C2, LD = D0 * D0 + D1 * D1 + D2 * D2;
    const float cd[3] = {c1 * d2 - c2 * d1, c2 * d0 - c0 * d2, c0 * d1 - c1 * d0};
    const float db[3] = {d1 * b2 - d2 * b1, d2 * b0 - d0 * b2, d0 * b1 - d1 * b0};
    const float bc[3] = {b1 * c2 - b2 * c1, b2 * c0 - b0 * c2, b0 * c1 - b1 * c0};
    const float pcd[3] = {fabsf(c1 * d2) + fabsf(c2 * d1), fabsf(c2 * d0) + fabsf(c0 * d2), fabsf(c0 * d1) + fabsf(c1 * d0)};
    const float pdb[3] = {fabsf(d1 * b2) + fabsf(d2 * b1), fabsf(d2 * b0) + fabsf(d0 * b2), fabsf(d0 * b1) + fabsf(d1 * b0)};
    const float pbc[3] = {fabsf(b1 * c2) + fabsf(b2 * c1), fabsf(b2 * c0) + fabsf(b0 * c2), fabsf(b0 * c1) + fabsf(b1 * c0)};
    const float PCD[3] = {C1 * D2 + C2 * D1, C2 * D0 + C0 * D2, C0 * D1 + C1 * D0};
    const float PDB[3] = {D1 * B2 + D2 * B1, D2 * B0 + D0 * B2, D0 * B1 + D1 * B0};
    const float PBC[3] = {B1 * C2 + B2 * C1, B2 * C0 + B0 * C2, B0 * C1 + B1 * C0};
    det = b0 * cd[0] + b1 * cd[1] + b2 * cd[2];
    const float p0d = fabsf(b0) * pcd[0] + fabsf(b1) * pcd[1] + fabsf(b2) * pcd[2];
    pdd = B0 * PCD[0] + B1 * PCD[1] + B2 * PCD[2];
    Edet = (pdd - p0d) + 1e-5f * pdd;
    for (int j = 0; j < 3; j++) {
      N[j] = lb * cd[j] + lc * db[j] + ld * bc[j];
      const float p0 = lb * pcd[j] + lc * pdb[j] + ld * pbc[j];
      const float pd = LB * PCD[j] + LC * PDB[j] + LD * PBC[j];
      EN[j] = (pd - p0) + 1e-5f * pd;
    }
  }
  if (!(pdd > F32_TINY && pdd < F32_HUGE) || !(fabsf(det) > 4.0f * Edet)) return false;
  const float adet = fabsf(det), inv = 0.5f / det;
  float r2 = 0, e2 = 0, cc[3] = {0, 0, 0};
  for (int j = 0; j < D; j++) {
    cc[j] = N[j] * inv;
    float e = 0.5f * (fabsf(N[j]) * Edet + adet * EN[j]) / (adet * (adet - Edet));
    e += 4e-7f * fabsf(cc[j]);
    r2 += cc[j] * cc[j];
    e2 += e * e;
  }
  const float r = sqrtf(r2), err = sqrtf(e2);
  if (!isfinite(r) || !isfinite(err)) return false;
  double cmag = 0;
  for (int j = 0; j < D; j++) {
    const double x = j == 0 ? a.x : (j == 1 ? a.y : a.z);
    S.c[j] = o[j] + (x + (double)cc[j]);
    cmag = fmax(cmag, fabs(S.c[j]));
  }
  for (int j = D; j < 3; j++) S.c[j] = 0;
  S.r = ((double)r * (1.0 + 1e-6) + 2.0 * (double)err * (1.0 + 1e-6) + (double)eta) * (1.0 + 1e-8) + 1e-14 * (1.0 + cmag);
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
  const float4* xs;        // FP32 copies of the points (one frame: origin xo, bound in w)
  const double* xo;
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
  const unsigned long long* others;   // per instance: partitions it is tested against (null: all others)
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
  unsigned long long others = A.others ? A.others[i]
                                       : (A.k >= 64 ? ~(1ull << i) : (((1ull << A.k) - 1) & ~(1ull << i)));
  if (!others) return;
  const bool gridded = A.prim == DT_PRIM_GRID || A.prim == DT_PRIM_POINTS;
  const bool points = A.prim == DT_PRIM_POINTS;
  if (g >= 0) {
    ghost_halfspace<D>(P, v, g, S);
    hit = gridded ? grid_query<D>(A.G, S, others, points) : bbox_query<D>(A.boxes, A.k, S, others, i);
  } else if (gridded && circumball_f32<D>(A.xs, A.xo, v, S)) {
    if (!grid_query<D>(A.G, S, others, points)) {
      hit = false;   // even the larger FP32 ball meets no other partition
    } else if (!points) {
      // the FP32 ball contains the FP64 one, so a hit is a (slightly larger)
      // superset of the grid test's border: no FP64 ball for the grid primitive
      hit = true;
    } else {
      // the point test decides point by point: take the tighter FP64 ball
      hit = circumball<D>(P, v, S) ? grid_query<D>(A.G, S, others, points) : true;
    }
  } else if (!circumball<D>(P, v, S)) {
    hit = true;
  } else {
    hit = gridded ? grid_query<D>(A.G, S, others, points) : bbox_query<D>(A.boxes, A.k, S, others, i);
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

// Level-0 cell of each point (the cell k_occupy assigns).
template <int D>
__global__ void k_point_cell(const typename PT<D>::T* P, int64_t n, GridView G, int* cell, int* count) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  long long id = 0;
  for (int c = D - 1; c >= 0; c--) {
    double f = (comp(P[i], c) - G.lo[c]) / G.h[0];
    int v = f < 0 ? 0 : (int)f;
    id = id * G.dims[0][c] + min(v, G.dims[0][c] - 1);
  }
  cell[i] = (int)id;
  atomicAdd(&count[id], 1);
}
__global__ void k_cell_scatter(const int* cell, int64_t n, const int* start, int* fill, int* pts) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int c = cell[i];
  pts[start[c] + atomicAdd(&fill[c], 1)] = (int)i;
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
                  int prim, unsigned char** bflag_out, unsigned char** vflag_out, int64_t* nborder,
                  const std::vector<unsigned long long>* others) {
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
  // FP32 copies in one frame for the exclusion stage
  float4* xs = nullptr;
  const double* xo = nullptr;
  std::vector<unsigned long long> hu;
  int rc = fp32_points(c, dim, Ps, nullptr, n, 1, "b.xs", &xs, &hu, &xo);
  if (rc) return rc;
  BorderArgs A;
  A.xs = xs;
  A.xo = xo;
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
  A.others = nullptr;
  if (others) {
    if ((int)others->size() < parts.ninst) return set_err(c, DT_E_INTERNAL, "partition masks");
    unsigned long long* om = (unsigned long long*)pool_get(c, "b.others", 8 * (size_t)parts.ninst);
    if (!om) return set_err(c, DT_E_NOMEM, "partition masks");
    CUDA_OK(cudaMemcpyAsync(om, others->data(), 8 * (size_t)parts.ninst, cudaMemcpyHostToDevice, s));
    A.others = om;
  }
  memset(&A.G, 0, sizeof(A.G));
  // per-partition boxes (bbox primitive and the grid's extent)
  CUDA_OK(cudaMemsetAsync(ubox, 0, 8 * 6 * (size_t)k, s));
  k_box_init<<<ceil_div(6 * k, 128), 128, (++c->launches, 0), s>>>(ubox, k);
  if (dim == 2) k_box_reduce<2><<<box_grid(n), 256, (++c->launches, 0), s>>>((const double2*)Ps, pinst, n, ubox);
  else k_box_reduce<3><<<box_grid(n), 256, (++c->launches, 0), s>>>((const double4_32a*)Ps, pinst, n, ubox);
  k_boxes_to_double<<<ceil_div(6 * k, 128), 128, (++c->launches, 0), s>>>(ubox, k, boxes);
  if (prim == DT_PRIM_GRID || prim == DT_PRIM_POINTS) {
    if (k > 64) return set_err(c, DT_E_ARG, "the grid and point primitives support k <= 64");
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
    G.inv_h0 = 1.0 / G.h[0];
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
    unsigned long long* dil = (unsigned long long*)pool_get(c, "b.dil", 8 * (size_t)total);
    if (!dil) return set_err(c, DT_E_NOMEM, "grid masks");
    for (int l = 0; l < G.levels; l++) {
      long long cells = (long long)G.dims[l][0] * G.dims[l][1] * G.dims[l][2];
      unsigned gl = (unsigned)ceil_div<long long>(cells, 256);
      if (dim == 2) k_dilate_mask<2><<<gl, 256, (++c->launches, 0), s>>>(G, l, mask, dil);
      else k_dilate_mask<3><<<gl, 256, (++c->launches, 0), s>>>(G, l, mask, dil);
    }
    G.dil = dil;
    G.cell_start = nullptr;
    G.cell_pts = nullptr;
    G.pts = Ps;
    G.label = pinst;
    if (prim == DT_PRIM_POINTS) {
      const long long ncell0 = (long long)G.dims[0][0] * G.dims[0][1] * G.dims[0][2];
      int* cstart = (int*)pool_get(c, "b.cstart", 4 * (size_t)(ncell0 + 1));
      int* ccount = (int*)pool_get(c, "b.ccount", 4 * (size_t)(ncell0 + 1));
      int* cfill = (int*)pool_get(c, "b.cfill", 4 * (size_t)(ncell0 + 1));
      int* ccell = (int*)pool_get(c, "b.ccell", 4 * (size_t)std::max<int64_t>(n, 1));
      int* cpts = (int*)pool_get(c, "b.cpts", 4 * (size_t)std::max<int64_t>(n, 1));
      if (!cstart || !ccount || !cfill || !ccell || !cpts) return set_err(c, DT_E_NOMEM, "cell lists");
      CUDA_OK(cudaMemsetAsync(ccount, 0, 4 * (size_t)(ncell0 + 1), s));
      CUDA_OK(cudaMemsetAsync(cfill, 0, 4 * (size_t)(ncell0 + 1), s));
      if (dim == 2) k_point_cell<2><<<g, 256, (++c->launches, 0), s>>>((const double2*)Ps, n, G, ccell, ccount);
      else k_point_cell<3><<<g, 256, (++c->launches, 0), s>>>((const double4_32a*)Ps, n, G, ccell, ccount);
      rc = exclusive_scan_i32(c, ccount, cstart, ncell0 + 1, nullptr);
      if (rc) return rc;
      k_cell_scatter<<<g, 256, (++c->launches, 0), s>>>(ccell, n, cstart, cfill, cpts);
      G.cell_start = cstart;
      G.cell_pts = cpts;
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
