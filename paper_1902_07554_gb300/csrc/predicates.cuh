// predicates.cuh -- exact geometric predicates on the GPU.
//
// orient and insphere are the signs of the determinants that define a
// Delaunay triangulation (Sec. 2.1).  Each is evaluated in two stages:
//   1. an FP64 semi-static filter: the determinant of coordinate differences
//      and a bound C * permanent on its rounding error (C derived from the
//      number of roundings along any monomial, with a factor >= 2 of slack);
//   2. when the filter cannot decide, the determinant is recomputed exactly in
//      fixed-width two's-complement integers: every coordinate difference is
//      split exactly into two doubles (TwoDiff), all of them are scaled by a
//      common power of two to integers, and the polynomial is evaluated modulo
//      2^(64*NL) with NL chosen so that no intermediate value can wrap.
// Exact zeros of insphere are resolved by a symbolic perturbation of the
// lifting map ranked by global point index (largest index dominates), which
// makes DT(P) unique for every duplicate-free input.
#pragma once
#include <cstdint>

namespace gdt {

// Per translation unit (no relocatable device code): each unit that uses the
// predicates exposes its own reader of these two words.  g_range_error counts
// exact evaluations that exceeded the widest integer format; it is never
// reset, so a caller compares its value before and after its own work (with
// several contexts at once an increase may come from another one: the error
// is then reported conservatively).
static __device__ unsigned long long g_exact_calls;
static __device__ int g_range_error;

// ---------------------------------------------------------------- filter
constexpr double TINY_PERM = 1e-270;   // below this, underflow could break the relative bound
constexpr double HUGE_PERM = 1e290;

static __device__ __forceinline__ int filt_sign(double det, double perm, double C) {
  if (!(perm > TINY_PERM && perm < HUGE_PERM)) return 0;
  double bound = C * perm;
  if (det > bound) return 1;
  if (det < -bound) return -1;
  return 0;
}

// ---------------------------------------------------------------- exact ints
template <int NL>
struct XI {
  uint64_t w[NL];
};

template <int NL>
static __device__ __forceinline__ void xi_zero(XI<NL>& r) {
#pragma unroll
  for (int i = 0; i < NL; i++) r.w[i] = 0;
}

template <int NL>
static __device__ __forceinline__ void xi_add(XI<NL>& r, const XI<NL>& a, const XI<NL>& b) {
  unsigned long long c = 0;
#pragma unroll
  for (int i = 0; i < NL; i++) {
    unsigned long long s = a.w[i] + b.w[i];
    unsigned long long c1 = s < a.w[i];
    unsigned long long s2 = s + c;
    unsigned long long c2 = s2 < s;
    r.w[i] = s2;
    c = c1 | c2;
  }
}

template <int NL>
static __device__ __forceinline__ void xi_neg(XI<NL>& r, const XI<NL>& a) {
  unsigned long long c = 1;
#pragma unroll
  for (int i = 0; i < NL; i++) {
    unsigned long long v = ~a.w[i];
    unsigned long long s = v + c;
    c = (s < v) ? 1ull : 0ull;
    r.w[i] = s;
  }
}

template <int NL>
static __device__ __forceinline__ void xi_sub(XI<NL>& r, const XI<NL>& a, const XI<NL>& b) {
  XI<NL> nb;
  xi_neg(nb, b);
  xi_add(r, a, nb);
}

// r = a * b mod 2^(64 NL); r must not alias a or b.
template <int NL>
__device__ __noinline__ void xi_mul(XI<NL>& r, const XI<NL>& a, const XI<NL>& b) {
  for (int i = 0; i < NL; i++) r.w[i] = 0;
  for (int i = 0; i < NL; i++) {
    unsigned long long carry = 0;
    uint64_t ai = a.w[i];
    for (int j = 0; i + j < NL; j++) {
      uint64_t lo = ai * b.w[j];
      uint64_t hi = __umul64hi(ai, b.w[j]);
      uint64_t t = r.w[i + j] + lo;
      hi += (t < lo);
      uint64_t t2 = t + carry;
      hi += (t2 < t);
      r.w[i + j] = t2;
      carry = hi;
    }
  }
}

template <int NL>
static __device__ __forceinline__ int xi_sign(const XI<NL>& a) {
  if ((int64_t)a.w[NL - 1] < 0) return -1;
  uint64_t o = 0;
#pragma unroll
  for (int i = 0; i < NL; i++) o |= a.w[i];
  return o ? 1 : 0;
}

// Decompose a finite double as m * 2^e with m a nonnegative integer < 2^53.
static __device__ __forceinline__ void dbl_split(double v, uint64_t& m, int& e, bool& neg) {
  uint64_t b = (uint64_t)__double_as_longlong(v);
  neg = (b >> 63) != 0;
  int E = (int)((b >> 52) & 0x7FF);
  m = b & ((1ull << 52) - 1);
  if (E == 0) {
    e = -1074;
  } else {
    m |= (1ull << 52);
    e = E - 1075;
  }
}

// r = v * 2^(-emin) exactly (v is a multiple of 2^emin).
template <int NL>
static __device__ __forceinline__ void xi_from_double(XI<NL>& r, double v, int emin) {
  xi_zero(r);
  uint64_t m; int e; bool neg;
  dbl_split(v, m, e, neg);
  if (m == 0) return;
  int sh = e - emin;
  if (sh < 0) { m >>= (-sh); sh = 0; }
  int limb = sh >> 6, bit = sh & 63;
  r.w[limb] = m << bit;
  if (bit && limb + 1 < NL) r.w[limb + 1] = m >> (64 - bit);
  if (neg) xi_neg(r, r);
}

// Exact difference a - b = s + t (TwoDiff; no multiplication, so FMA
// contraction cannot touch it).
static __device__ __forceinline__ void two_diff(double a, double b, double& s, double& t) {
  s = __dsub_rn(a, b);
  double bv = __dsub_rn(a, s);
  double av = __dadd_rn(s, bv);
  double br = __dsub_rn(bv, b);
  double ar = __dsub_rn(a, av);
  t = __dadd_rn(ar, br);
}

// Scale analysis over a list of doubles: lowest set bit (emin) and the
// number of magnitude bits above it.
struct Scale {
  int emin, emax;
};
static __device__ __forceinline__ void scale_init(Scale& s) { s.emin = 1 << 20; s.emax = -(1 << 20); }
static __device__ __forceinline__ void scale_add(Scale& s, double v) {
  uint64_t m; int e; bool neg;
  dbl_split(v, m, e, neg);
  if (m == 0) return;
  int lo = e + __ffsll((long long)m) - 1;
  int hi = e + 63 - __clzll((long long)m);
  s.emin = min(s.emin, lo);
  s.emax = max(s.emax, hi);
}
// Limb count for a polynomial of degree `deg` in differences whose parts
// have at most B = emax - emin + 1 bits: each difference (s + t) has at most
// B + 1 bits; products and sums of at most 2^6 monomials add deg*(B+1) + 6
// bits, plus a sign bit.
static __device__ __forceinline__ int limbs_for(const Scale& s, int deg) {
  if (s.emin > s.emax) return 1;   // everything is zero
  int B = s.emax - s.emin + 1;
  int bits = deg * (B + 2) + 16;
  return (bits + 63) / 64;
}

// ---------------------------------------------------------------- exact kernels
// Each takes the difference vectors as (s, t) pairs already scaled-checked.
// Vectors are stored as d[row][comp][0/1].

template <int NL>
static __device__ __forceinline__ void xi_diff(XI<NL>& r, const double* st, int emin) {
  XI<NL> a, b;
  xi_from_double(a, st[0], emin);
  xi_from_double(b, st[1], emin);
  xi_add(r, a, b);
}

template <int NL>
static __device__ __noinline__ int ex_orient(int D, const double* dv, int emin) {
  // dv: D rows x D comps x 2 doubles, det of the D x D matrix
  XI<NL> m[3][3];
  for (int i = 0; i < D; i++)
    for (int c = 0; c < D; c++) xi_diff(m[i][c], dv + (i * 3 + c) * 2, emin);
  XI<NL> r, t1, t2;
  if (D == 2) {
    xi_mul(t1, m[0][0], m[1][1]);
    xi_mul(t2, m[0][1], m[1][0]);
    xi_sub(r, t1, t2);
    return xi_sign(r);
  }
  XI<NL> acc, mn;
  xi_zero(acc);
  for (int j = 0; j < 3; j++) {
    int c1 = (j + 1) % 3, c2 = (j + 2) % 3;
    xi_mul(t1, m[1][c1], m[2][c2]);
    xi_mul(t2, m[1][c2], m[2][c1]);
    xi_sub(mn, t1, t2);           // cyclic cofactor: sign already folded in
    xi_mul(t1, m[0][j], mn);
    xi_add(acc, acc, t1);
  }
  return xi_sign(acc);
}

// rows: (r_i, |r_i|^2) for i = 0..D; returns (-1)^D det.
template <int NL>
static __device__ __noinline__ int ex_insphere(int D, const double* dv, int emin) {
  XI<NL> m[4][3], l[4], t1, t2;
  for (int i = 0; i <= D; i++) {
    xi_zero(l[i]);
    for (int c = 0; c < D; c++) {
      xi_diff(m[i][c], dv + (i * 3 + c) * 2, emin);
      xi_mul(t1, m[i][c], m[i][c]);
      xi_add(l[i], l[i], t1);
    }
  }
  XI<NL> acc;
  xi_zero(acc);
  if (D == 2) {
    // la (b x c) - lb (a x c) + lc (a x b)
    for (int i = 0; i < 3; i++) {
      int a = (i == 0) ? 1 : 0, b = (i == 2) ? 1 : 2;
      XI<NL> cr;
      xi_mul(t1, m[a][0], m[b][1]);
      xi_mul(t2, m[a][1], m[b][0]);
      xi_sub(cr, t1, t2);
      xi_mul(t1, l[i], cr);
      if (i == 1) xi_sub(acc, acc, t1); else xi_add(acc, acc, t1);
    }
    return xi_sign(acc);
  }
  // sum_i (-1)^i l_i M(rows != i), M the 3x3 determinant in row order
  for (int i = 0; i < 4; i++) {
    int r[3], k = 0;
    for (int j = 0; j < 4; j++) if (j != i) r[k++] = j;
    XI<NL> M, mn;
    xi_zero(M);
    for (int j = 0; j < 3; j++) {
      int c1 = (j + 1) % 3, c2 = (j + 2) % 3;
      xi_mul(t1, m[r[1]][c1], m[r[2]][c2]);
      xi_mul(t2, m[r[1]][c2], m[r[2]][c1]);
      xi_sub(mn, t1, t2);
      xi_mul(t1, m[r[0]][j], mn);
      xi_add(M, M, t1);
    }
    xi_mul(t1, l[i], M);
    if (i & 1) xi_sub(acc, acc, t1); else xi_add(acc, acc, t1);
  }
  return xi_sign(acc);
}

// sign of a . b for two difference vectors (2D)
template <int NL>
static __device__ __noinline__ int ex_dot2(const double* dv, int emin) {
  XI<NL> a0, a1, b0, b1, t1, t2, r;
  xi_diff(a0, dv + 0, emin); xi_diff(a1, dv + 2, emin);
  xi_diff(b0, dv + 6, emin); xi_diff(b1, dv + 8, emin);
  xi_mul(t1, a0, b0);
  xi_mul(t2, a1, b1);
  xi_add(r, t1, t2);
  return xi_sign(r);
}

template <int NL>
static __device__ __forceinline__ void xi_cross(XI<NL>* out, const XI<NL>* a, const XI<NL>* b) {
  XI<NL> t1, t2;
  for (int c = 0; c < 3; c++) {
    int c1 = (c + 1) % 3, c2 = (c + 2) % 3;
    xi_mul(t1, a[c1], b[c2]);
    xi_mul(t2, a[c2], b[c1]);
    xi_sub(out[c], t1, t2);
  }
}

// 3D, all points on one plane.  rows 0..2 = a - q, b - q, c - q.
//   mode 0: sign of [sum_cyc |a'|^2 (b' x c')] . n,  n = (b'-a') x (c'-a')
//           (> 0 iff q is inside the circumcircle of triangle abc)
//   mode 1: sign of n_x . n, where rows 3..5 hold a second triangle x
//           (in-plane orientation of x relative to abc)
template <int NL>
static __device__ __noinline__ int ex_coplanar(int mode, const double* dv, int emin) {
  XI<NL> r[6][3], t1, t2;
  int nrow = mode == 0 ? 3 : 6;
  for (int i = 0; i < nrow; i++)
    for (int c = 0; c < 3; c++) xi_diff(r[i][c], dv + (i * 3 + c) * 2, emin);
  XI<NL> e1[3], e2[3], n[3];
  for (int c = 0; c < 3; c++) { xi_sub(e1[c], r[1][c], r[0][c]); xi_sub(e2[c], r[2][c], r[0][c]); }
  xi_cross(n, e1, e2);
  XI<NL> acc;
  xi_zero(acc);
  if (mode == 0) {
    XI<NL> v[3];
    for (int c = 0; c < 3; c++) xi_zero(v[c]);
    for (int i = 0; i < 3; i++) {
      int j = (i + 1) % 3, k = (i + 2) % 3;
      XI<NL> cr[3], l;
      xi_cross(cr, r[j], r[k]);
      xi_zero(l);
      for (int c = 0; c < 3; c++) { xi_mul(t1, r[i][c], r[i][c]); xi_add(l, l, t1); }
      for (int c = 0; c < 3; c++) { xi_mul(t1, l, cr[c]); xi_add(v[c], v[c], t1); }
    }
    for (int c = 0; c < 3; c++) { xi_mul(t1, v[c], n[c]); xi_add(acc, acc, t1); }
    return xi_sign(acc);
  }
  XI<NL> f1[3], f2[3], nx[3];
  for (int c = 0; c < 3; c++) { xi_sub(f1[c], r[4][c], r[3][c]); xi_sub(f2[c], r[5][c], r[3][c]); }
  xi_cross(nx, f1, f2);
  for (int c = 0; c < 3; c++) { xi_mul(t2, nx[c], n[c]); xi_add(acc, acc, t2); }
  return xi_sign(acc);
}

// Dispatch on the required limb count.  kind: 0 orient, 1 insphere, 2 dot2,
// 3 coplanar incircle, 4 coplanar orientation.  dv holds TwoDiff pairs.
static __device__ __noinline__ int exact_dispatch(int kind, int D, const double* dv, int nvals) {
  atomicAdd(&g_exact_calls, 1ull);
  Scale s;
  scale_init(s);
  for (int i = 0; i < nvals; i++) scale_add(s, dv[i]);
  if (s.emin > s.emax) return 0;
  int deg = kind == 0 ? D : (kind == 1 ? D + 2 : (kind == 2 ? 2 : (kind == 3 ? 6 : 4)));
  int nl = limbs_for(s, deg);
  int emin = s.emin;
  if (nl <= 4) {
    switch (kind) {
      case 0: return ex_orient<4>(D, dv, emin);
      case 1: return ex_insphere<4>(D, dv, emin);
      case 2: return ex_dot2<4>(dv, emin);
      default: return ex_coplanar<4>(kind - 3, dv, emin);
    }
  } else if (nl <= 8) {
    switch (kind) {
      case 0: return ex_orient<8>(D, dv, emin);
      case 1: return ex_insphere<8>(D, dv, emin);
      case 2: return ex_dot2<8>(dv, emin);
      default: return ex_coplanar<8>(kind - 3, dv, emin);
    }
  } else if (nl <= 16) {
    switch (kind) {
      case 0: return ex_orient<16>(D, dv, emin);
      case 1: return ex_insphere<16>(D, dv, emin);
      case 2: return ex_dot2<16>(dv, emin);
      default: return ex_coplanar<16>(kind - 3, dv, emin);
    }
  }
  atomicAdd(&g_range_error, 1);
  return 1;
}

// ---------------------------------------------------------------- point types
template <int D> struct PT;
template <> struct PT<2> { using T = double2; };
template <> struct PT<3> { using T = double4_32a; };

static __device__ __forceinline__ double cx(const double2& p) { return p.x; }
static __device__ __forceinline__ double cy(const double2& p) { return p.y; }
static __device__ __forceinline__ double cz(const double2&) { return 0.0; }
static __device__ __forceinline__ double cx(const double4_32a& p) { return p.x; }
static __device__ __forceinline__ double cy(const double4_32a& p) { return p.y; }
static __device__ __forceinline__ double cz(const double4_32a& p) { return p.z; }
static __device__ __forceinline__ double comp(const double2& p, int c) { return c == 0 ? p.x : p.y; }
static __device__ __forceinline__ double comp(const double4_32a& p, int c) { return c == 0 ? p.x : (c == 1 ? p.y : p.z); }

// Build TwoDiff pairs of (P[i] - Q) for `rows` points into dv (row*3+c)*2.
template <typename P>
static __device__ __forceinline__ void diffs(double* dv, const P* pts, int rows, const P& q, int D) {
  for (int i = 0; i < rows; i++)
    for (int c = 0; c < D; c++) {
      double s, t;
      two_diff(comp(pts[i], c), comp(q, c), s, t);
      dv[(i * 3 + c) * 2] = s;
      dv[(i * 3 + c) * 2 + 1] = t;
    }
}

// ---------------------------------------------------------------- orient
static __device__ __noinline__ int orient2_exact(double2 a, double2 b, double2 c) {
  double dv[3 * 3 * 2] = {0};
  double2 rows[2] = {b, c};
  diffs(dv, rows, 2, a, 2);
  return exact_dispatch(0, 2, dv, 18);
}
static __device__ __forceinline__ int orient2(double2 a, double2 b, double2 c) {
  double bx = b.x - a.x, by = b.y - a.y, cxx = c.x - a.x, cyy = c.y - a.y;
  double det = bx * cyy - by * cxx;
  double perm = fabs(bx * cyy) + fabs(by * cxx);
  int s = filt_sign(det, perm, 1.2e-15);
  return s ? s : orient2_exact(a, b, c);
}

static __device__ __noinline__ int orient3_exact(double4_32a a, double4_32a b, double4_32a c, double4_32a d) {
  double dv[3 * 3 * 2] = {0};
  double4_32a rows[3] = {b, c, d};
  diffs(dv, rows, 3, a, 3);
  return exact_dispatch(0, 3, dv, 18);
}
static __device__ __forceinline__ int orient3(double4_32a a, double4_32a b, double4_32a c, double4_32a d) {
  double b0 = b.x - a.x, b1 = b.y - a.y, b2 = b.z - a.z;
  double c0 = c.x - a.x, c1 = c.y - a.y, c2 = c.z - a.z;
  double d0 = d.x - a.x, d1 = d.y - a.y, d2 = d.z - a.z;
  double m0 = c1 * d2 - c2 * d1, m1 = c2 * d0 - c0 * d2, m2 = c0 * d1 - c1 * d0;
  double det = b0 * m0 + b1 * m1 + b2 * m2;
  double p0 = fabs(c1 * d2) + fabs(c2 * d1), p1 = fabs(c2 * d0) + fabs(c0 * d2),
         p2 = fabs(c0 * d1) + fabs(c1 * d0);
  double perm = fabs(b0) * p0 + fabs(b1) * p1 + fabs(b2) * p2;
  int s = filt_sign(det, perm, 2.5e-15);
  return s ? s : orient3_exact(a, b, c, d);
}

// ---------------------------------------------------------------- insphere (raw)
static __device__ __noinline__ int insphere2_exact(double2 a, double2 b, double2 c, double2 q) {
  double dv[3 * 3 * 2] = {0};
  double2 rows[3] = {a, b, c};
  diffs(dv, rows, 3, q, 2);
  // fill unused third component slots with zero
  for (int i = 0; i < 3; i++) { dv[(i * 3 + 2) * 2] = 0; dv[(i * 3 + 2) * 2 + 1] = 0; }
  return exact_dispatch(1, 2, dv, 18);
}
// > 0 iff q is strictly inside the circumcircle of the positively oriented abc
static __device__ __forceinline__ int insphere2_raw(double2 a, double2 b, double2 c, double2 q) {
  double ax = a.x - q.x, ay = a.y - q.y, bx = b.x - q.x, by = b.y - q.y;
  double cx_ = c.x - q.x, cy_ = c.y - q.y;
  double la = ax * ax + ay * ay, lb = bx * bx + by * by, lc = cx_ * cx_ + cy_ * cy_;
  double m0 = bx * cy_ - by * cx_, m1 = ax * cy_ - ay * cx_, m2 = ax * by - ay * bx;
  double det = la * m0 - lb * m1 + lc * m2;
  double perm = la * (fabs(bx * cy_) + fabs(by * cx_)) + lb * (fabs(ax * cy_) + fabs(ay * cx_)) +
                lc * (fabs(ax * by) + fabs(ay * bx));
  int s = filt_sign(det, perm, 3.5e-15);
  return s ? s : insphere2_exact(a, b, c, q);
}

static __device__ __noinline__ int insphere3_exact(double4_32a a, double4_32a b, double4_32a c, double4_32a d, double4_32a q) {
  double dv[4 * 3 * 2] = {0};
  double4_32a rows[4] = {a, b, c, d};
  diffs(dv, rows, 4, q, 3);
  return exact_dispatch(1, 3, dv, 24);
}
// > 0 iff q is strictly inside the circumsphere of the positively oriented abcd
static __device__ __forceinline__ int insphere3_raw(double4_32a a, double4_32a b, double4_32a c, double4_32a d, double4_32a q) {
  double ax = a.x - q.x, ay = a.y - q.y, az = a.z - q.z;
  double bx = b.x - q.x, by = b.y - q.y, bz = b.z - q.z;
  double cxx = c.x - q.x, cyy = c.y - q.y, czz = c.z - q.z;
  double dx = d.x - q.x, dy = d.y - q.y, dz = d.z - q.z;
  double la = ax * ax + ay * ay + az * az;
  double lb = bx * bx + by * by + bz * bz;
  double lc = cxx * cxx + cyy * cyy + czz * czz;
  double ld = dx * dx + dy * dy + dz * dz;
  // 2x2 minors of the (x, y) columns and their absolute counterparts
  double ab = ax * by - ay * bx, ac = ax * cyy - ay * cxx, ad = ax * dy - ay * dx;
  double bc = bx * cyy - by * cxx, bd = bx * dy - by * dx, cd = cxx * dy - cyy * dx;
  double pab = fabs(ax * by) + fabs(ay * bx), pac = fabs(ax * cyy) + fabs(ay * cxx),
         pad = fabs(ax * dy) + fabs(ay * dx), pbc = fabs(bx * cyy) + fabs(by * cxx),
         pbd = fabs(bx * dy) + fabs(by * dx), pcd = fabs(cxx * dy) + fabs(cyy * dx);
  // 3x3 determinants M(u,v,w) = u_z*(v x w)_xy - v_z*(u x w)_xy + w_z*(u x v)_xy
  double Mbcd = bz * cd - czz * bd + dz * bc;
  double Macd = az * cd - czz * ad + dz * ac;
  double Mabd = az * bd - bz * ad + dz * ab;
  double Mabc = az * bc - bz * ac + czz * ab;
  double Pbcd = fabs(bz) * pcd + fabs(czz) * pbd + fabs(dz) * pbc;
  double Pacd = fabs(az) * pcd + fabs(czz) * pad + fabs(dz) * pac;
  double Pabd = fabs(az) * pbd + fabs(bz) * pad + fabs(dz) * pab;
  double Pabc = fabs(az) * pbc + fabs(bz) * pac + fabs(czz) * pab;
  double det = (la * Mbcd - lb * Macd) + (lc * Mabd - ld * Mabc);
  double perm = (la * Pbcd + lb * Pacd) + (lc * Pabd + ld * Pabc);
  int s = filt_sign(det, perm, 5e-15);
  return s ? s : insphere3_exact(a, b, c, d, q);
}

// ---------------------------------------------------------------- FP32 stage
// A first stage in front of the FP64 filter (GB300 issues FP32 at a far
// higher rate than FP64).  Every point carries X = fl32(fl64(x - o)) for the
// origin o of its instance and, in X.w, eta >= 2 (u32 + 2 u64) R with R the
// instance's largest |x_c - o_c| (u32 = 2^-24, u64 = 2^-53).  For two points
// of one instance the FP32 difference d = fl32(X_a - X_b) then satisfies
//   |d - d*| <= e(d) = eta + u32 |d| / (1 - u32)
// against the exact difference d* = x_a - x_b.  Write P for the permanent of
// a determinant (its monomials in absolute value) and D_i = |d_i| + e(d_i).
// Monomial by monomial, |det(d*) - det(d)| <= P(D) - P(|d|), and the FP32
// evaluation of det(d) is off by at most about 45 u32 P(|d|) (the roundings
// along one monomial); so the sign of the FP32 determinant is the exact sign
// when |det| > (P(D) - P(|d|)) + F32_C P(D).  F32_C = 1e-5 (about 168 u32)
// also covers the rounding of both permanents and of the bound itself.  Out
// of the range (F32_TINY, F32_HUGE), or when nothing is certain, the stage
// returns 0 and the FP64 filter decides.
constexpr float F32_C = 1e-5f;
constexpr float F32_TINY = 1e-25f, F32_HUGE = 1e30f;

static __device__ __forceinline__ float f32_up(float d, float eta) {
  // |d| + e(d), rounded upwards; 1.2e-7 > u32 / (1 - u32) with room for rounding
  return __fadd_ru(fabsf(d), __fadd_ru(eta, 1.2e-7f * fabsf(d)));
}
static __device__ __forceinline__ int f32_decide(float det, float pd, float p0) {
  if (!(pd > F32_TINY && pd < F32_HUGE)) return 0;
  float bound = (pd - p0) + F32_C * pd;
  if (det > bound) return 1;
  if (det < -bound) return -1;
  return 0;
}

static __device__ __forceinline__ int orient2_f(float4 a, float4 b, float4 c) {
  const float eta = a.w;
  float bx = b.x - a.x, by = b.y - a.y, cx_ = c.x - a.x, cy_ = c.y - a.y;
  float det = bx * cy_ - by * cx_;
  float p0 = fabsf(bx * cy_) + fabsf(by * cx_);
  float Bx = f32_up(bx, eta), By = f32_up(by, eta), Cx = f32_up(cx_, eta), Cy = f32_up(cy_, eta);
  float pd = Bx * Cy + By * Cx;
  return f32_decide(det, pd, p0);
}

static __device__ __forceinline__ int orient3_f(float4 a, float4 b, float4 c, float4 d) {
  const float eta = a.w;
  float b0 = b.x - a.x, b1 = b.y - a.y, b2 = b.z - a.z;
  float c0 = c.x - a.x, c1 = c.y - a.y, c2 = c.z - a.z;
  float d0 = d.x - a.x, d1 = d.y - a.y, d2 = d.z - a.z;
  float m0 = c1 * d2 - c2 * d1, m1 = c2 * d0 - c0 * d2, m2 = c0 * d1 - c1 * d0;
  float det = b0 * m0 + b1 * m1 + b2 * m2;
  float p0 = fabsf(b0) * (fabsf(c1 * d2) + fabsf(c2 * d1)) + fabsf(b1) * (fabsf(c2 * d0) + fabsf(c0 * d2)) +
             fabsf(b2) * (fabsf(c0 * d1) + fabsf(c1 * d0));
  float B0 = f32_up(b0, eta), B1 = f32_up(b1, eta), B2 = f32_up(b2, eta);
  float C0 = f32_up(c0, eta), C1 = f32_up(c1, eta), C2 = f32_up(c2, eta);
  float D0 = f32_up(d0, eta), D1 = f32_up(d1, eta), D2 = f32_up(d2, eta);
  float pd = B0 * (C1 * D2 + C2 * D1) + B1 * (C2 * D0 + C0 * D2) + B2 * (C0 * D1 + C1 * D0);
  return f32_decide(det, pd, p0);
}

// > 0: q inside the circumcircle of the positively oriented abc (0: undecided)
static __device__ __forceinline__ int insphere2_f(float4 a, float4 b, float4 c, float4 q) {
  const float eta = q.w;
  float ax = a.x - q.x, ay = a.y - q.y, bx = b.x - q.x, by = b.y - q.y, cx_ = c.x - q.x, cy_ = c.y - q.y;
  float la = ax * ax + ay * ay, lb = bx * bx + by * by, lc = cx_ * cx_ + cy_ * cy_;
  float det = la * (bx * cy_ - by * cx_) - lb * (ax * cy_ - ay * cx_) + lc * (ax * by - ay * bx);
  float p0 = la * (fabsf(bx * cy_) + fabsf(by * cx_)) + lb * (fabsf(ax * cy_) + fabsf(ay * cx_)) +
             lc * (fabsf(ax * by) + fabsf(ay * bx));
  float Ax = f32_up(ax, eta), Ay = f32_up(ay, eta), Bx = f32_up(bx, eta), By = f32_up(by, eta);
  float Cx = f32_up(cx_, eta), Cy = f32_up(cy_, eta);
  float pd = (Ax * Ax + Ay * Ay) * (Bx * Cy + By * Cx) + (Bx * Bx + By * By) * (Ax * Cy + Ay * Cx) +
             (Cx * Cx + Cy * Cy) * (Ax * By + Ay * Bx);
  return f32_decide(det, pd, p0);
}

// > 0: q inside the circumsphere of the positively oriented abcd (0: undecided)
static __device__ __forceinline__ int insphere3_f(float4 a, float4 b, float4 c, float4 d, float4 q) {
  const float eta = q.w;
  float ax = a.x - q.x, ay = a.y - q.y, az = a.z - q.z;
  float bx = b.x - q.x, by = b.y - q.y, bz = b.z - q.z;
  float cx_ = c.x - q.x, cy_ = c.y - q.y, cz_ = c.z - q.z;
  float dx = d.x - q.x, dy = d.y - q.y, dz = d.z - q.z;
  float la = ax * ax + ay * ay + az * az, lb = bx * bx + by * by + bz * bz;
  float lc = cx_ * cx_ + cy_ * cy_ + cz_ * cz_, ld = dx * dx + dy * dy + dz * dz;
  float ab = ax * by - ay * bx, ac = ax * cy_ - ay * cx_, ad = ax * dy - ay * dx;
  float bc = bx * cy_ - by * cx_, bd = bx * dy - by * dx, cd = cx_ * dy - cy_ * dx;
  float det = (la * (bz * cd - cz_ * bd + dz * bc) - lb * (az * cd - cz_ * ad + dz * ac)) +
              (lc * (az * bd - bz * ad + dz * ab) - ld * (az * bc - bz * ac + cz_ * ab));
  float pab = fabsf(ax * by) + fabsf(ay * bx), pac = fabsf(ax * cy_) + fabsf(ay * cx_);
  float pad = fabsf(ax * dy) + fabsf(ay * dx), pbc = fabsf(bx * cy_) + fabsf(by * cx_);
  float pbd = fabsf(bx * dy) + fabsf(by * dx), pcd = fabsf(cx_ * dy) + fabsf(cy_ * dx);
  float p0 = (la * (fabsf(bz) * pcd + fabsf(cz_) * pbd + fabsf(dz) * pbc) +
              lb * (fabsf(az) * pcd + fabsf(cz_) * pad + fabsf(dz) * pac)) +
             (lc * (fabsf(az) * pbd + fabsf(bz) * pad + fabsf(dz) * pab) +
              ld * (fabsf(az) * pbc + fabsf(bz) * pac + fabsf(cz_) * pab));
  float Ax = f32_up(ax, eta), Ay = f32_up(ay, eta), Az = f32_up(az, eta);
  float Bx = f32_up(bx, eta), By = f32_up(by, eta), Bz = f32_up(bz, eta);
  float Cx = f32_up(cx_, eta), Cy = f32_up(cy_, eta), Cz = f32_up(cz_, eta);
  float Dx = f32_up(dx, eta), Dy = f32_up(dy, eta), Dz = f32_up(dz, eta);
  float qab = Ax * By + Ay * Bx, qac = Ax * Cy + Ay * Cx, qad = Ax * Dy + Ay * Dx;
  float qbc = Bx * Cy + By * Cx, qbd = Bx * Dy + By * Dx, qcd = Cx * Dy + Cy * Dx;
  float pd = ((Ax * Ax + Ay * Ay + Az * Az) * (Bz * qcd + Cz * qbd + Dz * qbc) +
              (Bx * Bx + By * By + Bz * Bz) * (Az * qcd + Cz * qad + Dz * qac)) +
             ((Cx * Cx + Cy * Cy + Cz * Cz) * (Az * qbd + Bz * qad + Dz * qab) +
              (Dx * Dx + Dy * Dy + Dz * Dz) * (Az * qbc + Bz * qac + Cz * qab));
  return f32_decide(det, pd, p0);
}

// ---------------------------------------------------------------- helpers on indices
static __device__ __forceinline__ int orient_p(const double2* P, const int* v) {
  return orient2(P[v[0]], P[v[1]], P[v[2]]);
}
static __device__ __forceinline__ int orient_p(const double4_32a* P, const int* v) {
  return orient3(P[v[0]], P[v[1]], P[v[2]], P[v[3]]);
}
static __device__ __forceinline__ int insphere_raw_p(const double2* P, const int* v, int q) {
  return insphere2_raw(P[v[0]], P[v[1]], P[v[2]], P[q]);
}
static __device__ __forceinline__ int insphere_raw_p(const double4_32a* P, const int* v, int q) {
  return insphere3_raw(P[v[0]], P[v[1]], P[v[2]], P[v[3]], P[q]);
}

// Perturbed insphere of q against the positively oriented finite simplex v:
// +1 inside, -1 outside, never 0.  On an exact zero the point with the
// largest global index decides: q itself -> outside; a vertex v_i -> the
// sign of orient(v with v_i replaced by q), passing on to the next-largest
// index when that orientation vanishes too.
template <typename P>
static __device__ __noinline__ int insphere_sos_tail(const P* pts, const int* gid, const int* v, int q, int D) {
  int ids[5], slot[5];
  for (int i = 0; i <= D; i++) { ids[i] = v[i]; slot[i] = i; }
  ids[D + 1] = q; slot[D + 1] = -1;
  for (int a = 0; a < D + 2; a++)
    for (int b = a + 1; b < D + 2; b++)
      if (gid[ids[b]] > gid[ids[a]]) {
        int t = ids[a]; ids[a] = ids[b]; ids[b] = t;
        t = slot[a]; slot[a] = slot[b]; slot[b] = t;
      }
  for (int a = 0; a < D + 2; a++) {
    if (slot[a] < 0) return -1;
    int tmp[4];
    for (int i = 0; i <= D; i++) tmp[i] = v[i];
    tmp[slot[a]] = q;
    int o = orient_p(pts, tmp);
    if (o) return o;
  }
  return -1;
}

template <typename P>
static __device__ __forceinline__ int insphere_sos(const P* pts, const int* gid, const int* v, int q, int D) {
  int r = insphere_raw_p(pts, v, q);
  if (r) return r;
  return insphere_sos_tail(pts, gid, v, q, D);
}

// The same predicates with the FP32 stage first (X: the points' FP32 copies).
static __device__ __forceinline__ int orient_px(const double2* P, const float4* X, const int* v) {
  int s = orient2_f(X[v[0]], X[v[1]], X[v[2]]);
  return s ? s : orient2(P[v[0]], P[v[1]], P[v[2]]);
}
static __device__ __forceinline__ int orient_px(const double4_32a* P, const float4* X, const int* v) {
  int s = orient3_f(X[v[0]], X[v[1]], X[v[2]], X[v[3]]);
  return s ? s : orient3(P[v[0]], P[v[1]], P[v[2]], P[v[3]]);
}
static __device__ __forceinline__ int insphere_f_p(const double2*, const float4* X, const int* v, int q) {
  return insphere2_f(X[v[0]], X[v[1]], X[v[2]], X[q]);
}
static __device__ __forceinline__ int insphere_f_p(const double4_32a*, const float4* X, const int* v, int q) {
  return insphere3_f(X[v[0]], X[v[1]], X[v[2]], X[v[3]], X[q]);
}
template <typename P>
static __device__ __forceinline__ int insphere_sos_x(const P* pts, const float4* X, const int* gid, const int* v, int q,
                                                     int D) {
  int r = insphere_f_p(pts, X, v, q);
  if (r) return r;
  r = insphere_raw_p(pts, v, q);
  if (r) return r;
  return insphere_sos_tail(pts, gid, v, q, D);
}

// ---------------------------------------------------------------- ghost conflicts
// 2D: q on the line of hull edge (a, b): in conflict iff strictly between.
static __device__ __noinline__ int dot2_exact(double2 a, double2 b, double2 q) {
  double dv[3 * 3 * 2] = {0};
  double2 rows[2] = {a, b};
  diffs(dv, rows, 2, q, 2);
  return exact_dispatch(2, 2, dv, 12);
}
static __device__ __forceinline__ int dot2_sign(double2 a, double2 b, double2 q) {
  double ax = a.x - q.x, ay = a.y - q.y, bx = b.x - q.x, by = b.y - q.y;
  double det = ax * bx + ay * by;
  double perm = fabs(ax * bx) + fabs(ay * by);
  int s = filt_sign(det, perm, 1.2e-15);
  return s ? s : dot2_exact(a, b, q);
}

// 3D: q on the plane of hull facet (a, b, c).
static __device__ __noinline__ int coplanar_incircle3(double4_32a a, double4_32a b, double4_32a c, double4_32a q) {
  double dv[6 * 3 * 2] = {0};
  double4_32a rows[3] = {a, b, c};
  diffs(dv, rows, 3, q, 3);
  return exact_dispatch(3, 3, dv, 18);
}
static __device__ __noinline__ int coplanar_orient3(double4_32a a, double4_32a b, double4_32a c, double4_32a x0, double4_32a x1,
                                             double4_32a x2, double4_32a q) {
  double dv[6 * 3 * 2] = {0};
  double4_32a rows[6] = {a, b, c, x0, x1, x2};
  diffs(dv, rows, 6, q, 3);
  return exact_dispatch(4, 3, dv, 36);
}

static __device__ __noinline__ int ghost_coplanar3(const double4_32a* P, const int* gid, const int* f, int q) {
  double4_32a a = P[f[0]], b = P[f[1]], c = P[f[2]], x = P[q];
  int r = coplanar_incircle3(a, b, c, x);
  if (r) return r > 0;
  // cocircular: perturbed lifts of f and q decide (largest global index first)
  int ids[4] = {f[0], f[1], f[2], q}, slot[4] = {0, 1, 2, -1};
  for (int i = 0; i < 4; i++)
    for (int j = i + 1; j < 4; j++)
      if (gid[ids[j]] > gid[ids[i]]) {
        int t = ids[i]; ids[i] = ids[j]; ids[j] = t;
        t = slot[i]; slot[i] = slot[j]; slot[j] = t;
      }
  for (int i = 0; i < 4; i++) {
    if (slot[i] < 0) return 0;
    double4_32a t[3] = {a, b, c};
    t[slot[i]] = x;
    int o = coplanar_orient3(a, b, c, t[0], t[1], t[2], x);
    if (o) return o > 0;
  }
  return 0;
}

// Is the simplex with vertex tuple v (D+1 entries, at most one INF_V) in
// conflict with point q?  Finite: q inside the perturbed circumsphere.
// Ghost (stored so that an outside point in place of INF_V is positively
// oriented): q strictly beyond the hull facet, or on its hyperplane and
// inside the facet's own circumsphere.
static __device__ __forceinline__ bool in_conflict(const double2* P, const int* gid, const int* v, int q) {
  int g = -1;
#pragma unroll
  for (int i = 0; i < 3; i++) if (v[i] == INF_V) g = i;
  if (g < 0) return insphere_sos(P, gid, v, q, 2) > 0;
  int t[3] = {v[0], v[1], v[2]};
  t[g] = q;
  int o = orient_p(P, t);
  if (o) return o > 0;
  int a = v[(g + 1) % 3], b = v[(g + 2) % 3];
  return dot2_sign(P[a], P[b], P[q]) < 0;
}
static __device__ __forceinline__ bool in_conflict(const double4_32a* P, const int* gid, const int* v, int q) {
  int g = -1;
#pragma unroll
  for (int i = 0; i < 4; i++) if (v[i] == INF_V) g = i;
  if (g < 0) return insphere_sos(P, gid, v, q, 3) > 0;
  int t[4] = {v[0], v[1], v[2], v[3]};
  t[g] = q;
  int o = orient_p(P, t);
  if (o) return o > 0;
  int f[3], k = 0;
  for (int i = 0; i < 4; i++) if (i != g) f[k++] = v[i];
  return ghost_coplanar3(P, gid, f, q);
}

// in_conflict with the FP32 stage in front of the orientation and insphere tests.
template <typename P>
static __device__ __forceinline__ bool in_conflict_x(const P* pts, const float4* X, const int* gid, const int* v, int q,
                                                     int D) {
  int g = -1;
#pragma unroll
  for (int i = 0; i <= D; i++) if (v[i] == INF_V) g = i;
  if (g < 0) return insphere_sos_x(pts, X, gid, v, q, D) > 0;
  int t[4] = {v[0], v[1], v[2], D == 3 ? v[3] : 0};
  t[g] = q;
  int o = orient_px(pts, X, t);
  if (o) return o > 0;
  return in_conflict(pts, gid, v, q);   // q on the hull facet's hyperplane: exact path
}

// Exact sign of |p - a|^2 - |p - b|^2 (negative: a is closer).
template <int NL>
static __device__ __noinline__ int ex_closer(int D, const double* dv, int emin) {
  XI<NL> acc, t1, x;
  xi_zero(acc);
  for (int c = 0; c < D; c++) {
    xi_diff(x, dv + (0 * 3 + c) * 2, emin);
    xi_mul(t1, x, x);
    xi_add(acc, acc, t1);
    xi_diff(x, dv + (1 * 3 + c) * 2, emin);
    xi_mul(t1, x, x);
    xi_sub(acc, acc, t1);
  }
  return xi_sign(acc);
}
template <typename P>
static __device__ __noinline__ int closer_exact(P p, P a, P b, int D) {
  double dv[3 * 3 * 2] = {0};
  P rows[2] = {a, b};
  diffs(dv, rows, 2, p, D);
  Scale s;
  scale_init(s);
  for (int i = 0; i < 12; i++) scale_add(s, dv[i]);
  atomicAdd(&g_exact_calls, 1ull);
  if (s.emin > s.emax) return 0;
  int nl = limbs_for(s, 2);
  if (nl <= 4) return ex_closer<4>(D, dv, s.emin);
  if (nl <= 16) return ex_closer<16>(D, dv, s.emin);
  atomicAdd(&g_range_error, 1);
  return 0;
}
template <typename P>
static __device__ __forceinline__ int closer(P p, P a, P b, int D) {
  double da = 0, db = 0, pa = 0, pb = 0;
  for (int c = 0; c < D; c++) {
    double x = comp(a, c) - comp(p, c), y = comp(b, c) - comp(p, c);
    da += x * x; db += y * y;
  }
  pa = da; pb = db;
  double det = da - db;
  int s = filt_sign(det, pa + pb, 1.2e-15);
  return s ? s : closer_exact(p, a, b, D);
}

}  // namespace gdt
