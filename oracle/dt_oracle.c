/*
 * dt_oracle.c -- plain CPU reference for the Delaunay triangulation (DT).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file; only the tests, the package smoke check and the benchmark's
 * CPU-baseline leg use it.  It shares no code with the CUDA implementation.
 *
 * What it computes (Sec. 2.1 of the paper): DT(P), the triangulation of the
 * convex hull of P whose vertex set is P and whose simplices have circum-
 * spheres that contain no point of P.  The paper asserts uniqueness only for
 * points in general position; here every input is made "general" by a
 * symbolic perturbation of the lifting map (each point p with global index g
 * is lifted to |p|^2 + delta_g, where delta_g dominates every delta_h with
 * h < g).  With that reading DT(P) is unique for every duplicate-free input.
 *
 * Everything here is deliberately simple:
 *   - predicates are determinants written out from their definitions,
 *     evaluated first in interval arithmetic (directed rounding) and, when the
 *     interval contains zero, exactly in big-integer arithmetic on the
 *     coordinates scaled to integers;
 *   - the triangulation is built by incremental Bowyer-Watson insertion with
 *     an explicit infinite ("ghost") vertex, so hull simplices need no
 *     bounding super-simplex;
 *   - a brute-force enumerator (every (d+1)-subset tested against every
 *     point) serves as an independent check on tiny inputs.
 */
#define _GNU_SOURCE
#include <fenv.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>


#define EXPORT __attribute__((visibility("default")))

/* ======================================================================
 * Big integers: sign-magnitude, base 2^32, little-endian limbs.
 * Capacity covers a degree-5 polynomial in doubles spanning the whole
 * float64 exponent range (5 * 2100 bits plus carries).
 * ====================================================================== */
#define BL 340
typedef struct {
    int neg;           /* 1 if negative */
    int n;             /* used limbs; 0 means zero */
    uint32_t d[BL];
} bi;

static void bi_set0(bi *r) { r->neg = 0; r->n = 0; }

static void bi_trim(bi *r) {
    while (r->n > 0 && r->d[r->n - 1] == 0) r->n--;
    if (r->n == 0) r->neg = 0;
}

static int mag_cmp(const bi *a, const bi *b) {
    if (a->n != b->n) return a->n < b->n ? -1 : 1;
    for (int i = a->n - 1; i >= 0; i--)
        if (a->d[i] != b->d[i]) return a->d[i] < b->d[i] ? -1 : 1;
    return 0;
}

/* r = |a| + |b| (r may alias neither) */
static void mag_add(bi *r, const bi *a, const bi *b) {
    int n = a->n > b->n ? a->n : b->n;
    uint64_t c = 0;
    for (int i = 0; i < n; i++) {
        uint64_t s = c;
        if (i < a->n) s += a->d[i];
        if (i < b->n) s += b->d[i];
        r->d[i] = (uint32_t)s;
        c = s >> 32;
    }
    r->n = n;
    if (c) r->d[r->n++] = (uint32_t)c;
}

/* r = |a| - |b|, requires |a| >= |b| */
static void mag_sub(bi *r, const bi *a, const bi *b) {
    int64_t br = 0;
    for (int i = 0; i < a->n; i++) {
        int64_t s = (int64_t)a->d[i] - br - (i < b->n ? (int64_t)b->d[i] : 0);
        br = 0;
        if (s < 0) { s += ((int64_t)1 << 32); br = 1; }
        r->d[i] = (uint32_t)s;
    }
    r->n = a->n;
}

/* r = a + sb * b where sb is +1 or -1; r must not alias a or b */
static void bi_addsub(bi *r, const bi *a, const bi *b, int sb) {
    int bneg = b->n ? (b->neg ^ (sb < 0)) : 0;
    if (a->neg == bneg) {
        mag_add(r, a, b);
        r->neg = a->neg;
    } else {
        int c = mag_cmp(a, b);
        if (c >= 0) { mag_sub(r, a, b); r->neg = a->neg; }
        else        { mag_sub(r, b, a); r->neg = bneg; }
    }
    bi_trim(r);
}

static void bi_mul(bi *r, const bi *a, const bi *b) {
    if (a->n == 0 || b->n == 0) { bi_set0(r); return; }
    int n = a->n + b->n;
    memset(r->d, 0, sizeof(uint32_t) * (size_t)n);
    for (int i = 0; i < a->n; i++) {
        uint64_t c = 0;
        for (int j = 0; j < b->n; j++) {
            uint64_t t = (uint64_t)a->d[i] * b->d[j] + r->d[i + j] + c;
            r->d[i + j] = (uint32_t)t;
            c = t >> 32;
        }
        r->d[i + b->n] = (uint32_t)c;
    }
    r->n = n;
    r->neg = a->neg ^ b->neg;
    bi_trim(r);
}

static int bi_sign(const bi *a) { return a->n == 0 ? 0 : (a->neg ? -1 : 1); }

/* Exponent of the lowest set bit of a nonzero finite double (x = m * 2^e,
 * m odd).  Returns a large value for zero so it never lowers the minimum. */
static int low_bit_exp(double x) {
    if (x == 0.0) return 1 << 20;
    int e;
    double f = frexp(fabs(x), &e);          /* x = f * 2^e, 0.5 <= f < 1 */
    uint64_t m = (uint64_t)ldexp(f, 53);    /* exact 53-bit integer */
    e -= 53;
    while ((m & 1u) == 0) { m >>= 1; e++; }
    return e;
}

/* r = x * 2^(-emin), exact (x must be a multiple of 2^emin). */
static void bi_from_double(bi *r, double x, int emin) {
    bi_set0(r);
    if (x == 0.0) return;
    int e;
    double f = frexp(fabs(x), &e);
    uint64_t m = (uint64_t)ldexp(f, 53);
    int sh = e - 53 - emin;                  /* >= -(trailing zeros of m) */
    while (sh < 0) { m >>= 1; sh++; }
    /* place m shifted left by sh bits */
    int limb = sh / 32, bit = sh % 32;
    memset(r->d, 0, sizeof(uint32_t) * (size_t)(limb + 4));
    unsigned __int128 v = (unsigned __int128)m << bit;
    r->d[limb] = (uint32_t)v;
    r->d[limb + 1] = (uint32_t)(v >> 32);
    r->d[limb + 2] = (uint32_t)(v >> 64);
    r->d[limb + 3] = (uint32_t)(v >> 96);
    r->n = limb + 4;
    r->neg = x < 0;
    bi_trim(r);
}

/* Determinant of an n x n big-integer matrix (n <= 4) by cofactor expansion
 * along the first row -- the textbook definition, no pivoting. */
static void bi_det(bi *out, bi *m[4][4], int n, const int *rows, const int *cols) {
    if (n == 1) { *out = *m[rows[0]][cols[0]]; return; }
    bi acc, term, minor, tmp;
    bi_set0(&acc);
    int subc[4];
    for (int j = 0; j < n; j++) {
        int k = 0;
        for (int c = 0; c < n; c++) if (c != j) subc[k++] = cols[c];
        bi_det(&minor, m, n - 1, rows + 1, subc);
        bi_mul(&term, m[rows[0]][cols[j]], &minor);
        bi_addsub(&tmp, &acc, &term, (j % 2 == 0) ? 1 : -1);
        acc = tmp;
    }
    *out = acc;
}

/* ======================================================================
 * Interval arithmetic.  All bounds are computed with the FPU in round-up
 * mode; a lower bound is obtained as -(round_up(-(exact))).  A NaN in any
 * bound propagates so that the caller falls back to exact arithmetic.
 * ====================================================================== */
typedef struct { double lo, hi; } iv;

static inline double mx(double a, double b) { return (a != a || b != b) ? NAN : (a > b ? a : b); }
static inline double mn(double a, double b) { return (a != a || b != b) ? NAN : (a < b ? a : b); }

static inline iv iv_pt(double x) { iv r; r.lo = x; r.hi = x; return r; }
static inline iv iv_add(iv a, iv b) { iv r; r.hi = a.hi + b.hi; r.lo = -((-a.lo) - b.lo); return r; }
static inline iv iv_sub(iv a, iv b) { iv r; r.hi = a.hi - b.lo; r.lo = -(b.hi - a.lo); return r; }
static inline iv iv_neg(iv a) { iv r; r.lo = -a.hi; r.hi = -a.lo; return r; }
static inline iv iv_mul(iv a, iv b) {
    double h = mx(mx(a.lo * b.lo, a.lo * b.hi), mx(a.hi * b.lo, a.hi * b.hi));
    double l = mn(mn(-((-a.lo) * b.lo), -((-a.lo) * b.hi)),
                  mn(-((-a.hi) * b.lo), -((-a.hi) * b.hi)));
    iv r; r.lo = l; r.hi = h; return r;
}

static iv iv_det(iv m[4][4], int n, const int *rows, const int *cols) {
    if (n == 1) return m[rows[0]][cols[0]];
    iv acc = iv_pt(0.0);
    int subc[4];
    for (int j = 0; j < n; j++) {
        int k = 0;
        for (int c = 0; c < n; c++) if (c != j) subc[k++] = cols[c];
        iv t = iv_mul(m[rows[0]][cols[j]], iv_det(m, n - 1, rows + 1, subc));
        acc = (j % 2 == 0) ? iv_add(acc, t) : iv_sub(acc, t);
    }
    return acc;
}

/* ======================================================================
 * The predicate determinants.  `kind` selects the matrix:
 *   ORIENT  (npts = D+1): rows p_i - p_0, i = 1..D                 (D x D)
 *   INSPH   (npts = D+2): rows (p_i - q, |p_i - q|^2), i = 0..D,
 *                         q = the last point                        (D+1 x D+1)
 *   DOT2    (npts = 3, D = 2): (a - q).(b - q), a 1x1 "matrix"
 * Returned value is the sign of the determinant (times (-1)^D for INSPH,
 * so that INSPH > 0 means "q strictly inside the circumsphere of the
 * positively oriented simplex p_0..p_D").
 * ====================================================================== */
enum { K_ORIENT = 0, K_INSPH = 1, K_DOT2 = 2 };

__attribute__((noinline))
static int filter_sign(int kind, int D, const double *const *p) {
    iv m[4][4];
    int n;
    if (kind == K_ORIENT) {
        n = D;
        for (int i = 0; i < D; i++)
            for (int c = 0; c < D; c++)
                m[i][c] = iv_sub(iv_pt(p[i + 1][c]), iv_pt(p[0][c]));
    } else if (kind == K_INSPH) {
        n = D + 1;
        const double *q = p[D + 1];
        for (int i = 0; i <= D; i++) {
            iv s = iv_pt(0.0);
            for (int c = 0; c < D; c++) {
                m[i][c] = iv_sub(iv_pt(p[i][c]), iv_pt(q[c]));
                s = iv_add(s, iv_mul(m[i][c], m[i][c]));
            }
            m[i][D] = s;
        }
    } else {
        n = 1;
        iv s = iv_pt(0.0);
        for (int c = 0; c < 2; c++)
            s = iv_add(s, iv_mul(iv_sub(iv_pt(p[0][c]), iv_pt(p[2][c])),
                                 iv_sub(iv_pt(p[1][c]), iv_pt(p[2][c]))));
        m[0][0] = s;
    }
    int rows[4] = {0, 1, 2, 3}, cols[4] = {0, 1, 2, 3};
    iv d = iv_det(m, n, rows, cols);
    if (kind == K_INSPH && (D & 1)) d = iv_neg(d);
    if (d.lo > 0) return 1;
    if (d.hi < 0) return -1;
    return 0; /* undecided (or NaN) */
}

static long g_exact_calls = 0;
static int64_t g_dbg[4];
EXPORT int64_t or_debug(int i) { return g_dbg[i]; }

static int exact_sign(int kind, int D, const double *const *p, int npts) {
    g_exact_calls++;
    int emin = 1 << 20;
    for (int i = 0; i < npts; i++)
        for (int c = 0; c < D; c++) {
            int e = low_bit_exp(p[i][c]);
            if (e < emin) emin = e;
        }
    if (emin == (1 << 20)) emin = 0;
    static bi X[5][3];
    static bi store[4][4];
    bi *m[4][4];
    for (int i = 0; i < npts; i++)
        for (int c = 0; c < D; c++) bi_from_double(&X[i][c], p[i][c], emin);
    int n;
    bi t1, t2;
    if (kind == K_ORIENT) {
        n = D;
        for (int i = 0; i < D; i++)
            for (int c = 0; c < D; c++) {
                bi_addsub(&store[i][c], &X[i + 1][c], &X[0][c], -1);
                m[i][c] = &store[i][c];
            }
    } else if (kind == K_INSPH) {
        n = D + 1;
        for (int i = 0; i <= D; i++) {
            bi s; bi_set0(&s);
            for (int c = 0; c < D; c++) {
                bi_addsub(&store[i][c], &X[i][c], &X[D + 1][c], -1);
                m[i][c] = &store[i][c];
                bi_mul(&t1, &store[i][c], &store[i][c]);
                bi_addsub(&t2, &s, &t1, 1);
                s = t2;
            }
            store[i][D] = s;
            m[i][D] = &store[i][D];
        }
    } else {
        n = 1;
        bi s; bi_set0(&s);
        for (int c = 0; c < 2; c++) {
            bi a, b;
            bi_addsub(&a, &X[0][c], &X[2][c], -1);
            bi_addsub(&b, &X[1][c], &X[2][c], -1);
            bi_mul(&t1, &a, &b);
            bi_addsub(&t2, &s, &t1, 1);
            s = t2;
        }
        store[0][0] = s;
        m[0][0] = &store[0][0];
    }
    int rows[4] = {0, 1, 2, 3}, cols[4] = {0, 1, 2, 3};
    bi d;
    bi_det(&d, m, n, rows, cols);
    int s = bi_sign(&d);
    if (kind == K_INSPH && (D & 1)) s = -s;
    return s;
}

static int pred_sign(int kind, int D, const double *const *p, int npts) {
    int old = fegetround();
    fesetround(FE_UPWARD);
    int s = filter_sign(kind, D, p);
    fesetround(old);
    if (s) return s;
    return exact_sign(kind, D, p, npts);
}

/* ======================================================================
 * Triangulation state.  Vertex indices are local (0..n-1); -1 is the
 * infinite vertex; a dead simplex has v[0] == -2.  nb[s*(D+1)+i] is the
 * simplex across the facet opposite v[s*(D+1)+i].
 * Orientation: finite simplices have orient > 0; a ghost simplex is stored
 * so that putting any point strictly outside its hull facet in place of the
 * infinite vertex gives orient > 0.
 * ====================================================================== */
typedef struct {
    int D;
    int64_t n;
    const double *P;       /* n x D */
    const int64_t *gid;    /* global index used by the perturbation */
    int32_t *v, *nb;
    int64_t cap, ns;
    int32_t *freel; int64_t nfree, capfree;
    int32_t *stamp;        /* per-simplex visit stamp */
    int error;
} tri_t;

static inline const double *PT(const tri_t *T, int32_t i) { return T->P + (int64_t)i * T->D; }

static int orient_idx(const tri_t *T, const int32_t *ix) {
    const double *p[4];
    for (int i = 0; i <= T->D; i++) p[i] = PT(T, ix[i]);
    return pred_sign(K_ORIENT, T->D, p, T->D + 1);
}

/* Perturbed insphere: +1 if q is inside the circumsphere of the positively
 * oriented finite simplex s[0..D], -1 otherwise.  Never 0.
 * When the exact determinant vanishes, the lift of the point with the
 * largest global index decides: if it is q, q is outside; if it is a vertex
 * s_i, the answer is the sign of the barycentric coordinate of q w.r.t. s_i,
 * i.e. orient(s with s_i replaced by q); a zero there passes the decision to
 * the next-largest global index. */
static int insphere_sos(const tri_t *T, const int32_t *s, int32_t q) {
    const double *p[5];
    int D = T->D;
    for (int i = 0; i <= D; i++) p[i] = PT(T, s[i]);
    p[D + 1] = PT(T, q);
    int r = pred_sign(K_INSPH, D, p, D + 2);
    if (r) return r;
    /* order the D+2 points by global index, largest first */
    int32_t ids[5]; int slot[5];
    for (int i = 0; i <= D; i++) { ids[i] = s[i]; slot[i] = i; }
    ids[D + 1] = q; slot[D + 1] = -1;
    for (int a = 0; a < D + 2; a++)
        for (int b = a + 1; b < D + 2; b++)
            if (T->gid[ids[b]] > T->gid[ids[a]]) {
                int32_t t = ids[a]; ids[a] = ids[b]; ids[b] = t;
                int ts = slot[a]; slot[a] = slot[b]; slot[b] = ts;
            }
    for (int a = 0; a < D + 2; a++) {
        if (slot[a] < 0) return -1;
        int32_t tmp[4];
        for (int i = 0; i <= D; i++) tmp[i] = s[i];
        tmp[slot[a]] = q;
        int o = orient_idx(T, tmp);
        if (o) return o;
    }
    return -1;
}

/* q lies on the affine hull of the hull facet f (D points).  Returns 1 if q
 * is inside the facet's own (D-1)-dimensional circumsphere (perturbed the
 * same way), else 0.  D = 2: strictly between the two endpoints.  D = 3:
 * inside the circumcircle, tested through any sphere containing that circle,
 * namely the one through f and an auxiliary point off the facet's plane. */
static int ghost_coplanar_conflict(const tri_t *T, const int32_t *f, int32_t q) {
    if (T->D == 2) {
        const double *p[3] = {PT(T, f[0]), PT(T, f[1]), PT(T, q)};
        return pred_sign(K_DOT2, 2, p, 3) < 0;
    }
    const double *a = PT(T, f[0]), *b = PT(T, f[1]), *c = PT(T, f[2]), *x = PT(T, q);
    /* choose an axis k along which the facet's normal is nonzero: the
     * projection onto the other two axes is a nondegenerate triangle */
    int k = -1;
    for (int ax = 2; ax >= 0 && k < 0; ax--) {
        int u = (ax + 1) % 3, w = (ax + 2) % 3;
        double pa[2] = {a[u], a[w]}, pb[2] = {b[u], b[w]}, pc[2] = {c[u], c[w]};
        const double *pp[3] = {pa, pb, pc};
        if (pred_sign(K_ORIENT, 2, pp, 3) != 0) k = ax;
    }
    if (k < 0) { ((tri_t *)T)->error = 3; return 0; }
    double aux[3] = {a[0], a[1], a[2]};
    aux[k] = a[k] + (fabs(a[k]) + 1.0);
    const double *t4[4] = {a, b, c, aux};
    int s0 = pred_sign(K_ORIENT, 3, t4, 4);
    if (s0 == 0) { ((tri_t *)T)->error = 3; return 0; }
    const double *t5[5] = {a, b, c, aux, x};
    int r = pred_sign(K_INSPH, 3, t5, 5) * s0;
    if (r) return r > 0;
    /* cocircular: perturbed lifts of f[0..2] and q decide */
    int32_t ids[4] = {f[0], f[1], f[2], q}; int slot[4] = {0, 1, 2, -1};
    for (int i = 0; i < 4; i++)
        for (int j = i + 1; j < 4; j++)
            if (T->gid[ids[j]] > T->gid[ids[i]]) {
                int32_t t = ids[i]; ids[i] = ids[j]; ids[j] = t;
                int ts = slot[i]; slot[i] = slot[j]; slot[j] = ts;
            }
    for (int i = 0; i < 4; i++) {
        if (slot[i] < 0) return 0;
        const double *tt[4] = {a, b, c, aux};
        tt[slot[i]] = x;
        int o = pred_sign(K_ORIENT, 3, tt, 4) * s0;
        if (o) return o > 0;
    }
    return 0;
}

/* Is simplex s in conflict with point q (is q inside its perturbed
 * circumsphere; for a ghost: strictly beyond its hull facet, or on the
 * facet's hyperplane and inside the facet's circumsphere)? */
static int in_conflict(const tri_t *T, int64_t s, int32_t q) {
    int D = T->D;
    const int32_t *vv = T->v + s * (D + 1);
    int g = -1;
    for (int i = 0; i <= D; i++) if (vv[i] == -1) g = i;
    if (g < 0) return insphere_sos(T, vv, q) > 0;
    int32_t tmp[4];
    for (int i = 0; i <= D; i++) tmp[i] = vv[i];
    tmp[g] = q;
    int o = orient_idx(T, tmp);
    if (o) return o > 0;
    int32_t f[3]; int k = 0;
    for (int i = 0; i <= D; i++) if (i != g) f[k++] = vv[i];
    return ghost_coplanar_conflict(T, f, q);
}

/* ---------------- storage ---------------- */
static int64_t new_simplex(tri_t *T) {
    if (T->nfree > 0) return T->freel[--T->nfree];
    if (T->ns == T->cap) {
        int64_t nc = T->cap * 2 + 64;
        int D1 = T->D + 1;
        T->v = (int32_t *)realloc(T->v, sizeof(int32_t) * (size_t)(nc * D1));
        T->nb = (int32_t *)realloc(T->nb, sizeof(int32_t) * (size_t)(nc * D1));
        T->stamp = (int32_t *)realloc(T->stamp, sizeof(int32_t) * (size_t)nc);
        for (int64_t i = T->cap; i < nc; i++) T->stamp[i] = -1;
        T->cap = nc;
    }
    return T->ns++;
}

static void kill_simplex(tri_t *T, int64_t s) {
    T->v[s * (T->D + 1)] = -2;
    if (T->nfree == T->capfree) {
        T->capfree = T->capfree * 2 + 64;
        T->freel = (int32_t *)realloc(T->freel, sizeof(int32_t) * (size_t)T->capfree);
    }
    T->freel[T->nfree++] = (int32_t)s;
}

/* ---------------- point location: visibility walk ---------------- */
static int64_t locate(tri_t *T, int64_t start, int32_t q) {
    int D = T->D, D1 = D + 1;
    int64_t s = start;
    /* start from a finite simplex: step off a ghost through its hull facet */
    for (int i = 0; i < D1; i++)
        if (T->v[s * D1 + i] == -1) { s = T->nb[s * D1 + i]; break; }
    for (int64_t it = 0; it < 4 * T->ns + 1000; it++) {
        const int32_t *vv = T->v + s * D1;
        int ghost = 0;
        for (int i = 0; i < D1; i++) if (vv[i] == -1) ghost = 1;
        if (ghost) return s;      /* entered through its hull facet: q is beyond it */
        int moved = 0;
        for (int i = 0; i < D1; i++) {
            int32_t tmp[4];
            for (int j = 0; j < D1; j++) tmp[j] = vv[j];
            tmp[i] = q;
            if (orient_idx(T, tmp) < 0) { s = T->nb[s * D1 + i]; moved = 1; break; }
        }
        if (!moved) return s;     /* q lies in the closed simplex */
    }
    T->error = 2;
    return -1;
}

/* ---------------- Bowyer-Watson insertion ---------------- */
typedef struct { int32_t key[3]; int32_t simp; int32_t face; } ridge_t;

static int64_t *g_cav = NULL; static int64_t g_cavcap = 0;
static int64_t *g_bnd = NULL; static int64_t g_bndcap = 0;   /* packed (simplex, face) */
static ridge_t *g_rid = NULL; static int64_t g_ridcap = 0;
static int64_t *g_newt = NULL; static int64_t g_newcap = 0;
static int32_t *g_nv = NULL; static int64_t g_nvcap = 0;
static int32_t *g_outer = NULL; static int64_t g_outercap = 0;

static void grow(void **buf, int64_t *cap, int64_t need, size_t el) {
    if (need <= *cap) return;
    int64_t nc = *cap * 2 + 256;
    if (nc < need) nc = need;
    *buf = realloc(*buf, el * (size_t)nc);
    *cap = nc;
}

static int ridge_cmp(const void *x, const void *y) {
    const ridge_t *a = (const ridge_t *)x, *b = (const ridge_t *)y;
    for (int i = 0; i < 3; i++)
        if (a->key[i] != b->key[i]) return a->key[i] < b->key[i] ? -1 : 1;
    return 0;
}

/* Insert point q given a simplex `c0` in conflict with it.  Returns one of
 * the new simplices (a good start for the next walk). */
static int64_t bw_insert(tri_t *T, int64_t c0, int32_t q, int32_t stampval) {
    int D = T->D, D1 = D + 1;
    int64_t nc = 0, nbd = 0;
    grow((void **)&g_cav, &g_cavcap, 1, sizeof(int64_t));
    g_cav[nc++] = c0;
    T->stamp[c0] = stampval;
    /* breadth-first growth of the conflict region */
    for (int64_t h = 0; h < nc; h++) {
        int64_t s = g_cav[h];
        for (int i = 0; i < D1; i++) {
            int64_t t = T->nb[s * D1 + i];
            if (T->stamp[t] == stampval) continue;      /* already in the cavity */
            if (in_conflict(T, t, q)) {
                T->stamp[t] = stampval;
                grow((void **)&g_cav, &g_cavcap, nc + 1, sizeof(int64_t));
                g_cav[nc++] = t;
            } else {
                grow((void **)&g_bnd, &g_bndcap, nbd + 1, sizeof(int64_t));
                g_bnd[nbd++] = s * D1 + i;
            }
        }
    }
    /* one new simplex per boundary facet: the cavity simplex with the vertex
     * opposite that facet replaced by q (same orientation).  Vertex tuples
     * and outside neighbours are copied first, since cavity slots are reused. */
    grow((void **)&g_newt, &g_newcap, nbd, sizeof(int64_t));
    grow((void **)&g_nv, &g_nvcap, nbd * D1, sizeof(int32_t));
    grow((void **)&g_outer, &g_outercap, nbd, sizeof(int32_t));
    int32_t *nv = g_nv, *outer = g_outer;
    for (int64_t b = 0; b < nbd; b++) {
        int64_t s = g_bnd[b] / D1; int i = (int)(g_bnd[b] % D1);
        for (int j = 0; j < D1; j++) nv[b * D1 + j] = T->v[s * D1 + j];
        nv[b * D1 + i] = q;
        outer[b] = T->nb[s * D1 + i];
    }
    for (int64_t h = 0; h < nc; h++) kill_simplex(T, g_cav[h]);
    for (int64_t b = 0; b < nbd; b++) {
        int64_t ns = new_simplex(T);
        g_newt[b] = ns;
        T->stamp[ns] = -1;
        for (int j = 0; j < D1; j++) T->v[ns * D1 + j] = nv[b * D1 + j];
    }
    /* link across the boundary facet to the outside simplex */
    for (int64_t b = 0; b < nbd; b++) {
        int i = (int)(g_bnd[b] % D1);
        int64_t ns = g_newt[b], o = outer[b];
        T->nb[ns * D1 + i] = (int32_t)o;
        /* in the outside simplex, the facet shared with ns is the one whose
         * opposite vertex is not a vertex of ns */
        for (int j = 0; j < D1; j++) {
            int32_t w = T->v[o * D1 + j];
            int found = 0;
            for (int l = 0; l < D1; l++) if (T->v[ns * D1 + l] == w) found = 1;
            if (!found) { T->nb[o * D1 + j] = (int32_t)ns; break; }
        }
    }
    /* link new simplices to each other: facets through q, matched by the
     * (D-1) other vertices (the "ridge") */
    int64_t nr = 0;
    grow((void **)&g_rid, &g_ridcap, nbd * D, sizeof(ridge_t));
    for (int64_t b = 0; b < nbd; b++) {
        int i = (int)(g_bnd[b] % D1);
        int64_t ns = g_newt[b];
        for (int j = 0; j < D1; j++) {
            if (j == i) continue;
            ridge_t r; int k = 0;
            for (int l = 0; l < D1; l++) if (l != i && l != j) r.key[k++] = T->v[ns * D1 + l];
            while (k < 3) r.key[k++] = INT32_MIN;
            /* sort key */
            for (int x = 0; x < 3; x++)
                for (int y = x + 1; y < 3; y++)
                    if (r.key[y] < r.key[x]) { int32_t t = r.key[x]; r.key[x] = r.key[y]; r.key[y] = t; }
            r.simp = (int32_t)ns; r.face = j;
            g_rid[nr++] = r;
        }
    }
    qsort(g_rid, (size_t)nr, sizeof(ridge_t), ridge_cmp);
    for (int64_t a = 0; a + 1 < nr; a += 2) {
        if (ridge_cmp(&g_rid[a], &g_rid[a + 1]) != 0) { T->error = 4; break; }
        T->nb[(int64_t)g_rid[a].simp * D1 + g_rid[a].face] = g_rid[a + 1].simp;
        T->nb[(int64_t)g_rid[a + 1].simp * D1 + g_rid[a + 1].face] = g_rid[a].simp;
    }
    return nbd > 0 ? g_newt[0] : -1;
}

/* ---------------- insertion order: biased randomized rounds, Morton within ---------------- */
static uint64_t splitmix64(uint64_t x) {
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}

typedef struct { uint64_t key; int32_t idx; } ord_t;
static int ord_cmp(const void *a, const void *b) {
    const ord_t *x = (const ord_t *)a, *y = (const ord_t *)b;
    if (x->key != y->key) return x->key < y->key ? -1 : 1;
    return x->idx < y->idx ? -1 : (x->idx > y->idx);
}

static uint64_t spread_bits(uint64_t x, int D) {
    uint64_t r = 0;
    int nb = D == 2 ? 26 : 17;
    for (int b = 0; b < nb; b++) if (x & (1ull << b)) r |= 1ull << (b * D);
    return r;
}

static void insertion_order(const tri_t *T, int32_t *ord) {
    int D = T->D; int64_t n = T->n;
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t i = 0; i < n; i++)
        for (int c = 0; c < D; c++) {
            double x = T->P[i * D + c];
            if (x < lo[c]) lo[c] = x;
            if (x > hi[c]) hi[c] = x;
        }
    ord_t *o = (ord_t *)malloc(sizeof(ord_t) * (size_t)n);
    int nbits = D == 2 ? 26 : 17;
    double scale = (double)((1u << nbits) - 1);
    for (int64_t i = 0; i < n; i++) {
        /* round r: points with hash in [2^-(r+1), 2^-r) form round r; the
         * smallest rounds go first (a random sample grows by doubling) */
        uint64_t h = splitmix64((uint64_t)i ^ 0x5DEECE66Dull);
        int round = 0;
        while (round < 40 && !(h >> 63)) { h <<= 1; round++; }
        uint64_t m = 0;
        for (int c = 0; c < D; c++) {
            double w = hi[c] > lo[c] ? (T->P[i * D + c] - lo[c]) / (hi[c] - lo[c]) : 0.0;
            uint64_t qv = (uint64_t)(w * scale);
            m |= spread_bits(qv, D) << c;
        }
        int rk = 40 - round;
        o[i].key = ((uint64_t)rk << 58) | (m & ((1ull << 58) - 1));
        o[i].idx = (int32_t)i;
    }
    qsort(o, (size_t)n, sizeof(ord_t), ord_cmp);
    for (int64_t i = 0; i < n; i++) ord[i] = o[i].idx;
    free(o);
}

/* ---------------- building the triangulation ---------------- */
static void set_simplex(tri_t *T, int64_t s, const int32_t *vv) {
    for (int i = 0; i <= T->D; i++) T->v[s * (T->D + 1) + i] = vv[i];
}

/* Returns 0 on success; -1 degenerate (no D+1 affinely independent points);
 * other negative values on internal errors. */
static int build(tri_t *T) {
    int D = T->D, D1 = D + 1;
    int64_t n = T->n;
    if (n < D + 1) return -1;
    int32_t *ord = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    insertion_order(T, ord);
    /* first D+1 affinely independent points in insertion order */
    int64_t pick[4]; int np = 0;
    pick[np++] = 0;
    for (int64_t i = 1; i < n && np < D1; i++) {
        int32_t cand = ord[i];
        int ok;
        if (np == 1) ok = 1;
        else if (np == 2 && D == 3) {
            /* not collinear with the first two: some 2D projection is nondegenerate */
            ok = 0;
            for (int ax = 0; ax < 3 && !ok; ax++) {
                int u = (ax + 1) % 3, w = (ax + 2) % 3;
                const double *a = PT(T, ord[pick[0]]), *b = PT(T, ord[pick[1]]), *c = PT(T, cand);
                double pa[2] = {a[u], a[w]}, pb[2] = {b[u], b[w]}, pc[2] = {c[u], c[w]};
                const double *pp[3] = {pa, pb, pc};
                if (pred_sign(K_ORIENT, 2, pp, 3) != 0) ok = 1;
            }
        } else {
            int32_t tmp[4];
            for (int j = 0; j < np; j++) tmp[j] = ord[pick[j]];
            tmp[np] = cand;
            ok = orient_idx(T, tmp) != 0;
        }
        if (ok) pick[np++] = i;
    }
    if (np < D1) { free(ord); return -1; }
    int32_t v0[4];
    for (int j = 0; j < D1; j++) v0[j] = ord[pick[j]];
    if (orient_idx(T, v0) < 0) { int32_t t = v0[0]; v0[0] = v0[1]; v0[1] = t; }
    int64_t s0 = new_simplex(T);
    set_simplex(T, s0, v0);
    int64_t gh[4];
    for (int i = 0; i < D1; i++) {
        int32_t g[4];
        for (int j = 0; j < D1; j++) g[j] = v0[j];
        g[i] = -1;
        /* swapping two finite vertices turns "interior-positive" into the
         * ghost convention (outside point in place of -1 gives orient > 0) */
        int a = (i + 1) % D1, b = (i + 2) % D1;
        int32_t t = g[a]; g[a] = g[b]; g[b] = t;
        gh[i] = new_simplex(T);
        set_simplex(T, gh[i], g);
    }
    for (int i = 0; i < D1; i++) T->nb[s0 * D1 + i] = (int32_t)gh[i];
    /* ghost adjacency: ghost i touches s0 through its finite facet, and
     * ghost j (j != i) through the facet opposite the vertex v0[j] */
    for (int i = 0; i < D1; i++) {
        for (int j = 0; j < D1; j++) {
            int32_t w = T->v[gh[i] * D1 + j];
            if (w == -1) { T->nb[gh[i] * D1 + j] = (int32_t)s0; continue; }
            /* facet opposite w in ghost i: shared with the ghost whose -1 sits where w was in v0 */
            int other = -1;
            for (int l = 0; l < D1; l++) if (v0[l] == w) other = l;
            T->nb[gh[i] * D1 + j] = (int32_t)gh[other];
        }
    }
    int64_t last = s0;
    char *done = (char *)calloc((size_t)n, 1);
    for (int j = 0; j < D1; j++) done[v0[j]] = 1;
    int32_t stampval = 0;
    for (int64_t i = 0; i < n && !T->error; i++) {
        int32_t q = ord[i];
        if (done[q]) continue;
        int64_t c = locate(T, last, q);
        if (c < 0) break;
        /* a duplicate point would sit on a vertex of the located simplex */
        for (int j = 0; j < D1; j++) {
            int32_t w = T->v[c * D1 + j];
            if (w < 0) continue;
            int dup = 1;
            for (int cc = 0; cc < D; cc++) if (PT(T, w)[cc] != PT(T, q)[cc]) dup = 0;
            if (dup) T->error = 5;
        }
        if (T->error) break;
        if (!in_conflict(T, c, q)) { T->error = 6; g_dbg[0] = q; g_dbg[1] = c; break; }
        last = bw_insert(T, c, q, ++stampval);
        done[q] = 1;
    }
    free(done);
    free(ord);
    if (T->error == 5) return -2;
    return T->error ? -3 - T->error : 0;
}

/* ---------------- exported API ---------------- */
static int cmp_rows_D1;
static int row_cmp(const void *a, const void *b) {
    const int64_t *x = (const int64_t *)a, *y = (const int64_t *)b;
    for (int i = 0; i < cmp_rows_D1; i++)
        if (x[i] != y[i]) return x[i] < y[i] ? -1 : 1;
    return 0;
}

static void sort_small(int64_t *x, int m) {
    for (int i = 1; i < m; i++) {
        int64_t t = x[i]; int j = i - 1;
        while (j >= 0 && x[j] > t) { x[j + 1] = x[j]; j--; }
        x[j + 1] = t;
    }
}

static tri_t *g_last = NULL;

static void tri_free(tri_t *T) {
    if (!T) return;
    free(T->v); free(T->nb); free(T->freel); free(T->stamp);
    free(T);
}

/* Triangulate P (n x D, row-major) with perturbation ranks gid (or the
 * identity when gid is NULL).  Returns the number of finite simplices
 * (>= 0) or a negative error: -1 degenerate input, -2 duplicate point,
 * <= -3 internal error.  The result stays available for or_dt_fetch and
 * or_dt_fetch_mesh until the next call. */
EXPORT int64_t or_dt_build(int D, int64_t n, const double *P, const int64_t *gid) {
    tri_free(g_last);
    g_last = NULL;
    if (D != 2 && D != 3) return -3;
    tri_t *T = (tri_t *)calloc(1, sizeof(tri_t));
    T->D = D; T->n = n; T->P = P;
    int64_t *own = NULL;
    if (!gid) {
        own = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
        for (int64_t i = 0; i < n; i++) own[i] = i;
        gid = own;
    }
    T->gid = gid;
    int64_t cap0 = (D == 2 ? 3 : 8) * n + 64;
    T->cap = 0; T->ns = 0;
    T->v = NULL; T->nb = NULL; T->stamp = NULL;
    {
        int D1 = D + 1;
        T->v = (int32_t *)malloc(sizeof(int32_t) * (size_t)(cap0 * D1));
        T->nb = (int32_t *)malloc(sizeof(int32_t) * (size_t)(cap0 * D1));
        T->stamp = (int32_t *)malloc(sizeof(int32_t) * (size_t)cap0);
        for (int64_t i = 0; i < cap0; i++) T->stamp[i] = -1;
        T->cap = cap0;
    }
    int rc = build(T);
    int64_t cnt = 0;
    int D1 = D + 1;
    for (int64_t s = 0; s < T->ns; s++) {
        const int32_t *vv = T->v + s * D1;
        if (vv[0] == -2) continue;
        int fin = 1;
        for (int i = 0; i < D1; i++) if (vv[i] < 0) fin = 0;
        cnt += fin;
    }
    /* the perturbation ranks are only needed during the build */
    T->gid = NULL;
    free(own);
    g_last = T;
    if (rc < 0) return rc;
    return cnt;
}

/* Copy the finite simplices of the last build as gid tuples (or local
 * indices when gid is NULL), each tuple sorted ascending, rows sorted
 * lexicographically.  out has room for count*(D+1) int64. */
EXPORT int64_t or_dt_fetch(int64_t *out, int64_t count, const int64_t *gid) {
    tri_t *T = g_last;
    if (!T) return -1;
    int D1 = T->D + 1;
    int64_t k = 0;
    for (int64_t s = 0; s < T->ns && k < count; s++) {
        const int32_t *vv = T->v + s * D1;
        if (vv[0] == -2) continue;
        int fin = 1;
        for (int i = 0; i < D1; i++) if (vv[i] < 0) fin = 0;
        if (!fin) continue;
        for (int i = 0; i < D1; i++) out[k * D1 + i] = gid ? gid[vv[i]] : vv[i];
        sort_small(out + k * D1, D1);
        k++;
    }
    cmp_rows_D1 = D1;
    qsort(out, (size_t)k, sizeof(int64_t) * (size_t)D1, row_cmp);
    return k;
}

/* Raw mesh of the last build, including ghosts (vertex -1) and with
 * neighbour links, compacted to live simplices.  Returns the number of live
 * simplices; when v/nb are non-NULL they receive (live x (D+1)) entries. */
EXPORT int64_t or_dt_fetch_mesh(int32_t *v, int32_t *nb) {
    tri_t *T = g_last;
    if (!T) return -1;
    int D1 = T->D + 1;
    int32_t *remap = (int32_t *)malloc(sizeof(int32_t) * (size_t)(T->ns + 1));
    int64_t k = 0;
    for (int64_t s = 0; s < T->ns; s++) remap[s] = (T->v[s * D1] == -2) ? -1 : (int32_t)k++;
    if (v && nb) {
        for (int64_t s = 0; s < T->ns; s++) {
            if (remap[s] < 0) continue;
            for (int i = 0; i < D1; i++) {
                v[(int64_t)remap[s] * D1 + i] = T->v[s * D1 + i];
                nb[(int64_t)remap[s] * D1 + i] = remap[T->nb[s * D1 + i]];
            }
        }
    }
    free(remap);
    return k;
}

/* Exact sign of |p-a|^2 - |p-b|^2 (negative: a is closer). */
static int closer_sign(int D, const double *p, const double *a, const double *b) {
    /* round-to-nearest filter: each squared difference carries a relative
     * error below 4u and the sums below (D+3)u of their magnitude, so
     * 1e-12 of the magnitude bound is far above the worst case */
    double da = 0, db = 0, mag = 0;
    for (int c = 0; c < D; c++) {
        double x = p[c] - a[c], y = p[c] - b[c];
        da += x * x; db += y * y;
        mag += p[c] * p[c] + a[c] * a[c] + b[c] * b[c];
    }
    double diff = da - db;
    if (diff > 1e-12 * mag) return 1;
    if (-diff > 1e-12 * mag) return -1;
    int emin = 1 << 20;
    const double *pp[3] = {p, a, b};
    for (int i = 0; i < 3; i++)
        for (int c = 0; c < D; c++) { int e = low_bit_exp(pp[i][c]); if (e < emin) emin = e; }
    if (emin == (1 << 20)) emin = 0;
    bi acc, t1, t2, X, Y, d1;
    bi_set0(&acc);
    for (int c = 0; c < D; c++) {
        bi_from_double(&X, p[c], emin);
        bi_from_double(&Y, a[c], emin);
        bi_addsub(&d1, &X, &Y, -1);
        bi_mul(&t1, &d1, &d1);
        bi_addsub(&t2, &acc, &t1, 1); acc = t2;
        bi_from_double(&Y, b[c], emin);
        bi_addsub(&d1, &X, &Y, -1);
        bi_mul(&t1, &d1, &d1);
        bi_addsub(&t2, &acc, &t1, -1); acc = t2;
    }
    return bi_sign(&acc);
}

/* ---------------- predicates on index tuples (for tests) ---------------- */
/* kind 0: orient of (D+1) points; kind 1: perturbed insphere of D+1 simplex
 * points (any orientation is normalised first) and a query; kind 2: raw
 * (unperturbed) insphere determinant sign of D+2 points in the given order;
 * kind 3: exact sign of |p-a|^2 - |p-b|^2 (tuple = p, a, b).
 * Returns 0 on success. */
EXPORT int or_predicates(int D, int64_t n, const double *P, const int64_t *gid,
                         int kind, int64_t m, const int32_t *tuples, int8_t *out) {
    tri_t T; memset(&T, 0, sizeof(T));
    T.D = D; T.n = n; T.P = P;
    int64_t *own = NULL;
    if (!gid) {
        own = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
        for (int64_t i = 0; i < n; i++) own[i] = i;
        gid = own;
    }
    T.gid = gid;
    int w = (kind == 0) ? D + 1 : (kind == 3 ? 3 : D + 2);
    for (int64_t r = 0; r < m; r++) {
        const int32_t *t = tuples + r * w;
        if (kind == 0) {
            out[r] = (int8_t)orient_idx(&T, t);
        } else if (kind == 1) {
            int32_t s[4];
            for (int i = 0; i <= D; i++) s[i] = t[i];
            int o = orient_idx(&T, s);
            if (o == 0) { out[r] = 0; continue; }
            if (o < 0) { int32_t x = s[0]; s[0] = s[1]; s[1] = x; }
            out[r] = (int8_t)insphere_sos(&T, s, t[D + 1]);
        } else if (kind == 2) {
            const double *p[5];
            for (int i = 0; i < D + 2; i++) p[i] = PT(&T, t[i]);
            out[r] = (int8_t)pred_sign(K_INSPH, D, p, D + 2);
        } else {
            out[r] = (int8_t)closer_sign(D, PT(&T, t[0]), PT(&T, t[1]), PT(&T, t[2]));
        }
    }
    free(own);
    return 0;
}

/* Brute force: every (D+1)-subset with nonzero orientation whose perturbed
 * circumsphere contains no other point.  Tuples are returned as sorted local
 * indices, rows in lexicographic order.  Returns the count, or -1 if more
 * than `cap` simplices were found. */
EXPORT int64_t or_dt_bruteforce(int D, int64_t n, const double *P, const int64_t *gid,
                                int64_t *out, int64_t cap) {
    tri_t T; memset(&T, 0, sizeof(T));
    T.D = D; T.n = n; T.P = P;
    int64_t *own = NULL;
    if (!gid) {
        own = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
        for (int64_t i = 0; i < n; i++) own[i] = i;
        gid = own;
    }
    T.gid = gid;
    int D1 = D + 1;
    int64_t k = 0;
    int32_t idx[4];
    /* enumerate combinations i0 < i1 < ... < iD */
    for (int i = 0; i < D1; i++) idx[i] = i;
    if (n < D1) { free(own); return 0; }
    for (;;) {
        int32_t s[4];
        for (int i = 0; i < D1; i++) s[i] = idx[i];
        int o = orient_idx(&T, s);
        if (o != 0) {
            if (o < 0) { int32_t x = s[0]; s[0] = s[1]; s[1] = x; }
            int empty = 1;
            for (int64_t q = 0; q < n && empty; q++) {
                int mine = 0;
                for (int i = 0; i < D1; i++) if (idx[i] == q) mine = 1;
                if (mine) continue;
                if (insphere_sos(&T, s, (int32_t)q) > 0) empty = 0;
            }
            if (empty) {
                if (k >= cap) { free(own); return -1; }
                for (int i = 0; i < D1; i++) out[k * D1 + i] = idx[i];
                k++;
            }
        }
        /* next combination */
        int p = D;
        while (p >= 0 && idx[p] == n - D1 + p) p--;
        if (p < 0) break;
        idx[p]++;
        for (int i = p + 1; i < D1; i++) idx[i] = idx[i - 1] + 1;
    }
    free(own);
    return k;
}

/* Exact nearest site (Alg. 2, nearest-sample assignment): for each query
 * point, the site with the smallest exact squared distance, ties broken by
 * the smaller site rank.  Brute force over all sites. */
EXPORT int or_nearest(int D, int64_t nq, const double *Q, int64_t ns, const double *S,
                      const int64_t *srank, int32_t *out) {
    for (int64_t i = 0; i < nq; i++) {
        const double *p = Q + i * D;
        int64_t best = 0;
        for (int64_t j = 1; j < ns; j++) {
            int s = closer_sign(D, p, S + j * D, S + best * D);
            if (s < 0 || (s == 0 && srank[j] < srank[best])) best = j;
        }
        out[i] = (int32_t)best;
    }
    return 0;
}

EXPORT long or_exact_calls(void) { return g_exact_calls; }

/* Self-check of the rounding-mode machinery: in round-up mode the interval
 * product of [1/3,1/3] with itself must have lo < hi and must contain the
 * round-to-nearest product. */
__attribute__((noinline)) static iv selftest_ops(double t, iv *sum) {
    *sum = iv_add(iv_pt(0.1), iv_pt(0.2));
    return iv_mul(iv_pt(t), iv_pt(t));
}

EXPORT int or_interval_selftest(void) {
    volatile double third = 1.0 / 3.0;
    iv s;
    int old = fegetround();
    fesetround(FE_UPWARD);
    iv r = selftest_ops(third, &s);
    fesetround(old);
    double rn = third * third;
    double sn = 0.1 + 0.2;
    return (r.lo < r.hi) && (r.lo <= rn) && (rn <= r.hi) && (s.lo < s.hi) &&
           (s.lo <= sn) && (sn <= s.hi);
}
