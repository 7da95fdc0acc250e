/*
 * FP64 CPU oracle for segment / triangle-mesh intersection.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file; only the test-suite, the smoke check and the CPU-baseline
 * leg of the benchmark do.  It shares no code, header or constant with the
 * CUDA implementation.
 *
 * Compile with -O2 -ffp-contract=off (no FMA contraction: every product and
 * sum is rounded exactly where it is written), optionally -fopenmp.
 *
 * What it computes (paper: Sec. 1 problem statement, Sec. 2 Moller-Trumbore
 * test, Sec. 2.4 output modes):
 *
 *   segment  l_i : a + s d,  d = b - a,  s in [0,1]
 *   triangle j   : v0 + u e1 + v e2,  e1 = v1 - v0,  e2 = v2 - v0
 *
 *   Moller-Trumbore, division free, every quantity in double from the float
 *   inputs widened exactly:
 *     p = d x e2, det = e1 . p, s0 = a - v0, q = s0 x e1,
 *     nU = s0 . p, nV = d . q, nT = e2 . q;
 *     if det < 0 negate det, nU, nV, nT;
 *     hit  <=>  det > 0 && nU >= 0 && nV >= 0 && nU + nV <= det
 *               && nT >= 0 && nT <= det          (closed intervals)
 *     t = nT/det, u = nU/det, v = nV/det, P = a + t d, dist = t |d|.
 *   Dot products sum left to right: x.y = (x0*y0 + x1*y1) + x2*y2.
 *   Cross products: (x1*y2 - x2*y1, x2*y0 - x0*y2, x0*y1 - x1*y0).
 *
 *   boolean mode  : flag_i  = exists j hit_ij            (Sec. 1, y in {0,1})
 *   count mode    : count_i = #{ j : hit_ij }            (Sec. 2.4 intercept_count)
 *   nearest mode  : argmin_j t_ij over hits, ties to the smaller j, with
 *                   (j, t, u, v, P, dist)                (Sec. 2.4 barycentric)
 *
 *   A segment or triangle with a non-finite coordinate never hits (the paper
 *   is silent; without this rule infinities give hits with t = NaN).
 *
 *   near-degenerate segment: some triangle with det != 0 has
 *   m = min(u, v, 1-u-v, t, 1-t) in [-1e-6, 1e-6], or the segment is exactly
 *   parallel to and coplanar with a triangle whose box it touches.
 *
 * Also here: a simple CPU BVH (median split, FP64 boxes grown by a margin)
 * used only to enumerate candidates faster than brute force; the FP64 adjoint
 * of the nearest-hit outputs; a fixed-triangle FP64 evaluator for finite
 * differences; and a plain-definition LBVH build (Sec. 2: centroids,
 * quantisation, Morton codes, sort, binary radix tree, bottom-up boxes).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define NEAR_BAND 1e-6

/* ------------------------------------------------------------------ */
/* vector helpers (double)                                             */
/* ------------------------------------------------------------------ */
static void sub3(const double* x, const double* y, double* r) {
    r[0] = x[0] - y[0];
    r[1] = x[1] - y[1];
    r[2] = x[2] - y[2];
}
static double dot3(const double* x, const double* y) {
    double s = x[0] * y[0];
    s = s + x[1] * y[1];
    s = s + x[2] * y[2];
    return s;
}
static void cross3(const double* x, const double* y, double* r) {
    r[0] = x[1] * y[2] - x[2] * y[1];
    r[1] = x[2] * y[0] - x[0] * y[2];
    r[2] = x[0] * y[1] - x[1] * y[0];
}
static void widen3(const float* f, double* d) {
    d[0] = (double)f[0];
    d[1] = (double)f[1];
    d[2] = (double)f[2];
}

typedef struct {
    double det, nu, nv, nt; /* sign-normalised */
    double raw_det;         /* before normalisation */
    int hit;
} mt_t;

/* Moller-Trumbore, division free, as in the header comment. */
static void mt_test(const double* a, const double* b, const double* v0,
                    const double* v1, const double* v2, mt_t* r) {
    double d[3], e1[3], e2[3], s0[3], p[3], q[3];
    sub3(b, a, d);
    sub3(v1, v0, e1);
    sub3(v2, v0, e2);
    cross3(d, e2, p);
    double det = dot3(e1, p);
    sub3(a, v0, s0);
    cross3(s0, e1, q);
    double nu = dot3(s0, p);
    double nv = dot3(d, q);
    double nt = dot3(e2, q);
    r->raw_det = det;
    if (det < 0) {
        det = -det;
        nu = -nu;
        nv = -nv;
        nt = -nt;
    }
    r->det = det;
    r->nu = nu;
    r->nv = nv;
    r->nt = nt;
    r->hit = (det > 0) && (nu >= 0) && (nv >= 0) && (nu + nv <= det) &&
             (nt >= 0) && (nt <= det);
}

static void load_tri(const float* V, const int32_t* T, long j, double* v0,
                     double* v1, double* v2) {
    widen3(V + 3 * (long)T[3 * j + 0], v0);
    widen3(V + 3 * (long)T[3 * j + 1], v1);
    widen3(V + 3 * (long)T[3 * j + 2], v2);
}

/* Is the segment exactly parallel to the triangle plane, inside that plane,
 * and touching the triangle's box?  (coplanar-overlap part of near-degeneracy) */
static int coplanar_touch(const double* a, const double* b, const double* v0,
                          const double* v1, const double* v2) {
    double e1[3], e2[3], n[3], s0[3], s1[3];
    sub3(v1, v0, e1);
    sub3(v2, v0, e2);
    cross3(e1, e2, n);
    sub3(a, v0, s0);
    sub3(b, v0, s1);
    if (dot3(n, s0) != 0.0 || dot3(n, s1) != 0.0) return 0;
    for (int k = 0; k < 3; ++k) {
        double lo = fmin(v0[k], fmin(v1[k], v2[k]));
        double hi = fmax(v0[k], fmax(v1[k], v2[k]));
        double slo = fmin(a[k], b[k]), shi = fmax(a[k], b[k]);
        if (shi < lo || slo > hi) return 0;
    }
    return 1;
}

/* per-segment accumulator for all three modes */
typedef struct {
    int count;
    long best;
    double bt, bu, bv;
    int neardeg;
} acc_t;

static void acc_init(acc_t* s) {
    s->count = 0;
    s->best = -1;
    s->bt = s->bu = s->bv = 0.0;
    s->neardeg = 0;
}

static int finite3(const double* x) {
    return isfinite(x[0]) && isfinite(x[1]) && isfinite(x[2]);
}

static void acc_add(acc_t* s, const double* a, const double* b, const double* v0,
                    const double* v1, const double* v2, long j) {
    /* a segment or triangle with a non-finite coordinate never hits */
    if (!finite3(a) || !finite3(b) || !finite3(v0) || !finite3(v1) || !finite3(v2))
        return;
    mt_t r;
    mt_test(a, b, v0, v1, v2, &r);
    if (r.det != 0.0) {
        double t = r.nt / r.det, u = r.nu / r.det, v = r.nv / r.det;
        double w = 1.0 - u - v;
        double m = fmin(fmin(fmin(u, v), fmin(w, t)), 1.0 - t);
        if (m >= -NEAR_BAND && m <= NEAR_BAND) s->neardeg = 1;
    } else if (coplanar_touch(a, b, v0, v1, v2)) {
        s->neardeg = 1;
    }
    if (!r.hit) return;
    s->count += 1;
    double t = r.nt / r.det;
    if (s->best < 0 || t < s->bt || (t == s->bt && j < s->best)) {
        s->best = j;
        s->bt = t;
        s->bu = r.nu / r.det;
        s->bv = r.nv / r.det;
    }
}

static void acc_store(const acc_t* s, const double* a, const double* b, long i,
                      uint8_t* flag, int32_t* count, int32_t* tri, double* tuv,
                      double* point, double* dist, uint8_t* neardeg) {
    if (flag) flag[i] = (uint8_t)(s->count > 0);
    if (count) count[i] = s->count;
    if (neardeg) neardeg[i] = (uint8_t)s->neardeg;
    if (tri) tri[i] = (int32_t)s->best;
    double d[3];
    sub3(b, a, d);
    if (tuv) {
        tuv[3 * i + 0] = s->best >= 0 ? s->bt : 0.0;
        tuv[3 * i + 1] = s->best >= 0 ? s->bu : 0.0;
        tuv[3 * i + 2] = s->best >= 0 ? s->bv : 0.0;
    }
    if (point) {
        for (int k = 0; k < 3; ++k)
            point[3 * i + k] = s->best >= 0 ? a[k] + s->bt * d[k] : 0.0;
    }
    if (dist) dist[i] = s->best >= 0 ? s->bt * sqrt(dot3(d, d)) : 0.0;
}

static void set_threads(int nthreads) {
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
}

int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Single segment / triangle test, exported for the hand-built cases.
 * out5 = {hit, det, nU, nV, nT} (det.. sign-normalised). */
void orc_mt(const float* a, const float* b, const float* p0, const float* p1,
            const float* p2, double* out5) {
    double A[3], B[3], v0[3], v1[3], v2[3];
    widen3(a, A);
    widen3(b, B);
    widen3(p0, v0);
    widen3(p1, v1);
    widen3(p2, v2);
    mt_t r;
    mt_test(A, B, v0, v1, v2, &r);
    out5[0] = r.hit;
    out5[1] = r.det;
    out5[2] = r.nu;
    out5[3] = r.nv;
    out5[4] = r.nt;
}

/* Brute force over all N_t x N_r pairs.  Every output pointer may be NULL. */
int orc_brute(const float* V, long nV, const int32_t* T, long nT, const float* A,
              const float* B, long nR, int nthreads, uint8_t* flag, int32_t* count,
              int32_t* tri, double* tuv, double* point, double* dist,
              uint8_t* neardeg) {
    for (long j = 0; j < 3 * nT; ++j)
        if (T[j] < 0 || T[j] >= nV) return 1;
    set_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 64)
    for (long i = 0; i < nR; ++i) {
        double a[3], b[3], v0[3], v1[3], v2[3];
        widen3(A + 3 * i, a);
        widen3(B + 3 * i, b);
        acc_t s;
        acc_init(&s);
        for (long j = 0; j < nT; ++j) {
            load_tri(V, T, j, v0, v1, v2);
            acc_add(&s, a, b, v0, v1, v2, j);
        }
        acc_store(&s, a, b, i, flag, count, tri, tuv, point, dist, neardeg);
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* simple CPU BVH: median split on the longest centroid axis, leaves of  */
/* at most 4 triangles, FP64 boxes grown by `margin`.  Only a candidate  */
/* filter: every candidate then goes through the same mt_test.           */
/* ------------------------------------------------------------------ */
typedef struct {
    double lo[3], hi[3];
    long left, right; /* children, or -1 for a leaf */
    long first, cnt;  /* leaf range into idx[] */
} cnode_t;

typedef struct {
    cnode_t* nodes;
    long n_nodes;
    long* idx;
    long nT;
} cbvh_t;

static double* g_cent; /* qsort context (single-threaded build) */
static int g_axis;
static int cmp_cent(const void* x, const void* y) {
    long i = *(const long*)x, j = *(const long*)y;
    double ci = g_cent[3 * i + g_axis], cj = g_cent[3 * j + g_axis];
    if (ci < cj) return -1;
    if (ci > cj) return 1;
    return (i > j) - (i < j);
}

void* orc_bvh_build(const float* V, long nV, const int32_t* T, long nT, double margin) {
    (void)nV;
    cbvh_t* h = (cbvh_t*)calloc(1, sizeof(cbvh_t));
    h->nT = nT;
    h->idx = (long*)malloc(sizeof(long) * (nT > 0 ? nT : 1));
    h->nodes = (cnode_t*)malloc(sizeof(cnode_t) * (2 * (nT > 0 ? nT : 1)));
    double* cent = (double*)malloc(sizeof(double) * 3 * (nT > 0 ? nT : 1));
    double* tlo = (double*)malloc(sizeof(double) * 3 * (nT > 0 ? nT : 1));
    double* thi = (double*)malloc(sizeof(double) * 3 * (nT > 0 ? nT : 1));
    for (long j = 0; j < nT; ++j) {
        double v0[3], v1[3], v2[3];
        load_tri(V, T, j, v0, v1, v2);
        for (int k = 0; k < 3; ++k) {
            cent[3 * j + k] = (v0[k] + v1[k] + v2[k]) / 3.0;
            tlo[3 * j + k] = fmin(v0[k], fmin(v1[k], v2[k])) - margin;
            thi[3 * j + k] = fmax(v0[k], fmax(v1[k], v2[k])) + margin;
        }
        h->idx[j] = j;
    }
    if (nT == 0) {
        h->n_nodes = 0;
        free(cent); free(tlo); free(thi);
        return h;
    }
    /* explicit work stack of (node, first, cnt) */
    long cap = 2 * nT + 8;
    long* stk = (long*)malloc(sizeof(long) * 3 * cap);
    long sp = 0, nn = 1;
    stk[0] = 0; stk[1] = 0; stk[2] = nT; sp = 1;
    g_cent = cent;
    while (sp > 0) {
        --sp;
        long node = stk[3 * sp], first = stk[3 * sp + 1], cnt = stk[3 * sp + 2];
        cnode_t* nd = &h->nodes[node];
        for (int k = 0; k < 3; ++k) { nd->lo[k] = INFINITY; nd->hi[k] = -INFINITY; }
        double clo[3] = {INFINITY, INFINITY, INFINITY}, chi[3] = {-INFINITY, -INFINITY, -INFINITY};
        for (long q = first; q < first + cnt; ++q) {
            long j = h->idx[q];
            for (int k = 0; k < 3; ++k) {
                nd->lo[k] = fmin(nd->lo[k], tlo[3 * j + k]);
                nd->hi[k] = fmax(nd->hi[k], thi[3 * j + k]);
                clo[k] = fmin(clo[k], cent[3 * j + k]);
                chi[k] = fmax(chi[k], cent[3 * j + k]);
            }
        }
        if (cnt <= 4) {
            nd->left = nd->right = -1;
            nd->first = first;
            nd->cnt = cnt;
            continue;
        }
        int ax = 0;
        for (int k = 1; k < 3; ++k)
            if (chi[k] - clo[k] > chi[ax] - clo[ax]) ax = k;
        g_axis = ax;
        qsort(h->idx + first, (size_t)cnt, sizeof(long), cmp_cent);
        long half = cnt / 2;
        nd->left = nn++;
        nd->right = nn++;
        nd->first = first;
        nd->cnt = cnt;
        stk[3 * sp] = nd->left; stk[3 * sp + 1] = first; stk[3 * sp + 2] = half; ++sp;
        stk[3 * sp] = nd->right; stk[3 * sp + 1] = first + half; stk[3 * sp + 2] = cnt - half; ++sp;
    }
    h->n_nodes = nn;
    free(stk); free(cent); free(tlo); free(thi);
    return h;
}

void orc_bvh_free(void* p) {
    cbvh_t* h = (cbvh_t*)p;
    if (!h) return;
    free(h->nodes);
    free(h->idx);
    free(h);
}

long orc_bvh_nodes(void* p) { return ((cbvh_t*)p)->n_nodes; }

static int box_touch(const cnode_t* nd, const double* slo, const double* shi) {
    for (int k = 0; k < 3; ++k)
        if (shi[k] < nd->lo[k] || slo[k] > nd->hi[k]) return 0;
    return 1;
}

/* Same outputs as orc_brute, candidates enumerated by the CPU BVH: a node is
 * entered when the segment's own box touches it (node boxes already contain
 * every triangle's box grown by `margin`). */
int orc_bvh_query(void* p, const float* V, long nV, const int32_t* T, const float* A,
                  const float* B, long nR, int nthreads, uint8_t* flag, int32_t* count,
                  int32_t* tri, double* tuv, double* point, double* dist,
                  uint8_t* neardeg) {
    cbvh_t* h = (cbvh_t*)p;
    for (long j = 0; j < 3 * h->nT; ++j)
        if (T[j] < 0 || T[j] >= nV) return 1;
    set_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 64)
    for (long i = 0; i < nR; ++i) {
        double a[3], b[3], v0[3], v1[3], v2[3], slo[3], shi[3];
        widen3(A + 3 * i, a);
        widen3(B + 3 * i, b);
        for (int k = 0; k < 3; ++k) {
            slo[k] = fmin(a[k], b[k]);
            shi[k] = fmax(a[k], b[k]);
        }
        acc_t s;
        acc_init(&s);
        long stack[256];
        int sp = 0;
        if (h->n_nodes > 0) stack[sp++] = 0;
        while (sp > 0) {
            const cnode_t* nd = &h->nodes[stack[--sp]];
            if (!box_touch(nd, slo, shi)) continue;
            if (nd->left < 0) {
                for (long q = nd->first; q < nd->first + nd->cnt; ++q) {
                    long j = h->idx[q];
                    load_tri(V, T, j, v0, v1, v2);
                    acc_add(&s, a, b, v0, v1, v2, j);
                }
            } else {
                stack[sp++] = nd->left;
                stack[sp++] = nd->right;
            }
        }
        acc_store(&s, a, b, i, flag, count, tri, tuv, point, dist, neardeg);
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* nearest-hit adjoint (FP64)                                          */
/*                                                                     */
/* The hit solves a + t d = v0 + u e1 + v e2 with x = (t,u,v) and       */
/* M = [-d, e1, e2]:  M x = a - v0.  With the triangle held fixed,     */
/* outputs (P, t, u, v), P = (1-t) a + t b, and incoming gradients      */
/* gP, gt, gu, gv:                                                     */
/*   g_x    = (gt + gP.d, gu, gv)                                      */
/*   lambda = M^-T g_x                                                 */
/*          = (g_x0 (e1 x e2) + g_x1 (e2 x -d) + g_x2 (-d x e1)) / det M */
/*   dL/da  = (1-t)(gP + lambda),  dL/db = t (gP + lambda)             */
/*   dL/dv0 = -(1-u-v) lambda, dL/dv1 = -u lambda, dL/dv2 = -v lambda    */
/* (implicit differentiation of the hit equation; the paper has no     */
/* backward pass).  (t,u,v) are recomputed in FP64 from the geometry.  */
/* ------------------------------------------------------------------ */
int orc_backward(const float* V, long nV, const int32_t* T, long nT, const float* A,
                 const float* B, long nR, const int32_t* tri, const double* gP,
                 const double* gtuv, double* gV, double* gA, double* gB) {
    for (long i = 0; i < nR; ++i) {
        long j = tri[i];
        for (int k = 0; k < 3; ++k) {
            if (gA) gA[3 * i + k] = 0.0;
            if (gB) gB[3 * i + k] = 0.0;
        }
        if (j < 0) continue;
        if (j >= nT) return 1;
        double a[3], b[3], v0[3], v1[3], v2[3], d[3], e1[3], e2[3], s0[3], nd[3];
        widen3(A + 3 * i, a);
        widen3(B + 3 * i, b);
        load_tri(V, T, j, v0, v1, v2);
        sub3(b, a, d);
        sub3(v1, v0, e1);
        sub3(v2, v0, e2);
        sub3(a, v0, s0);
        nd[0] = -d[0]; nd[1] = -d[1]; nd[2] = -d[2];
        double c12[3], c20[3], c01[3];
        cross3(e1, e2, c12);
        cross3(e2, nd, c20);
        cross3(nd, e1, c01);
        double detM = dot3(nd, c12);
        if (detM == 0.0) continue;
        /* x = M^-1 (a - v0): rows of M^-1 are c12, c20, c01 over detM */
        double t = dot3(c12, s0) / detM;
        double u = dot3(c20, s0) / detM;
        double v = dot3(c01, s0) / detM;
        const double* gp = gP ? gP + 3 * i : NULL;
        double gpd = gp ? dot3(gp, d) : 0.0;
        double gx0 = (gtuv ? gtuv[3 * i + 0] : 0.0) + gpd;
        double gx1 = gtuv ? gtuv[3 * i + 1] : 0.0;
        double gx2 = gtuv ? gtuv[3 * i + 2] : 0.0;
        double lam[3];
        for (int k = 0; k < 3; ++k)
            lam[k] = (gx0 * c12[k] + gx1 * c20[k] + gx2 * c01[k]) / detM;
        double w = 1.0 - u - v;
        for (int k = 0; k < 3; ++k) {
            double gpk = gp ? gp[k] : 0.0;
            if (gA) gA[3 * i + k] = (1.0 - t) * (gpk + lam[k]);
            if (gB) gB[3 * i + k] = t * (gpk + lam[k]);
            if (gV) {
                long i0 = T[3 * j + 0], i1 = T[3 * j + 1], i2 = T[3 * j + 2];
                if (i0 < 0 || i0 >= nV || i1 < 0 || i1 >= nV || i2 < 0 || i2 >= nV) return 1;
                gV[3 * i0 + k] += -w * lam[k];
                gV[3 * i1 + k] += -u * lam[k];
                gV[3 * i2 + k] += -v * lam[k];
            }
        }
    }
    return 0;
}

/* Fixed-triangle evaluation in FP64 from FP64 inputs (finite differences):
 * for each listed segment i with triangle tri[i] >= 0, solve M x = a - v0 by
 * Cramer's rule and return (t, u, v, P).  Segments with tri < 0 give zeros. */
int orc_eval_fixed(const double* V, long nV, const int32_t* T, const double* A,
                   const double* B, long nR, const int32_t* tri, double* tuvp) {
    for (long i = 0; i < nR; ++i) {
        long j = tri[i];
        double* o = tuvp + 6 * i;
        for (int k = 0; k < 6; ++k) o[k] = 0.0;
        if (j < 0) continue;
        long i0 = T[3 * j], i1 = T[3 * j + 1], i2 = T[3 * j + 2];
        if (i0 < 0 || i0 >= nV || i1 < 0 || i1 >= nV || i2 < 0 || i2 >= nV) return 1;
        const double *a = A + 3 * i, *b = B + 3 * i;
        const double *v0 = V + 3 * i0, *v1 = V + 3 * i1, *v2 = V + 3 * i2;
        double d[3], e1[3], e2[3], s0[3], nd[3], c12[3], c20[3], c01[3];
        sub3(b, a, d);
        sub3(v1, v0, e1);
        sub3(v2, v0, e2);
        sub3(a, v0, s0);
        nd[0] = -d[0]; nd[1] = -d[1]; nd[2] = -d[2];
        cross3(e1, e2, c12);
        cross3(e2, nd, c20);
        cross3(nd, e1, c01);
        double detM = dot3(nd, c12);
        if (detM == 0.0) continue;
        double t = dot3(c12, s0) / detM;
        o[0] = t;
        o[1] = dot3(c20, s0) / detM;
        o[2] = dot3(c01, s0) / detM;
        for (int k = 0; k < 3; ++k) o[3 + k] = a[k] + t * d[k];
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* LBVH build by its plain definition (Sec. 2):                         */
/*  1. centroid c_j = ((v_a + v_b) + v_c) / 3 in float;                 */
/*  2. support interval [lo, hi] of {c_j} per axis;                     */
/*  3. q = clamp(floor(((c - lo) / (hi - lo)) * 1024), 0, 1023) in      */
/*     float (q = 0 on an axis of zero extent);                          */
/*  4. 30-bit Morton code: bit 3k+2 = bit k of qx, 3k+1 of qy, 3k of qz;  */
/*  5. sort (code, j) ascending; sorted position i gets the distinct     */
/*     64-bit key K_i = code << 32 | i;                                  */
/*  6. binary radix tree over K: the node over leaves [f, l] (f < l)     */
/*     splits after the last leaf whose key shares more leading bits     */
/*     with K_f than K_l does.  Node numbering: the root is 0, a left    */
/*     child is numbered by its last leaf, a right child by its first;   */
/*     a child range of one leaf is that leaf;                           */
/*  7. boxes: leaf = min/max of the triangle's vertices, internal =      */
/*     min/max of its children (float, exact).                           */
/* ------------------------------------------------------------------ */
static uint32_t interleave10(uint32_t x, uint32_t y, uint32_t z) {
    uint32_t c = 0;
    for (int k = 0; k < 10; ++k) {
        c |= ((x >> k) & 1u) << (3 * k + 2);
        c |= ((y >> k) & 1u) << (3 * k + 1);
        c |= ((z >> k) & 1u) << (3 * k);
    }
    return c;
}

uint32_t orc_morton3(uint32_t x, uint32_t y, uint32_t z) { return interleave10(x, y, z); }

/* Height-field variant (not in the paper, an option of the library): the
 * centroid coordinate along the height axis is left out and the two others
 * are quantised to 15 bits each, interleaved first-axis-high:
 * bit 2k+1 = bit k of the first kept axis, bit 2k = bit k of the second. */
static uint32_t interleave15x2(uint32_t x, uint32_t y) {
    uint32_t c = 0;
    for (int k = 0; k < 15; ++k) {
        c |= ((x >> k) & 1u) << (2 * k + 1);
        c |= ((y >> k) & 1u) << (2 * k);
    }
    return c;
}

uint32_t orc_morton2(uint32_t x, uint32_t y) { return interleave15x2(x, y); }

static uint64_t* g_keys;
static int cmp_key(const void* x, const void* y) {
    uint64_t a = g_keys[*(const uint32_t*)x], b = g_keys[*(const uint32_t*)y];
    return (a > b) - (a < b);
}

static int clz64(uint64_t x) {
    int n = 0;
    if (x == 0) return 64;
    while (!(x & 0x8000000000000000ull)) {
        x <<= 1;
        ++n;
    }
    return n;
}

/* outputs (all caller allocated):
 *   bounds[6]       lo xyz, hi xyz of the centroids
 *   codes[nT]       Morton code of triangle j (input order)
 *   order[nT]       sorted position -> triangle index
 *   left,right[nT-1] child of internal node: >= 0 internal index,
 *                   < 0 leaf -(pos+1)
 *   range[2(nT-1)]  first, last leaf of each internal node
 *   nbox[6(nT-1)]   internal node boxes (lo xyz, hi xyz)
 *   lbox[6 nT]      leaf boxes by sorted position                      */
/* height_axis: 0 = the paper's code over x, y, z; 1, 2, 3 = leave out x, y
 * or z (the height-field variant above). */
int orc_lbvh_h(const float* V, long nV, const int32_t* T, long nT, int height_axis,
               float* bounds, uint32_t* codes, uint32_t* order, int32_t* left, int32_t* right,
               int32_t* range, float* nbox, float* lbox) {
    if (height_axis < 0 || height_axis > 3) return 2;
    if (nT <= 0) return 0;
    for (long j = 0; j < 3 * nT; ++j)
        if (T[j] < 0 || T[j] >= nV) return 1;
    float* c = (float*)malloc(sizeof(float) * 3 * nT);
    for (long j = 0; j < nT; ++j)
        for (int k = 0; k < 3; ++k) {
            float va = V[3 * (long)T[3 * j] + k], vb = V[3 * (long)T[3 * j + 1] + k];
            float vc = V[3 * (long)T[3 * j + 2] + k];
            float s = va + vb;
            s = s + vc;
            c[3 * j + k] = s / 3.0f;
        }
    float lo[3], hi[3];
    for (int k = 0; k < 3; ++k) {
        lo[k] = c[k];
        hi[k] = c[k];
    }
    for (long j = 1; j < nT; ++j)
        for (int k = 0; k < 3; ++k) {
            if (c[3 * j + k] < lo[k]) lo[k] = c[3 * j + k];
            if (c[3 * j + k] > hi[k]) hi[k] = c[3 * j + k];
        }
    for (int k = 0; k < 3; ++k) {
        bounds[k] = lo[k];
        bounds[3 + k] = hi[k];
    }
    uint64_t* key = (uint64_t*)malloc(sizeof(uint64_t) * nT);
    const float levels = height_axis ? 32768.0f : 1024.0f;
    for (long j = 0; j < nT; ++j) {
        uint32_t q[3];
        for (int k = 0; k < 3; ++k) {
            float ext = hi[k] - lo[k];
            if (ext > 0.0f) {
                float s = (c[3 * j + k] - lo[k]) / ext;
                s = s * levels;
                float f = floorf(s);
                if (f < 0.0f) f = 0.0f;
                if (f > levels - 1.0f) f = levels - 1.0f;
                q[k] = (uint32_t)f;
            } else {
                q[k] = 0;
            }
        }
        if (height_axis == 0) {
            codes[j] = interleave10(q[0], q[1], q[2]);
        } else {
            const int a = height_axis == 1 ? 1 : 0, b = height_axis == 3 ? 1 : 2;
            codes[j] = interleave15x2(q[a], q[b]);
        }
        key[j] = ((uint64_t)codes[j] << 32) | (uint64_t)j;
        order[j] = (uint32_t)j;
    }
    g_keys = key;
    qsort(order, (size_t)nT, sizeof(uint32_t), cmp_key);
    /* distinct keys by sorted position */
    uint64_t* K = (uint64_t*)malloc(sizeof(uint64_t) * nT);
    for (long i = 0; i < nT; ++i) K[i] = ((uint64_t)codes[order[i]] << 32) | (uint64_t)i;
    for (long i = 0; i < nT; ++i) {
        long j = order[i];
        float* bx = lbox + 6 * i;
        for (int k = 0; k < 3; ++k) {
            float a0 = V[3 * (long)T[3 * j] + k], a1 = V[3 * (long)T[3 * j + 1] + k];
            float a2 = V[3 * (long)T[3 * j + 2] + k];
            float mn = a0 < a1 ? a0 : a1;
            mn = mn < a2 ? mn : a2;
            float mx = a0 > a1 ? a0 : a1;
            mx = mx > a2 ? mx : a2;
            bx[k] = mn;
            bx[3 + k] = mx;
        }
    }
    if (nT >= 2) {
        /* top-down: stack of (node index, f, l) */
        long* stk = (long*)malloc(sizeof(long) * 3 * (nT + 2));
        long sp = 0;
        stk[0] = 0; stk[1] = 0; stk[2] = nT - 1; sp = 1;
        /* post-order box pass needs children first: record visit order */
        long* visit = (long*)malloc(sizeof(long) * (nT - 1));
        long nvis = 0;
        while (sp > 0) {
            --sp;
            long node = stk[3 * sp], f = stk[3 * sp + 1], l = stk[3 * sp + 2];
            visit[nvis++] = node;
            int dfl = clz64(K[f] ^ K[l]);
            long g = f;
            for (long k = f; k < l; ++k)
                if (clz64(K[f] ^ K[k]) > dfl) g = k;
            range[2 * node] = (int32_t)f;
            range[2 * node + 1] = (int32_t)l;
            if (g == f) {
                left[node] = (int32_t)(-(f + 1));
            } else {
                left[node] = (int32_t)g;
                stk[3 * sp] = g; stk[3 * sp + 1] = f; stk[3 * sp + 2] = g; ++sp;
            }
            if (g + 1 == l) {
                right[node] = (int32_t)(-(l + 1));
            } else {
                right[node] = (int32_t)(g + 1);
                stk[3 * sp] = g + 1; stk[3 * sp + 1] = g + 1; stk[3 * sp + 2] = l; ++sp;
            }
        }
        /* children are visited after their parent: reverse order is bottom-up */
        for (long q = nvis - 1; q >= 0; --q) {
            long node = visit[q];
            const float* cb[2];
            int32_t ch[2] = {left[node], right[node]};
            for (int s = 0; s < 2; ++s)
                cb[s] = ch[s] < 0 ? lbox + 6 * (long)(-ch[s] - 1) : nbox + 6 * (long)ch[s];
            for (int k = 0; k < 3; ++k) {
                float mn = cb[0][k] < cb[1][k] ? cb[0][k] : cb[1][k];
                float mx = cb[0][3 + k] > cb[1][3 + k] ? cb[0][3 + k] : cb[1][3 + k];
                nbox[6 * node + k] = mn;
                nbox[6 * node + 3 + k] = mx;
            }
        }
        free(visit);
        free(stk);
    }
    free(K);
    free(key);
    free(c);
    return 0;
}

int orc_lbvh(const float* V, long nV, const int32_t* T, long nT, float* bounds,
             uint32_t* codes, uint32_t* order, int32_t* left, int32_t* right,
             int32_t* range, float* nbox, float* lbox) {
    return orc_lbvh_h(V, nV, T, nT, 0, bounds, codes, order, left, right, range, nbox, lbox);
}
