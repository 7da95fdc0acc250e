// Per-segment stack traversal (arXiv 2209.02878, Sec. 3.2 bvhTraverse /
// bvhFindCollisions and Sec. 3.3 bvhIntersectionKernel), redesigned:
//  - each node holds both child boxes, so one 64-byte fetch tests both
//    children (the paper loads each child node to test its box);
//  - the boxes are tested against the segment itself with a conservative
//    slab test (the paper tests the segment's bounding box, rbxKernel);
//  - triangles are tested inline when a leaf is reached, so there is no
//    collision buffer (CollisionList / bvhInsert) and no restart logic;
//  - BOOL stops at the first crossing (as detected[rayIdx] does), COUNT
//    visits every candidate, NEAREST shrinks the segment to the best t.
#pragma once

#include "rsi_internal.cuh"

namespace rsi {

constexpr int kNoRoot = 0x7fffffff;  // empty mesh: every segment misses

struct TravOut {
    uint8_t* flag;
    int32_t* count;
    int32_t* tri;
    float* tuv;
    float* point;
    float* dist;
    int32_t* hit_idx;
    int64_t hit_cap;
    int64_t* n_hits;
    int32_t* hit_tri;
    float* hit_dist;
    float* hit_point;
    int32_t* hit_count;
};

// Counters of a STATS launch, in this order: segments, node visits, triangle
// tests, FP64 decisions, double-float refinements, stack overflows, FP64
// value recomputations.
constexpr int kStatCounters = 7;

struct TravStats {
    // refines: nearest outputs recomputed in double-float; exact: recomputed
    // with the FP64 definition (grazing crossings, out-of-range directions)
    unsigned long long visits, tests, fp64, refines, overflows, exact;
};

struct Result {
    int count;   // crossings found (BOOL: 0 / 1)
    int best;    // NEAREST: original triangle index, -1 = none
    int bpos;    // NEAREST: leaf-order position of best
    float bt, bu, bv, berr;
    double bt64;  // exact t of best when known
    bool b64;
};

// t of the FP64 definition for the triangle at leaf position pos.
static __device__ __noinline__ double exact_t(const float* A, const float* B, int64_t i,
                                       const float4* __restrict__ tris, int pos) {
    double tuv[3] = {0.0, 0.0, 0.0};
    mt64(A[3 * i], A[3 * i + 1], A[3 * i + 2], B[3 * i], B[3 * i + 1], B[3 * i + 2],
         ld4(tris + 3 * (int64_t)pos), ld4(tris + 3 * (int64_t)pos + 1),
         ld4(tris + 3 * (int64_t)pos + 2), tuv);
    return tuv[0];
}

// Test the triangles at leaf positions [first, first + cnt) and then
// [first1, first1 + cnt1) in one loop (so lanes whose leaf is either child of
// a node test together).  Returns true when BOOL found a crossing.
template <int MODE, bool STATS>
__device__ __forceinline__ bool leaf_test(const Seg& s, const float* A, const float* B, int64_t i,
                                          const float4* __restrict__ tris, int first, int cnt,
                                          int first1, int cnt1, Result& res, float& tlim,
                                          TravStats& st) {
    const int tot = cnt + cnt1;
    for (int k = 0; k < tot; ++k) {
        const int pos = k < cnt ? first + k : first1 + (k - cnt);
        const float4 a = ld4(tris + 3 * (int64_t)pos);
        const float4 b = ld4(tris + 3 * (int64_t)pos + 1);
        const float4 c = ld4(tris + 3 * (int64_t)pos + 2);
        float t = 0.f, u = 0.f, v = 0.f, err = 0.f;
        if (STATS) ++st.tests;
        int r = mt32(s, a, b, c, MODE == RSI_MODE_NEAREST, t, u, v, err);
        bool has64 = false;
        double t64 = 0.0;
        if (r == 2) {
            if (STATS) ++st.fp64;
            double tuv[3];
            r = mt64(A[3 * i], A[3 * i + 1], A[3 * i + 2], B[3 * i], B[3 * i + 1], B[3 * i + 2],
                     a, b, c, MODE == RSI_MODE_NEAREST ? tuv : nullptr);
            if (r && MODE == RSI_MODE_NEAREST) {
                t64 = tuv[0];
                t = (float)tuv[0];
                u = (float)tuv[1];
                v = (float)tuv[2];
                err = 0x1p-23f;
                has64 = true;
            }
        }
        if (!r) continue;
        if (MODE == RSI_MODE_BOOL) {
            res.count = 1;
            return true;
        }
        ++res.count;
        if (MODE == RSI_MODE_NEAREST) {
            const int j = f2i(a.w);
            bool take;
            if (res.best < 0) {
                take = true;
            } else if (t + err < res.bt - res.berr) {
                take = true;
            } else if (t - err > res.bt + res.berr) {
                take = false;
            } else {
                // intervals overlap: compare the FP64 definition's t exactly,
                // ties to the lower triangle index
                const double tn = has64 ? t64 : exact_t(A, B, i, tris, pos);
                const double tb = res.b64 ? res.bt64 : exact_t(A, B, i, tris, res.bpos);
                res.bt64 = tb;
                res.b64 = true;
                take = tn < tb || (tn == tb && j < res.best);
                t64 = tn;
                has64 = true;
            }
            if (take) {
                res.best = j;
                res.bpos = pos;
                res.bt = t;
                res.bu = u;
                res.bv = v;
                res.berr = err;
                res.b64 = has64;
                res.bt64 = t64;
                tlim = fminf(1.f, t + err);
            }
        }
    }
    return false;
}

// One 64 B node record in two 256-bit read-only loads (the record is 64 B
// aligned).
__device__ __forceinline__ void ld_node(const float4* rec, ulonglong2& q0, ulonglong2& q1,
                                        ulonglong2& q2, int4& rc) {
    unsigned long long r0, r1;
    asm("ld.global.nc.v4.u64 {%0, %1, %2, %3}, [%4];"
        : "=l"(q0.x), "=l"(q0.y), "=l"(q1.x), "=l"(q1.y)
        : "l"(rec));
    asm("ld.global.nc.v4.u64 {%0, %1, %2, %3}, [%4];"
        : "=l"(q2.x), "=l"(q2.y), "=l"(r0), "=l"(r1)
        : "l"(rec + 2));
    rc.x = (int)(unsigned)r0;
    rc.y = (int)(unsigned)(r0 >> 32);
    rc.z = (int)(unsigned)r1;
    rc.w = (int)(unsigned)(r1 >> 32);
}

// Everything one traversal launch needs (by value in registers / params).
struct TraceCtx {
    const float* A;
    const float* B;
    int64_t nR;
    int root;   // treelet node ~0, a global root slot, or kNoRoot
    int root4;  // root slot for 4-wide traversal
    const float4* nodes;
    const float4* nodes4;  // 4-wide records (see rsi_internal.cuh)
    const float4* tris;
    const float4* treelet;
    const float4* snodes;  // shared-memory copy of treelet[0..S)
    int S;
    int max_visits;
    int fetch;             // segments a warp takes from the counter at once
    const int32_t* ready;  // streamed input: chunk c of ready_chunk segments is in
    int64_t ready_chunk;   // place once ready[c] != 0 (nullptr: all in place)
    int wait_polls;        // polls of a ready flag before giving up
    const int32_t* order;  // optional processing order of the segments
    int32_t* status;
    TravOut out;
};

// One node visit of segment i: test both child boxes, test the triangles of
// child leaves, then descend (near child first, far child pushed) or pop.
// Returns true when the segment is finished (stack empty, a BOOL crossing,
// a stack overflow, or the visit bound).  TL: the tree has a top treelet
// (negative node ids, children flagged by a negative count); without one
// every node is a global slot and those tests are compiled out.
template <int MODE, int STACK, bool STATS, bool TL>
__device__ __forceinline__ bool node_step(const TraceCtx& C, const Seg& s, int64_t i, int& node,
                                          int& sp, int* stack, float& tlim, Result& res,
                                          int& visits, bool& overflow, TravStats& st) {
    if (++visits > C.max_visits) {
        atomicCAS(C.status, 0, RSI_ERR_INTERNAL);
        return true;
    }
    ulonglong2 q0, q1, q2;
    int4 rc;
    if (TL && node < 0) {
        const int k = ~node;
        if (k < C.S) {
            const ulonglong2* p = (const ulonglong2*)(C.snodes + 4 * k);
            q0 = p[0];
            q1 = p[1];
            q2 = p[2];
            rc = ((const int4*)p)[3];
        } else {
            ld_node(C.treelet + 4 * (int64_t)k, q0, q1, q2, rc);
        }
    } else {
        ld_node(C.nodes + 4 * (int64_t)node, q0, q1, q2, rc);
    }
    if (STATS) ++st.visits;
    float t0, t1;
    bool h0, h1;
    slab2(s, q0, q1, q2, tlim, h0, t0, h1, t1);
    const int r0 = rc.x, r1 = rc.y, c0 = rc.z, c1 = rc.w;
    // one loop over both leaves for BOOL and COUNT; NEAREST keeps two (its
    // merged loop measured slower: more live state across the loop)
    if (MODE == RSI_MODE_NEAREST) {
        if (h0 && c0 > 0)
            leaf_test<MODE, STATS>(s, C.A, C.B, i, C.tris, r0, c0, 0, 0, res, tlim, st);
        if (h1 && c1 > 0)
            leaf_test<MODE, STATS>(s, C.A, C.B, i, C.tris, r1, c1, 0, 0, res, tlim, st);
    } else {
        const int n0 = h0 && c0 > 0 ? c0 : 0, n1 = h1 && c1 > 0 ? c1 : 0;
        if ((n0 | n1) &&
            leaf_test<MODE, STATS>(s, C.A, C.B, i, C.tris, r0, n0, r1, n1, res, tlim, st))
            return true;
    }
    const bool g0 = h0 && c0 <= 0, g1 = h1 && c1 <= 0;
    const int x0 = TL && c0 < 0 ? ~r0 : r0, x1 = TL && c1 < 0 ? ~r1 : r1;
    if (g0 && g1) {
        if (sp >= STACK) {
            overflow = true;
            return true;
        }
        const bool near0 = t0 <= t1;
        stack[sp++] = near0 ? x1 : x0;
        node = near0 ? x0 : x1;
    } else if (g0) {
        node = x0;
    } else if (g1) {
        node = x1;
    } else {
        if (sp == 0) return true;
        node = stack[--sp];
    }
    return false;
}

// Compare-exchange of (key, value) pairs, ascending by key.
__device__ __forceinline__ void cswap(float& ka, int& va, float& kb, int& vb) {
    const bool sw = kb < ka;
    const float k = sw ? kb : ka;
    kb = sw ? ka : kb;
    ka = k;
    const int v = sw ? vb : va;
    vb = sw ? va : vb;
    va = v;
}

// One visit of a 4-wide node (the grandchildren of binary slot `node`):
// test the four child boxes, test the triangles of child leaves, continue
// with the nearest internal child and push the others farthest first.
// Returns true when the segment is finished.
template <int MODE, int STACK, bool STATS>
__device__ __forceinline__ bool node_step4(const TraceCtx& C, const Seg& s, int64_t i, int& node,
                                           int& sp, int* stack, float& tlim, Result& res,
                                           int& visits, bool& overflow, TravStats& st) {
    if (++visits > C.max_visits) {
        atomicCAS(C.status, 0, RSI_ERR_INTERNAL);
        return true;
    }
    const ulonglong2* p = (const ulonglong2*)(C.nodes4 + 8 * (int64_t)node);
    const ulonglong2 lx = __ldg(p), ly = __ldg(p + 1), lz = __ldg(p + 2);
    const ulonglong2 hx = __ldg(p + 3), hy = __ldg(p + 4), hz = __ldg(p + 5);
    const int4 rf = __ldg((const int4*)p + 6), ct = __ldg((const int4*)p + 7);
    if (STATS) ++st.visits;
    const int r[4] = {rf.x, rf.y, rf.z, rf.w};
    const int c[4] = {ct.x, ct.y, ct.z, ct.w};
    float t[4];
    bool h[4];
    // children 0,1 and 2,3 as two packed pairs (SoA words split in halves)
    slab2(s, make_ulonglong2(lx.x, ly.x), make_ulonglong2(lz.x, hx.x),
          make_ulonglong2(hy.x, hz.x), tlim, h[0], t[0], h[1], t[1]);
    slab2(s, make_ulonglong2(lx.y, ly.y), make_ulonglong2(lz.y, hx.y),
          make_ulonglong2(hy.y, hz.y), tlim, h[2], t[2], h[3], t[3]);
#pragma unroll
    for (int q = 0; q < 4; ++q)
        if (h[q] && c[q] > 0 &&
            leaf_test<MODE, STATS>(s, C.A, C.B, i, C.tris, r[q], c[q], 0, 0, res, tlim, st))
            return true;
    // internal children, sorted by entry parameter (misses keyed +inf)
    float k0 = (h[0] && c[0] == 0) ? t[0] : INFINITY, k1 = (h[1] && c[1] == 0) ? t[1] : INFINITY;
    float k2 = (h[2] && c[2] == 0) ? t[2] : INFINITY, k3 = (h[3] && c[3] == 0) ? t[3] : INFINITY;
    int v0 = r[0], v1 = r[1], v2 = r[2], v3 = r[3];
    const int n_int = (k0 < INFINITY) + (k1 < INFINITY) + (k2 < INFINITY) + (k3 < INFINITY);
    if (n_int == 0) {
        if (sp == 0) return true;
        node = stack[--sp];
        return false;
    }
    if (n_int > 1) {
        cswap(k0, v0, k1, v1);
        cswap(k2, v2, k3, v3);
        cswap(k0, v0, k2, v2);
        cswap(k1, v1, k3, v3);
        cswap(k1, v1, k2, v2);
        if (sp + n_int - 1 > STACK) {
            overflow = true;
            return true;
        }
        if (n_int > 3) stack[sp++] = v3;
        if (n_int > 2) stack[sp++] = v2;
        stack[sp++] = v1;
    } else {
        // the single internal child: move it to slot 0
        v0 = k0 < INFINITY ? v0 : k1 < INFINITY ? v1 : k2 < INFINITY ? v2 : v3;
    }
    node = v0;
    return false;
}

// Whole traversal of one segment from `root` (used for the deep-stack
// re-run).  Returns false when the stack overflowed (result incomplete).
template <int MODE, int STACK, bool STATS, bool TL>
__device__ __forceinline__ bool trace(const TraceCtx& C, const Seg& s, int64_t i, int root,
                                      Result& res, TravStats& st) {
    int stack[STACK];
    int sp = 0, node = root, visits = 0;
    float tlim = 1.f;
    bool overflow = false;
    while (!node_step<MODE, STACK, STATS, TL>(C, s, i, node, sp, stack, tlim, res, visits, overflow,
                                              st)) {
    }
    return !overflow;
}

// Deep-stack re-run for segments whose stack overflowed (a radix tree over
// 62-bit keys is at most 63 levels deep, so 64 entries always suffice), on
// binary nodes from `root`: the treelet root ~0 needs TL, a global slot not.
template <int MODE, bool STATS, bool TL>
__device__ __noinline__ void trace_deep(const TraceCtx& C, const Seg& s, int64_t i, int root,
                                        Result& res, TravStats& st) {
    res.count = 0;
    res.best = -1;
    res.b64 = false;
    trace<MODE, 64, STATS, TL>(C, s, i, root, res, st);
}

__device__ __forceinline__ void result_init(Result& r) {
    r.count = 0;
    r.best = -1;
    r.bpos = 0;
    r.bt = r.bu = r.bv = r.berr = 0.f;
    r.bt64 = 0.0;
    r.b64 = false;
}

// Nearest outputs recomputed with the FP64 definition (its operation order
// for t, u, v; the point a + t d and the distance t |d| in FP64 as well),
// rounded to FP32 and written to o[0..6] = t, u, v, P, dist.  The
// recomputations are out of line and return through the caller's local
// array: inlined, or returning a structure in registers, they cost the
// traversal loop registers (measured: a quarter slower nearest traversals).
static __device__ __noinline__ void values64(const float* A, const float* B, int64_t i,
                                             float4 v0, float4 v1, float4 v2, float* o) {
    double tuv[3] = {0.0, 0.0, 0.0};
    mt64(A[3 * i], A[3 * i + 1], A[3 * i + 2], B[3 * i], B[3 * i + 1], B[3 * i + 2], v0, v1, v2,
         tuv);
    double dd = 0.0;
    for (int k = 0; k < 3; ++k) {
        const double a = A[3 * i + k], d = __dsub_rn((double)B[3 * i + k], a);
        o[3 + k] = (float)__dadd_rn(a, __dmul_rn(tuv[0], d));
        dd = __dadd_rn(dd, __dmul_rn(d, d));
    }
    o[0] = (float)tuv[0];
    o[1] = (float)tuv[1];
    o[2] = (float)tuv[2];
    o[6] = (float)__dmul_rn(tuv[0], __dsqrt_rn(dd));
}

// (t, u, v) recomputed in double-float and rounded to FP32, written to
// tuv[0..2] (out of line; returns through the caller's local array).
static __device__ __noinline__ void values_df(const float* a3, const float* b3, float4 v0,
                                              float4 v1, float4 v2, float* tuv) {
    dfl t;
    mt_df(a3, b3, v0, v1, v2, t, tuv[1], tuv[2]);
    tuv[0] = df_float(t);
}

// Nearest outputs.  (t, u, v) keep their FP32 values when a rigorous bound
// (first the filter's, then a tighter one for this triangle) shows them, and
// the point, within the tolerance.  Otherwise they are recomputed: in
// double-float (t, u, v rounded to FP32, the point fma(t, fl(d), a)) while
// the tight bound still keeps det away from zero, the double-float error of
// t (below 2^-20 of that bound; measured: 2e-8) times |d| stays within half
// the tolerance, and |d| < 64 (so that the rounding of t and of fl(b - a),
// |d| 2u t, plus the point's own rounding stays below 0.8e-5); with the FP64
// definition where it does not (a crossing at a grazing angle, or a long
// segment), or where the segment's direction is outside the FP32 filter's
// range.
//
// Thresholds: the output tolerance is 1e-5 relative to max(1, |x|), and the
// bounds are rigorous.  u and v: their bound (which includes their FP32
// rounding) below 0.95e-5.  t: the point fma(t, fl(d), a) is off by at most
// |d| (err_t + u) (the error of t, and the rounding of fl(b - a), t <= 1)
// plus its own rounding u max(1, |P|), so err_t below
// 0.95 ((1e-5 - u) / max(1, |d|) - u) keeps the point, the distance and t
// itself within the tolerance (u = 2^-24); for |d| beyond about 160 no FP32
// t qualifies and the outputs are always recomputed.
template <bool STATS>
__device__ __forceinline__ void nearest_values(const Seg& s, const float* A, const float* B,
                                               int64_t i, const float4* __restrict__ tris,
                                               const Result& res, float& t, float& u, float& v,
                                               float P[3], float& dist, TravStats& st) {
    t = res.bt;
    u = res.bu;
    v = res.bv;
    const float dlen = sqrtf(fmaf(s.dx, s.dx, fmaf(s.dy, s.dy, s.dz * s.dz))) * 1.0001f;
    const float thresh = 0.95f * ((1e-5f - 0x1p-24f) / fmaxf(1.f, dlen) - 0x1p-24f);
    const float thresh_uv = 0.95e-5f;
    const int p = res.bpos;
    bool exact = s.fp64only;
    bool refine = !exact && res.berr > thresh;  // berr bounds t, u and v together
    if (refine) {  // tighter bounds for this one triangle first, t and (u, v) apart
        float t2, u2, v2, euv;
        const float et = mt32_tight(s, ld4(tris + 3 * (int64_t)p), ld4(tris + 3 * (int64_t)p + 1),
                                    ld4(tris + 3 * (int64_t)p + 2), t2, u2, v2, euv);
        if (et <= thresh && euv <= thresh_uv) {
            t = t2;
            u = u2;
            v = v2;
            refine = false;
        } else if (!(et < INFINITY && dlen * et <= 4.f && euv <= 4.f) || dlen >= 64.f) {
            exact = true;
        }
    }
    if (exact) {
        if (STATS) ++st.exact;
        float o[7];
        values64(A, B, i, ld4(tris + 3 * (int64_t)p), ld4(tris + 3 * (int64_t)p + 1),
                 ld4(tris + 3 * (int64_t)p + 2), o);
        t = o[0];
        u = o[1];
        v = o[2];
        P[0] = o[3];
        P[1] = o[4];
        P[2] = o[5];
        dist = o[6];
        return;
    }
    if (refine) {
        if (STATS) ++st.refines;
        const float a3[3] = {s.ax(), s.ay(), s.az()};
        const float b3[3] = {B[3 * i], B[3 * i + 1], B[3 * i + 2]};
        float tuv[3];
        values_df(a3, b3, ld4(tris + 3 * (int64_t)p), ld4(tris + 3 * (int64_t)p + 1),
                  ld4(tris + 3 * (int64_t)p + 2), tuv);
        t = tuv[0];
        u = tuv[1];
        v = tuv[2];
    }
    P[0] = fmaf(t, s.dx, s.ax());
    P[1] = fmaf(t, s.dy, s.ay());
    P[2] = fmaf(t, s.dz, s.az());
    dist = t * sqrtf(fmaf(s.dx, s.dx, fmaf(s.dy, s.dy, s.dz * s.dz)));
}

// Dense output writes of one segment.
template <int MODE, bool STATS>
__device__ __forceinline__ void write_result(const TravOut& o, const Seg& s, bool seg_ok,
                                             const float* A, const float* B, int64_t i,
                                             const float4* __restrict__ tris, const Result& res,
                                             float& dist_out, float P[3], TravStats& st) {
    if (MODE == RSI_MODE_BOOL) {
        o.flag[i] = (uint8_t)(res.count > 0);
    } else if (MODE == RSI_MODE_COUNT) {
        o.count[i] = res.count;
    } else {
        float t = 0.f, u = 0.f, v = 0.f, dist = 0.f;
        P[0] = P[1] = P[2] = 0.f;
        if (seg_ok && res.best >= 0) nearest_values<STATS>(s, A, B, i, tris, res, t, u, v, P, dist, st);
        o.tri[i] = res.best;
        if (o.tuv) {
            o.tuv[3 * i] = t;
            o.tuv[3 * i + 1] = u;
            o.tuv[3 * i + 2] = v;
        }
        if (o.point) {
            o.point[3 * i] = P[0];
            o.point[3 * i + 1] = P[1];
            o.point[3 * i + 2] = P[2];
        }
        if (o.dist) o.dist[i] = dist;
        dist_out = dist;
    }
}

// Warp-aggregated append of the segments with a crossing (one atomic per
// warp).  Must be called by all 32 lanes.
template <int MODE>
__device__ __forceinline__ void compact(const TravOut& o, bool has, int64_t i, const Result& res,
                                        float dist, const float P[3]) {
    const unsigned m = __ballot_sync(0xffffffffu, has);
    if (m == 0u) return;
    const int lane = threadIdx.x & 31;
    unsigned long long b0 = 0ull;
    if (lane == 0) b0 = atomicAdd((unsigned long long*)o.n_hits, (unsigned long long)__popc(m));
    b0 = __shfl_sync(0xffffffffu, b0, 0);
    if (!has) return;
    const int64_t p = (int64_t)b0 + __popc(m & ((1u << lane) - 1u));
    if (p >= o.hit_cap) return;
    o.hit_idx[p] = (int32_t)i;
    if (MODE == RSI_MODE_COUNT) {
        if (o.hit_count) o.hit_count[p] = res.count;
    } else if (MODE == RSI_MODE_NEAREST) {
        if (o.hit_tri) o.hit_tri[p] = res.best;
        if (o.hit_dist) o.hit_dist[p] = dist;
        if (o.hit_point) {
            o.hit_point[3 * p] = P[0];
            o.hit_point[3 * p + 1] = P[1];
            o.hit_point[3 * p + 2] = P[2];
        }
    }
}

// Segments a warp takes from the global counter at once: kFetchChunk for
// large launches (one atomic per 4 segments per lane), down to kFetchMin so
// that a launch of few segments still gives every resident warp work.
constexpr int kFetchChunk = 128;
constexpr int kFetchMin = 32;
constexpr int kRefillMin = 8;     // idle lanes that trigger a refill of a busy warp
constexpr int kWaitPolls = 1 << 22;  // polls of a ready flag (~1 s) before RSI_ERR_TIMEOUT

// Bounded wait of a whole warp for *flag != 0 (written by a copy on another
// stream): every lane polls with an acquire load, so its later loads of the
// flagged data are ordered after it.  Gives up after `polls` polls, or as
// soon as *status holds RSI_ERR_TIMEOUT (another warp's wait already gave
// up), latches RSI_ERR_TIMEOUT and returns false; the caller then stops
// taking work (its results are not to be trusted, which the status says).
// Must be called by all 32 lanes.
__device__ __forceinline__ bool wait_flag(const int32_t* flag, int32_t* status, int polls) {
    for (int q = 0; q < polls; ++q) {
        int v;
        asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(flag) : "memory");
        if (__all_sync(0xffffffffu, v != 0)) return true;
        if ((q & 255) == 255) {
            int st;
            asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(st) : "l"(status) : "memory");
            if (__any_sync(0xffffffffu, st == RSI_ERR_TIMEOUT)) break;
        }
        __nanosleep(256);
    }
    if ((threadIdx.x & 31) == 0) atomicCAS(status, 0, RSI_ERR_TIMEOUT);
    return false;
}

// Persistent per-warp traversal loop over segments [lo, hi).  Every lane
// holds one segment and advances it by one node per iteration; lanes whose
// segments finish take the next ones from the warp's pool as soon as
// kRefillMin of them are free, so the warp does not idle behind its slowest
// lane and the divergent segment setup runs for several lanes at once.  A
// finished lane keeps its result until that refill and writes it then,
// together with the other finished lanes.  The pool is refilled with
// C.fetch segments from *counter (one atomic per chunk), or, with
// counter == nullptr, holds the whole range [lo, hi) from the start.  When
// `order` is given, pool position k processes segment order[k] (a coherent
// ordering of the segments); outputs still go to the segment's own index.
// Dense outputs are written as segments finish; compaction is
// warp-aggregated.  Must be called by all 32 lanes of the warp.
template <int MODE, int STACK, bool STATS, int W, bool TL>
__device__ __forceinline__ void trace_loop(const TraceCtx& C, unsigned long long* counter,
                                           int64_t lo, int64_t hi, TravStats& st,
                                           unsigned long long& segs) {
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    int64_t pool = lo, pool_end = counter ? lo : hi;
    bool more = counter != nullptr;
    int64_t i = -1;
    Seg s;
    int node = 0, sp = 0, visits = 0;
    float tlim = 1.f;
    Result res;
    result_init(res);
    int stack[STACK];
    bool done = false;  // segment i finished, its outputs not yet written
    while (true) {
        unsigned idle = __ballot_sync(FULL, i < 0 || done);
        // Refill in batches: the setup of a new segment and the writes of a
        // finished one run divergently, so wait until kRefillMin lanes are
        // free (or the whole warp is).
        if (__popc(idle) < kRefillMin && idle != FULL) idle = 0u;
        const bool refill = idle != 0u;  // warp-uniform
        if (idle) {  // outputs of the finished segments first
            float dist = 0.f, P[3] = {0.f, 0.f, 0.f};
            if (done)
                write_result<MODE, STATS>(C.out, s, true, C.A, C.B, i, C.tris, res, dist, P, st);
            if (MODE != RSI_MODE_BOOL && C.out.hit_idx)
                compact<MODE>(C.out, done && res.count > 0, i, res, dist, P);
            if (done) {
                i = -1;
                done = false;
            }
        }
        while (idle) {
            if (pool >= pool_end) {
                if (!more) break;
                unsigned long long b = 0ull;
                if (lane == 0) b = atomicAdd(counter, (unsigned long long)C.fetch);
                b = __shfl_sync(FULL, b, 0);
                if (b >= (unsigned long long)hi) {
                    more = false;
                    break;
                }
                pool = (int64_t)b;
                pool_end = pool + C.fetch < hi ? pool + C.fetch : hi;
                // streamed input: the chunks holding [pool, pool_end) have
                // landed once the flag of the last one is set (copies in order).
                // A wait that gives up ends the launch: this warp skips its
                // chunk and the counter is run out, so that no warp takes
                // (and waits for) another one.
                if (C.ready &&
                    !wait_flag(C.ready + (pool_end - 1) / C.ready_chunk, C.status, C.wait_polls)) {
                    if (lane == 0) atomicMax(counter, (unsigned long long)hi);
                    pool = pool_end;
                    more = false;
                    break;
                }
            }
            const int64_t left = pool_end - pool;
            const int avail = left < (int64_t)__popc(idle) ? (int)left : __popc(idle);
            if (i < 0 && (int)__popc(idle & lt) < avail) {
                int64_t k = pool + __popc(idle & lt);
                bool known = true;
                if (C.order) {  // a caller's order: entries outside [0, nR) are skipped
                    k = C.order[k];
                    known = k >= 0 && k < C.nR;
                    if (!known) atomicCAS(C.status, 0, RSI_ERR_BAD_INDEX);
                }
                if (STATS) ++segs;
                result_init(res);
                if (known && seg_setup(C.A, C.B, k, s) && C.root != kNoRoot) {
                    i = k;
                    node = W == 4 ? C.root4 : C.root;
                    sp = 0;
                    visits = 0;
                    tlim = 1.f;
                } else if (known) {  // non-finite segment or empty mesh: a miss
                    float dist, P[3];
                    write_result<MODE, STATS>(C.out, s, false, C.A, C.B, k, C.tris, res, dist, P,
                                              st);
                }
            }
            pool += avail;
            idle = __ballot_sync(FULL, i < 0);
        }
        // without a refill some lane is still busy: the warp goes on
        if (refill && __ballot_sync(FULL, i >= 0) == 0u) break;
        if (i >= 0 && !done) {
            bool overflow = false;
            if (W == 4)
                done = node_step4<MODE, STACK, STATS>(C, s, i, node, sp, stack, tlim, res, visits,
                                                      overflow, st);
            else
                done = node_step<MODE, STACK, STATS, TL>(C, s, i, node, sp, stack, tlim, res, visits,
                                                     overflow, st);
            if (done && (STACK < 64 || W == 4) && overflow) {
                if (STATS) ++st.overflows;
                // 4-wide traversal re-runs on binary nodes from the global root
                trace_deep<MODE, STATS, TL && W != 4>(C, s, i, W == 4 ? C.root4 : C.root, res,
                                                      st);
            }
        }
    }
}

// Sum the per-thread counters of a warp into the global stats.
__device__ __forceinline__ void flush_stats(const TravStats& st, unsigned long long* g,
                                            unsigned long long segs) {
    unsigned long long v[kStatCounters] = {segs,     st.visits,    st.tests, st.fp64,
                                           st.refines, st.overflows, st.exact};
#pragma unroll
    for (int k = 0; k < kStatCounters; ++k) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
    }
    if ((threadIdx.x & 31) == 0)
        for (int k = 0; k < kStatCounters; ++k) atomicAdd(g + k, v[k]);
}

}  // namespace rsi
