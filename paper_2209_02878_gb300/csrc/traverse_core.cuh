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

struct TravStats {
    unsigned long long visits, tests, fp64, refines, overflows;
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

// Test the cnt triangles of a leaf.  Returns true when BOOL found a crossing.
template <int MODE, bool STATS>
__device__ __forceinline__ bool leaf_test(const Seg& s, const float* A, const float* B, int64_t i,
                                          const float4* __restrict__ tris, int first, int cnt,
                                          Result& res, float& tlim, TravStats& st) {
    for (int k = 0; k < cnt; ++k) {
        const int pos = first + k;
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

// Returns false when the stack overflowed (result incomplete).
template <int MODE, int STACK, bool STATS>
__device__ __forceinline__ bool trace(const Seg& s, const float* A, const float* B, int64_t i,
                                      int root, const float4* __restrict__ nodes,
                                      const float4* __restrict__ tris,
                                      const float4* __restrict__ treelet, const float4* snodes,
                                      int S, int max_visits, int32_t* status, Result& res,
                                      TravStats& st) {
    int stack[STACK];
    int sp = 0;
    int node = root;
    float tlim = 1.f;
    // each node of a tree is visited at most once per segment
    for (int visits = 0;; ++visits) {
        if (visits > max_visits) {
            atomicCAS(status, 0, RSI_ERR_INTERNAL);
            break;
        }
        float4 n0, n1, n2, n3;
        if (node < 0) {
            const int k = ~node;
            if (k < S) {
                n0 = snodes[4 * k];
                n1 = snodes[4 * k + 1];
                n2 = snodes[4 * k + 2];
                n3 = snodes[4 * k + 3];
            } else {
                const float4* p = treelet + 4 * (int64_t)k;
                n0 = ld4(p);
                n1 = ld4(p + 1);
                n2 = ld4(p + 2);
                n3 = ld4(p + 3);
            }
        } else {
            const float4* p = nodes + 4 * (int64_t)node;
            n0 = ld4(p);
            n1 = ld4(p + 1);
            n2 = ld4(p + 2);
            n3 = ld4(p + 3);
        }
        if (STATS) ++st.visits;
        float t0, t1;
        const bool h0 = slab(s, n0.x, n0.y, n0.z, n0.w, n1.x, n1.y, tlim, t0);
        const bool h1 = slab(s, n1.z, n1.w, n2.x, n2.y, n2.z, n2.w, tlim, t1);
        const int r0 = f2i(n3.x), r1 = f2i(n3.y), c0 = f2i(n3.z), c1 = f2i(n3.w);
        if (h0 && c0 > 0) {
            if (leaf_test<MODE, STATS>(s, A, B, i, tris, r0, c0, res, tlim, st)) return true;
        }
        if (h1 && c1 > 0) {
            if (leaf_test<MODE, STATS>(s, A, B, i, tris, r1, c1, res, tlim, st)) return true;
        }
        const bool g0 = h0 && c0 <= 0, g1 = h1 && c1 <= 0;
        const int x0 = c0 < 0 ? ~r0 : r0, x1 = c1 < 0 ? ~r1 : r1;
        if (g0 && g1) {
            const bool near0 = t0 <= t1;
            if (sp >= STACK) return false;
            stack[sp++] = near0 ? x1 : x0;
            node = near0 ? x0 : x1;
        } else if (g0) {
            node = x0;
        } else if (g1) {
            node = x1;
        } else {
            if (sp == 0) break;
            node = stack[--sp];
        }
    }
    return true;
}

// Deep-stack re-run for segments whose stack overflowed (a radix tree over
// 62-bit keys is at most 63 levels deep, so 64 entries always suffice).
template <int MODE, bool STATS>
__device__ __noinline__ void trace_deep(const Seg& s, const float* A, const float* B, int64_t i,
                                        int root, const float4* __restrict__ nodes,
                                        const float4* __restrict__ tris,
                                        const float4* __restrict__ treelet, const float4* snodes,
                                        int S, int max_visits, int32_t* status, Result& res,
                                        TravStats& st) {
    res.count = 0;
    res.best = -1;
    res.b64 = false;
    trace<MODE, 64, STATS>(s, A, B, i, root, nodes, tris, treelet, snodes, S, max_visits, status,
                           res, st);
}

__device__ __forceinline__ void result_init(Result& r) {
    r.count = 0;
    r.best = -1;
    r.bpos = 0;
    r.bt = r.bu = r.bv = r.berr = 0.f;
    r.bt64 = 0.0;
    r.b64 = false;
}

// Nearest outputs; (t, u, v) are recomputed in FP64 when their FP32 error
// bound could move the point by more than about 2^-21.
template <bool STATS>
__device__ __forceinline__ void nearest_values(const Seg& s, const float* A, const float* B,
                                               int64_t i, const float4* __restrict__ tris,
                                               const Result& res, float& t, float& u, float& v,
                                               float P[3], float& dist, TravStats& st) {
    t = res.bt;
    u = res.bu;
    v = res.bv;
    const float thresh = 0x1p-21f / fmaxf(1.f, s.md * 1.7320508f);
    if (res.berr > thresh || s.fp64only) {
        if (STATS) ++st.refines;
        double tuv[3] = {0.0, 0.0, 0.0};
        const int p = res.bpos;
        mt64(A[3 * i], A[3 * i + 1], A[3 * i + 2], B[3 * i], B[3 * i + 1], B[3 * i + 2],
             ld4(tris + 3 * (int64_t)p), ld4(tris + 3 * (int64_t)p + 1),
             ld4(tris + 3 * (int64_t)p + 2), tuv);
        t = (float)tuv[0];
        u = (float)tuv[1];
        v = (float)tuv[2];
        if (s.fp64only) {
            double dd = 0.0;
            for (int k = 0; k < 3; ++k) {
                const double a = A[3 * i + k], d = (double)B[3 * i + k] - a;
                P[k] = (float)(a + tuv[0] * d);
                dd += d * d;
            }
            dist = (float)(tuv[0] * sqrt(dd));
            return;
        }
    }
    P[0] = fmaf(t, s.dx, s.ax);
    P[1] = fmaf(t, s.dy, s.ay);
    P[2] = fmaf(t, s.dz, s.az);
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

// One segment end to end: setup, traversal (+ deep re-run), dense outputs,
// compaction.  All lanes of the warp call it (i >= nR for idle lanes).
template <int MODE, int STACK, bool STATS>
__device__ __forceinline__ void process_segment(const float* A, const float* B, int64_t nR,
                                                int64_t i, int root,
                                                const float4* __restrict__ nodes,
                                                const float4* __restrict__ tris,
                                                const float4* __restrict__ treelet,
                                                const float4* snodes, int S, int max_visits,
                                                int32_t* status, const TravOut& o,
                                                TravStats& st) {
    Result res;
    result_init(res);
    float dist = 0.f, P[3] = {0.f, 0.f, 0.f};
    const bool valid = i < nR;
    if (valid) {
        Seg s;
        const bool seg_ok = seg_setup(A, B, i, s);
        if (seg_ok && root != kNoRoot) {
            const bool ok = trace<MODE, STACK, STATS>(s, A, B, i, root, nodes, tris, treelet,
                                                      snodes, S, max_visits, status, res, st);
            if (STACK < 64 && !ok) {
                if (STATS) ++st.overflows;
                trace_deep<MODE, STATS>(s, A, B, i, root, nodes, tris, treelet, snodes, S,
                                        max_visits, status, res, st);
            }
        }
        write_result<MODE, STATS>(o, s, seg_ok, A, B, i, tris, res, dist, P, st);
    }
    if (MODE != RSI_MODE_BOOL && o.hit_idx) compact<MODE>(o, valid && res.count > 0, i, res, dist, P);
}

// Sum the per-thread counters of a warp into the global stats.
__device__ __forceinline__ void flush_stats(const TravStats& st, unsigned long long* g,
                                            unsigned long long segs) {
    unsigned long long v[5] = {st.visits, st.tests, st.fp64, st.refines, st.overflows};
#pragma unroll
    for (int k = 0; k < 5; ++k) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(g + 0, segs);
        for (int k = 0; k < 5; ++k) atomicAdd(g + 1 + k, v[k]);
    }
}

}  // namespace rsi
