// Traversal with deferred leaf tests (BOOL and COUNT): a lane that reaches a
// leaf does not test its triangles at once -- that path would run for the
// one or two lanes of the warp that reached a leaf while the others wait --
// but appends (leaf, lane) to a per-warp queue in shared memory and keeps
// traversing.  When the queue holds kDrain entries, or when lanes whose
// traversal has ended wait on their queued tests, the whole warp drains it:
// each lane takes one entry, fetches the owner lane's segment with shuffles
// and runs the segment / triangle test (Sec. 2), so the tests run 32 at a
// time.  The results go back to their owners: COUNT adds them up, BOOL ends
// the owner's traversal at its first crossing (later than the inline test
// would, by the entries waiting in the queue).  Same decisions, same
// outputs as the inline traversal.
#pragma once

#include "traverse_core.cuh"

namespace rsi {

constexpr int kQueueCap = 96;  // entries per warp: < kDrain + 64 (two leaves per lane per visit)

struct WarpQueue {
    uint2 e[kQueueCap];  // {first leaf position, count << 5 | owner lane}
    int32_t res[32];     // per owner lane: crossings found by the last drain
};

template <int MODE>
struct QueueDrain {  // entries that trigger a drain
    static constexpr int value = MODE == RSI_MODE_BOOL ? 8 : 32;
};

// Test every queued (owner segment, leaf) pair, up to 32 at a time, and
// return this lane's crossings found.  (ax, ay, az, dx, dy, dz, md, fp64only,
// i) are this lane's segment, which the lanes testing its entries fetch by
// shuffles.  Out of line: inlined, its state would cost the traversal loop
// registers.  Must be called by all 32 lanes with the same qn; clears the
// queue and the result slots.
template <int MODE, bool STATS>
__device__ __noinline__ int drain_queue(const float* A, const float* B,
                                        const float4* __restrict__ tris, WarpQueue* q, int qn,
                                        float ax_, float ay_, float az_, float dx_, float dy_,
                                        float dz_, float md_, int fp64only_, long long i,
                                        unsigned long long* st_tests,
                                        unsigned long long* st_fp64) {
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    __syncwarp();  // the appends of every lane are visible
    while (qn > 0) {
        const int take = qn < 32 ? qn : 32;
        const bool act = lane < take;
        const uint2 e = act ? q->e[qn - take + lane] : make_uint2(0u, 0u);
        const int owner = (int)(e.y & 31u);
        const float ax = __shfl_sync(FULL, ax_, owner);
        const float ay = __shfl_sync(FULL, ay_, owner);
        const float az = __shfl_sync(FULL, az_, owner);
        Seg so;
        so.pax = pk2(ax, ax);
        so.pay = pk2(ay, ay);
        so.paz = pk2(az, az);
        so.pix = so.piy = so.piz = 0ull;
        so.dx = __shfl_sync(FULL, dx_, owner);
        so.dy = __shfl_sync(FULL, dy_, owner);
        so.dz = __shfl_sync(FULL, dz_, owner);
        so.md = __shfl_sync(FULL, md_, owner);
        so.fp64only = __shfl_sync(FULL, fp64only_, owner) != 0;
        so.tiny = false;
        const long long io = __shfl_sync(FULL, i, owner);
        if (act) {
            int hits = 0;
            const int cnt = (int)(e.y >> 5);
            for (int k = 0; k < cnt; ++k) {
                const int pos = (int)e.x + k;
                const float4 a = ld4(tris + 3 * (int64_t)pos);
                const float4 b = ld4(tris + 3 * (int64_t)pos + 1);
                const float4 c = ld4(tris + 3 * (int64_t)pos + 2);
                float t, u, v, err;
                if (STATS) ++*st_tests;
                int r = mt32(so, a, b, c, false, t, u, v, err);
                if (r == 2) {
                    if (STATS) ++*st_fp64;
                    r = mt64(A[3 * io], A[3 * io + 1], A[3 * io + 2], B[3 * io], B[3 * io + 1],
                             B[3 * io + 2], a, b, c, nullptr);
                }
                hits += r;
                if (MODE == RSI_MODE_BOOL && hits) break;
            }
            if (hits) {
                if (MODE == RSI_MODE_BOOL)
                    q->res[owner] = 1;
                else
                    atomicAdd(&q->res[owner], hits);
            }
        }
        qn -= take;
    }
    __syncwarp();
    const int f = q->res[lane];
    q->res[lane] = 0;
    __syncwarp();
    return f;
}

template <int MODE, bool STATS>
__device__ __forceinline__ int drain(const TraceCtx& C, WarpQueue& q, int& qn, const Seg& s,
                                     int64_t i, TravStats& st) {
    const int f = drain_queue<MODE, STATS>(C.A, C.B, C.tris, &q, qn, s.ax(), s.ay(), s.az(),
                                           s.dx, s.dy, s.dz, s.md, (int)s.fp64only,
                                           (long long)i, &st.tests, &st.fp64);
    qn = 0;
    return f;
}

// One node visit of the deferred-test traversal: test both child boxes,
// report child leaves to queue (first position and count, or cnt 0), then
// descend or pop.  Returns true when the traversal of segment i has ended.
template <int STACK, bool STATS>
__device__ __forceinline__ bool node_step_q(const TraceCtx& C, const Seg& s, int& node, int& sp,
                                            int* stack, int& visits, int2& l0, int2& l1,
                                            TravStats& st) {
    if (++visits > C.max_visits) {
        atomicCAS(C.status, 0, RSI_ERR_INTERNAL);
        return true;
    }
    ulonglong2 q0, q1, q2;
    int4 rc;
    ld_node(C.nodes + 4 * (int64_t)node, q0, q1, q2, rc);
    if (STATS) ++st.visits;
    float t0, t1;
    bool h0, h1;
    slab2(s, q0, q1, q2, 1.f, h0, t0, h1, t1);
    const int r0 = rc.x, r1 = rc.y, c0 = rc.z, c1 = rc.w;
    l0 = make_int2(r0, h0 && c0 > 0 ? c0 : 0);
    l1 = make_int2(r1, h1 && c1 > 0 ? c1 : 0);
    const bool g0 = h0 && c0 <= 0, g1 = h1 && c1 <= 0;
    if (g0 && g1) {
        const bool near0 = t0 <= t1;
        stack[sp++] = near0 ? r1 : r0;  // STACK is 64: a radix tree never overflows it
        node = near0 ? r0 : r1;
    } else if (g0) {
        node = r0;
    } else if (g1) {
        node = r1;
    } else {
        if (sp == 0) return true;
        node = stack[--sp];
    }
    return false;
}

// Persistent per-warp loop of the deferred-test traversal: the refill,
// output and compaction logic of trace_loop, binary nodes without a
// treelet, a 64-entry stack.  A lane's segment is finished once its
// traversal has ended and its queued tests have drained (BOOL: or a drained
// test found a crossing).  Must be called by all 32 lanes of the warp.
template <int MODE, bool STATS>
__device__ __forceinline__ void trace_loop_q(const TraceCtx& C, WarpQueue& q,
                                             unsigned long long* counter, int64_t lo, int64_t hi,
                                             TravStats& st, unsigned long long& segs) {
    constexpr int STACK = 64;
    constexpr int kDrain = QueueDrain<MODE>::value;
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    int64_t pool = lo, pool_end = counter ? lo : hi;
    bool more = counter != nullptr;
    int64_t i = -1;
    Seg s;
    int node = 0, sp = 0, visits = 0;
    Result res;
    result_init(res);
    int stack[STACK];
    bool done = false;     // segment i finished, its outputs not yet written
    bool waiting = false;  // traversal ended, some of its tests still queued
    int pend = 0;          // entries of this lane in the queue
    int qn = 0;            // queue length (the same in every lane)
    q.res[lane] = 0;
    __syncwarp();
    // take the results of a drain: counts add up, a BOOL crossing ends the
    // traversal, and lanes that waited on their tests are finished
    auto apply = [&](int f) {
        if (i >= 0 && !done) {
            if (MODE == RSI_MODE_BOOL) {
                if (f) {
                    res.count = 1;
                    done = true;
                }
            } else {
                res.count += f;
            }
            if (waiting) done = true;
        }
        waiting = false;
        pend = 0;
    };
    while (true) {
        unsigned idle = __ballot_sync(FULL, i < 0 || done);
        const unsigned waitm = __ballot_sync(FULL, waiting);
        if (waitm) {
            const unsigned trav = __ballot_sync(FULL, i >= 0 && !done && !waiting);
            if (trav == 0u || __popc(idle | waitm) >= kRefillMin) {
                apply(drain<MODE, STATS>(C, q, qn, s, i, st));
                idle = __ballot_sync(FULL, i < 0 || done);
            }
        }
        if (__popc(idle) < kRefillMin && idle != FULL) idle = 0u;
        if (idle) {
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
                if (C.order) k = C.order[k];
                if (STATS) ++segs;
                result_init(res);
                if (seg_setup(C.A, C.B, k, s) && C.root != kNoRoot) {
                    i = k;
                    node = C.root;
                    sp = 0;
                    visits = 0;
                } else {  // non-finite segment or empty mesh: a miss
                    float dist, P[3];
                    write_result<MODE, STATS>(C.out, s, false, C.A, C.B, k, C.tris, res, dist, P,
                                              st);
                }
            }
            pool += avail;
            idle = __ballot_sync(FULL, i < 0);
        }
        if (__ballot_sync(FULL, i >= 0) == 0u) break;
        int2 l0 = make_int2(0, 0), l1 = make_int2(0, 0);
        bool fin = false;
        if (i >= 0 && !done && !waiting)
            fin = node_step_q<STACK, STATS>(C, s, node, sp, stack, visits, l0, l1, st);
        const unsigned m0 = __ballot_sync(FULL, l0.y > 0), m1 = __ballot_sync(FULL, l1.y > 0);
        if (m0 | m1) {
            if (l0.y > 0)
                q.e[qn + __popc(m0 & lt)] = make_uint2((unsigned)l0.x, ((unsigned)l0.y << 5) | lane);
            if (l1.y > 0)
                q.e[qn + __popc(m0) + __popc(m1 & lt)] =
                    make_uint2((unsigned)l1.x, ((unsigned)l1.y << 5) | lane);
            qn += __popc(m0) + __popc(m1);
            pend += (l0.y > 0) + (l1.y > 0);
        }
        if (fin) {
            if (pend > 0)
                waiting = true;
            else
                done = true;
        }
        if (qn >= kDrain) apply(drain<MODE, STATS>(C, q, qn, s, i, st));
    }
}

}  // namespace rsi
