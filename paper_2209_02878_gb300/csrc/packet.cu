// Warp-cooperative ("packet") traversal, the alternative to one stack per
// segment for coherent segments (the divergence remark of Sec. 4.1 on
// Morton-sorted rays; launch option `packet`).
//
// A warp takes 32 consecutive segments in processing order (input order, or
// the coherent order of sort_bits) and walks the tree once for all of them:
//  - every node is fetched once per warp (all lanes load the same record, a
//    broadcast), and each lane slab-tests its own segment against the two
//    child boxes;
//  - each lane tests the triangles of the leaves its own segment enters
//    (BOOL lanes stop at their first crossing, NEAREST lanes shrink their own
//    t limit);
//  - the warp descends into a child when any active lane enters it, the near
//    child first by majority vote of the lanes entering both, and keeps the
//    other on one warp-uniform stack (held by every lane at the same index,
//    so its local-memory accesses are coalesced);
//  - the warp stops when the stack is empty or no lane is active.
// The results are the per-segment results (the same leaf tests, in a
// different order); the cost is the union of the 32 paths, so it pays off
// only when a warp's segments are close in space and direction.
#include <cuda_runtime.h>

#include "rsi_trace.h"
#include "traverse_core.cuh"

namespace rsi {

constexpr int kPacketBlock = 128;
constexpr int kPacketStack = 64;  // a radix tree over 62-bit keys is at most 63 deep

template <int MODE>
struct PacketRegs {
    static constexpr int value = MODE == RSI_MODE_NEAREST ? 80 : 72;
};

template <int MODE, bool STATS>
__global__ void __maxnreg__(PacketRegs<MODE>::value) k_trace_packet(TraceParams P) {
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    TraceCtx C;
    C.A = P.A;
    C.B = P.B;
    C.nR = P.nR;
    C.root = P.root;
    C.root4 = P.root4;
    C.nodes = P.nodes;
    C.nodes4 = P.nodes4;
    C.tris = P.tris;
    C.treelet = P.treelet;
    C.snodes = nullptr;
    C.S = 0;
    C.max_visits = P.max_visits;
    C.fetch = 32;  // packets take 32 segments per warp themselves
    C.ready = nullptr;
    C.ready_chunk = 1;
    C.wait_polls = kWaitPolls;
    C.order = P.order;
    C.status = P.status;
    C.out = P.out;
    TravStats st = {0ull, 0ull, 0ull, 0ull, 0ull, 0ull};
    unsigned long long segs = 0;
    int stack[kPacketStack];
    while (true) {
        unsigned long long b = 0ull;
        if (lane == 0) b = atomicAdd(P.work, 32ull);
        b = __shfl_sync(FULL, b, 0);
        if (b >= (unsigned long long)P.nR) break;
        const int64_t pos = (int64_t)b + lane;
        bool valid = pos < P.nR;
        int64_t i = pos;
        if (valid && C.order) {  // a caller's order: entries outside [0, nR) are skipped
            i = C.order[pos];
            if (i < 0 || i >= P.nR) {
                atomicCAS(C.status, 0, RSI_ERR_BAD_INDEX);
                valid = false;
            }
        }
        if (!valid) i = 0;
        Seg s;
        Result res;
        result_init(res);
        float tlim = 1.f;
        bool ok = false;
        if (valid) {
            if (STATS) ++segs;
            ok = seg_setup(C.A, C.B, i, s) && C.root != kNoRoot;
        }
        bool act = ok;
        int node = C.root, sp = 0, visits = 0;
        while (__ballot_sync(FULL, act)) {
            if (++visits > C.max_visits) {  // warp-uniform: a corrupt tree
                if (lane == 0) atomicCAS(C.status, 0, RSI_ERR_INTERNAL);
                break;
            }
            ulonglong2 q0, q1, q2;
            int4 rc;
            if (node < 0)
                ld_node(C.treelet + 4 * (int64_t)(~node), q0, q1, q2, rc);
            else
                ld_node(C.nodes + 4 * (int64_t)node, q0, q1, q2, rc);
            bool h0 = false, h1 = false;
            float t0 = 0.f, t1 = 0.f;
            if (act) {
                if (STATS) ++st.visits;
                slab2(s, q0, q1, q2, tlim, h0, t0, h1, t1);
            }
            const int r0 = rc.x, r1 = rc.y, c0 = rc.z, c1 = rc.w;
            if (MODE == RSI_MODE_NEAREST) {
                if (h0 && c0 > 0)
                    leaf_test<MODE, STATS>(s, C.A, C.B, i, C.tris, r0, c0, 0, 0, res, tlim, st);
                if (h1 && c1 > 0)
                    leaf_test<MODE, STATS>(s, C.A, C.B, i, C.tris, r1, c1, 0, 0, res, tlim, st);
            } else {
                const int n0 = h0 && c0 > 0 ? c0 : 0, n1 = h1 && c1 > 0 ? c1 : 0;
                if ((n0 | n1) &&
                    leaf_test<MODE, STATS>(s, C.A, C.B, i, C.tris, r0, n0, r1, n1, res, tlim, st))
                    act = false;  // BOOL: the first crossing decides
            }
            const bool g0 = act && h0 && c0 <= 0, g1 = act && h1 && c1 <= 0;
            const unsigned m0 = __ballot_sync(FULL, g0), m1 = __ballot_sync(FULL, g1);
            const int x0 = c0 < 0 ? ~r0 : r0, x1 = c1 < 0 ? ~r1 : r1;
            if (m0 && m1) {
                const unsigned both = m0 & m1;
                const unsigned near0 = __ballot_sync(FULL, g0 && g1 && t0 <= t1);
                const bool first0 = both ? 2 * __popc(near0) >= __popc(both)
                                         : __popc(m0) >= __popc(m1);
                if (sp >= kPacketStack) {  // deeper than any radix tree: a corrupt tree
                    if (lane == 0) atomicCAS(C.status, 0, RSI_ERR_INTERNAL);
                    break;
                }
                stack[sp++] = first0 ? x1 : x0;
                node = first0 ? x0 : x1;
            } else if (m0) {
                node = x0;
            } else if (m1) {
                node = x1;
            } else {
                if (sp == 0) break;
                node = stack[--sp];
            }
        }
        float dist = 0.f, Pt[3] = {0.f, 0.f, 0.f};
        if (valid) write_result<MODE, STATS>(C.out, s, ok, C.A, C.B, i, C.tris, res, dist, Pt, st);
        if (MODE != RSI_MODE_BOOL && C.out.hit_idx)
            compact<MODE>(C.out, valid && ok && res.count > 0, i, res, dist, Pt);
    }
    if (STATS) flush_stats(st, P.stats, segs);
}

using PacketFn = void (*)(TraceParams);

static PacketFn packet_kernel(int mode, bool stats) {
    if (mode == RSI_MODE_BOOL)
        return stats ? k_trace_packet<RSI_MODE_BOOL, true> : k_trace_packet<RSI_MODE_BOOL, false>;
    if (mode == RSI_MODE_COUNT)
        return stats ? k_trace_packet<RSI_MODE_COUNT, true> : k_trace_packet<RSI_MODE_COUNT, false>;
    return stats ? k_trace_packet<RSI_MODE_NEAREST, true> : k_trace_packet<RSI_MODE_NEAREST, false>;
}

cudaError_t launch_trace_packet(const TraceParams& P, int mode, bool stats, cudaStream_t s) {
    PacketFn fn = packet_kernel(mode, stats);
    int grid = 0;
    cudaError_t e = occupancy_grid((const void*)fn, kPacketBlock, 0, &grid);
    if (e != cudaSuccess) return e;
    const int64_t warps_needed = (P.nR + 31) / 32;
    const int64_t blocks_needed = (warps_needed + kPacketBlock / 32 - 1) / (kPacketBlock / 32);
    if (blocks_needed < grid) grid = (int)blocks_needed;
    if (grid < 1) grid = 1;
    e = cudaMemsetAsync(P.work, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    if (P.out.hit_idx) {
        e = cudaMemsetAsync(P.out.n_hits, 0, sizeof(int64_t), s);
        if (e != cudaSuccess) return e;
    }
    fn<<<grid, kPacketBlock, 0, s>>>(P);
    return cudaGetLastError();
}

}  // namespace rsi
