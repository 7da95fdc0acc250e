// Batched traversal: many independent (mesh, segments, mode) problems in one
// persistent launch.  The work is a list of tiles (up to kBatchTile segments
// of one item) ordered by decreasing estimated cost per segment (log2 N_t,
// NEAREST and COUNT weighted above BOOL) so the expensive tiles start first;
// each warp pulls the next tile from one atomic counter and runs the same
// per-lane refill traversal as the single-mesh kernel over the tile, in that
// item's mode.  All meshes live in one concatenated node / triangle storage
// built by one multi-mesh build.
#include <cuda_runtime.h>

#include "rsi_trace.h"

namespace rsi {

// All three modes are inlined into one kernel; without a cap it needs ~170
// registers (two warps per scheduler).  128 measured fastest on the 64-mesh
// mix (8.37 ms against 8.79 ms at 96 and 9.52 ms at 72, where the nearest
// path spills).
template <int STACK>
__global__ void __maxnreg__(128) k_batch(BatchParams P) {
    TravStats st = {0ull, 0ull, 0ull, 0ull, 0ull, 0ull};
    unsigned long long segs = 0;
    const int lane = threadIdx.x & 31;
    while (true) {
        unsigned long long t = 0ull;
        if (lane == 0) t = atomicAdd(P.work, 1ull);
        t = __shfl_sync(0xffffffffu, t, 0);
        if (t >= (unsigned long long)P.n_tiles) break;
        const BatchTile tile = P.tiles[t];
        const BatchItemDev& it = P.items[tile.item];
        TraceCtx C;
        C.A = it.A;
        C.B = it.B;
        C.nR = it.nR;
        C.root = it.root;
        C.root4 = it.root;
        C.nodes = P.nodes;
        C.nodes4 = P.nodes4;
        C.tris = P.tris;
        C.treelet = nullptr;
        C.snodes = nullptr;
        C.S = 0;
        C.max_visits = P.max_visits;
        C.fetch = kFetchChunk;  // unused: each tile is one warp's whole pool
        C.ready = nullptr;
        C.ready_chunk = 1;
        C.wait_polls = kWaitPolls;
        C.order = nullptr;
        C.status = P.status;
        C.out = it.out;
        switch (it.mode) {
            case RSI_MODE_BOOL:
                trace_loop<RSI_MODE_BOOL, STACK, false, 2, false>(C, nullptr, tile.lo, tile.hi, st,
                                                                  segs);
                break;
            case RSI_MODE_COUNT:
                trace_loop<RSI_MODE_COUNT, STACK, false, 2, false>(C, nullptr, tile.lo, tile.hi, st,
                                                                   segs);
                break;
            default:
                trace_loop<RSI_MODE_NEAREST, STACK, false, 2, false>(C, nullptr, tile.lo, tile.hi,
                                                                     st, segs);
                break;
        }
    }
}

// Zero the compaction counters of the items that compact.
__global__ void k_zero_counts(const BatchItemDev* items, int n) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n && items[k].out.hit_idx) *items[k].out.n_hits = 0;
}

const void* batch_kernel(int stack) {
    switch (stack) {
        case 8: return (const void*)k_batch<8>;
        case 32: return (const void*)k_batch<32>;
        default: return (const void*)k_batch<64>;
    }
}

cudaError_t launch_batch(const BatchParams& P, int block, int stack, cudaStream_t s) {
    if (P.n_tiles == 0) return cudaSuccess;
    const void* fn = batch_kernel(stack);
    block = max_block(fn, block);
    int grid = 0;
    cudaError_t e = occupancy_grid(fn, block, 0, &grid);
    if (e != cudaSuccess) return e;
    const int64_t blocks_needed = (P.n_tiles + block / 32 - 1) / (block / 32);
    if (blocks_needed < grid) grid = (int)blocks_needed;
    e = cudaMemsetAsync(P.work, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    k_zero_counts<<<(P.n_items + 255) / 256, 256, 0, s>>>(P.items, P.n_items);
    switch (stack) {
        case 8: k_batch<8><<<grid, block, 0, s>>>(P); break;
        case 32: k_batch<32><<<grid, block, 0, s>>>(P); break;
        default: k_batch<64><<<grid, block, 0, s>>>(P); break;
    }
    return cudaGetLastError();
}

}  // namespace rsi
