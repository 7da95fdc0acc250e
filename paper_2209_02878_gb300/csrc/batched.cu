// Batched traversal: many independent (mesh, segments, mode) problems in one
// persistent launch.  The work is a list of 32-segment chunks; items are laid
// out in decreasing estimated cost per segment (log2 N_t, NEAREST and COUNT
// weighted above BOOL) so the expensive chunks start first, and each warp
// pulls the next chunk from one atomic counter, finds its item by binary
// search over the items' first chunks and runs the same per-segment
// traversal as the single-mesh kernel in that item's mode.  All meshes live
// in one concatenated node / triangle storage built by one multi-mesh build.
#include <cuda_runtime.h>

#include "rsi_trace.h"

namespace rsi {

template <int STACK>
__global__ void k_batch(BatchParams P) {
    TravStats st = {0ull, 0ull, 0ull, 0ull, 0ull};
    const int lane = threadIdx.x & 31;
    while (true) {
        unsigned long long c = 0ull;
        if (lane == 0) c = atomicAdd(P.work, 1ull);
        c = __shfl_sync(0xffffffffu, c, 0);
        if (c >= (unsigned long long)P.n_chunks) break;
        int lo = 0, hi = P.n_items - 1;  // last item with chunk0 <= c
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if ((unsigned long long)P.items[mid].chunk0 <= c)
                lo = mid;
            else
                hi = mid - 1;
        }
        const BatchItemDev& it = P.items[lo];
        const int64_t i = ((int64_t)c - it.chunk0) * 32 + lane;
        switch (it.mode) {
            case RSI_MODE_BOOL:
                process_segment<RSI_MODE_BOOL, STACK, false>(it.A, it.B, it.nR, i, it.root,
                                                             P.nodes, P.tris, nullptr, nullptr,
                                                             0, P.max_visits, P.status,
                                                             it.out, st);
                break;
            case RSI_MODE_COUNT:
                process_segment<RSI_MODE_COUNT, STACK, false>(it.A, it.B, it.nR, i, it.root,
                                                              P.nodes, P.tris, nullptr, nullptr,
                                                              0, P.max_visits, P.status,
                                                              it.out, st);
                break;
            default:
                process_segment<RSI_MODE_NEAREST, STACK, false>(it.A, it.B, it.nR, i, it.root,
                                                                P.nodes, P.tris, nullptr,
                                                                nullptr, 0, P.max_visits,
                                                                P.status, it.out, st);
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
        case 16: return (const void*)k_batch<16>;
        case 32: return (const void*)k_batch<32>;
        default: return (const void*)k_batch<64>;
    }
}

cudaError_t launch_batch(const BatchParams& P, int block, int stack, cudaStream_t s) {
    if (P.n_chunks == 0) return cudaSuccess;
    const void* fn = batch_kernel(stack);
    int grid = 0;
    cudaError_t e = occupancy_grid(fn, block, 0, &grid);
    if (e != cudaSuccess) return e;
    const int64_t blocks_needed = (P.n_chunks + block / 32 - 1) / (block / 32);
    if (blocks_needed < grid) grid = (int)blocks_needed;
    e = cudaMemsetAsync(P.work, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    k_zero_counts<<<(P.n_items + 255) / 256, 256, 0, s>>>(P.items, P.n_items);
    switch (stack) {
        case 16: k_batch<16><<<grid, block, 0, s>>>(P); break;
        case 32: k_batch<32><<<grid, block, 0, s>>>(P); break;
        default: k_batch<64><<<grid, block, 0, s>>>(P); break;
    }
    return cudaGetLastError();
}

}  // namespace rsi
