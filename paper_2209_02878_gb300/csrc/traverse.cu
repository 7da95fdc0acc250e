// Single-mesh traversal launch (arXiv 2209.02878, Sec. 3.3
// bvhIntersectionKernel): a persistent grid sized from the occupancy query
// (the paper's N_grid lesson, Sec. 3.3: fill the machine), each warp pulling
// a chunk of segments at a time from an atomic counter, optionally the top
// treelet staged once per block in shared memory.
#include <cuda_runtime.h>

#include <mutex>

#include "rsi_trace.h"
#include "traverse_core.cuh"

namespace rsi {

// Register caps per mode, measured on the paper-scale workload: BOOL gains
// more from resident warps (hiding the dependent node fetches) than it loses
// to a few spills; NEAREST carries more state and spills badly below 80.
template <int MODE>
struct TraceRegs {
    static constexpr int value = MODE == RSI_MODE_BOOL ? 64 : (MODE == RSI_MODE_COUNT ? 72 : 80);
};

template <int MODE, int STACK, bool STATS, int W, bool TL>
__global__ void __maxnreg__(TraceRegs<MODE>::value) k_trace(TraceParams P) {
    extern __shared__ float4 snodes[];
    int S = 0;
    if (P.smem_nodes > 0) {
        S = min(P.smem_nodes, *P.treelet_n);
        for (int q = threadIdx.x; q < 4 * S; q += blockDim.x) snodes[q] = P.treelet[q];
        __syncthreads();
    }
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
    C.snodes = snodes;
    C.S = S;
    C.max_visits = P.max_visits;
    C.fetch = P.fetch;
    C.ready = P.ready;
    C.ready_chunk = P.ready_chunk;
    C.wait_polls = P.wait_polls > 0 ? P.wait_polls : kWaitPolls;
    C.order = P.order;
    C.status = P.status;
    C.out = P.out;
    TravStats st = {0ull, 0ull, 0ull, 0ull, 0ull, 0ull};
    unsigned long long segs = 0;
    trace_loop<MODE, STACK, STATS, W, TL>(C, P.work, 0, P.nR, st, segs);
    if (STATS) flush_stats(st, P.stats, segs);
}

using KernelFn = void (*)(TraceParams);

template <int MODE, bool STATS, int W, bool TL>
static KernelFn pick_stack(int stack) {
    switch (stack) {
        case 8: return k_trace<MODE, 8, STATS, W, TL>;
        case 32: return k_trace<MODE, 32, STATS, W, TL>;
        default: return k_trace<MODE, 64, STATS, W, TL>;
    }
}

// Without a treelet, BOOL and COUNT take the variant with the treelet tests
// compiled out (1-2 % faster on the paper-scale heightfield); binary NEAREST
// always takes the general one, which the register allocator handles better
// (2.22 against 2.39 ms there).
template <bool STATS, int W, bool TL>
static KernelFn pick_mode(int mode, int stack) {
    if (mode == RSI_MODE_BOOL) return pick_stack<RSI_MODE_BOOL, STATS, W, TL>(stack);
    if (mode == RSI_MODE_COUNT) return pick_stack<RSI_MODE_COUNT, STATS, W, TL>(stack);
    return pick_stack<RSI_MODE_NEAREST, STATS, W, TL || W == 2>(stack);
}

// The treelet variant for binary traversal from a treelet root (~0); 4-wide
// traversal starts at the global root.
KernelFn trace_kernel(int mode, int stack, bool stats, int width, bool treelet) {
    if (width != 2)
        return stats ? pick_mode<true, 4, false>(mode, stack) : pick_mode<false, 4, false>(mode, stack);
    if (treelet)
        return stats ? pick_mode<true, 2, true>(mode, stack) : pick_mode<false, 2, true>(mode, stack);
    return stats ? pick_mode<true, 2, false>(mode, stack) : pick_mode<false, 2, false>(mode, stack);
}

struct OccKey {
    const void* fn;
    int block, smem, dev;
};
static std::mutex g_occ_mu;
static OccKey g_occ_key[64];
static int g_occ_val[64];
static int g_occ_n = 0;

int sm_count(int dev) {
    static int cache[64] = {0};
    if (dev < 0 || dev >= 64) return 1;
    if (cache[dev] == 0) {
        int n = 0;
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        cache[dev] = n > 0 ? n : 1;
    }
    return cache[dev];
}

cudaError_t occupancy_grid(const void* fn, int block, int smem, int* grid) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    {
        std::lock_guard<std::mutex> lk(g_occ_mu);
        for (int k = 0; k < g_occ_n; ++k)
            if (g_occ_key[k].fn == fn && g_occ_key[k].block == block &&
                g_occ_key[k].smem == smem && g_occ_key[k].dev == dev) {
                *grid = g_occ_val[k];
                return cudaSuccess;
            }
    }
    if (smem > 48 * 1024) {
        e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
    }
    int nb = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, block, smem);
    if (e != cudaSuccess) return e;
    if (nb < 1) return cudaErrorInvalidConfiguration;
    const int g = nb * sm_count(dev);
    std::lock_guard<std::mutex> lk(g_occ_mu);
    if (g_occ_n < 64) {
        g_occ_key[g_occ_n] = OccKey{fn, block, smem, dev};
        g_occ_val[g_occ_n] = g;
        ++g_occ_n;
    }
    *grid = g;
    return cudaSuccess;
}

int max_block(const void* fn, int block) {
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, fn) != cudaSuccess) return block;
    const int cap = (fa.maxThreadsPerBlock / 32) * 32;
    return block > cap ? cap : block;
}

cudaError_t launch_trace(const TraceParams& P, int mode, int stack, bool stats, int block,
                         int width, cudaStream_t s) {
    KernelFn fn = trace_kernel(mode, stack, stats, width, P.root < 0);
    block = max_block((const void*)fn, block);  // register-limited kernels cap the block
    const int smem = P.smem_nodes > 0 ? P.smem_nodes * 64 : 0;
    int grid = 0;
    cudaError_t e = occupancy_grid((const void*)fn, block, smem, &grid);
    if (e != cudaSuccess) return e;
    // chunk size: about four chunks per resident warp, a multiple of 32 in
    // [kFetchMin, kFetchChunk]
    const int64_t warps = (int64_t)grid * (block / 32);
    int64_t f = P.nR / (4 * warps);
    f = f < kFetchMin ? kFetchMin : f > kFetchChunk ? kFetchChunk : f / 32 * 32;
    TraceParams Q = P;
    Q.fetch = (int)f;
    const int64_t warps_needed = (P.nR + f - 1) / f;
    const int64_t blocks_needed = (warps_needed + block / 32 - 1) / (block / 32);
    if (blocks_needed < grid) grid = (int)blocks_needed;
    if (grid < 1) grid = 1;
    e = cudaMemsetAsync(P.work, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    if (P.out.hit_idx) {
        e = cudaMemsetAsync(P.out.n_hits, 0, sizeof(int64_t), s);
        if (e != cudaSuccess) return e;
    }
    fn<<<grid, block, smem, s>>>(Q);
    return cudaGetLastError();
}

}  // namespace rsi
