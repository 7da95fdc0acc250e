// Host-side traversal / backward / batch launchers shared between the
// translation units of librsi.
#pragma once

#include <cuda_runtime.h>

#include "traverse_core.cuh"

namespace rsi {

// Device allocator in effect (rsi_set_allocator); null hooks mean
// cudaMallocAsync / cudaFreeAsync.  alloc.cu.
struct AllocHooks {
    rsi_alloc_fn alloc;
    rsi_free_fn free;
    void* ctx;
};
AllocHooks current_hooks();
cudaError_t dev_alloc(const AllocHooks& h, void** p, size_t bytes, cudaStream_t s);
cudaError_t dev_free(const AllocHooks& h, void* p, cudaStream_t s);

struct TraceParams {
    const float* A;
    const float* B;
    int64_t nR;
    int root;   // treelet node ~0, a global root slot, or kNoRoot
    int root4;  // root slot for 4-wide traversal
    const float4* nodes;
    const float4* nodes4;
    const float4* tris;
    const float4* treelet;
    const int32_t* treelet_n;
    int smem_nodes;
    unsigned long long* work;   // zeroed before each launch
    unsigned long long* stats;  // 6 counters (STATS launches)
    int max_visits;             // node fetches per segment before giving up
    int fetch;                  // segments per warp fetch (set by launch_trace)
    const int32_t* ready;       // streamed input flags (see TraceCtx), or nullptr
    int64_t ready_chunk;
    int wait_polls;             // polls of a ready flag before giving up (0: kWaitPolls)
    const int32_t* order;       // optional coherent processing order (nullptr = identity)
    int32_t* status;
    TravOut out;
};

// Enqueue one traversal (2 memsets + 1 kernel).
cudaError_t launch_trace(const TraceParams& P, int mode, int stack, bool stats, int block,
                         int width, cudaStream_t s);

// Enqueue one warp-cooperative (packet) traversal (packet.cu).
cudaError_t launch_trace_packet(const TraceParams& P, int mode, bool stats, cudaStream_t s);

// Persistent grid size for a kernel / block size / dynamic smem (cached).
cudaError_t occupancy_grid(const void* fn, int block, int smem, int* grid);
int sm_count(int dev);
// Largest multiple of 32 <= block that the kernel can launch with.
int max_block(const void* fn, int block);

// Workspace of the segment ordering (keys / values ping-pong, histograms).
struct SegOrderWs {
    uint32_t* keys[2];
    uint32_t* vals[2];
    uint32_t* hist;
    uint32_t* totals;
    int64_t cap;  // segments
};

// Enqueue the coherent order of n segments (keys + radix sort); *order
// points into ws when the stream reaches it.
cudaError_t segment_order(const float* A, const float* B, int n, const float4* rootbox, int bits,
                          SegOrderWs& ws, cudaStream_t s, const int32_t** order);

// Odd-parity classification helpers (inside.cu).
cudaError_t launch_inside_segments(const float* P, int64_t n, const float4* rootbox, float* B,
                                   cudaStream_t s);
cudaError_t launch_parity(const int32_t* count, int64_t n, uint8_t* out, cudaStream_t s);

// Adjoint of the nearest outputs (2 kernels + stream-ordered FP64 scratch).
cudaError_t launch_backward(const float* V, int64_t nV, const int32_t* T, int64_t nT,
                            const float* A, const float* B, int64_t nR, const int32_t* tri,
                            const float* gP, const float* gtuv, float* gV, float* gA, float* gB,
                            cudaStream_t s);

// Batched traversal over items (see batched.cu).
struct BatchItemDev {
    const float* A;
    const float* B;
    int64_t nR;
    int root;  // root slot of the item's mesh, or kNoRoot
    int mode;
    TravOut out;
};

struct BatchTile {  // a range of one item's segments, handed to one warp
    int32_t item;
    int32_t pad;
    int64_t lo, hi;
};

constexpr int kBatchTile = 1024;  // segments per tile

struct BatchParams {
    const BatchItemDev* items;
    int n_items;
    const BatchTile* tiles;
    int64_t n_tiles;
    const float4* nodes;
    const float4* nodes4;
    const float4* tris;
    unsigned long long* work;
    int max_visits;
    int32_t* status;
};

cudaError_t launch_batch(const BatchParams& P, int block, int stack, cudaStream_t s);
const void* batch_kernel(int stack);

}  // namespace rsi
