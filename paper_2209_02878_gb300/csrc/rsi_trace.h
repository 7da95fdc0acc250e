// Host-side traversal / backward / batch launchers shared between the
// translation units of librsi.
#pragma once

#include <cuda_runtime.h>

#include "traverse_core.cuh"

namespace rsi {

struct TraceParams {
    const float* A;
    const float* B;
    int64_t nR;
    int root;  // treelet node ~0, a global root slot, or kNoRoot
    const float4* nodes;
    const float4* tris;
    const float4* treelet;
    const int32_t* treelet_n;
    int smem_nodes;
    unsigned long long* work;   // zeroed before each launch
    unsigned long long* stats;  // 6 counters (STATS launches)
    int max_visits;             // node fetches per segment before giving up
    int32_t* status;
    TravOut out;
};

// Enqueue one traversal (2 memsets + 1 kernel).
cudaError_t launch_trace(const TraceParams& P, int mode, int stack, bool stats, int block,
                         cudaStream_t s);

// Persistent grid size for a kernel / block size / dynamic smem (cached).
cudaError_t occupancy_grid(const void* fn, int block, int smem, int* grid);
int sm_count(int dev);

cudaError_t launch_backward(const float* V, int64_t nV, const int32_t* T, int64_t nT,
                            const float* A, const float* B, int64_t nR, const int32_t* tri,
                            const float* tuv, const float* gP, const float* gtuv, float* gV,
                            float* gA, float* gB, cudaStream_t s);

// Batched traversal over items (see batched.cu).
struct BatchItemDev {
    const float* A;
    const float* B;
    int64_t nR;
    int root;  // root slot of the item's mesh, or kNoRoot
    int mode;
    int64_t chunk0;  // first 32-segment chunk of this item in the work order
    TravOut out;
};

struct BatchParams {
    const BatchItemDev* items;
    int n_items;
    int64_t n_chunks;
    const float4* nodes;
    const float4* tris;
    unsigned long long* work;
    int max_visits;
    int32_t* status;
};

cudaError_t launch_batch(const BatchParams& P, int block, int stack, cudaStream_t s);
const void* batch_kernel(int stack);

}  // namespace rsi
