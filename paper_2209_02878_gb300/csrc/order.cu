// Coherent processing order of the segments (the paper's v2.2, Sec. 4.1:
// Morton-sorted rays halve the traversal time by reducing divergence).
//
// Key of a segment: Morton code of its midpoint quantised over the mesh box
// grown by its own extent on every side (p bits per axis), then the octant of
// its direction (3 bits) as the lowest bits, so a warp receives segments that
// start near each other and point the same way.  The order only changes
// which lane processes which segment when; every output is still written to
// the segment's own index, so results do not depend on it.
#include <cuda_runtime.h>
#include <stdint.h>

#include "rsi_trace.h"
#include "sort.cuh"

namespace rsi {

__device__ __forceinline__ uint32_t spread_bits3(uint32_t x) {
    x &= 0x3ffu;
    x = (x | (x << 16)) & 0x030000ffu;
    x = (x | (x << 8)) & 0x0300f00fu;
    x = (x | (x << 4)) & 0x030c30c3u;
    x = (x | (x << 2)) & 0x09249249u;
    return x;
}

__global__ void k_seg_keys(const float* __restrict__ A, const float* __restrict__ B, int n,
                           const float4* __restrict__ rootbox, int pbits,
                           uint32_t* __restrict__ keys, uint32_t* __restrict__ vals) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float4 lo = rootbox[0], hi = rootbox[1];
    const float levels = (float)(1u << pbits);
    float a[3], b[3], l[3] = {lo.x, lo.y, lo.z}, h[3] = {hi.x, hi.y, hi.z};
    uint32_t q[3];
    uint32_t oct = 0;
    bool ok = true;
    for (int k = 0; k < 3; ++k) {
        a[k] = A[3 * (int64_t)i + k];
        b[k] = B[3 * (int64_t)i + k];
        const float ext = fmaxf(h[k] - l[k], 1e-30f);
        const float m = 0.5f * (a[k] + b[k]);
        float x = (m - (l[k] - ext)) / (3.f * ext) * levels;
        ok = ok && isfinite(x);
        x = fminf(fmaxf(x, 0.f), levels - 1.f);
        q[k] = ok ? (uint32_t)x : 0u;
        oct |= (b[k] < a[k] ? 1u : 0u) << (2 - k);
    }
    const uint32_t code = (spread_bits3(q[0]) << 2) | (spread_bits3(q[1]) << 1) | spread_bits3(q[2]);
    keys[i] = ok ? ((code << 3) | oct) : 0xffffffffu;
    vals[i] = (uint32_t)i;
}

cudaError_t segment_order(const float* A, const float* B, int n, const float4* rootbox, int bits,
                          SegOrderWs& ws, cudaStream_t s, const int32_t** order) {
    const int pbits = (bits - 3) / 3;
    k_seg_keys<<<(n + 255) / 256, 256, 0, s>>>(A, B, n, rootbox, pbits, ws.keys[0], ws.vals[0]);
    int shifts[4], np = 0;
    for (int sh = 0; sh < 3 * pbits + 3; sh += 8) shifts[np++] = sh;
    int cur = 0;
    cudaError_t e = radix_sort<uint32_t>(ws.keys, ws.vals, n, shifts, np, ws.hist, ws.totals, s,
                                         &cur);
    *order = (const int32_t*)ws.vals[cur];
    return e;
}

}  // namespace rsi
