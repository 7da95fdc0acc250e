// Odd-parity point classification (paper Sec. 2.6: the number of crossings
// returned by the intercept_count mode identifies segment starting points
// inside a closed surface).  Each point p gets the segment p -> p + L u, u a
// fixed direction with no zero or repeated component (so the segment is not
// axis-aligned and does not run along a grid diagonal) and L long enough to
// leave the mesh box; an odd crossing count means p is inside.
#include <cuda_runtime.h>
#include <stdint.h>

#include "rsi_trace.h"

namespace rsi {

__global__ void k_inside_segments(const float* __restrict__ P, int64_t n,
                                  const float4* __restrict__ rootbox, float* __restrict__ B) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float4 lo = rootbox[0], hi = rootbox[1];
    const float u[3] = {0.5773503f, 0.5773113f, 0.5773892f};
    const float c[3] = {0.5f * (lo.x + hi.x), 0.5f * (lo.y + hi.y), 0.5f * (lo.z + hi.z)};
    const float e = fmaxf(fmaxf(hi.x - lo.x, hi.y - lo.y), hi.z - lo.z);
    float far2 = 0.f;
    for (int k = 0; k < 3; ++k) {
        const float d = P[3 * i + k] - c[k];
        far2 += d * d;
    }
    // |p - c| + 2 * (largest extent) reaches beyond the box from any point
    const float L = sqrtf(far2) + 2.f * e + 1.f;
    for (int k = 0; k < 3; ++k) B[3 * i + k] = P[3 * i + k] + L * u[k];
}

__global__ void k_parity(const int32_t* __restrict__ count, int64_t n, uint8_t* __restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = (uint8_t)(count[i] & 1);
}

cudaError_t launch_inside_segments(const float* P, int64_t n, const float4* rootbox, float* B,
                                   cudaStream_t s) {
    k_inside_segments<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(P, n, rootbox, B);
    return cudaGetLastError();
}

cudaError_t launch_parity(const int32_t* count, int64_t n, uint8_t* out, cudaStream_t s) {
    k_parity<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(count, n, out);
    return cudaGetLastError();
}

}  // namespace rsi
