// Adjoint of the nearest-crossing outputs (not in the paper): with the
// crossing triangle held fixed, the crossing solves
//     a + t d = v0 + u e1 + v e2,   i.e.  M x = a - v0,  M = [-d, e1, e2],
// x = (t, u, v).  For outputs P = (1-t) a + t b, t, u, v with incoming
// gradients gP, gt, gu, gv, implicit differentiation gives
//     g_x = (gt + gP.d, gu, gv),   lambda = M^-T g_x
//         = (g_x0 (e1 x e2) + g_x1 (e2 x -d) + g_x2 (-d x e1)) / det M,
//     dL/da = (1-t)(gP + lambda),  dL/db = t (gP + lambda),
//     dL/dv0 = -(1-u-v) lambda, dL/dv1 = -u lambda, dL/dv2 = -v lambda.
// One thread per segment; vertex gradients are scattered with atomicAdd
// (the only cross-segment reduction).  FP32.
#include <cuda_runtime.h>

#include "rsi_trace.h"

namespace rsi {

__global__ void k_backward(const float* __restrict__ V, int64_t nV, const int32_t* __restrict__ T,
                           int64_t nT, const float* __restrict__ A, const float* __restrict__ B,
                           int64_t nR, const int32_t* __restrict__ tri,
                           const float* __restrict__ tuv, const float* __restrict__ gP,
                           const float* __restrict__ gtuv, float* __restrict__ gV,
                           float* __restrict__ gA, float* __restrict__ gB) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nR) return;
    const int j = tri[i];
    float ga[3] = {0.f, 0.f, 0.f}, gb[3] = {0.f, 0.f, 0.f};
    if (j >= 0 && j < nT) {
        const int64_t i0 = T[3 * (int64_t)j], i1 = T[3 * (int64_t)j + 1], i2 = T[3 * (int64_t)j + 2];
        if (i0 >= 0 && i0 < nV && i1 >= 0 && i1 < nV && i2 >= 0 && i2 < nV) {
            float a[3], d[3], e1[3], e2[3];
            for (int k = 0; k < 3; ++k) {
                a[k] = A[3 * i + k];
                d[k] = B[3 * i + k] - a[k];
                const float v0 = V[3 * i0 + k];
                e1[k] = V[3 * i1 + k] - v0;
                e2[k] = V[3 * i2 + k] - v0;
            }
            const float nd[3] = {-d[0], -d[1], -d[2]};
            const float c12[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2],
                                  e1[0] * e2[1] - e1[1] * e2[0]};
            const float c20[3] = {e2[1] * nd[2] - e2[2] * nd[1], e2[2] * nd[0] - e2[0] * nd[2],
                                  e2[0] * nd[1] - e2[1] * nd[0]};
            const float c01[3] = {nd[1] * e1[2] - nd[2] * e1[1], nd[2] * e1[0] - nd[0] * e1[2],
                                  nd[0] * e1[1] - nd[1] * e1[0]};
            const float detM = nd[0] * c12[0] + nd[1] * c12[1] + nd[2] * c12[2];
            if (detM != 0.f) {
                const float t = tuv[3 * i], u = tuv[3 * i + 1], v = tuv[3 * i + 2];
                float gp[3] = {0.f, 0.f, 0.f};
                if (gP) {
                    gp[0] = gP[3 * i];
                    gp[1] = gP[3 * i + 1];
                    gp[2] = gP[3 * i + 2];
                }
                float gx0 = gp[0] * d[0] + gp[1] * d[1] + gp[2] * d[2];
                float gx1 = 0.f, gx2 = 0.f;
                if (gtuv) {
                    gx0 += gtuv[3 * i];
                    gx1 = gtuv[3 * i + 1];
                    gx2 = gtuv[3 * i + 2];
                }
                const float inv = 1.f / detM;
                const float w = 1.f - u - v;
                for (int k = 0; k < 3; ++k) {
                    const float lam = (gx0 * c12[k] + gx1 * c20[k] + gx2 * c01[k]) * inv;
                    const float s = gp[k] + lam;
                    ga[k] = (1.f - t) * s;
                    gb[k] = t * s;
                    if (gV) {
                        atomicAdd(gV + 3 * i0 + k, -w * lam);
                        atomicAdd(gV + 3 * i1 + k, -u * lam);
                        atomicAdd(gV + 3 * i2 + k, -v * lam);
                    }
                }
            }
        }
    }
    if (gA)
        for (int k = 0; k < 3; ++k) gA[3 * i + k] = ga[k];
    if (gB)
        for (int k = 0; k < 3; ++k) gB[3 * i + k] = gb[k];
}

cudaError_t launch_backward(const float* V, int64_t nV, const int32_t* T, int64_t nT,
                            const float* A, const float* B, int64_t nR, const int32_t* tri,
                            const float* tuv, const float* gP, const float* gtuv, float* gV,
                            float* gA, float* gB, cudaStream_t s) {
    if (nR == 0) return cudaSuccess;
    const int block = 256;
    const int64_t grid = (nR + block - 1) / block;
    k_backward<<<(unsigned)grid, block, 0, s>>>(V, nV, T, nT, A, B, nR, tri, tuv, gP, gtuv, gV,
                                                gA, gB);
    return cudaGetLastError();
}

}  // namespace rsi
