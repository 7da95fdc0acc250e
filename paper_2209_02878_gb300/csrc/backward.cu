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
// (the only cross-segment reduction).  The per-segment algebra and the
// vertex accumulation run in FP64 -- (t, u, v) recomputed from the geometry
// as in the definition -- because a vertex gradient is a sum of a few
// contributions that can cancel, and FP32 atomics would leave an absolute
// error proportional to the sum of their magnitudes; the total is rounded
// to FP32 once.
#include <cuda_runtime.h>

#include "rsi_trace.h"

namespace rsi {

__global__ void k_backward(const float* __restrict__ V, int64_t nV, const int32_t* __restrict__ T,
                           int64_t nT, const float* __restrict__ A, const float* __restrict__ B,
                           int64_t nR, const int32_t* __restrict__ tri,
                           const float* __restrict__ gP, const float* __restrict__ gtuv,
                           double* __restrict__ gV64, float* __restrict__ gA,
                           float* __restrict__ gB) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nR) return;
    const int j = tri[i];
    double ga[3] = {0.0, 0.0, 0.0}, gb[3] = {0.0, 0.0, 0.0};
    if (j >= 0 && j < nT) {
        const int64_t i0 = T[3 * (int64_t)j], i1 = T[3 * (int64_t)j + 1], i2 = T[3 * (int64_t)j + 2];
        if (i0 >= 0 && i0 < nV && i1 >= 0 && i1 < nV && i2 >= 0 && i2 < nV) {
            double d[3], e1[3], e2[3], s0[3], nd[3];
            for (int k = 0; k < 3; ++k) {
                const double a = A[3 * i + k], v0 = V[3 * i0 + k];
                d[k] = (double)B[3 * i + k] - a;
                nd[k] = -d[k];
                e1[k] = (double)V[3 * i1 + k] - v0;
                e2[k] = (double)V[3 * i2 + k] - v0;
                s0[k] = a - v0;
            }
            const double c12[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2],
                                   e1[0] * e2[1] - e1[1] * e2[0]};
            const double c20[3] = {e2[1] * nd[2] - e2[2] * nd[1], e2[2] * nd[0] - e2[0] * nd[2],
                                   e2[0] * nd[1] - e2[1] * nd[0]};
            const double c01[3] = {nd[1] * e1[2] - nd[2] * e1[1], nd[2] * e1[0] - nd[0] * e1[2],
                                   nd[0] * e1[1] - nd[1] * e1[0]};
            const double detM = nd[0] * c12[0] + nd[1] * c12[1] + nd[2] * c12[2];
            if (detM != 0.0) {
                // x = M^-1 (a - v0): the rows of M^-1 are c12, c20, c01 over det M
                const double inv = 1.0 / detM;
                const double t = (c12[0] * s0[0] + c12[1] * s0[1] + c12[2] * s0[2]) * inv;
                const double u = (c20[0] * s0[0] + c20[1] * s0[1] + c20[2] * s0[2]) * inv;
                const double v = (c01[0] * s0[0] + c01[1] * s0[1] + c01[2] * s0[2]) * inv;
                double gp[3] = {0.0, 0.0, 0.0};
                if (gP) {
                    gp[0] = gP[3 * i];
                    gp[1] = gP[3 * i + 1];
                    gp[2] = gP[3 * i + 2];
                }
                double gx0 = gp[0] * d[0] + gp[1] * d[1] + gp[2] * d[2];
                double gx1 = 0.0, gx2 = 0.0;
                if (gtuv) {
                    gx0 += gtuv[3 * i];
                    gx1 = gtuv[3 * i + 1];
                    gx2 = gtuv[3 * i + 2];
                }
                const double w = 1.0 - u - v;
                for (int k = 0; k < 3; ++k) {
                    const double lam = (gx0 * c12[k] + gx1 * c20[k] + gx2 * c01[k]) * inv;
                    const double sk = gp[k] + lam;
                    ga[k] = (1.0 - t) * sk;
                    gb[k] = t * sk;
                    if (gV64) {
                        atomicAdd(gV64 + 3 * i0 + k, -w * lam);
                        atomicAdd(gV64 + 3 * i1 + k, -u * lam);
                        atomicAdd(gV64 + 3 * i2 + k, -v * lam);
                    }
                }
            }
        }
    }
    if (gA)
        for (int k = 0; k < 3; ++k) gA[3 * i + k] = (float)ga[k];
    if (gB)
        for (int k = 0; k < 3; ++k) gB[3 * i + k] = (float)gb[k];
}

// dGradV += the FP64 accumulator, rounded once.
__global__ void k_add_grad(float* __restrict__ gV, const double* __restrict__ gV64, int64_t n) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) gV[k] = (float)((double)gV[k] + gV64[k]);
}

cudaError_t launch_backward(const float* V, int64_t nV, const int32_t* T, int64_t nT,
                            const float* A, const float* B, int64_t nR, const int32_t* tri,
                            const float* gP, const float* gtuv, float* gV, float* gA, float* gB,
                            cudaStream_t s) {
    if (nR == 0) return cudaSuccess;
    const int block = 256;
    double* acc = nullptr;
    const size_t bytes = sizeof(double) * 3 * (size_t)(nV > 0 ? nV : 1);
    cudaError_t e = cudaSuccess;
    const AllocHooks hooks = current_hooks();
    if (gV) {
        e = dev_alloc(hooks, (void**)&acc, bytes, s);
        if (e != cudaSuccess) return e;
        e = cudaMemsetAsync(acc, 0, bytes, s);
        if (e != cudaSuccess) {
            dev_free(hooks, acc, s);
            return e;
        }
    }
    k_backward<<<(unsigned)((nR + block - 1) / block), block, 0, s>>>(V, nV, T, nT, A, B, nR, tri,
                                                                     gP, gtuv, acc, gA, gB);
    e = cudaGetLastError();
    if (gV && e == cudaSuccess && nV > 0) {
        k_add_grad<<<(unsigned)((3 * nV + block - 1) / block), block, 0, s>>>(gV, acc, 3 * nV);
        e = cudaGetLastError();
    }
    if (acc) {
        const cudaError_t f = dev_free(hooks, acc, s);
        if (e == cudaSuccess) e = f;
    }
    return e;
}

}  // namespace rsi
