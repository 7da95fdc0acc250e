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
// (the only cross-segment reduction).  The per-segment algebra runs in
// double-float (pairs of floats from the error-free transformations, about
// 44 significant bits: the input differences are exact, (t, u, v) are
// recomputed from the geometry as in the definition) -- GB300's FP64 rate is
// a small fraction of its FP32 rate and the FP64 version of this kernel kept
// its FP64 pipe 83 % busy -- except where det M is small against its
// componentwise magnitude (|det M| <= 2^-16 sum |d_i| (|e1_j||e2_k| +
// |e1_k||e2_j|), a crossing at a grazing angle): lambda grows like 1/det M
// and the double-float cancellation error with it, so those segments run the
// whole algebra in FP64, in the same operation order as the closed form
// above.  The vertex accumulation uses FP64 atomics (done in L2), because a
// vertex gradient is a sum of a few contributions that can cancel; the total
// is rounded to FP32 once.
#include <cuda_runtime.h>

#include "rsi_trace.h"

namespace rsi {

namespace {

__device__ __forceinline__ dfl df_from(float x) { return {x, 0.f}; }

__device__ __forceinline__ dfl df_sub(dfl a, dfl b) { return df_add(a, df_neg(b)); }

__device__ __forceinline__ void df_cross(const dfl* x, const dfl* y, dfl* r) {
    r[0] = df_sub(df_mul(x[1], y[2]), df_mul(x[2], y[1]));
    r[1] = df_sub(df_mul(x[2], y[0]), df_mul(x[0], y[2]));
    r[2] = df_sub(df_mul(x[0], y[1]), df_mul(x[1], y[0]));
}

__device__ __forceinline__ dfl df_dot(const dfl* x, const dfl* y) {
    return df_add(df_add(df_mul(x[0], y[0]), df_mul(x[1], y[1])), df_mul(x[2], y[2]));
}

__device__ __forceinline__ double df_double(dfl a) { return (double)a.h + (double)a.l; }

// |det M| / (componentwise magnitude of det M) below which the algebra runs
// in FP64 (see above).
constexpr float kAdjointFp64Ratio = 0x1p-16f;

__device__ __forceinline__ void cross64(const double* x, const double* y, double* r) {
    r[0] = __dsub_rn(__dmul_rn(x[1], y[2]), __dmul_rn(x[2], y[1]));
    r[1] = __dsub_rn(__dmul_rn(x[2], y[0]), __dmul_rn(x[0], y[2]));
    r[2] = __dsub_rn(__dmul_rn(x[0], y[1]), __dmul_rn(x[1], y[0]));
}

__device__ __forceinline__ double dot64(const double* x, const double* y) {
    return __dadd_rn(__dadd_rn(__dmul_rn(x[0], y[0]), __dmul_rn(x[1], y[1])),
                     __dmul_rn(x[2], y[2]));
}

// The adjoint of one segment in FP64 (no contraction, every operation
// rounded where written): x = M^-1 (a - v0) by the rows c12, c20, c01 of
// the adjugate, lambda = (g_x0 c12 + g_x1 c20 + g_x2 c01) / det M, then the
// endpoint gradients written to gA / gB (each may be null) and the vertex
// sums added to gV64.  A zero or non-finite det M contributes nothing (zero
// endpoint gradients).
__device__ __noinline__ void adjoint64(const float* V, int64_t i0, int64_t i1, int64_t i2,
                                       const float* A, const float* B, int64_t i, const float* gP,
                                       const float* gtuv, double* gV64, float* gA, float* gB) {
    double a[3], d[3], nd[3], e1[3], e2[3], s0[3];
    for (int k = 0; k < 3; ++k) {
        a[k] = A[3 * i + k];
        const double v0 = V[3 * i0 + k];
        d[k] = __dsub_rn((double)B[3 * i + k], a[k]);
        nd[k] = -d[k];
        e1[k] = __dsub_rn((double)V[3 * i1 + k], v0);
        e2[k] = __dsub_rn((double)V[3 * i2 + k], v0);
        s0[k] = __dsub_rn(a[k], v0);
    }
    double c12[3], c20[3], c01[3];
    cross64(e1, e2, c12);
    cross64(e2, nd, c20);
    cross64(nd, e1, c01);
    const double detM = dot64(nd, c12);
    if (detM == 0.0 || !isfinite(detM)) {
        for (int k = 0; k < 3; ++k) {
            if (gA) gA[3 * i + k] = 0.f;
            if (gB) gB[3 * i + k] = 0.f;
        }
        return;
    }
    const double t = __ddiv_rn(dot64(c12, s0), detM);
    const double u = __ddiv_rn(dot64(c20, s0), detM);
    const double v = __ddiv_rn(dot64(c01, s0), detM);
    double gp[3] = {0.0, 0.0, 0.0};
    if (gP)
        for (int k = 0; k < 3; ++k) gp[k] = gP[3 * i + k];
    const double gpd = gP ? dot64(gp, d) : 0.0;
    const double gx0 = __dadd_rn(gtuv ? (double)gtuv[3 * i] : 0.0, gpd);
    const double gx1 = gtuv ? (double)gtuv[3 * i + 1] : 0.0;
    const double gx2 = gtuv ? (double)gtuv[3 * i + 2] : 0.0;
    const double w = __dsub_rn(__dsub_rn(1.0, u), v);
    const double omt = __dsub_rn(1.0, t);
    for (int k = 0; k < 3; ++k) {
        const double num = __dadd_rn(__dadd_rn(__dmul_rn(gx0, c12[k]), __dmul_rn(gx1, c20[k])),
                                     __dmul_rn(gx2, c01[k]));
        const double lam = __ddiv_rn(num, detM);
        const double sk = __dadd_rn(gp[k], lam);
        if (gA) gA[3 * i + k] = (float)__dmul_rn(omt, sk);
        if (gB) gB[3 * i + k] = (float)__dmul_rn(t, sk);
        if (gV64) {
            atomicAdd(gV64 + 3 * i0 + k, __dmul_rn(-w, lam));
            atomicAdd(gV64 + 3 * i1 + k, __dmul_rn(-u, lam));
            atomicAdd(gV64 + 3 * i2 + k, __dmul_rn(-v, lam));
        }
    }
}

}  // namespace

__global__ void k_backward(const float* __restrict__ V, int64_t nV, const int32_t* __restrict__ T,
                           int64_t nT, const float* __restrict__ A, const float* __restrict__ B,
                           int64_t nR, const int32_t* __restrict__ tri,
                           const float* __restrict__ gP, const float* __restrict__ gtuv,
                           double* __restrict__ gV64, float* __restrict__ gA,
                           float* __restrict__ gB) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nR) return;
    const int j = tri[i];
    float ga[3] = {0.f, 0.f, 0.f}, gb[3] = {0.f, 0.f, 0.f};
    if (j >= 0 && j < nT) {
        const int64_t i0 = T[3 * (int64_t)j], i1 = T[3 * (int64_t)j + 1], i2 = T[3 * (int64_t)j + 2];
        if (i0 >= 0 && i0 < nV && i1 >= 0 && i1 < nV && i2 >= 0 && i2 < nV) {
            dfl d[3], nd[3], e1[3], e2[3], s0[3];
            for (int k = 0; k < 3; ++k) {
                const float a = A[3 * i + k], v0 = V[3 * i0 + k];
                d[k] = df_two_sum(B[3 * i + k], -a);
                nd[k] = df_neg(d[k]);
                e1[k] = df_two_sum(V[3 * i1 + k], -v0);
                e2[k] = df_two_sum(V[3 * i2 + k], -v0);
                s0[k] = df_two_sum(a, -v0);
            }
            dfl c12[3], c20[3], c01[3];
            df_cross(e1, e2, c12);
            df_cross(e2, nd, c20);
            df_cross(nd, e1, c01);
            const dfl detM = df_dot(nd, c12);
            // componentwise magnitude of det M = -d . (e1 x e2)
            float mag = 0.f;
            for (int k = 0; k < 3; ++k) {
                const int k1 = k == 2 ? 0 : k + 1, k2 = k == 0 ? 2 : k - 1;
                mag = fmaf(fabsf(d[k].h),
                           fmaf(fabsf(e1[k1].h), fabsf(e2[k2].h), fabsf(e1[k2].h) * fabsf(e2[k1].h)),
                           mag);
            }
            if (!(fabsf(detM.h) > kAdjointFp64Ratio * mag)) {
                // grazing crossing (or det M zero / not finite): FP64, which
                // writes this segment's endpoint gradients itself
                adjoint64(V, i0, i1, i2, A, B, i, gP, gtuv, gV64, gA, gB);
                return;
            } else {
                // x = M^-1 (a - v0): the rows of M^-1 are c12, c20, c01 over det M
                const float r = rcp_approx(detM.h);
                const dfl t = df_div(df_dot(c12, s0), detM, r);
                const dfl u = df_div(df_dot(c20, s0), detM, r);
                const dfl v = df_div(df_dot(c01, s0), detM, r);
                float gp[3] = {0.f, 0.f, 0.f};
                if (gP) {
                    gp[0] = gP[3 * i];
                    gp[1] = gP[3 * i + 1];
                    gp[2] = gP[3 * i + 2];
                }
                const dfl gpd[3] = {df_from(gp[0]), df_from(gp[1]), df_from(gp[2])};
                dfl gx0 = df_dot(gpd, d), gx1 = df_from(0.f), gx2 = df_from(0.f);
                if (gtuv) {
                    gx0 = df_add(gx0, df_from(gtuv[3 * i]));
                    gx1 = df_from(gtuv[3 * i + 1]);
                    gx2 = df_from(gtuv[3 * i + 2]);
                }
                const dfl w = df_sub(df_sub(df_from(1.f), u), v);
                const dfl omt = df_sub(df_from(1.f), t);
                for (int k = 0; k < 3; ++k) {
                    const dfl num =
                        df_add(df_add(df_mul(gx0, c12[k]), df_mul(gx1, c20[k])), df_mul(gx2, c01[k]));
                    const dfl lam = df_div(num, detM, r);
                    const dfl sk = df_add(gpd[k], lam);
                    ga[k] = df_float(df_mul(omt, sk));
                    gb[k] = df_float(df_mul(t, sk));
                    if (gV64) {
                        atomicAdd(gV64 + 3 * i0 + k, -df_double(df_mul(w, lam)));
                        atomicAdd(gV64 + 3 * i1 + k, -df_double(df_mul(u, lam)));
                        atomicAdd(gV64 + 3 * i2 + k, -df_double(df_mul(v, lam)));
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
