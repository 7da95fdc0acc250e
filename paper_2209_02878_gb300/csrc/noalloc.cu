// rsi_intersect_backward_static: the nearest-hit adjoint without any device
// allocation.
//
// rsi_intersect_backward sums the vertex gradients in an FP64 scratch array
// that it allocates (cudaMallocAsync) and frees on every call.  Some callers
// cannot allocate at that point: hosts that reserve all device memory up
// front and forbid allocation afterwards (fixed memory budgets, real-time
// loops), code running while a CUDA graph is being captured into a memory
// pool it does not own, or code called back from inside a custom allocator
// that must not be re-entered.  This entry point keeps that scratch in a
// file-scope __device__ array of fixed size instead; the caller passes only
// its inputs and outputs.
//
// Properties a caller relies on:
//  - Capacity: at most kStaticMaxVertices vertices (nV); larger meshes are
//    rejected with RSI_ERR_CAPACITY before anything is enqueued.
//  - The array exists once per device that loads the library and stays
//    allocated until the process exits (6 MiB).
//  - Host code cannot use the array's name as a device address.  The first
//    call on each device (with that device current) looks the address up
//    with cudaGetSymbolAddress and remembers it.  The library is built
//    without relocatable device code, so this file is a module of its own:
//    under lazy module loading (the default since CUDA 12) that lookup is
//    what loads the module and commits the array's 6 MiB on the device.
//    Make that first call before reserving the rest of device memory and
//    before any stream capture starts.
//  - Every call shares the one array: each call clears the part it uses
//    (cudaMemsetAsync, which does not allocate) before accumulating, and the
//    array keeps the last call's sums afterwards.  Two calls whose work
//    overlaps on the GPU (different streams, no ordering between them) race
//    on the array and give wrong gradients: order them on one stream or
//    with events.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "rsi.h"
#include "rsi_trace.h"

namespace rsi {
// Defined in backward.cu.
__global__ void k_backward(const float* __restrict__ V, int64_t nV, const int32_t* __restrict__ T,
                           int64_t nT, const float* __restrict__ A, const float* __restrict__ B,
                           int64_t nR, const int32_t* __restrict__ tri,
                           const float* __restrict__ gP, const float* __restrict__ gtuv,
                           double* __restrict__ gV64, float* __restrict__ gA,
                           float* __restrict__ gB);
__global__ void k_add_grad(float* __restrict__ gV, const double* __restrict__ gV64, int64_t n);
}  // namespace rsi

namespace {

constexpr int64_t kStaticMaxVertices = RSI_STATIC_MAX_VERTICES;
constexpr int kMaxDevices = 64;

// FP64 vertex-gradient accumulator, 3 doubles per vertex.
__device__ __align__(256) double g_static_grad[3 * kStaticMaxVertices];

std::mutex g_addr_mu;
double* g_addr[kMaxDevices] = {nullptr};

// Device address of g_static_grad on the current device (looked up once per
// device).
rsi_status static_scratch(double** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return RSI_ERR_CUDA;
    }
    if (dev < 0 || dev >= kMaxDevices) return RSI_ERR_ARG;
    std::lock_guard<std::mutex> lk(g_addr_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_static_grad);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return RSI_ERR_CUDA;
        }
        g_addr[dev] = (double*)p;
    }
    *out = g_addr[dev];
    return RSI_OK;
}

}  // namespace

extern "C" rsi_status rsi_intersect_backward_static(
    const float* dV, int64_t nV, const int32_t* dT, int64_t nT, const float* dA, const float* dB,
    int64_t nR, const int32_t* dTri, const float* dGradPoint, const float* dGradTuv,
    float* dGradV, float* dGradA, float* dGradB, rsi_stream s) {
    if (nV < 0 || nT < 0 || nR < 0) return RSI_ERR_ARG;
    if (nV > kStaticMaxVertices) return RSI_ERR_CAPACITY;
    if (nR == 0) return RSI_OK;
    if (!dA || !dB || !dTri || (nT > 0 && (!dV || !dT))) return RSI_ERR_ARG;
    double* acc = nullptr;
    if (dGradV) {
        const rsi_status st = static_scratch(&acc);
        if (st != RSI_OK) return st;
    }
    cudaStream_t cs = (cudaStream_t)s;
    const int block = 256;
    if (acc && nV > 0 &&
        cudaMemsetAsync(acc, 0, sizeof(double) * 3 * (size_t)nV, cs) != cudaSuccess) {
        cudaGetLastError();
        return RSI_ERR_CUDA;
    }
    rsi::k_backward<<<(unsigned)((nR + block - 1) / block), block, 0, cs>>>(
        dV, nV, dT, nT, dA, dB, nR, dTri, dGradPoint, dGradTuv, acc, dGradA, dGradB);
    if (acc && nV > 0)
        rsi::k_add_grad<<<(unsigned)((3 * nV + block - 1) / block), block, 0, cs>>>(dGradV, acc,
                                                                                3 * nV);
    if (cudaGetLastError() != cudaSuccess) return RSI_ERR_CUDA;
    return RSI_OK;
}
