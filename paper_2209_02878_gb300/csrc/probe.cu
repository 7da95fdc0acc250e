// Measurement and self-test utilities (not part of the paper's method).
//
// FP32 peak probe: the FP32 ceiling against which the traversal's box and
// triangle arithmetic is compared (the traversal's own roofline is HBM
// bandwidth nominally, issue rate in practice; this gives the third
// ceiling).  Not part of the paper's method.
//
// Every thread runs kChains independent FMA chains for `iters` rounds, so
// the FMA pipes never wait on a dependency; the grid fills every SM.  The
// result is written only if it equals a value it cannot reach, which keeps
// the chains live without memory traffic.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include "rsi.h"
#include "rsi_trace.h"

namespace {

constexpr int kChains = 8;
constexpr int kProbeBlock = 256;

__global__ void k_fma_probe(int64_t iters, float a, float b, float* sink) {
    float x[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = (float)(threadIdx.x + k);
    for (int64_t r = 0; r < iters; ++r) {
#pragma unroll
        for (int k = 0; k < kChains; ++k) x[k] = fmaf(x[k], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += x[k];
    if (s == -1.2345f) sink[0] = s;  // never true for the arguments used
}

// One warp waits on a flag that nothing sets, with the traversal's bounded
// wait; the wait gives up after `polls` polls and latches the status.
__global__ void k_wait_selftest(const int32_t* flag, int32_t* status, int polls) {
    rsi::wait_flag(flag, status, polls);
}

}  // namespace

extern "C" rsi_status rsi_selftest_wait(int32_t polls, rsi_stream s, int32_t* status_out) {
    if (polls < 1 || !status_out) return RSI_ERR_ARG;
    cudaStream_t cs = (cudaStream_t)s;
    const rsi::AllocHooks hooks = rsi::current_hooks();
    int32_t* mem = nullptr;  // [0] the flag, [1] the status word
    if (rsi::dev_alloc(hooks, (void**)&mem, 2 * sizeof(int32_t), cs) != cudaSuccess) {
        cudaGetLastError();
        return RSI_ERR_OOM;
    }
    rsi_status st = RSI_OK;
    if (cudaMemsetAsync(mem, 0, 2 * sizeof(int32_t), cs) != cudaSuccess) st = RSI_ERR_CUDA;
    if (st == RSI_OK) {
        k_wait_selftest<<<1, 32, 0, cs>>>(mem, mem + 1, polls);
        if (cudaGetLastError() != cudaSuccess ||
            cudaMemcpyAsync(status_out, mem + 1, sizeof(int32_t), cudaMemcpyDeviceToHost, cs) !=
                cudaSuccess ||
            cudaStreamSynchronize(cs) != cudaSuccess)
            st = RSI_ERR_CUDA;
    }
    rsi::dev_free(hooks, mem, cs);
    if (st != RSI_OK) cudaGetLastError();
    return st;
}

extern "C" rsi_status rsi_selftest_stream_wait(int32_t polls, int64_t nR, rsi_stream s,
                                               int32_t* status_out, float* ms_out) {
    if (polls < 1 || nR < 1 || nR > (int64_t(1) << 26) || !status_out || !ms_out)
        return RSI_ERR_ARG;
    cudaStream_t cs = (cudaStream_t)s;
    const rsi::AllocHooks hooks = rsi::current_hooks();
    // segments (all zero), flags, the per-chunk ready flags that no copy
    // ever sets, the work counter and the status word
    const int64_t chunk = 32;
    const int64_t nc = (nR + chunk - 1) / chunk;
    const size_t seg_b = (12 * (size_t)nR + 255) / 256 * 256;
    const size_t flag_b = ((size_t)nR + 255) / 256 * 256;
    const size_t ready_b = (4 * (size_t)nc + 255) / 256 * 256;
    const size_t bytes = seg_b + flag_b + ready_b + 256;
    char* mem = nullptr;
    if (rsi::dev_alloc(hooks, (void**)&mem, bytes, cs) != cudaSuccess) {
        cudaGetLastError();
        return RSI_ERR_OOM;
    }
    rsi_status st = RSI_OK;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaMemsetAsync(mem, 0, bytes, cs) != cudaSuccess ||
        cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        st = RSI_ERR_CUDA;
    if (st == RSI_OK) {
        rsi::TraceParams P;
        memset(&P, 0, sizeof(P));
        P.A = (const float*)mem;  // A and B alias: zero-length segments
        P.B = (const float*)mem;
        P.nR = nR;
        P.root = rsi::kNoRoot;  // no mesh: a segment, once its chunk is in, misses
        P.root4 = rsi::kNoRoot;
        P.out.flag = (uint8_t*)(mem + seg_b);
        P.ready = (const int32_t*)(mem + seg_b + flag_b);
        P.ready_chunk = chunk;
        P.wait_polls = polls;
        P.work = (unsigned long long*)(mem + seg_b + flag_b + ready_b);
        P.status = (int32_t*)(mem + seg_b + flag_b + ready_b + 128);
        P.max_visits = 2;
        if (cudaEventRecord(e0, cs) != cudaSuccess ||
            rsi::launch_trace(P, RSI_MODE_BOOL, 64, false, 128, 2, cs) != cudaSuccess ||
            cudaEventRecord(e1, cs) != cudaSuccess ||
            cudaMemcpyAsync(status_out, P.status, sizeof(int32_t), cudaMemcpyDeviceToHost, cs) !=
                cudaSuccess ||
            cudaStreamSynchronize(cs) != cudaSuccess ||
            cudaEventElapsedTime(ms_out, e0, e1) != cudaSuccess)
            st = RSI_ERR_CUDA;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    rsi::dev_free(hooks, mem, cs);
    if (st != RSI_OK) cudaGetLastError();
    return st;
}

extern "C" rsi_status rsi_fp32_peak(int64_t iters, double* tflops, rsi_stream s) {
    if (iters < 1 || !tflops) return RSI_ERR_ARG;
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fma_probe, kProbeBlock, 0) !=
            cudaSuccess) {
        cudaGetLastError();
        return RSI_ERR_CUDA;
    }
    const int grid = sms * (per_sm > 0 ? per_sm : 1);
    cudaStream_t cs = (cudaStream_t)s;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    float* sink = nullptr;
    rsi_status st = RSI_OK;
    const rsi::AllocHooks hooks = rsi::current_hooks();
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess ||
        rsi::dev_alloc(hooks, (void**)&sink, sizeof(float), cs) != cudaSuccess) {
        st = RSI_ERR_CUDA;
    } else {
        // a,b keep the chains finite: x -> 0.5 x + 0.25 converges to 0.5
        k_fma_probe<<<grid, kProbeBlock, 0, cs>>>(iters / 8 + 1, 0.5f, 0.25f, sink);  // warm-up
        cudaEventRecord(e0, cs);
        k_fma_probe<<<grid, kProbeBlock, 0, cs>>>(iters, 0.5f, 0.25f, sink);
        cudaEventRecord(e1, cs);
        float ms = 0.f;
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) !=
                                                           cudaSuccess || ms <= 0.f) {
            st = RSI_ERR_CUDA;
        } else {
            const double flops = 2.0 * kChains * (double)iters * grid * kProbeBlock;
            *tflops = flops / (ms * 1e-3) / 1e12;
        }
    }
    if (sink) rsi::dev_free(hooks, sink, cs);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (cudaGetLastError() != cudaSuccess && st == RSI_OK) st = RSI_ERR_CUDA;
    return st;
}
