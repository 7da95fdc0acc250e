// Device-memory hooks: every device buffer the library allocates (handle
// storage, workspaces, staging, the adjoint's accumulator) goes through
// dev_alloc / dev_free, which call the caller's allocator when one is set
// (rsi_set_allocator; e.g. PyTorch's caching allocator, so the memory shows
// up in its pools) and stream-ordered cudaMallocAsync / cudaFreeAsync
// otherwise.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "rsi.h"
#include "rsi_trace.h"

namespace rsi {

namespace {
std::mutex g_hooks_mu;
AllocHooks g_hooks = {nullptr, nullptr, nullptr};
}  // namespace

AllocHooks current_hooks() {
    std::lock_guard<std::mutex> lk(g_hooks_mu);
    return g_hooks;
}

cudaError_t dev_alloc(const AllocHooks& h, void** p, size_t bytes, cudaStream_t s) {
    *p = nullptr;
    if (!h.alloc) return cudaMallocAsync(p, bytes, s);
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    void* q = h.alloc(bytes > 0 ? bytes : 1, dev, (rsi_stream)s, h.ctx);
    if (!q) return cudaErrorMemoryAllocation;
    if (((uintptr_t)q & 255) != 0) {  // the layouts inside assume 256-byte alignment
        h.free(q, dev, (rsi_stream)s, h.ctx);
        return cudaErrorMisalignedAddress;
    }
    *p = q;
    return cudaSuccess;
}

cudaError_t dev_free(const AllocHooks& h, void* p, cudaStream_t s) {
    if (!p) return cudaSuccess;
    if (!h.free) return cudaFreeAsync(p, s);
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    h.free(p, dev, (rsi_stream)s, h.ctx);
    return cudaSuccess;
}

}  // namespace rsi

extern "C" rsi_status rsi_set_allocator(rsi_alloc_fn alloc, rsi_free_fn free_fn, void* ctx) {
    if ((alloc == nullptr) != (free_fn == nullptr)) return RSI_ERR_ARG;
    std::lock_guard<std::mutex> lk(rsi::g_hooks_mu);
    rsi::g_hooks = rsi::AllocHooks{alloc, free_fn, ctx};
    return RSI_OK;
}
