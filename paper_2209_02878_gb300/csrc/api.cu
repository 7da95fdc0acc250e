// C ABI of librsi (declarations and documentation in include/rsi.h).
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "rsi.h"
#include "rsi_build.h"
#include "rsi_trace.h"

using rsi::MeshArgs;
using rsi::MeshDesc;
using rsi::TreeBufs;

#define RSI_CK(call)                                                                   \
    do {                                                                               \
        cudaError_t e_ = (call);                                                       \
        if (e_ != cudaSuccess) {                                                       \
            cudaGetLastError();                                                        \
            return e_ == cudaErrorMemoryAllocation ? RSI_ERR_OOM : RSI_ERR_CUDA;       \
        }                                                                              \
    } while (0)

namespace {

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

constexpr int kDefaultBlock = 128;
constexpr int64_t kHostChunk = (int64_t)1 << 21;  // segments per pipeline chunk
constexpr int64_t kHostChunkInPlace = (int64_t)1 << 24;  // the same, BOOL read in place
constexpr int64_t kStreamChunk = (int64_t)1 << 20;  // segments per streamed copy (BOOL)
constexpr int64_t kStreamMaxChunks = 256;
constexpr int64_t kStreamMax = (int64_t)1 << 28;      // larger inputs take the chunked path

// Carves the device buffers of a tree over N triangles and M meshes out of
// one allocation.  With base == nullptr only the total size is computed.
size_t carve(TreeBufs& tb, int64_t N, int M, int nblk, char* base) {
    size_t off = 0;
    auto take = [&](size_t bytes) -> char* {
        char* p = base ? base + off : nullptr;
        off += align256(bytes > 0 ? bytes : 1);
        return p;
    };
    const int64_t n1 = N > 0 ? N : 1;
    tb.N = (int32_t)N;
    tb.M = M;
    tb.ntiles = (int32_t)((N + rsi::kSortTileMin - 1) / rsi::kSortTileMin);
    tb.nblk = nblk;
    tb.keys[0] = (uint64_t*)take(8 * n1);
    tb.keys[1] = (uint64_t*)take(8 * n1);
    tb.vals[0] = (uint32_t*)take(4 * n1);
    tb.vals[1] = (uint32_t*)take(4 * n1);
    tb.hist = (uint32_t*)take(4 * (size_t)rsi::kSortBins * (tb.ntiles > 0 ? tb.ntiles : 1));
    tb.totals = (uint32_t*)take(4 * (size_t)rsi::kSortBins);
    tb.partial = (float*)take(4 * 6 * (size_t)(nblk > 0 ? nblk : 1));
    tb.bounds = (float*)take(4 * 6 * (size_t)M);
    tb.rootbox = (float4*)take(16 * 2 * (size_t)M);
    tb.child = (int32_t*)take(4 * 2 * n1);
    tb.range = (int32_t*)take(4 * 2 * n1);
    tb.span = (int4*)take(16 * n1);
    tb.nspan = (int32_t*)take(4);
    tb.pre = (float4*)take(16 * 2 * n1);
    tb.suf = (float4*)take(16 * 2 * n1);
    tb.nbox = (float4*)take(16 * 2 * n1);
    tb.lbox = (float4*)take(16 * 2 * n1);
    tb.nodes = (float4*)take(16 * 4 * n1);
    tb.nodes4 = (float4*)take(16 * 8 * n1);
    tb.tris = (float4*)take(16 * 3 * n1);
    tb.treelet = (float4*)take(M == 1 ? 16 * 4 * (size_t)rsi::kTreeletMax : 16);
    tb.treelet_n = (int32_t*)take(4);
    tb.status = (int32_t*)take(4);
    return off;
}

rsi_status check_build_opts(const rsi_build_opts* o, int32_t* leaf, int32_t* levels,
                            int32_t* height) {
    *leaf = 1;
    *levels = 0;
    *height = 0;
    if (!o) return RSI_OK;
    if (o->leaf_size < 0 || o->leaf_size > rsi::kMaxLeaf) return RSI_ERR_ARG;
    if (o->top_levels < -1 || o->top_levels > 12) return RSI_ERR_ARG;
    if (o->height_axis < 0 || o->height_axis > 3) return RSI_ERR_ARG;
    *height = o->height_axis;
    if (o->leaf_size > 0) *leaf = o->leaf_size;
    if (o->top_levels > 0) *levels = o->top_levels;
    return RSI_OK;
}

struct LaunchCfg {
    int block, stack, smem_nodes, sort_bits, width;
    bool stats, packet;
    const int32_t* order;
};

rsi_status check_launch_opts(const rsi_launch_opts* lo, bool has_treelet, LaunchCfg* c) {
    c->block = kDefaultBlock;
    c->stack = 64;
    c->smem_nodes = 0;
    c->sort_bits = 0;
    c->width = 2;
    c->stats = false;
    c->packet = false;
    c->order = nullptr;
    int sm = 0;
    if (lo) {
        c->order = lo->order;
        if (lo->block_size != 0) {
            if (lo->block_size < 32 || lo->block_size > 1024 || lo->block_size % 32) return RSI_ERR_ARG;
            c->block = lo->block_size;
        }
        if (lo->stack_depth != 0) {
            if (lo->stack_depth != 8 && lo->stack_depth != 32 && lo->stack_depth != 64)
                return RSI_ERR_ARG;
            c->stack = lo->stack_depth;
        }
        if (lo->smem_nodes < -1 || lo->smem_nodes > rsi::kTreeletMax) return RSI_ERR_ARG;
        sm = lo->smem_nodes;
        if (lo->sort_bits != 0 && lo->sort_bits != -1 && (lo->sort_bits < 6 || lo->sort_bits > 30))
            return RSI_ERR_ARG;
        c->sort_bits = lo->sort_bits;
        if (lo->node_width != 0 && lo->node_width != 2 && lo->node_width != 4) return RSI_ERR_ARG;
        if (lo->node_width != 0) c->width = lo->node_width;
        c->stats = lo->stats != 0;
        if (lo->packet != 0 && lo->packet != 1) return RSI_ERR_ARG;
        if (lo->packet == 1 && (lo->node_width == 4 || lo->smem_nodes > 0)) return RSI_ERR_ARG;
        c->packet = lo->packet == 1;
    }
    if (has_treelet && sm > 0) c->smem_nodes = sm;
    if (c->smem_nodes > 0) c->width = 2;  // the treelet holds binary nodes
    return RSI_OK;
}

rsi_status check_output(rsi_mode mode, const rsi_output* out) {
    if (!out) return RSI_ERR_ARG;
    if (mode == RSI_MODE_BOOL && !out->flag) return RSI_ERR_ARG;
    if (mode == RSI_MODE_COUNT && !out->count) return RSI_ERR_ARG;
    if (mode == RSI_MODE_NEAREST && !out->tri) return RSI_ERR_ARG;
    if (mode != RSI_MODE_BOOL && out->hit_idx && (!out->n_hits || out->hit_cap < 0))
        return RSI_ERR_ARG;
    return RSI_OK;
}

rsi::TravOut trav_out(rsi_mode mode, const rsi_output* o) {
    rsi::TravOut t;
    memset(&t, 0, sizeof(t));
    t.flag = o->flag;
    t.count = o->count;
    t.tri = o->tri;
    t.tuv = o->tuv;
    t.point = o->point;
    t.dist = o->dist;
    if (mode != RSI_MODE_BOOL && o->hit_idx) {
        t.hit_idx = o->hit_idx;
        t.hit_cap = o->hit_cap;
        t.n_hits = o->n_hits;
        t.hit_tri = o->hit_tri;
        t.hit_dist = o->hit_dist;
        t.hit_point = o->hit_point;
        t.hit_count = o->hit_count;
    }
    return t;
}

}  // namespace

struct rsi_bvh_s {
    int device = 0;
    int64_t nV = 0, nT = 0;
    int32_t leaf = 1, levels = 0;
    TreeBufs tb;
    char* mem = nullptr;
    size_t bytes = 0;
    unsigned long long* scratch = nullptr;  // [0] work counter, [1..7] stats, [8..9] streamed counters
    bool built = false;
    bool nodes4_valid = false;  // 4-wide records built for the current tree
    // stream of the last call that queued work on the handle's memory: calls
    // on a handle are ordered (header), so it follows every earlier use, and
    // memory is released stream-ordered on it (on reallocation the current
    // call's stream plays that role)
    cudaStream_t stream = nullptr;
    char* seg_mem = nullptr;  // segment-order workspace (grown on demand)
    rsi::SegOrderWs seg_ws{};
    // host-buffer pipeline (rsi_intersect_host): two streams, double buffers
    cudaStream_t pst[2] = {nullptr, nullptr};
    cudaEvent_t pev_start = nullptr, pev_done[2] = {nullptr, nullptr};
    char* pipe_mem = nullptr;
    size_t pipe_bytes = 0;
    int32_t* one = nullptr;  // pinned host 1: the value of a streamed chunk's ready flag
    // streamed path: two staging slots used in turn; slot q is free again
    // once sev_free[q] (recorded after the traversal and copy back of the
    // last streamed call that used it) completes
    cudaEvent_t sev_free[2] = {nullptr, nullptr}, sev_reset = nullptr;
    bool sfree_valid[2] = {false, false};
    int sslot = 0;
    // odd-parity workspace (rsi_points_inside): segment ends + counts
    char* in_mem = nullptr;
    int64_t in_cap = 0;
    rsi::AllocHooks hooks{};  // device allocator of all this handle's memory
};

namespace {
// Grow the segment-order workspace of h to n segments (stream-ordered).
rsi_status ensure_seg_ws(rsi_bvh h, int64_t n, cudaStream_t s) {
    if (h->seg_mem && h->seg_ws.cap >= n) return RSI_OK;
    if (h->seg_mem) {
        rsi::dev_free(h->hooks, h->seg_mem, s);
        h->seg_mem = nullptr;
    }
    const int64_t ntiles = (n + rsi::kSortTileMin - 1) / rsi::kSortTileMin;
    const size_t b1 = align256(4 * (size_t)n);
    const size_t bh = align256(4 * (size_t)rsi::kSortBins * (size_t)(ntiles > 0 ? ntiles : 1));
    const size_t bytes = 4 * b1 + bh + align256(4 * rsi::kSortBins);
    cudaError_t e = rsi::dev_alloc(h->hooks, (void**)&h->seg_mem, bytes, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        h->seg_mem = nullptr;
        return e == cudaErrorMemoryAllocation ? RSI_ERR_OOM : RSI_ERR_CUDA;
    }
    char* p = h->seg_mem;
    h->seg_ws.keys[0] = (uint32_t*)p;
    h->seg_ws.keys[1] = (uint32_t*)(p + b1);
    h->seg_ws.vals[0] = (uint32_t*)(p + 2 * b1);
    h->seg_ws.vals[1] = (uint32_t*)(p + 3 * b1);
    h->seg_ws.hist = (uint32_t*)(p + 4 * b1);
    h->seg_ws.totals = (uint32_t*)(p + 4 * b1 + bh);
    h->seg_ws.cap = n;
    return RSI_OK;
}
}  // namespace

extern "C" {

const char* rsi_version(void) { return "librsi 1.0 (sm_103a)"; }

const char* rsi_status_string(rsi_status s) {
    switch (s) {
        case RSI_OK: return "ok";
        case RSI_ERR_ARG: return "invalid argument";
        case RSI_ERR_CUDA: return "CUDA runtime error";
        case RSI_ERR_OOM: return "device out of memory";
        case RSI_ERR_BAD_INDEX: return "triangle index out of range";
        case RSI_ERR_STACK_OVERFLOW: return "traversal stack overflow";
        case RSI_ERR_TIMEOUT: return "device-side wait timed out";
        case RSI_ERR_NOT_BUILT: return "tree not built";
        case RSI_ERR_INTERNAL: return "device-side consistency bound hit";
        case RSI_ERR_CAPACITY: return "problem exceeds the static scratch capacity";
    }
    return "unknown status";
}

rsi_status rsi_bvh_create(int64_t nV, int64_t nT, const rsi_build_opts* opt, rsi_stream s,
                          rsi_bvh* out) {
    if (!out) return RSI_ERR_ARG;
    *out = nullptr;
    if (nV < 0 || nT < 0 || nT >= (int64_t)1 << 31) return RSI_ERR_ARG;
    int32_t leaf, levels, height;
    rsi_status st = check_build_opts(opt, &leaf, &levels, &height);
    if (st != RSI_OK) return st;
    int device = 0;
    RSI_CK(cudaGetDevice(&device));
    RSI_CK(rsi::build_prepare());
    rsi_bvh h = new rsi_bvh_s();
    h->hooks = rsi::current_hooks();
    h->device = device;
    h->nV = nV;
    h->nT = nT;
    h->leaf = leaf;
    h->levels = levels;
    const int nblk = (int)((nT + rsi::kBuildChunk - 1) / rsi::kBuildChunk);
    TreeBufs tb;
    memset(&tb, 0, sizeof(tb));
    size_t bytes = carve(tb, nT, 1, nblk, nullptr) + 256;
    cudaStream_t cs = (cudaStream_t)s;
    cudaError_t e = rsi::dev_alloc(h->hooks, (void**)&h->mem, bytes, cs);
    if (e != cudaSuccess) {
        cudaGetLastError();
        delete h;
        return e == cudaErrorMemoryAllocation ? RSI_ERR_OOM : RSI_ERR_CUDA;
    }
    carve(tb, nT, 1, nblk, h->mem);
    h->scratch = (unsigned long long*)(h->mem + bytes - 256);
    tb.leaf_size = leaf;
    tb.height_axis = height;
    tb.top_levels = levels;
    tb.sorted = 0;
    h->tb = tb;
    h->bytes = bytes;
    h->stream = cs;
    e = cudaMemsetAsync(tb.status, 0, 4, cs);
    if (e == cudaSuccess) e = cudaMemsetAsync(tb.treelet_n, 0, 4, cs);
    if (e != cudaSuccess) {
        cudaGetLastError();
        rsi::dev_free(h->hooks, h->mem, cs);
        delete h;
        return RSI_ERR_CUDA;
    }
    *out = h;
    return RSI_OK;
}

rsi_status rsi_bvh_build(rsi_bvh h, const float* dV, const int32_t* dT, rsi_stream s) {
    if (!h) return RSI_ERR_ARG;
    if (h->nT > 0 && (!dV || !dT)) return RSI_ERR_ARG;
    MeshArgs ma;
    memset(&ma, 0, sizeof(ma));
    ma.M = 1;
    ma.one.V = dV;
    ma.one.T = dT;
    ma.one.nV = h->nV;
    ma.one.n = (int32_t)h->nT;
    ma.one.off = 0;
    ma.one.blk0 = 0;
    ma.one.nblk = h->tb.nblk;
    ma.one.height_axis = h->tb.height_axis;
    h->tb.leaf_size = h->leaf;
    h->tb.top_levels = h->levels;
    RSI_CK(rsi::build_tree(h->tb, ma, (cudaStream_t)s, false));
    h->built = true;
    h->nodes4_valid = false;
    h->stream = (cudaStream_t)s;
    return RSI_OK;
}

rsi_status rsi_build_bvh(const float* dV, int64_t nV, const int32_t* dT, int64_t nT,
                         const rsi_build_opts* opt, rsi_stream s, rsi_bvh* out) {
    rsi_status st = rsi_bvh_create(nV, nT, opt, s, out);
    if (st != RSI_OK) return st;
    st = rsi_bvh_build(*out, dV, dT, s);
    if (st != RSI_OK) {
        rsi_bvh_destroy(*out);
        *out = nullptr;
    }
    return st;
}

rsi_status rsi_refit(rsi_bvh h, const float* dV, const int32_t* dT, rsi_stream s) {
    if (!h || (h->nT > 0 && (!dV || !dT))) return RSI_ERR_ARG;
    if (!h->built) return RSI_ERR_NOT_BUILT;
    MeshArgs ma;
    memset(&ma, 0, sizeof(ma));
    ma.M = 1;
    ma.one.V = dV;
    ma.one.T = dT;
    ma.one.nV = h->nV;
    ma.one.n = (int32_t)h->nT;
    ma.one.nblk = h->tb.nblk;
    RSI_CK(rsi::build_tree(h->tb, ma, (cudaStream_t)s, true));
    h->nodes4_valid = false;
    h->stream = (cudaStream_t)s;
    return RSI_OK;
}

rsi_status rsi_bvh_status(rsi_bvh h, rsi_stream s) {
    if (!h) return RSI_ERR_ARG;
    int32_t v = 0;
    RSI_CK(cudaMemcpyAsync(&v, h->tb.status, 4, cudaMemcpyDeviceToHost, (cudaStream_t)s));
    RSI_CK(cudaStreamSynchronize((cudaStream_t)s));
    RSI_CK(cudaMemsetAsync(h->tb.status, 0, 4, (cudaStream_t)s));
    RSI_CK(cudaStreamSynchronize((cudaStream_t)s));
    return (rsi_status)v;
}

rsi_status rsi_bvh_get_info(rsi_bvh h, rsi_bvh_info* info) {
    if (!h || !info) return RSI_ERR_ARG;
    info->n_vertices = h->nV;
    info->n_triangles = h->nT;
    info->leaf_size = h->leaf;
    int32_t tn = 0;
    if (h->built && h->levels > 0) {
        RSI_CK(cudaStreamSynchronize(h->stream));
        RSI_CK(cudaMemcpy(&tn, h->tb.treelet_n, 4, cudaMemcpyDeviceToHost));
    }
    info->treelet_nodes = tn;
    info->device_bytes = (int64_t)h->bytes;
    return RSI_OK;
}

rsi_status rsi_bvh_destroy(rsi_bvh h) {
    if (!h) return RSI_ERR_ARG;
    int cur = 0;
    cudaGetDevice(&cur);
    if (cur != h->device) cudaSetDevice(h->device);
    // the internal streams of the host path are the handle's own: let their
    // work end before the memory they use goes back, on the stream of the
    // last call (which every use of the memory precedes)
    for (int q = 0; q < 2; ++q)
        if (h->pst[q]) cudaStreamSynchronize(h->pst[q]);
    if (h->seg_mem) rsi::dev_free(h->hooks, h->seg_mem, h->stream);
    if (h->pipe_mem) rsi::dev_free(h->hooks, h->pipe_mem, h->stream);
    if (h->in_mem) rsi::dev_free(h->hooks, h->in_mem, h->stream);
    for (int q = 0; q < 2; ++q) {
        if (h->pst[q]) cudaStreamDestroy(h->pst[q]);
        if (h->pev_done[q]) cudaEventDestroy(h->pev_done[q]);
    }
    if (h->pev_start) cudaEventDestroy(h->pev_start);
    for (int q = 0; q < 2; ++q)
        if (h->sev_free[q]) cudaEventDestroy(h->sev_free[q]);
    if (h->sev_reset) cudaEventDestroy(h->sev_reset);
    if (h->one) cudaFreeHost(h->one);
    cudaError_t e = rsi::dev_free(h->hooks, h->mem, h->stream);
    if (cur != h->device) cudaSetDevice(cur);
    delete h;
    if (e != cudaSuccess) {
        cudaGetLastError();
        return RSI_ERR_CUDA;
    }
    return RSI_OK;
}

rsi_status rsi_bvh_export(rsi_bvh h, rsi_stream s, float* bounds, uint32_t* codes, int32_t* order,
                          int32_t* left, int32_t* right, int32_t* range, float* nbox, float* lbox,
                          float* nodes) {
    if (!h) return RSI_ERR_ARG;
    if (!h->built) return RSI_ERR_NOT_BUILT;
    RSI_CK(cudaStreamSynchronize((cudaStream_t)s));
    RSI_CK(cudaStreamSynchronize(h->stream));
    const int64_t N = h->nT;
    const TreeBufs& tb = h->tb;
    if (bounds) RSI_CK(cudaMemcpy(bounds, tb.bounds, 24, cudaMemcpyDeviceToHost));
    if (N == 0) return RSI_OK;
    if (codes) {
        std::vector<uint64_t> k(N);
        RSI_CK(cudaMemcpy(k.data(), tb.keys[tb.sorted], 8 * N, cudaMemcpyDeviceToHost));
        for (int64_t i = 0; i < N; ++i) codes[i] = (uint32_t)k[i];
    }
    if (order) RSI_CK(cudaMemcpy(order, tb.vals[tb.sorted], 4 * N, cudaMemcpyDeviceToHost));
    if (left || right || range) {
        std::vector<int32_t> c(2 * N), r(2 * N);
        RSI_CK(cudaMemcpy(c.data(), tb.child, 8 * N, cudaMemcpyDeviceToHost));
        RSI_CK(cudaMemcpy(r.data(), tb.range, 8 * N, cudaMemcpyDeviceToHost));
        for (int64_t i = 0; i + 1 < N; ++i) {
            if (left) left[i] = c[2 * i];
            if (right) right[i] = c[2 * i + 1];
            if (range) {
                range[2 * i] = r[2 * i];
                range[2 * i + 1] = r[2 * i + 1];
            }
        }
    }
    auto boxes = [&](const float4* src, int64_t n, float* dst) -> rsi_status {
        std::vector<float4> b(2 * (n > 0 ? n : 1));
        if (n > 0) RSI_CK(cudaMemcpy(b.data(), src, 32 * n, cudaMemcpyDeviceToHost));
        for (int64_t i = 0; i < n; ++i) {
            dst[6 * i + 0] = b[2 * i].x;
            dst[6 * i + 1] = b[2 * i].y;
            dst[6 * i + 2] = b[2 * i].z;
            dst[6 * i + 3] = b[2 * i + 1].x;
            dst[6 * i + 4] = b[2 * i + 1].y;
            dst[6 * i + 5] = b[2 * i + 1].z;
        }
        return RSI_OK;
    };
    if (nbox) {
        rsi_status st = boxes(tb.nbox, N - 1, nbox);
        if (st != RSI_OK) return st;
    }
    if (lbox) {
        rsi_status st = boxes(tb.lbox, N, lbox);
        if (st != RSI_OK) return st;
    }
    if (nodes) RSI_CK(cudaMemcpy(nodes, tb.nodes, 64 * N, cudaMemcpyDeviceToHost));
    return RSI_OK;
}

static rsi_status intersect_impl(rsi_bvh h, const float* dA, const float* dB, int64_t nR,
                                 rsi_mode mode, const rsi_output* out, const rsi_launch_opts* lo,
                                 rsi_stream s, bool force_stats,
                                 unsigned long long* work = nullptr,
                                 const int32_t* ready = nullptr, int64_t ready_chunk = 1) {
    if (!h || nR < 0) return RSI_ERR_ARG;
    if (mode != RSI_MODE_BOOL && mode != RSI_MODE_COUNT && mode != RSI_MODE_NEAREST)
        return RSI_ERR_ARG;
    if (!out) return RSI_ERR_ARG;
    if (!h->built) return RSI_ERR_NOT_BUILT;
    LaunchCfg c;
    rsi_status st = check_launch_opts(lo, h->levels > 0 && h->nT > 0, &c);
    if (st != RSI_OK) return st;
    if (force_stats) c.stats = true;
    if (nR == 0) {  // no-op (the output arrays may be empty)
        if (mode != RSI_MODE_BOOL && out->hit_idx && out->n_hits)
            RSI_CK(cudaMemsetAsync(out->n_hits, 0, 8, (cudaStream_t)s));
        return RSI_OK;
    }
    st = check_output(mode, out);
    if (st != RSI_OK) return st;
    if (!dA || !dB) return RSI_ERR_ARG;
    rsi::TraceParams P;
    memset(&P, 0, sizeof(P));
    P.A = dA;
    P.B = dB;
    P.nR = nR;
    if (h->nT == 0)
        P.root = rsi::kNoRoot;
    else if (h->levels > 0)
        P.root = ~0;
    else
        P.root = (int)(h->nT - 1);
    P.root4 = h->nT > 0 ? (int)(h->nT - 1) : rsi::kNoRoot;
    P.nodes = h->tb.nodes;
    P.nodes4 = h->tb.nodes4;
    P.tris = h->tb.tris;
    P.treelet = h->tb.treelet;
    P.treelet_n = h->tb.treelet_n;
    P.smem_nodes = c.smem_nodes;
    P.work = work ? work : h->scratch;
    P.stats = h->scratch + 1;
    P.max_visits = (int)h->nT + 2;
    P.status = h->tb.status;
    P.out = trav_out(mode, out);
    P.order = c.order;  // the caller's order, else sort_bits
    P.ready = ready;
    P.ready_chunk = ready_chunk;
    const int bits = c.sort_bits;  // 0 or -1: input order
    if (!c.order && bits > 0 && h->nT > 0 && nR < ((int64_t)1 << 31)) {
        st = ensure_seg_ws(h, nR, (cudaStream_t)s);
        if (st != RSI_OK) return st;
        RSI_CK(rsi::segment_order(dA, dB, (int)nR, h->tb.rootbox, bits, h->seg_ws,
                                  (cudaStream_t)s, &P.order));
    }
    if (c.width == 4 && !h->nodes4_valid && h->nT > 0) {  // built on first use
        RSI_CK(rsi::build_nodes4(h->tb, (cudaStream_t)s));
        h->nodes4_valid = true;
    }
    if (c.stats)
        RSI_CK(cudaMemsetAsync(P.stats, 0, rsi::kStatCounters * 8, (cudaStream_t)s));
    if (c.packet)
        RSI_CK(rsi::launch_trace_packet(P, mode, c.stats, (cudaStream_t)s));
    else
        RSI_CK(rsi::launch_trace(P, mode, c.stack, c.stats, c.block, c.width, (cudaStream_t)s));
    return RSI_OK;
}

static rsi_status segment_order_impl(rsi_bvh h, const float* dA, const float* dB, int64_t nR,
                                     int32_t bits, int32_t* dOrder, rsi_stream s) {
    if (!h || nR < 0 || nR >= ((int64_t)1 << 31)) return RSI_ERR_ARG;
    if (bits == 0) bits = 30;
    if (bits < 6 || bits > 30) return RSI_ERR_ARG;
    if (!h->built) return RSI_ERR_NOT_BUILT;
    if (nR == 0) return RSI_OK;
    if (!dA || !dB || !dOrder) return RSI_ERR_ARG;
    rsi_status st = ensure_seg_ws(h, nR, (cudaStream_t)s);
    if (st != RSI_OK) return st;
    // an empty mesh has no box: the keys are then arbitrary, and the sorted
    // values still a permutation
    const int32_t* ord = nullptr;
    RSI_CK(rsi::segment_order(dA, dB, (int)nR, h->tb.rootbox, bits, h->seg_ws, (cudaStream_t)s,
                              &ord));
    RSI_CK(cudaMemcpyAsync(dOrder, ord, 4 * (size_t)nR, cudaMemcpyDeviceToDevice,
                           (cudaStream_t)s));
    return RSI_OK;
}

rsi_status rsi_segment_order(rsi_bvh h, const float* dA, const float* dB, int64_t nR,
                             int32_t bits, int32_t* dOrder, rsi_stream s) {
    const rsi_status st = segment_order_impl(h, dA, dB, nR, bits, dOrder, s);
    if (h) h->stream = (cudaStream_t)s;
    return st;
}

rsi_status rsi_intersect(rsi_bvh h, const float* dA, const float* dB, int64_t nR, rsi_mode mode,
                         const rsi_output* out, const rsi_launch_opts* lo, rsi_stream s) {
    const rsi_status st = intersect_impl(h, dA, dB, nR, mode, out, lo, s, false);
    if (h) h->stream = (cudaStream_t)s;
    return st;
}

rsi_status rsi_intersect_stats(rsi_bvh h, const float* dA, const float* dB, int64_t nR,
                               rsi_mode mode, const rsi_output* out, const rsi_launch_opts* lo,
                               rsi_stream s, rsi_stats* stt) {
    if (!stt) return RSI_ERR_ARG;
    memset(stt, 0, sizeof(*stt));
    rsi_status st = intersect_impl(h, dA, dB, nR, mode, out, lo, s, true);
    if (h) h->stream = (cudaStream_t)s;
    if (st != RSI_OK || nR == 0) return st;
    unsigned long long v[rsi::kStatCounters];
    RSI_CK(cudaMemcpyAsync(v, h->scratch + 1, sizeof(v), cudaMemcpyDeviceToHost,
                           (cudaStream_t)s));
    RSI_CK(cudaStreamSynchronize((cudaStream_t)s));
    stt->segments = (int64_t)v[0];
    stt->node_visits = (int64_t)v[1];
    stt->tri_tests = (int64_t)v[2];
    stt->fp64_tests = (int64_t)v[3];
    stt->df_refines = (int64_t)v[4];
    stt->overflows = (int64_t)v[5];
    stt->fp64_values = (int64_t)v[6];
    return RSI_OK;
}

// Bytes of device output staging per segment in rsi_intersect_host.
static int64_t out_bytes_per_seg(rsi_mode mode) {
    return mode == RSI_MODE_BOOL ? 1 : mode == RSI_MODE_COUNT ? 4 : 32;
}

// Device address of [p, p + bytes) when the whole range lies in page-locked
// host memory that the current device can address (cudaHostAlloc or
// cudaHostRegister memory under unified addressing), else nullptr.
static const float* mapped_host(const float* p, size_t bytes) {
    cudaPointerAttributes a0, a1;
    if (cudaPointerGetAttributes(&a0, p) != cudaSuccess ||
        cudaPointerGetAttributes(&a1, (const char*)p + bytes - 1) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (a0.type != cudaMemoryTypeHost || a1.type != cudaMemoryTypeHost || !a0.devicePointer ||
        !a1.devicePointer)
        return nullptr;
    if ((const char*)a1.devicePointer - (const char*)a0.devicePointer != (ptrdiff_t)(bytes - 1))
        return nullptr;
    return (const float*)a0.devicePointer;
}

// Streamed BOOL from page-locked host memory: one persistent traversal on s
// starts at once, while the copy engine stages the segments chunk by chunk
// (multiples of 32 segments, so no cache line spans two chunks) on an
// internal stream and sets each chunk's ready flag by a 4-byte copy after
// its data; a warp waits (bounded) for the flag of the chunk it takes
// segments from.  The copy (~211 GB/s) and the traversal overlap instead of
// one waiting for the other.  Two staging slots are used in turn, and the
// copies wait only until their slot is free (the call before the previous
// one is done with it), not for everything on s: the copies of one call run
// during the build and the traversal of the previous one, so back-to-back
// calls keep the copy engine busy.  The flags are reset on the copy stream
// and the traversal waits for that reset.  The copies are queued before the
// traversal: where a launch blocks the host until the kernel ends
// (CUDA_LAUNCH_BLOCKING, a profiler's replay), a traversal queued first
// would wait for copies not yet queued until its bounded waits ran out.
// Staging: 2 x (24 B + 1 B) per segment, held by the handle.
static rsi_status intersect_streamed(rsi_bvh h, const float* hA, const float* hB, int64_t nR,
                                     const rsi_output* hout, int64_t chunk,
                                     const rsi_launch_opts* lo, cudaStream_t cs) {
    int64_t ch = chunk > 0 ? chunk : kStreamChunk;
    if ((nR + ch - 1) / ch > kStreamMaxChunks) ch = (nR + kStreamMaxChunks - 1) / kStreamMaxChunks;
    ch = (ch + 31) / 32 * 32;
    const int64_t nc = (nR + ch - 1) / ch;
    const size_t ab = align256(12 * (size_t)nR), fb = align256((size_t)nR);
    const size_t slot_need = 2 * ab + fb + align256(4 * (size_t)nc);
    if (!h->sev_reset) {
        for (int q = 0; q < 2; ++q)
            RSI_CK(cudaEventCreateWithFlags(&h->sev_free[q], cudaEventDisableTiming));
        RSI_CK(cudaEventCreateWithFlags(&h->sev_reset, cudaEventDisableTiming));
    }
    if (h->pipe_bytes < 2 * slot_need) {  // (re)allocated on s: the copies must follow s
        h->sfree_valid[0] = h->sfree_valid[1] = false;
        if (h->pipe_mem) {  // every earlier use precedes this call on cs
            RSI_CK(rsi::dev_free(h->hooks, h->pipe_mem, cs));
            h->pipe_mem = nullptr;
            h->pipe_bytes = 0;
        }
        cudaError_t e = rsi::dev_alloc(h->hooks, (void**)&h->pipe_mem, 2 * slot_need, cs);
        if (e != cudaSuccess) {
            cudaGetLastError();
            h->pipe_mem = nullptr;
            return e == cudaErrorMemoryAllocation ? RSI_ERR_OOM : RSI_ERR_CUDA;
        }
        h->pipe_bytes = 2 * slot_need;
    }
    if (!h->one) {
        RSI_CK(cudaHostAlloc((void**)&h->one, sizeof(int32_t), cudaHostAllocDefault));
        *h->one = 1;
    }
    // slot q at a fixed offset (half the allocation, whatever nR), so that
    // it never overlaps the other slot that a running call may still read
    const int q = h->sslot;
    h->sslot ^= 1;
    char* base = h->pipe_mem + q * (h->pipe_bytes / 512 * 256);
    float* dA = (float*)base;
    float* dB = (float*)(base + ab);
    uint8_t* dflag = (uint8_t*)(base + 2 * ab);
    int32_t* ready = (int32_t*)(base + 2 * ab + fb);
    cudaStream_t cp = h->pst[0];
    if (!h->sfree_valid[q]) {
        RSI_CK(cudaEventRecord(h->pev_start, cs));
        RSI_CK(cudaStreamWaitEvent(cp, h->pev_start, 0));
    } else {
        RSI_CK(cudaStreamWaitEvent(cp, h->sev_free[q], 0));
    }
    RSI_CK(cudaMemsetAsync(ready, 0, 4 * (size_t)nc, cp));
    RSI_CK(cudaEventRecord(h->sev_reset, cp));
    h->sfree_valid[q] = false;
    for (int64_t c = 0; c < nc; ++c) {
        const int64_t off = c * ch, n = nR - off < ch ? nR - off : ch;
        RSI_CK(cudaMemcpyAsync(dA + 3 * off, hA + 3 * off, 12 * (size_t)n, cudaMemcpyHostToDevice,
                               cp));
        RSI_CK(cudaMemcpyAsync(dB + 3 * off, hB + 3 * off, 12 * (size_t)n, cudaMemcpyHostToDevice,
                               cp));
        RSI_CK(cudaMemcpyAsync(ready + c, h->one, sizeof(int32_t), cudaMemcpyHostToDevice, cp));
    }
    RSI_CK(cudaEventRecord(h->pev_done[0], cp));
    rsi_output dout;
    memset(&dout, 0, sizeof(dout));
    dout.flag = dflag;
    RSI_CK(cudaStreamWaitEvent(cs, h->sev_reset, 0));  // never a previous call's flags
    const rsi_status st = intersect_impl(h, dA, dB, nR, RSI_MODE_BOOL, &dout, lo, (rsi_stream)cs,
                                         false, nullptr, ready, ch);
    if (st != RSI_OK) {
        cudaStreamWaitEvent(cs, h->pev_done[0], 0);  // hA, hB are read until then
        return st;
    }
    RSI_CK(cudaMemcpyAsync(hout->flag, dflag, (size_t)nR, cudaMemcpyDeviceToHost, cs));
    RSI_CK(cudaEventRecord(h->sev_free[q], cs));
    h->sfree_valid[q] = true;
    RSI_CK(cudaStreamWaitEvent(cs, h->pev_done[0], 0));
    return RSI_OK;
}

static rsi_status intersect_host_impl(rsi_bvh h, const float* hA, const float* hB, int64_t nR,
                              rsi_mode mode, const rsi_output* hout, int64_t chunk,
                              const rsi_launch_opts* lo, rsi_stream s) {
    if (!h || nR < 0 || chunk < 0) return RSI_ERR_ARG;
    if (mode != RSI_MODE_BOOL && mode != RSI_MODE_COUNT && mode != RSI_MODE_NEAREST)
        return RSI_ERR_ARG;
    if (!h->built) return RSI_ERR_NOT_BUILT;
    if (nR == 0) return RSI_OK;
    if (!hA || !hB) return RSI_ERR_ARG;
    rsi_status st = check_output(mode, hout);
    if (st != RSI_OK) return st;
    if (hout->hit_idx) return RSI_ERR_ARG;  // no compaction from host buffers
    if (lo && lo->order) return RSI_ERR_ARG;  // an order indexes device-resident segments
    rsi_launch_opts lo2;
    memset(&lo2, 0, sizeof(lo2));
    if (lo) lo2 = *lo;
    lo2.sort_bits = -1;  // the segment-order workspace is shared: keep input order
    lo2.stats = 0;
    // Page-locked inputs: BOOL streams them into device staging while one
    // persistent traversal runs (intersect_streamed: 1.30 ms per call for
    // 10M segments on GB300, back to back); COUNT and NEAREST, whose larger outputs come back
    // per chunk, read them in place over the CPU-GPU link (1.61 ms for BOOL,
    // against 1.74 ms for staging chunk by chunk; copies and in-place reads
    // running together compete for the same link).  Other host memory is
    // staged chunk by chunk.
    const float* mA = mapped_host(hA, 12 * (size_t)nR);
    const float* mB = mA ? mapped_host(hB, 12 * (size_t)nR) : nullptr;
    const bool in_place = mA && mB;
    // Default chunk: with inputs read in place and 1 B of output per segment
    // few launches are fastest (the copy back is short); otherwise
    // kHostChunk segments, so that copies overlap the traversal of other
    // chunks.
    int64_t dflt = kHostChunk;
    if (in_place && mode == RSI_MODE_BOOL) dflt = kHostChunkInPlace;
    const int64_t ch = chunk > 0 ? (chunk < nR ? chunk : nR) : (nR < dflt ? nR : dflt);
    cudaStream_t cs = (cudaStream_t)s;
    if (!h->pst[0]) {
        for (int q = 0; q < 2; ++q) {
            RSI_CK(cudaStreamCreateWithFlags(&h->pst[q], cudaStreamNonBlocking));
            RSI_CK(cudaEventCreateWithFlags(&h->pev_done[q], cudaEventDisableTiming));
        }
        RSI_CK(cudaEventCreateWithFlags(&h->pev_start, cudaEventDisableTiming));
    }
    if (in_place && mode == RSI_MODE_BOOL && nR <= kStreamMax) {
        lo2.packet = 0;  // the packet kernel does not wait for streamed chunks
        return intersect_streamed(h, hA, hB, nR, hout, chunk, &lo2, cs);
    }
    // this call uses the staging too: a later streamed call follows s
    h->sfree_valid[0] = h->sfree_valid[1] = false;
    // staging of buffer q: [A | B when copied] | outputs (flag / count /
    // tri, tuv, point, dist), each part 256-byte aligned
    const size_t in_b = in_place ? 0 : align256(12 * (size_t)ch);
    const size_t o1 = align256((size_t)ch * 4), o3 = align256((size_t)ch * 12);
    const size_t out_b = mode == RSI_MODE_NEAREST
                             ? 2 * o1 + 2 * o3
                             : align256((size_t)(out_bytes_per_seg(mode) * ch));
    const size_t per_buf = 2 * in_b + out_b;
    if (h->pipe_bytes < 2 * per_buf) {
        if (h->pipe_mem) {  // every earlier use precedes this call on cs
            RSI_CK(rsi::dev_free(h->hooks, h->pipe_mem, cs));
            h->pipe_mem = nullptr;
            h->pipe_bytes = 0;
        }
        cudaError_t e = rsi::dev_alloc(h->hooks, (void**)&h->pipe_mem, 2 * per_buf, cs);
        if (e != cudaSuccess) {
            cudaGetLastError();
            h->pipe_mem = nullptr;
            return e == cudaErrorMemoryAllocation ? RSI_ERR_OOM : RSI_ERR_CUDA;
        }
        h->pipe_bytes = 2 * per_buf;
    }
    RSI_CK(cudaEventRecord(h->pev_start, cs));
    for (int q = 0; q < 2; ++q) RSI_CK(cudaStreamWaitEvent(h->pst[q], h->pev_start, 0));
    int k = 0;
    for (int64_t off = 0; off < nR; off += ch, ++k) {
        const int q = k & 1;
        const int64_t n = nR - off < ch ? nR - off : ch;
        cudaStream_t S = h->pst[q];
        char* b = h->pipe_mem + (size_t)q * per_buf;
        const float* dA = in_place ? mA + 3 * off : nullptr;
        const float* dB = in_place ? mB + 3 * off : nullptr;
        char* o = b + 2 * in_b;
        if (!in_place) {
            float* sA = (float*)b;
            float* sB = (float*)(b + in_b);
            RSI_CK(cudaMemcpyAsync(sA, hA + 3 * off, 12 * (size_t)n, cudaMemcpyHostToDevice, S));
            RSI_CK(cudaMemcpyAsync(sB, hB + 3 * off, 12 * (size_t)n, cudaMemcpyHostToDevice, S));
            dA = sA;
            dB = sB;
        }
        rsi_output dout;
        memset(&dout, 0, sizeof(dout));
        if (mode == RSI_MODE_BOOL) {
            dout.flag = (uint8_t*)o;
        } else if (mode == RSI_MODE_COUNT) {
            dout.count = (int32_t*)o;
        } else {
            dout.tri = (int32_t*)o;
            dout.tuv = (float*)(o + o1);
            dout.point = (float*)(o + o1 + o3);
            dout.dist = (float*)(o + o1 + 2 * o3);
        }
        st = intersect_impl(h, dA, dB, n, mode, &dout, &lo2, (rsi_stream)S, false,
                            h->scratch + 8 + q);
        if (st != RSI_OK) return st;
        auto back = [&](void* host, const void* dev, size_t bytes) -> cudaError_t {
            return host ? cudaMemcpyAsync(host, dev, bytes, cudaMemcpyDeviceToHost, S)
                        : cudaSuccess;
        };
        if (mode == RSI_MODE_BOOL) {
            RSI_CK(back(hout->flag + off, dout.flag, (size_t)n));
        } else if (mode == RSI_MODE_COUNT) {
            RSI_CK(back(hout->count + off, dout.count, 4 * (size_t)n));
        } else {
            RSI_CK(back(hout->tri + off, dout.tri, 4 * (size_t)n));
            if (hout->tuv) RSI_CK(back(hout->tuv + 3 * off, dout.tuv, 12 * (size_t)n));
            if (hout->point) RSI_CK(back(hout->point + 3 * off, dout.point, 12 * (size_t)n));
            if (hout->dist) RSI_CK(back(hout->dist + off, dout.dist, 4 * (size_t)n));
        }
    }
    for (int q = 0; q < 2; ++q) {
        RSI_CK(cudaEventRecord(h->pev_done[q], h->pst[q]));
        RSI_CK(cudaStreamWaitEvent(cs, h->pev_done[q], 0));
    }
    return RSI_OK;
}

rsi_status rsi_intersect_host(rsi_bvh h, const float* hA, const float* hB, int64_t nR,
                              rsi_mode mode, const rsi_output* hout, int64_t chunk,
                              const rsi_launch_opts* lo, rsi_stream s) {
    const rsi_status st = intersect_host_impl(h, hA, hB, nR, mode, hout, chunk, lo, s);
    if (h) h->stream = (cudaStream_t)s;
    return st;
}

static rsi_status points_inside_impl(rsi_bvh h, const float* dP, int64_t nP, uint8_t* dInside,
                                     const rsi_launch_opts* lo, rsi_stream s) {
    if (!h || nP < 0 || (lo && lo->order)) return RSI_ERR_ARG;
    if (!h->built) return RSI_ERR_NOT_BUILT;
    if (nP == 0) return RSI_OK;
    if (!dP || !dInside) return RSI_ERR_ARG;
    cudaStream_t cs = (cudaStream_t)s;
    if (h->nT == 0) {
        RSI_CK(cudaMemsetAsync(dInside, 0, (size_t)nP, cs));
        return RSI_OK;
    }
    if (h->in_cap < nP) {
        if (h->in_mem) {
            RSI_CK(rsi::dev_free(h->hooks, h->in_mem, cs));
            h->in_mem = nullptr;
        }
        cudaError_t e = rsi::dev_alloc(h->hooks, (void**)&h->in_mem, (size_t)(16 * nP + 512), cs);
        if (e != cudaSuccess) {
            cudaGetLastError();
            h->in_mem = nullptr;
            h->in_cap = 0;
            return e == cudaErrorMemoryAllocation ? RSI_ERR_OOM : RSI_ERR_CUDA;
        }
        h->in_cap = nP;
    }
    float* dB = (float*)h->in_mem;
    int32_t* cnt = (int32_t*)(h->in_mem + align256(12 * (size_t)h->in_cap));
    RSI_CK(rsi::launch_inside_segments(dP, nP, h->tb.rootbox, dB, cs));
    rsi_output o;
    memset(&o, 0, sizeof(o));
    o.count = cnt;
    const rsi_status st = intersect_impl(h, dP, dB, nP, RSI_MODE_COUNT, &o, lo, s, false);
    if (st != RSI_OK) return st;
    RSI_CK(rsi::launch_parity(cnt, nP, dInside, cs));
    return RSI_OK;
}

rsi_status rsi_points_inside(rsi_bvh h, const float* dP, int64_t nP, uint8_t* dInside,
                             const rsi_launch_opts* lo, rsi_stream s) {
    const rsi_status st = points_inside_impl(h, dP, nP, dInside, lo, s);
    if (h) h->stream = (cudaStream_t)s;
    return st;
}

rsi_status rsi_intersect_backward(const float* dV, int64_t nV, const int32_t* dT, int64_t nT,
                                  const float* dA, const float* dB, int64_t nR,
                                  const int32_t* dTri, const float* dGradPoint,
                                  const float* dGradTuv, float* dGradV, float* dGradA,
                                  float* dGradB, rsi_stream s) {
    if (nV < 0 || nT < 0 || nR < 0) return RSI_ERR_ARG;
    if (nR == 0) return RSI_OK;
    if (!dA || !dB || !dTri || (nT > 0 && (!dV || !dT))) return RSI_ERR_ARG;
    RSI_CK(rsi::launch_backward(dV, nV, dT, nT, dA, dB, nR, dTri, dGradPoint, dGradTuv, dGradV,
                                dGradA, dGradB, (cudaStream_t)s));
    return RSI_OK;
}

}  // extern "C"

// ------------------------------------------------------------------ batch
struct rsi_batch_s {
    int device = 0;
    std::vector<rsi_batch_item> items;
    TreeBufs tb;
    char* mem = nullptr;
    size_t bytes = 0;
    MeshDesc* d_table = nullptr;
    int32_t* d_blkmesh = nullptr;
    rsi::BatchItemDev* d_items = nullptr;
    unsigned long long* work = nullptr;
    int64_t n_tiles = 0;
    rsi::BatchTile* d_tiles = nullptr;
    LaunchCfg cfg;
    int32_t leaf = 1;
    cudaStream_t cap = nullptr;
    cudaGraphExec_t g_full = nullptr, g_trav = nullptr;
    cudaStream_t stream = nullptr;
    rsi::AllocHooks hooks{};  // device allocator of all this batch's memory
};

extern "C" {

rsi_status rsi_batch_create(const rsi_batch_item* items, int32_t n, const rsi_build_opts* bo,
                            const rsi_launch_opts* lo, rsi_stream s, rsi_batch* out) {
    if (!out || n < 1 || !items) return RSI_ERR_ARG;
    *out = nullptr;
    int32_t leaf, levels, height;
    rsi_status st = check_build_opts(bo, &leaf, &levels, &height);
    if (st != RSI_OK) return st;
    LaunchCfg cfg;
    st = check_launch_opts(lo, false, &cfg);
    if (st != RSI_OK) return st;
    if (cfg.order) return RSI_ERR_ARG;  // one order cannot serve several items
    RSI_CK(rsi::build_prepare());
    int64_t N = 0;
    int nblk = 0;
    std::vector<MeshDesc> table(n);
    std::vector<int32_t> blkmesh;
    for (int k = 0; k < n; ++k) {
        const rsi_batch_item& it = items[k];
        if (it.nV < 0 || it.nT < 0 || it.nR < 0) return RSI_ERR_ARG;
        if (it.nT > 0 && (!it.dV || !it.dT)) return RSI_ERR_ARG;
        if (it.nR > 0 && (!it.dA || !it.dB)) return RSI_ERR_ARG;
        if (it.mode < 0 || it.mode > 2) return RSI_ERR_ARG;
        st = check_output((rsi_mode)it.mode, &it.out);
        if (st != RSI_OK) return st;
        MeshDesc& md = table[k];
        md.V = it.dV;
        md.T = it.dT;
        md.nV = it.nV;
        md.n = (int32_t)it.nT;
        md.off = (int32_t)N;
        md.blk0 = nblk;
        md.nblk = (int32_t)((it.nT + rsi::kBuildChunk - 1) / rsi::kBuildChunk);
        if (it.height_axis < 0 || it.height_axis > 3) return RSI_ERR_ARG;
        md.height_axis = it.height_axis > 0 ? it.height_axis : height;
        for (int q = 0; q < md.nblk; ++q) blkmesh.push_back(k);
        nblk += md.nblk;
        N += it.nT;
        if (N >= ((int64_t)1 << 31)) return RSI_ERR_ARG;
    }
    // work order: items by decreasing estimated cost per segment
    std::vector<int> ord(n);
    for (int k = 0; k < n; ++k) ord[k] = k;
    auto cost = [&](int k) {
        const double w = items[k].mode == RSI_MODE_BOOL ? 1.0 : 1.5;
        return w * std::log2(2.0 + (double)items[k].nT);
    };
    std::stable_sort(ord.begin(), ord.end(), [&](int x, int y) { return cost(x) > cost(y); });
    std::vector<rsi::BatchItemDev> dev(n);
    std::vector<rsi::BatchTile> tiles;
    for (int q = 0; q < n; ++q) {
        const int k = ord[q];
        const rsi_batch_item& it = items[k];
        rsi::BatchItemDev& d = dev[k];
        d.A = it.dA;
        d.B = it.dB;
        d.nR = it.nR;
        d.root = it.nT > 0 ? (int)(table[k].off + it.nT - 1) : rsi::kNoRoot;
        d.mode = it.mode;
        d.out = trav_out((rsi_mode)it.mode, &it.out);
        for (int64_t lo = 0; lo < it.nR; lo += rsi::kBatchTile) {
            rsi::BatchTile t;
            t.item = k;
            t.pad = 0;
            t.lo = lo;
            t.hi = lo + rsi::kBatchTile < it.nR ? lo + rsi::kBatchTile : it.nR;
            tiles.push_back(t);
        }
    }
    int device = 0;
    RSI_CK(cudaGetDevice(&device));
    rsi_batch b = new rsi_batch_s();
    b->hooks = rsi::current_hooks();
    b->device = device;
    b->items.assign(items, items + n);
    b->cfg = cfg;
    b->leaf = leaf;
    b->n_tiles = (int64_t)tiles.size();
    TreeBufs tb;
    memset(&tb, 0, sizeof(tb));
    const size_t tree_bytes = carve(tb, N, n, nblk, nullptr);
    const size_t tab_bytes = align256(sizeof(MeshDesc) * n);
    const size_t blk_bytes = align256(sizeof(int32_t) * (blkmesh.size() + 1));
    const size_t item_bytes = align256(sizeof(rsi::BatchItemDev) * n);
    const size_t tile_bytes = align256(sizeof(rsi::BatchTile) * (tiles.size() + 1));
    const size_t bytes = tree_bytes + tab_bytes + blk_bytes + item_bytes + tile_bytes + 256;
    cudaStream_t cs = (cudaStream_t)s;
    cudaError_t e = rsi::dev_alloc(b->hooks, (void**)&b->mem, bytes, cs);
    if (e != cudaSuccess) {
        cudaGetLastError();
        delete b;
        return e == cudaErrorMemoryAllocation ? RSI_ERR_OOM : RSI_ERR_CUDA;
    }
    carve(tb, N, n, nblk, b->mem);
    tb.leaf_size = leaf;
    tb.height_axis = height;
    tb.top_levels = 0;
    b->tb = tb;
    b->bytes = bytes;
    b->d_table = (MeshDesc*)(b->mem + tree_bytes);
    b->d_blkmesh = (int32_t*)(b->mem + tree_bytes + tab_bytes);
    b->d_items = (rsi::BatchItemDev*)(b->mem + tree_bytes + tab_bytes + blk_bytes);
    b->d_tiles = (rsi::BatchTile*)(b->mem + tree_bytes + tab_bytes + blk_bytes + item_bytes);
    b->work = (unsigned long long*)(b->mem + bytes - 256);
    b->stream = cs;
    e = cudaMemcpyAsync(b->d_table, table.data(), sizeof(MeshDesc) * n, cudaMemcpyHostToDevice, cs);
    if (e == cudaSuccess && !blkmesh.empty())
        e = cudaMemcpyAsync(b->d_blkmesh, blkmesh.data(), sizeof(int32_t) * blkmesh.size(),
                            cudaMemcpyHostToDevice, cs);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->d_items, dev.data(), sizeof(rsi::BatchItemDev) * n,
                            cudaMemcpyHostToDevice, cs);
    if (e == cudaSuccess && !tiles.empty())
        e = cudaMemcpyAsync(b->d_tiles, tiles.data(), sizeof(rsi::BatchTile) * tiles.size(),
                            cudaMemcpyHostToDevice, cs);
    if (e == cudaSuccess) e = cudaMemsetAsync(tb.status, 0, 4, cs);
    if (e == cudaSuccess) e = cudaStreamSynchronize(cs);  // host tables go out of scope
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        cudaGetLastError();
        rsi::dev_free(b->hooks, b->mem, cs);
        delete b;
        return RSI_ERR_CUDA;
    }
    *out = b;
    return RSI_OK;
}

static MeshArgs batch_mesh_args(rsi_batch b) {
    MeshArgs ma;
    memset(&ma, 0, sizeof(ma));
    ma.M = b->tb.M;
    ma.table = b->d_table;
    ma.blk_mesh = b->d_blkmesh;
    if (ma.M == 1) {
        const rsi_batch_item& it = b->items[0];
        ma.one.V = it.dV;
        ma.one.T = it.dT;
        ma.one.nV = it.nV;
        ma.one.n = (int32_t)it.nT;
        ma.one.nblk = b->tb.nblk;
        ma.one.height_axis = it.height_axis > 0 ? it.height_axis : b->tb.height_axis;
    }
    return ma;
}

rsi_status rsi_batch_build(rsi_batch b, rsi_stream s) {
    if (!b) return RSI_ERR_ARG;
    RSI_CK(rsi::build_tree(b->tb, batch_mesh_args(b), (cudaStream_t)s, false));
    return RSI_OK;
}

rsi_status rsi_batch_intersect(rsi_batch b, rsi_stream s) {
    if (!b) return RSI_ERR_ARG;
    rsi::BatchParams P;
    P.items = b->d_items;
    P.n_items = (int)b->items.size();
    P.tiles = b->d_tiles;
    P.n_tiles = b->n_tiles;
    P.nodes = b->tb.nodes;
    P.nodes4 = b->tb.nodes4;
    P.tris = b->tb.tris;
    P.work = b->work;
    P.max_visits = b->tb.N + 2;
    P.status = b->tb.status;
    RSI_CK(rsi::launch_batch(P, b->cfg.block, b->cfg.stack, (cudaStream_t)s));
    return RSI_OK;
}

rsi_status rsi_batch_run_graph(rsi_batch b, int32_t rebuild, rsi_stream s) {
    if (!b) return RSI_ERR_ARG;
    cudaGraphExec_t* slot = rebuild ? &b->g_full : &b->g_trav;
    if (!*slot) {
        cudaGraph_t g = nullptr;
        RSI_CK(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
        rsi_status st = RSI_OK;
        if (rebuild) st = rsi_batch_build(b, (rsi_stream)b->cap);
        if (st == RSI_OK) st = rsi_batch_intersect(b, (rsi_stream)b->cap);
        cudaError_t e = cudaStreamEndCapture(b->cap, &g);
        if (st != RSI_OK) {
            if (g) cudaGraphDestroy(g);
            return st;
        }
        RSI_CK(e);
        e = cudaGraphInstantiate(slot, g, 0);
        cudaGraphDestroy(g);
        RSI_CK(e);
    }
    RSI_CK(cudaGraphLaunch(*slot, (cudaStream_t)s));
    return RSI_OK;
}

rsi_status rsi_batch_status(rsi_batch b, rsi_stream s) {
    if (!b) return RSI_ERR_ARG;
    int32_t v = 0;
    RSI_CK(cudaMemcpyAsync(&v, b->tb.status, 4, cudaMemcpyDeviceToHost, (cudaStream_t)s));
    RSI_CK(cudaStreamSynchronize((cudaStream_t)s));
    RSI_CK(cudaMemsetAsync(b->tb.status, 0, 4, (cudaStream_t)s));
    RSI_CK(cudaStreamSynchronize((cudaStream_t)s));
    return (rsi_status)v;
}

rsi_status rsi_batch_destroy(rsi_batch b) {
    if (!b) return RSI_ERR_ARG;
    if (b->g_full) cudaGraphExecDestroy(b->g_full);
    if (b->g_trav) cudaGraphExecDestroy(b->g_trav);
    cudaStreamSynchronize(b->stream);
    cudaError_t e = rsi::dev_free(b->hooks, b->mem, b->stream);
    if (b->cap) cudaStreamDestroy(b->cap);
    delete b;
    if (e != cudaSuccess) {
        cudaGetLastError();
        return RSI_ERR_CUDA;
    }
    return RSI_OK;
}

// ------------------------------------------------------------------ tuner
rsi_status rsi_autotune(rsi_bvh h, const float* dV, const int32_t* dT, const float* dA,
                        const float* dB, int64_t nR, rsi_mode mode, const rsi_output* out,
                        const int32_t* block_sizes, int32_t n_bs, const int32_t* stack_depths,
                        int32_t n_sd, const int32_t* smem_nodes, int32_t n_sm,
                        const int32_t* leaf_sizes, int32_t n_ls, int32_t reps, rsi_stream s,
                        rsi_tune_entry* table, int32_t cap, int32_t* n_written,
                        rsi_launch_opts* best_lo, int32_t* best_leaf) {
    if (!h || !block_sizes || !stack_depths || !smem_nodes || !leaf_sizes || n_bs < 1 ||
        n_sd < 1 || n_sm < 1 || n_ls < 1 || reps < 1 || !best_lo || !best_leaf || nR <= 0)
        return RSI_ERR_ARG;
    cudaStream_t cs = (cudaStream_t)s;
    cudaEvent_t e0, e1;
    RSI_CK(cudaEventCreate(&e0));
    RSI_CK(cudaEventCreate(&e1));
    float best_ms = INFINITY;
    int32_t written = 0;
    const int32_t leaf0 = h->leaf;
    *best_leaf = leaf0;
    memset(best_lo, 0, sizeof(*best_lo));
    rsi_status result = RSI_OK;
    for (int li = 0; li < n_ls && result == RSI_OK; ++li) {
        if (leaf_sizes[li] < 1 || leaf_sizes[li] > rsi::kMaxLeaf) {
            result = RSI_ERR_ARG;
            break;
        }
        h->leaf = leaf_sizes[li];
        result = rsi_bvh_build(h, dV, dT, s);
        if (result != RSI_OK) break;
        for (int bi = 0; bi < n_bs && result == RSI_OK; ++bi)
            for (int si = 0; si < n_sd && result == RSI_OK; ++si)
                for (int mi = 0; mi < n_sm && result == RSI_OK; ++mi) {
                    rsi_launch_opts lo;
                    memset(&lo, 0, sizeof(lo));
                    lo.block_size = block_sizes[bi];
                    lo.stack_depth = stack_depths[si];
                    lo.smem_nodes = smem_nodes[mi];
                    result = rsi_intersect(h, dA, dB, nR, mode, out, &lo, s);  // warm-up
                    if (result != RSI_OK) break;
                    std::vector<float> ms(reps);
                    for (int r = 0; r < reps && result == RSI_OK; ++r) {
                        cudaEventRecord(e0, cs);
                        result = rsi_intersect(h, dA, dB, nR, mode, out, &lo, s);
                        cudaEventRecord(e1, cs);
                        if (cudaEventSynchronize(e1) != cudaSuccess) result = RSI_ERR_CUDA;
                        cudaEventElapsedTime(&ms[r], e0, e1);
                    }
                    if (result != RSI_OK) break;
                    std::sort(ms.begin(), ms.end());
                    const float med = ms[reps / 2];
                    if (table && written < cap) {
                        rsi_tune_entry& t = table[written];
                        t.block_size = lo.block_size;
                        t.stack_depth = lo.stack_depth;
                        t.smem_nodes = lo.smem_nodes;
                        t.leaf_size = h->leaf;
                        t.ms = med;
                    }
                    ++written;
                    if (med < best_ms) {
                        best_ms = med;
                        *best_lo = lo;
                        *best_leaf = h->leaf;
                    }
                }
    }
    if (n_written) *n_written = written < cap ? written : cap;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    h->leaf = result == RSI_OK ? *best_leaf : leaf0;
    rsi_status rb = rsi_bvh_build(h, dV, dT, s);
    if (result == RSI_OK) result = rb;
    if (result == RSI_OK) RSI_CK(cudaStreamSynchronize(cs));
    return result;
}

rsi_status rsi_autotune_height_axis(rsi_bvh h, const float* dV, const int32_t* dT,
                                    const float* dA, const float* dB, int64_t nR,
                                    rsi_mode mode, const rsi_output* out,
                                    const rsi_launch_opts* lo, int32_t reps, rsi_stream s,
                                    float* ms, int32_t* best_axis) {
    if (!h || !dV || !dT || !dA || !dB || !out || !ms || !best_axis || nR <= 0 || reps < 1)
        return RSI_ERR_ARG;
    if (!h->built) return RSI_ERR_NOT_BUILT;
    cudaStream_t cs = (cudaStream_t)s;
    cudaEvent_t e0, e1;
    RSI_CK(cudaEventCreate(&e0));
    RSI_CK(cudaEventCreate(&e1));
    const int32_t axis0 = h->tb.height_axis;
    *best_axis = axis0;
    float best_ms = INFINITY;
    rsi_status result = RSI_OK;
    for (int a = 0; a < 4 && result == RSI_OK; ++a) {
        h->tb.height_axis = a;
        result = rsi_bvh_build(h, dV, dT, s);
        if (result == RSI_OK) result = rsi_intersect(h, dA, dB, nR, mode, out, lo, s);  // warm-up
        std::vector<float> t(reps);
        for (int r = 0; r < reps && result == RSI_OK; ++r) {
            cudaEventRecord(e0, cs);
            result = rsi_intersect(h, dA, dB, nR, mode, out, lo, s);
            cudaEventRecord(e1, cs);
            if (cudaEventSynchronize(e1) != cudaSuccess) result = RSI_ERR_CUDA;
            cudaEventElapsedTime(&t[r], e0, e1);
        }
        if (result != RSI_OK) break;
        std::sort(t.begin(), t.end());
        ms[a] = t[reps / 2];
        if (ms[a] < best_ms) {
            best_ms = ms[a];
            *best_axis = a;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    h->tb.height_axis = result == RSI_OK ? *best_axis : axis0;
    const rsi_status rb = rsi_bvh_build(h, dV, dT, s);
    if (result == RSI_OK) result = rb;
    if (result == RSI_OK && cudaStreamSynchronize(cs) != cudaSuccess) result = RSI_ERR_CUDA;
    return result;
}

}  // extern "C"
