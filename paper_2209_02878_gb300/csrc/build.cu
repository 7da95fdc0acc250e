// LBVH construction on the device (arXiv 2209.02878, Sec. 2 and Sec. 3.1).
//
//   a1  k_bounds / k_morton : centroid c_j = ((v_a + v_b) + v_c) / 3 and its
//                             support interval per mesh (Sec. 2, first step)
//   a2  k_morton            : q = clamp(floor(((c - lo) / (hi - lo)) 1024),
//                             0, 1023), 30-bit Morton code, sort key
//                             mesh << 32 | code, value = triangle index
//   a3  k_sort_*            : stable LSD radix sort, 8-bit digits
//   a4  k_karras            : binary radix tree over the distinct keys
//                             code << 32 | sorted position (Karras 2012, as
//                             cited in Sec. 2), one thread per internal node
//   a5  k_climb             : bottom-up boxes, one thread per leaf, the
//                             second child to arrive at a node merges (the
//                             per-node `atomic` of Sec. 3.1); writes the
//                             64-byte traversal nodes and the triangles in
//                             leaf order; optional leaf collapse
//       k_treelet           : breadth-first copy of the top levels
//
// All kernels work on a concatenation of M meshes (M = 1 for a single
// handle), so a batch of meshes builds with the same number of launches.
#include <cuda_runtime.h>
#include <stdint.h>

#include "rsi_build.h"
#include "rsi_internal.cuh"
#include "sort.cuh"

namespace rsi {

__device__ __forceinline__ void latch(int32_t* status, int code) {
    atomicCAS(status, 0, code);
}

// atomicAdd with acquire-release semantics at device scope (no separate
// fences): writes before it are visible to the thread that later reads the
// value it produced, and writes made visible by earlier releases are seen
// after it.
__device__ __forceinline__ int atomic_add_acq_rel(int32_t* p, int v) {
    int old;
    asm volatile("atom.acq_rel.gpu.global.add.s32 %0, [%1], %2;"
                 : "=r"(old)
                 : "l"(p), "r"(v)
                 : "memory");
    return old;
}

// Loads triangle j of mesh md; an index outside [0, nV) latches
// RSI_ERR_BAD_INDEX and yields vertex 0 (the triangle is then discarded).
__device__ __forceinline__ bool tri_vertices(const MeshDesc& md, int j, int32_t* status,
                                             float3& a, float3& b, float3& c) {
    const int64_t i0 = md.T[3 * (int64_t)j], i1 = md.T[3 * (int64_t)j + 1],
                  i2 = md.T[3 * (int64_t)j + 2];
    const bool ok = i0 >= 0 && i0 < md.nV && i1 >= 0 && i1 < md.nV && i2 >= 0 && i2 < md.nV;
    if (!ok) {
        latch(status, RSI_ERR_BAD_INDEX);
        a = b = c = make_float3(0.f, 0.f, 0.f);
        return false;
    }
    a = make_float3(md.V[3 * i0], md.V[3 * i0 + 1], md.V[3 * i0 + 2]);
    b = make_float3(md.V[3 * i1], md.V[3 * i1 + 1], md.V[3 * i1 + 2]);
    c = make_float3(md.V[3 * i2], md.V[3 * i2 + 1], md.V[3 * i2 + 2]);
    return finite3(a.x, a.y, a.z) && finite3(b.x, b.y, b.z) && finite3(c.x, c.y, c.z);
}

__device__ __forceinline__ float3 centroid(float3 a, float3 b, float3 c) {
    return make_float3(__fdiv_rn(__fadd_rn(__fadd_rn(a.x, b.x), c.x), 3.0f),
                       __fdiv_rn(__fadd_rn(__fadd_rn(a.y, b.y), c.y), 3.0f),
                       __fdiv_rn(__fadd_rn(__fadd_rn(a.z, b.z), c.z), 3.0f));
}

__device__ __forceinline__ int block_mesh(const MeshArgs& ma, int b) {
    return ma.M == 1 ? 0 : ma.blk_mesh[b];
}

// Block-wide min / max of 6 values (lo xyz, hi xyz); result valid in thread 0.
__device__ __forceinline__ void block_minmax6(float v[6]) {
    __shared__ float red[6][kBuildThreads / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        float x = v[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float y = __shfl_xor_sync(0xffffffffu, x, o);
            x = k < 3 ? fminf(x, y) : fmaxf(x, y);
        }
        if (lane == 0) red[k][w] = x;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            float x = red[k][0];
            for (int q = 1; q < kBuildThreads / 32; ++q)
                x = k < 3 ? fminf(x, red[k][q]) : fmaxf(x, red[k][q]);
            v[k] = x;
        }
    }
}

// a1: per-block support interval of the (finite) centroids.
__global__ void __launch_bounds__(kBuildThreads) k_bounds(MeshArgs ma, TreeBufs tb) {
    const int b = blockIdx.x;
    const MeshDesc md = mesh_of(ma, block_mesh(ma, b));
    const int j0 = (b - md.blk0) * kBuildChunk;
    const int j1 = min(md.n, j0 + kBuildChunk);
    float v[6] = {INFINITY, INFINITY, INFINITY, -INFINITY, -INFINITY, -INFINITY};
    for (int j = j0 + threadIdx.x; j < j1; j += blockDim.x) {
        float3 a, bb, c;
        if (!tri_vertices(md, j, tb.status, a, bb, c)) continue;
        const float3 ce = centroid(a, bb, c);
        if (!finite3(ce.x, ce.y, ce.z)) continue;
        v[0] = fminf(v[0], ce.x); v[1] = fminf(v[1], ce.y); v[2] = fminf(v[2], ce.z);
        v[3] = fmaxf(v[3], ce.x); v[4] = fmaxf(v[4], ce.y); v[5] = fmaxf(v[5], ce.z);
    }
    block_minmax6(v);
    if (threadIdx.x == 0)
        for (int k = 0; k < 6; ++k) tb.partial[6 * b + k] = v[k];
}

// 10-bit value -> bits at positions 3k (k = 0..9).
__device__ __forceinline__ uint32_t spread3(uint32_t x) {
    x &= 0x3ffu;
    x = (x | (x << 16)) & 0x030000ffu;
    x = (x | (x << 8)) & 0x0300f00fu;
    x = (x | (x << 4)) & 0x030c30c3u;
    x = (x | (x << 2)) & 0x09249249u;
    return x;
}

__device__ __forceinline__ uint32_t quant(float c, float lo, float hi) {
    const float ext = __fsub_rn(hi, lo);
    if (!(ext > 0.f)) return 0u;
    float s = __fmul_rn(__fdiv_rn(__fsub_rn(c, lo), ext), 1024.0f);
    s = floorf(s);
    s = fminf(fmaxf(s, 0.f), 1023.f);
    return (uint32_t)s;
}

// a2: mesh interval from the partials, quantisation, Morton code, sort key.
__global__ void __launch_bounds__(kBuildThreads) k_morton(MeshArgs ma, TreeBufs tb) {
    const int b = blockIdx.x;
    const int m = block_mesh(ma, b);
    const MeshDesc md = mesh_of(ma, m);
    float v[6] = {INFINITY, INFINITY, INFINITY, -INFINITY, -INFINITY, -INFINITY};
    for (int q = threadIdx.x; q < md.nblk; q += blockDim.x) {
        const float* p = tb.partial + 6 * (md.blk0 + q);
        v[0] = fminf(v[0], p[0]); v[1] = fminf(v[1], p[1]); v[2] = fminf(v[2], p[2]);
        v[3] = fmaxf(v[3], p[3]); v[4] = fmaxf(v[4], p[4]); v[5] = fmaxf(v[5], p[5]);
    }
    block_minmax6(v);
    __shared__ float bnd[6];
    if (threadIdx.x == 0)
        for (int k = 0; k < 6; ++k) bnd[k] = v[k];
    __syncthreads();
    if (b == md.blk0 && threadIdx.x < 6) tb.bounds[6 * m + threadIdx.x] = bnd[threadIdx.x];
    const int j0 = (b - md.blk0) * kBuildChunk;
    const int j1 = min(md.n, j0 + kBuildChunk);
    for (int j = j0 + threadIdx.x; j < j1; j += blockDim.x) {
        float3 a, bb, c;
        uint32_t code = 0;
        if (tri_vertices(md, j, tb.status, a, bb, c)) {
            const float3 ce = centroid(a, bb, c);
            if (finite3(ce.x, ce.y, ce.z))
                code = (spread3(quant(ce.x, bnd[0], bnd[3])) << 2) |
                       (spread3(quant(ce.y, bnd[1], bnd[4])) << 1) |
                       spread3(quant(ce.z, bnd[2], bnd[5]));
        }
        tb.keys[0][md.off + j] = ((uint64_t)m << 32) | code;
        tb.vals[0][md.off + j] = (uint32_t)(md.off + j);
    }
}

// ---------------------------------------------------------------- a4
// Length of the common prefix of K_i = code_i << 32 | i and K_j (local
// indices of one mesh); -1 outside [0, n).
__device__ __forceinline__ int kdelta(const uint64_t* __restrict__ keys, int off, int n, int i,
                                      int j) {
    if (j < 0 || j >= n) return -1;
    const uint32_t ci = (uint32_t)keys[off + i], cj = (uint32_t)keys[off + j];
    if (ci != cj) return __clz(ci ^ cj);
    return 32 + __clz((unsigned)(i ^ j));
}

__global__ void k_karras(MeshArgs ma, TreeBufs tb, const uint64_t* __restrict__ keys) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= tb.N) return;
    const MeshDesc md = mesh_of(ma, (int)(keys[g] >> 32));
    const int off = md.off, n = md.n, i = g - off, N = tb.N;
    tb.flag[g] = 0;
    if (i == n - 1) {  // root slot of this mesh
        if (n == 1)
            tb.parent[N + g] = g;
        else
            tb.parent[off] = g;
        return;
    }
    const int d = kdelta(keys, off, n, i, i + 1) > kdelta(keys, off, n, i, i - 1) ? 1 : -1;
    const int dmin = kdelta(keys, off, n, i, i - d);
    int64_t lmax = 2;  // stops once i + lmax d leaves [0, n)
    while (kdelta(keys, off, n, i, (int)max((int64_t)-1, min((int64_t)n, i + lmax * d))) > dmin)
        lmax <<= 1;
    int l = 0;
    for (int64_t t = lmax >> 1; t >= 1; t >>= 1)
        if (l + t < n && kdelta(keys, off, n, i, i + (int)(l + t) * d) > dmin) l += (int)t;
    const int j = i + l * d;
    const int dn = kdelta(keys, off, n, i, j);
    int s = 0, t = l;
    do {
        t = (t + 1) >> 1;
        if (kdelta(keys, off, n, i, i + (s + t) * d) > dn) s += t;
    } while (t > 1);
    const int gam = i + s * d + min(d, 0);
    const int lo = min(i, j), hi = max(i, j);
    const int left = (lo == gam) ? -(off + gam + 1) : off + gam;
    const int right = (hi == gam + 1) ? -(off + gam + 2) : off + gam + 1;
    tb.child[2 * g] = left;
    tb.child[2 * g + 1] = right;
    tb.range[2 * g] = off + lo;
    tb.range[2 * g + 1] = off + hi;
    if (left < 0)
        tb.parent[N + off + gam] = g;
    else
        tb.parent[off + gam] = g;
    if (right < 0)
        tb.parent[N + off + gam + 1] = g;
    else
        tb.parent[off + gam + 1] = g;
}

// ---------------------------------------------------------------- a5
// A box with lo > hi (no valid triangle below) is stored in a traversal node
// as lo = hi = +inf, which the slab test never enters.
__device__ __forceinline__ void store_child_box(float4 lo, float4 hi, float* dst) {
    if (lo.x > hi.x || lo.y > hi.y || lo.z > hi.z) {
        lo = hi = make_float4(INFINITY, INFINITY, INFINITY, 0.f);
    }
    dst[0] = lo.x; dst[1] = lo.y; dst[2] = lo.z;
    dst[3] = hi.x; dst[4] = hi.y; dst[5] = hi.z;
}

__device__ __forceinline__ void write_node(float4* nodes, int slot, float4 l0, float4 h0,
                                           int ref0, int cnt0, float4 l1, float4 h1, int ref1,
                                           int cnt1) {
    float f[16];
    store_child_box(l0, h0, f);
    store_child_box(l1, h1, f + 6);
    f[12] = i2f(ref0);
    f[13] = i2f(ref1);
    f[14] = i2f(cnt0);
    f[15] = i2f(cnt1);
    // the two children's coordinates interleaved in pairs (see rsi_internal.cuh)
    float4* o = nodes + 4 * (int64_t)slot;
    __stcg(o + 0, make_float4(f[0], f[6], f[1], f[7]));
    __stcg(o + 1, make_float4(f[2], f[8], f[3], f[9]));
    __stcg(o + 2, make_float4(f[4], f[10], f[5], f[11]));
    __stcg(o + 3, make_float4(f[12], f[13], f[14], f[15]));
}

__device__ __forceinline__ void write_root(float4* nodes, int slot, float4 lo, float4 hi, int ref,
                                           int cnt) {
    const float4 e = make_float4(INFINITY, INFINITY, INFINITY, 0.f);
    write_node(nodes, slot, lo, hi, ref, cnt, e, e, -1, 0);
}

// 4-wide traversal node of slot `slot` (8 x float4 = 128 B, one record per
// binary slot): the grandchildren of the binary node, i.e. each internal
// child is replaced by its own two children, a leaf child is kept.  Layout:
// {lo.x[4]}, {lo.y[4]}, {lo.z[4]}, {hi.x[4]}, {hi.y[4]}, {hi.z[4]},
// {ref[4]}, {cnt[4]}; an empty slot has lo = hi = +inf, ref -1, cnt 0.
struct Slot4 {
    float lo[3], hi[3];
    int ref, cnt;
};

__device__ __forceinline__ void binary_children(const float4* __restrict__ nodes, int slot,
                                                Slot4& a, Slot4& b) {
    const float4* p = nodes + 4 * (int64_t)slot;
    const float4 f0 = __ldcg(p), f1 = __ldcg(p + 1), f2 = __ldcg(p + 2), f3 = __ldcg(p + 3);
    a.lo[0] = f0.x; a.lo[1] = f0.z; a.lo[2] = f1.x;
    a.hi[0] = f1.z; a.hi[1] = f2.x; a.hi[2] = f2.z;
    b.lo[0] = f0.y; b.lo[1] = f0.w; b.lo[2] = f1.y;
    b.hi[0] = f1.w; b.hi[1] = f2.y; b.hi[2] = f2.w;
    a.ref = f2i(f3.x);
    b.ref = f2i(f3.y);
    a.cnt = f2i(f3.z);
    b.cnt = f2i(f3.w);
}

// Expand binary slot `slot` (whose own record is already written) into its
// 4-wide record.
__device__ __forceinline__ void write_node4(const float4* __restrict__ nodes, float4* nodes4,
                                            int slot) {
    Slot4 c[2], o[4];
    binary_children(nodes, slot, c[0], c[1]);
    int k = 0;
    for (int q = 0; q < 2; ++q) {
        if (c[q].cnt == 0 && c[q].ref >= 0) {  // internal: take its two children
            binary_children(nodes, c[q].ref, o[k], o[k + 1]);
            k += 2;
        } else if (c[q].cnt > 0) {
            o[k++] = c[q];
        }
    }
    for (; k < 4; ++k) {
        for (int a = 0; a < 3; ++a) o[k].lo[a] = o[k].hi[a] = INFINITY;
        o[k].ref = -1;
        o[k].cnt = 0;
    }
    float4* d = nodes4 + 8 * (int64_t)slot;
    for (int a = 0; a < 3; ++a) {
        __stcg(d + a, make_float4(o[0].lo[a], o[1].lo[a], o[2].lo[a], o[3].lo[a]));
        __stcg(d + 3 + a, make_float4(o[0].hi[a], o[1].hi[a], o[2].hi[a], o[3].hi[a]));
    }
    __stcg(d + 6, make_float4(i2f(o[0].ref), i2f(o[1].ref), i2f(o[2].ref), i2f(o[3].ref)));
    __stcg(d + 7, make_float4(i2f(o[0].cnt), i2f(o[1].cnt), i2f(o[2].cnt), i2f(o[3].cnt)));
}

__global__ void k_climb(MeshArgs ma, TreeBufs tb, const uint64_t* __restrict__ keys,
                        const uint32_t* __restrict__ vals) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= tb.N) return;
    const MeshDesc md = mesh_of(ma, (int)(keys[g] >> 32));
    const int off = md.off, n = md.n, N = tb.N, L = tb.leaf_size;
    const int root_slot = off + n - 1;
    const int j = (int)vals[g] - off;
    float3 a, b, c;
    const bool ok = tri_vertices(md, j, tb.status, a, b, c);
    if (!ok) a = b = c = make_float3(0.f, 0.f, 0.f);  // never hits (zero edges)
    tb.tris[3 * (int64_t)g + 0] = make_float4(a.x, a.y, a.z, i2f(j));
    tb.tris[3 * (int64_t)g + 1] = make_float4(b.x, b.y, b.z, 0.f);
    tb.tris[3 * (int64_t)g + 2] = make_float4(c.x, c.y, c.z, 0.f);
    float4 lo, hi;
    if (ok) {
        lo = make_float4(fminf(fminf(a.x, b.x), c.x), fminf(fminf(a.y, b.y), c.y),
                         fminf(fminf(a.z, b.z), c.z), 0.f);
        hi = make_float4(fmaxf(fmaxf(a.x, b.x), c.x), fmaxf(fmaxf(a.y, b.y), c.y),
                         fmaxf(fmaxf(a.z, b.z), c.z), 0.f);
    } else {
        lo = make_float4(INFINITY, INFINITY, INFINITY, 0.f);
        hi = make_float4(-INFINITY, -INFINITY, -INFINITY, 0.f);
    }
    __stcg(tb.lbox + 2 * (int64_t)g, lo);
    __stcg(tb.lbox + 2 * (int64_t)g + 1, hi);
    const int m = (int)(keys[g] >> 32);
    if (n == 1) {
        write_root(tb.nodes, root_slot, lo, hi, g, 1);
        tb.rootbox[2 * m] = lo;
        tb.rootbox[2 * m + 1] = hi;
        return;
    }
    int node = tb.parent[N + g];
    // The climbing thread carries its own subtree (child code, box, first
    // leaf, size), so after the atomic only the sibling's box and range are
    // loaded; the node's child pair and parent (written by k_karras) are
    // loaded before the atomic so that their latency overlaps it.
    int me = -g - 1;
    float4 mlo = lo, mhi = hi;
    int mfirst = g, msize = 1;
    // a radix tree over 62-bit keys is at most 63 levels deep
    for (int climb = 0;; ++climb) {
        if (climb > 70 || node < off || node >= off + n - 1) {
            latch(tb.status, RSI_ERR_INTERNAL);
            return;
        }
        const int2 cc = *(const int2*)(tb.child + 2 * (int64_t)node);
        const int par = tb.parent[node];
        // acquire-release: the first arrival publishes its child's box and
        // node record, the second arrival sees them
        if (atomic_add_acq_rel(&tb.flag[node], 1) == 0) return;  // the sibling finishes it
        const bool mine0 = cc.x == me;
        const int x = mine0 ? cc.y : cc.x;  // the sibling
        float4 slo, shi;
        int sfirst, ssize;
        if (x < 0) {
            const int leaf = -x - 1;
            slo = __ldcg(tb.lbox + 2 * (int64_t)leaf);
            shi = __ldcg(tb.lbox + 2 * (int64_t)leaf + 1);
            sfirst = leaf;
            ssize = 1;
        } else {
            slo = __ldcg(tb.nbox + 2 * (int64_t)x);
            shi = __ldcg(tb.nbox + 2 * (int64_t)x + 1);
            const int2 rg = *(const int2*)(tb.range + 2 * (int64_t)x);
            sfirst = rg.x;
            ssize = rg.y - rg.x + 1;
        }
        // children in the node's order: 0 = cc.x, 1 = cc.y
        const float4 l0 = mine0 ? mlo : slo, h0 = mine0 ? mhi : shi;
        const float4 l1 = mine0 ? slo : mlo, h1 = mine0 ? shi : mhi;
        const int f0 = mine0 ? mfirst : sfirst, z0 = mine0 ? msize : ssize;
        const int f1 = mine0 ? sfirst : mfirst, z1 = mine0 ? ssize : msize;
        const int ref0 = z0 <= L ? f0 : cc.x, cnt0 = z0 <= L ? z0 : 0;
        const int ref1 = z1 <= L ? f1 : cc.y, cnt1 = z1 <= L ? z1 : 0;
        const float4 ulo = make_float4(fminf(l0.x, l1.x), fminf(l0.y, l1.y), fminf(l0.z, l1.z), 0.f);
        const float4 uhi = make_float4(fmaxf(h0.x, h1.x), fmaxf(h0.y, h1.y), fmaxf(h0.z, h1.z), 0.f);
        __stcg(tb.nbox + 2 * (int64_t)node, ulo);
        __stcg(tb.nbox + 2 * (int64_t)node + 1, uhi);
        write_node(tb.nodes, node, l0, h0, ref0, cnt0, l1, h1, ref1, cnt1);
        if (node == off) {  // Karras root: fill the root slot
            tb.rootbox[2 * m] = ulo;
            tb.rootbox[2 * m + 1] = uhi;
            if (n <= L)
                write_root(tb.nodes, root_slot, ulo, uhi, off, n);
            else
                write_root(tb.nodes, root_slot, ulo, uhi, off, 0);
            return;
        }
        me = node;
        mlo = ulo;
        mhi = uhi;
        mfirst = f0 < f1 ? f0 : f1;
        msize = z0 + z1;
        node = par;
    }
}

// 4-wide records for every slot of the built tree (one thread per slot, after
// the climb has written all binary records).  Only needed by 4-wide
// traversal, so it runs on first use.
__global__ void k_nodes4(const float4* __restrict__ nodes, float4* __restrict__ nodes4, int N) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g < N) write_node4(nodes, nodes4, g);
}

// ---------------------------------------------------------------- treelet
__device__ __forceinline__ int block_excl_scan(int x, int& total) {
    __shared__ int ws[32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int incl = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) ws[w] = incl;
    __syncthreads();
    if (w == 0) {
        const int nw = blockDim.x >> 5;
        int v = lane < nw ? ws[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += y;
        }
        ws[lane] = v;
    }
    __syncthreads();
    total = ws[(blockDim.x >> 5) - 1];
    const int r = incl - x + (w > 0 ? ws[w - 1] : 0);
    __syncthreads();
    return r;
}

// Breadth-first copy of the top `levels` levels below the root slot, at most
// kTreeletMax nodes; children inside the copy are re-pointed to it
// (cnt = -1, ref = treelet index).  One block of 1024 threads.
__global__ void __launch_bounds__(1024) k_treelet(TreeBufs tb, int root_slot, int levels) {
    __shared__ int ids[kTreeletMax];
    __shared__ int kid[2 * kTreeletMax];
    for (int q = threadIdx.x; q < 2 * kTreeletMax; q += blockDim.x) kid[q] = -1;
    if (threadIdx.x == 0) ids[0] = root_slot;
    __syncthreads();
    int head = 0, tail = 1;
    for (int lev = 0; lev < levels && head < tail; ++lev) {
        int next = tail;
        for (int base = head; base < tail; base += blockDim.x) {
            const int e = base + threadIdx.x;
            int c0 = 0, c1 = 0, r0 = 0, r1 = 0;
            if (e < tail) {
                const float4 n3 = tb.nodes[4 * (int64_t)ids[e] + 3];
                r0 = f2i(n3.x);
                r1 = f2i(n3.y);
                c0 = (f2i(n3.z) == 0 && r0 >= 0) ? 1 : 0;
                c1 = (f2i(n3.w) == 0 && r1 >= 0) ? 1 : 0;
            }
            int total;
            const int pos = block_excl_scan(c0 + c1, total);
            if (e < tail) {
                int idx = next + pos;
                if (c0) {
                    if (idx < kTreeletMax) {
                        ids[idx] = r0;
                        kid[2 * e] = idx;
                    }
                    ++idx;
                }
                if (c1 && idx < kTreeletMax) {
                    ids[idx] = r1;
                    kid[2 * e + 1] = idx;
                }
            }
            next += total;
            __syncthreads();
        }
        head = tail;
        tail = min(next, kTreeletMax);
    }
    __syncthreads();
    for (int e = threadIdx.x; e < tail; e += blockDim.x) {
        const float4* src = tb.nodes + 4 * (int64_t)ids[e];
        float4* dst = tb.treelet + 4 * (int64_t)e;
        dst[0] = src[0];
        dst[1] = src[1];
        dst[2] = src[2];
        float4 n3 = src[3];
        if (kid[2 * e] >= 0) {
            n3.x = i2f(kid[2 * e]);
            n3.z = i2f(-1);
        }
        if (kid[2 * e + 1] >= 0) {
            n3.y = i2f(kid[2 * e + 1]);
            n3.w = i2f(-1);
        }
        dst[3] = n3;
    }
    if (threadIdx.x == 0) *tb.treelet_n = tail;
}

// ---------------------------------------------------------------- host
static inline int cdiv(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

cudaError_t build_tree(TreeBufs& tb, const MeshArgs& ma, cudaStream_t s, bool refit) {
    const int N = tb.N;
    if (N == 0) return cudaSuccess;
    if (!refit) {
        k_bounds<<<tb.nblk, kBuildThreads, 0, s>>>(ma, tb);
        k_morton<<<tb.nblk, kBuildThreads, 0, s>>>(ma, tb);
        int shifts[8], np = 0;
        for (int sh = 0; sh < 32; sh += 8) shifts[np++] = sh;
        for (int sh = 32; sh < 64 && ((int64_t)(tb.M - 1) >> (sh - 32)) > 0; sh += 8)
            shifts[np++] = sh;
        int cur = 0;
        cudaError_t e = radix_sort<uint64_t>(tb.keys, tb.vals, N, shifts, np, tb.hist, tb.totals,
                                             s, &cur);
        if (e != cudaSuccess) return e;
        tb.sorted = cur;
        k_karras<<<cdiv(N, 256), 256, 0, s>>>(ma, tb, tb.keys[cur]);
    } else {
        cudaError_t e = cudaMemsetAsync(tb.flag, 0, sizeof(int32_t) * (size_t)N, s);
        if (e != cudaSuccess) return e;
    }
    k_climb<<<cdiv(N, 256), 256, 0, s>>>(ma, tb, tb.keys[tb.sorted], tb.vals[tb.sorted]);
    if (tb.M == 1 && tb.top_levels > 0) k_treelet<<<1, 1024, 0, s>>>(tb, N - 1, tb.top_levels);
    return cudaGetLastError();
}

cudaError_t build_nodes4(const TreeBufs& tb, cudaStream_t s) {
    if (tb.N == 0) return cudaSuccess;
    k_nodes4<<<cdiv(tb.N, 256), 256, 0, s>>>(tb.nodes, tb.nodes4, tb.N);
    return cudaGetLastError();
}

}  // namespace rsi
