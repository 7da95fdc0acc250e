// LBVH construction on the device (arXiv 2209.02878, Sec. 2 and Sec. 3.1).
//
//   a1  k_bounds / k_morton : centroid c_j = ((v_a + v_b) + v_c) / 3 and its
//                             support interval per mesh (Sec. 2, first step)
//   a2  k_morton            : q = clamp(floor(((c - lo) / (hi - lo)) 1024),
//                             0, 1023), 30-bit Morton code, sort key
//                             mesh << 32 | code, value = triangle index
//                             (option height_axis: that axis left out, the
//                             other two quantised to 2^15 levels)
//   a3  k_sort_*            : stable LSD radix sort, 8-bit digits
//   a4  k_karras            : binary radix tree over the distinct keys
//                             code << 32 | sorted position (Karras 2012, as
//                             cited in Sec. 2), one thread per internal node
//   a5  k_boxes_local       : boxes (the bottom-up pass of Sec. 3.1): one
//                             block per kBoxBlock sorted leaves writes the
//                             triangles in leaf order, the leaf boxes, a
//                             shared-memory sparse table of them, and from
//                             it every node whose leaf range lies inside
//                             the block, and prefix / suffix unions
//       k_boxes_span        : the nodes whose leaf range crosses a block
//                             boundary, from those unions; both write the
//                             64-byte traversal nodes, with the optional
//                             leaf collapse
//       k_treelet           : breadth-first copy of the top levels
//
// All kernels work on a concatenation of M meshes (M = 1 for a single
// handle), so a batch of meshes builds with the same number of launches.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "rsi_build.h"
#include "rsi_internal.cuh"
#include "sort.cuh"

namespace rsi {

__device__ __forceinline__ void latch(int32_t* status, int code) {
    atomicCAS(status, 0, code);
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

// q = clamp(floor(((c - lo) / (hi - lo)) * levels), 0, levels - 1); 0 for a
// zero extent (levels = 1024 for the paper's code, 2^15 for the height-field
// option's two axes).
__device__ __forceinline__ uint32_t quant(float c, float lo, float hi, float levels) {
    const float ext = __fsub_rn(hi, lo);
    if (!(ext > 0.f)) return 0u;
    float s = __fmul_rn(__fdiv_rn(__fsub_rn(c, lo), ext), levels);
    s = floorf(s);
    s = fminf(fmaxf(s, 0.f), levels - 1.f);
    return (uint32_t)s;
}

// 15-bit x -> bit k at bit 2k.
__device__ __forceinline__ uint32_t spread2(uint32_t x) {
    x &= 0x7fffu;
    x = (x | (x << 8)) & 0x00ff00ffu;
    x = (x | (x << 4)) & 0x0f0f0f0fu;
    x = (x | (x << 2)) & 0x33333333u;
    x = (x | (x << 1)) & 0x55555555u;
    return x;
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
            if (finite3(ce.x, ce.y, ce.z)) {
                if (md.height_axis == 0) {
                    code = (spread3(quant(ce.x, bnd[0], bnd[3], 1024.f)) << 2) |
                           (spread3(quant(ce.y, bnd[1], bnd[4], 1024.f)) << 1) |
                           spread3(quant(ce.z, bnd[2], bnd[5], 1024.f));
                } else {  // height field: the other two axes, the first one high
                    const float cc[3] = {ce.x, ce.y, ce.z};
                    const int a = md.height_axis == 1 ? 1 : 0, b = md.height_axis == 3 ? 1 : 2;
                    code = (spread2(quant(cc[a], bnd[a], bnd[3 + a], 32768.f)) << 1) |
                           spread2(quant(cc[b], bnd[b], bnd[3 + b], 32768.f));
                }
            }
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
    const int off = md.off, n = md.n, i = g - off;
    if (g == 0) *tb.nspan = 0;  // the box pass lists the slots that span its blocks
    if (i == n - 1) return;  // root slot of this mesh
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

// Merges box (lo, hi) into (l, h).
__device__ __forceinline__ void merge_box(float l[3], float h[3], float4 lo, float4 hi) {
    l[0] = fminf(l[0], lo.x);
    l[1] = fminf(l[1], lo.y);
    l[2] = fminf(l[2], lo.z);
    h[0] = fmaxf(h[0], hi.x);
    h[1] = fmaxf(h[1], hi.y);
    h[2] = fmaxf(h[2], hi.z);
}

__device__ __forceinline__ float4 f4(const float v[3]) { return make_float4(v[0], v[1], v[2], 0.f); }

// Traversal record of internal slot `node` from its two children's boxes and
// leaf ranges (children of at most leaf_size triangles become leaf ranges);
// also the slot's own box, and the mesh's root slot when `node` is the Karras
// root.
__device__ __forceinline__ void finish_node(const TreeBufs& tb, const MeshDesc& md, int m, int node,
                                            int2 cc, const float l0[3], const float h0[3],
                                            int f0, int z0, const float l1[3], const float h1[3],
                                            int f1, int z1) {
    const int L = tb.leaf_size;
    const int ref0 = z0 <= L ? f0 : cc.x, cnt0 = z0 <= L ? z0 : 0;
    const int ref1 = z1 <= L ? f1 : cc.y, cnt1 = z1 <= L ? z1 : 0;
    float ul[3] = {l0[0], l0[1], l0[2]}, uh[3] = {h0[0], h0[1], h0[2]};
    merge_box(ul, uh, f4(l1), f4(h1));
    __stcg(tb.nbox + 2 * (int64_t)node, f4(ul));
    __stcg(tb.nbox + 2 * (int64_t)node + 1, f4(uh));
    write_node(tb.nodes, node, f4(l0), f4(h0), ref0, cnt0, f4(l1), f4(h1), ref1, cnt1);
    if (node == md.off) {  // Karras root: fill the root slot
        const int root_slot = md.off + md.n - 1;
        tb.rootbox[2 * m] = f4(ul);
        tb.rootbox[2 * m + 1] = f4(uh);
        write_root(tb.nodes, root_slot, f4(ul), f4(uh), md.off, md.n <= L ? md.n : 0);
    }
}

// Shared-memory sparse table of one block's leaf boxes: level k holds the
// union of the 2^k boxes starting at each position (kBoxBlock - 2^k + 1
// entries), levels packed one after another, six float planes (lo xyz,
// hi xyz).  The union over any range [a, b] of the block is that of two
// overlapping entries of level floor(log2(b - a + 1)).
constexpr int kBoxLevels = 10;  // log2(kBoxBlock) + 1
static_assert(1 << (kBoxLevels - 1) == kBoxBlock, "kBoxBlock is a power of two");
__host__ __device__ constexpr int st_level(int k) { return k * (kBoxBlock + 1) - ((1 << k) - 1); }
constexpr int kStEntries = st_level(kBoxLevels);
constexpr size_t kBoxSmem = sizeof(float) * 6 * kStEntries + 2 * sizeof(int2) * kBoxBlock;

// Union of the leaf boxes at block positions [a, b] (a <= b).
__device__ __forceinline__ void st_query(const float* st, int a, int b, float l[3], float h[3]) {
    const int k = 31 - __clz(b - a + 1);
    const int i = st_level(k) + a, j = st_level(k) + b - (1 << k) + 1;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        l[c] = fminf(st[c * kStEntries + i], st[c * kStEntries + j]);
        h[c] = fmaxf(st[(3 + c) * kStEntries + i], st[(3 + c) * kStEntries + j]);
    }
}

// a5, first pass.  One block per kBoxBlock consecutive sorted leaves, one
// thread per leaf.  Each thread writes its triangle in leaf order and its
// leaf box; the block builds a sparse table of its leaf boxes in shared
// memory, from which it writes the prefix and suffix unions of every leaf
// (tb.pre / tb.suf, for the second pass) and the traversal record of every
// slot whose leaf range lies inside the block: each child's box is the
// union over the child's leaf range, so no slot waits for another (the
// paper's bottom-up pass with its per-node counters, Sec. 3.1, gives the
// same boxes: min / max are exact in any order).  Slots whose range crosses
// a block boundary are finished by k_boxes_span; with `list` (a build, not
// a refit) they are appended to tb.span.
__global__ void __launch_bounds__(kBoxBlock) k_boxes_local(MeshArgs ma, TreeBufs tb,
                                                           const uint64_t* __restrict__ keys,
                                                           const uint32_t* __restrict__ vals,
                                                           int list) {
    extern __shared__ float4 smem4[];
    float* st = (float*)smem4;
    int2* sch = (int2*)(st + 6 * kStEntries);  // children of slots base ..
    int2* srg = sch + kBoxBlock;               // leaf ranges of slots base ..
    const int tid = threadIdx.x, lane = tid & 31;
    const int base = blockIdx.x * kBoxBlock, g = base + tid, N = tb.N;
    float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    MeshDesc md;
    md.off = 0;
    md.n = 0;
    int m = 0;
    if (g < N) {
        m = (int)(keys[g] >> 32);
        md = mesh_of(ma, m);
        sch[tid] = *(const int2*)(tb.child + 2 * (int64_t)g);
        srg[tid] = *(const int2*)(tb.range + 2 * (int64_t)g);
        const int j = (int)vals[g] - md.off;
        float3 a, b, c;
        const bool ok = tri_vertices(md, j, tb.status, a, b, c);
        if (!ok) a = b = c = make_float3(0.f, 0.f, 0.f);  // never hits (zero edges)
        tb.tris[3 * (int64_t)g + 0] = make_float4(a.x, a.y, a.z, i2f(j));
        tb.tris[3 * (int64_t)g + 1] = make_float4(b.x, b.y, b.z, 0.f);
        tb.tris[3 * (int64_t)g + 2] = make_float4(c.x, c.y, c.z, 0.f);
        if (ok) {  // an invalid triangle keeps the empty box (lo > hi)
            lo[0] = fminf(fminf(a.x, b.x), c.x);
            lo[1] = fminf(fminf(a.y, b.y), c.y);
            lo[2] = fminf(fminf(a.z, b.z), c.z);
            hi[0] = fmaxf(fmaxf(a.x, b.x), c.x);
            hi[1] = fmaxf(fmaxf(a.y, b.y), c.y);
            hi[2] = fmaxf(fmaxf(a.z, b.z), c.z);
        }
        __stcg(tb.lbox + 2 * (int64_t)g, f4(lo));
        __stcg(tb.lbox + 2 * (int64_t)g + 1, f4(hi));
        if (md.n == 1) {
            write_root(tb.nodes, md.off, f4(lo), f4(hi), g, 1);
            tb.rootbox[2 * m] = f4(lo);
            tb.rootbox[2 * m + 1] = f4(hi);
        }
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        st[c * kStEntries + tid] = lo[c];
        st[(3 + c) * kStEntries + tid] = hi[c];
    }
    // slots whose range crosses a block boundary, for the second pass
    const bool inner = g < N && g - md.off < md.n - 1;  // an internal slot, not a root slot
    const bool local = inner && srg[tid].x >= base && srg[tid].y < base + kBoxBlock;
    if (list) {
        const bool span = inner && !local;
        const unsigned bal = __ballot_sync(0xffffffffu, span);
        if (bal) {
            int p0 = 0;
            if (lane == 0) p0 = atomicAdd(tb.nspan, __popc(bal));
            p0 = __shfl_sync(0xffffffffu, p0, 0);
            if (span) {
                const int2 rg = srg[tid], cc = sch[tid];
                tb.span[p0 + __popc(bal & ((1u << lane) - 1u))] =
                    make_int4(g, rg.x, rg.y, cc.x >= 0 ? cc.x : -cc.x - 1);
            }
        }
    }
    for (int k = 1; k < kBoxLevels; ++k) {
        __syncthreads();
        const int h = 1 << (k - 1);
        if (tid <= kBoxBlock - 2 * h) {
            const int s = st_level(k - 1) + tid, d = st_level(k) + tid;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                st[c * kStEntries + d] = fminf(st[c * kStEntries + s], st[c * kStEntries + s + h]);
                st[(3 + c) * kStEntries + d] =
                    fmaxf(st[(3 + c) * kStEntries + s], st[(3 + c) * kStEntries + s + h]);
            }
        }
    }
    __syncthreads();
    if (g >= N) return;
    float l0[3], h0[3];
    st_query(st, 0, tid, l0, h0);
    __stcg(tb.pre + 2 * (int64_t)g, f4(l0));
    __stcg(tb.pre + 2 * (int64_t)g + 1, f4(h0));
    st_query(st, tid, kBoxBlock - 1, l0, h0);
    __stcg(tb.suf + 2 * (int64_t)g, f4(l0));
    __stcg(tb.suf + 2 * (int64_t)g + 1, f4(h0));
    if (!local) return;
    // the record of slot g: children [first, gam] and [gam + 1, last]
    const int2 rg = srg[tid], cc = sch[tid];
    const int gam = cc.x >= 0 ? cc.x : -cc.x - 1;
    if (gam < rg.x || gam >= rg.y) {
        latch(tb.status, RSI_ERR_INTERNAL);
        return;
    }
    float l1[3], h1[3];
    st_query(st, rg.x - base, gam - base, l0, h0);
    st_query(st, gam + 1 - base, rg.y - base, l1, h1);
    finish_node(tb, md, m, g, cc, l0, h0, rg.x, gam - rg.x + 1, l1, h1, gam + 1, rg.y - gam);
}

// Union of the leaf boxes at sorted positions [a, b], a and b in different
// blocks of the first pass: the suffix of a's block from a, every whole block
// in between (the suffix of its first leaf), the prefix of b's block up to b.
// All 32 lanes call it (want == false: no range).  The lanes' whole blocks
// are laid end to end and loaded 32 per round, one per lane; a segmented
// scan over the lanes then merges each round's boxes into their owner's.
__device__ __forceinline__ void span_box(const TreeBufs& tb, bool want, int a, int b, float l[3],
                                         float h[3]) {
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    l[0] = l[1] = l[2] = INFINITY;
    h[0] = h[1] = h[2] = -INFINITY;
    int q0 = 0, cnt = 0;  // whole blocks [q0, q0 + cnt)
    if (want) {
        merge_box(l, h, __ldcg(tb.suf + 2 * (int64_t)a), __ldcg(tb.suf + 2 * (int64_t)a + 1));
        merge_box(l, h, __ldcg(tb.pre + 2 * (int64_t)b), __ldcg(tb.pre + 2 * (int64_t)b + 1));
        q0 = a / kBoxBlock + 1;
        cnt = b / kBoxBlock - q0;
        if (cnt < 0) cnt = 0;
    }
    int inc = cnt;  // items [inc - cnt, inc) of the laid-out list are this lane's
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(FULL, inc, o);
        if (lane >= o) inc += y;
    }
    const int total = __shfl_sync(FULL, inc, 31);
    const int exc = inc - cnt;
    for (int r0 = 0; r0 < total; r0 += 32) {
        const int j = r0 + lane;
        int own = 0;  // the lane whose items hold j: lanes with inc <= j come before it
#pragma unroll
        for (int step = 16; step > 0; step >>= 1)
            if (__shfl_sync(FULL, inc, own + step - 1) <= j) own += step;
        const int oq0 = __shfl_sync(FULL, q0, own), oexc = __shfl_sync(FULL, exc, own);
        float wl[3] = {INFINITY, INFINITY, INFINITY}, wh[3] = {-INFINITY, -INFINITY, -INFINITY};
        if (j < total) {
            const int64_t p = 2 * (int64_t)(oq0 + (j - oexc)) * kBoxBlock;
            merge_box(wl, wh, __ldcg(tb.suf + p), __ldcg(tb.suf + p + 1));
        }
        // inclusive scan within each owner's run of lanes
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int oo = __shfl_up_sync(FULL, own, o);
            float yl[3], yh[3];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                yl[k] = __shfl_up_sync(FULL, wl[k], o);
                yh[k] = __shfl_up_sync(FULL, wh[k], o);
            }
            if (lane >= o && oo == own) merge_box(wl, wh, f4(yl), f4(yh));
        }
        // each owner takes the union from the last lane of its run
        const bool mine = cnt > 0 && exc < r0 + 32 && inc > r0;
        const int src = mine ? min(inc, r0 + 32) - 1 - r0 : lane;
        float tl[3], th[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            tl[k] = __shfl_sync(FULL, wl[k], src);
            th[k] = __shfl_sync(FULL, wh[k], src);
        }
        if (mine) merge_box(l, h, f4(tl), f4(th));
    }
}

// Box of the child of a second-pass slot that covers leaves [a, b] (code c:
// Karras child code): a leaf box, the box of a slot the first pass finished,
// or the union over the blocks its range crosses.  All 32 lanes call it.
__device__ __forceinline__ void child_box(const TreeBufs& tb, bool act, int c, int a, int b,
                                          float l[3], float h[3]) {
    const bool wide = act && a / kBoxBlock != b / kBoxBlock;
    if (act && !wide) {
        const float4* p = c < 0 ? tb.lbox + 2 * (int64_t)a : tb.nbox + 2 * (int64_t)c;
        const float4 lo = __ldcg(p), hi = __ldcg(p + 1);
        l[0] = lo.x; l[1] = lo.y; l[2] = lo.z;
        h[0] = hi.x; h[1] = hi.y; h[2] = hi.z;
    }
    float wl[3], wh[3];
    span_box(tb, wide, a, b, wl, wh);
    if (wide) {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            l[k] = wl[k];
            h[k] = wh[k];
        }
    }
}

// a5, second pass: the slots listed by the first pass (leaf range across a
// block boundary), each independently.  A list entry holds the slot, its
// leaf range [first, last] and its split g (the last leaf of the left
// child): the left child is leaf g when first == g, else slot g; the right
// child leaf g + 1 when last == g + 1, else slot g + 1 (Karras numbering).
// The children's boxes come from the first pass (leaf boxes, finished
// slots) or from the prefix / suffix unions (children that cross a boundary
// themselves); no slot waits for another.
__global__ void __launch_bounds__(128) k_boxes_span(MeshArgs ma, TreeBufs tb,
                                                    const uint64_t* __restrict__ keys) {
    const int cnt = *tb.nspan;
    const int lane = threadIdx.x & 31;
    const int wg = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int k0 = wg * 32; k0 < cnt; k0 += nw * 32) {  // warp-uniform
        const int k = k0 + lane;
        const bool act = k < cnt;
        int4 e = make_int4(0, 0, 0, 0);
        if (act) e = __ldcg(tb.span + k);
        const int node = e.x, first = e.y, last = e.z, gam = e.w;
        const bool ok = act && first >= 0 && gam >= first && gam < last && last < tb.N;
        if (act && !ok) latch(tb.status, RSI_ERR_INTERNAL);
        const int2 cc = make_int2(first == gam ? -gam - 1 : gam,
                                  last == gam + 1 ? -gam - 2 : gam + 1);
        float l0[3], h0[3], l1[3], h1[3];
        child_box(tb, ok, cc.x, first, gam, l0, h0);
        child_box(tb, ok, cc.y, gam + 1, last, l1, h1);
        if (!ok) continue;
        const int m = (int)(keys[first] >> 32);
        const MeshDesc md = mesh_of(ma, m);
        if (node < md.off || node >= md.off + md.n - 1) {
            latch(tb.status, RSI_ERR_INTERNAL);
            continue;
        }
        finish_node(tb, md, m, node, cc, l0, h0, first, gam - first + 1, l1, h1, gam + 1,
                    last - gam);
    }
}

// 4-wide records for every slot of the built tree (one thread per slot, after
// the box passes have written all binary records).  Only needed by 4-wide
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

// The first box pass takes more than the default 48 KB of dynamic shared
// memory; its limit is raised once per device.
static std::mutex g_box_mu;
static uint64_t g_box_dev = 0;  // bit d: raised on device d

cudaError_t build_prepare() {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(g_box_mu);
    if (dev < 64 && ((g_box_dev >> dev) & 1ull)) return cudaSuccess;
    e = cudaFuncSetAttribute(k_boxes_local, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kBoxSmem);
    if (e == cudaSuccess && dev < 64) g_box_dev |= 1ull << dev;
    return e;
}

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
    }
    cudaError_t e = build_prepare();
    if (e != cudaSuccess) return e;
    k_boxes_local<<<cdiv(N, kBoxBlock), kBoxBlock, kBoxSmem, s>>>(ma, tb, tb.keys[tb.sorted],
                                                         tb.vals[tb.sorted], refit ? 0 : 1);
    k_boxes_span<<<cdiv(N, 4096), 128, 0, s>>>(ma, tb, tb.keys[tb.sorted]);
    if (tb.M == 1 && tb.top_levels > 0) k_treelet<<<1, 1024, 0, s>>>(tb, N - 1, tb.top_levels);
    return cudaGetLastError();
}

cudaError_t build_nodes4(const TreeBufs& tb, cudaStream_t s) {
    if (tb.N == 0) return cudaSuccess;
    k_nodes4<<<cdiv(tb.N, 256), 256, 0, s>>>(tb.nodes, tb.nodes4, tb.N);
    return cudaGetLastError();
}

}  // namespace rsi
