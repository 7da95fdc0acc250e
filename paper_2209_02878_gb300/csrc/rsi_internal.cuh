// Internal declarations of librsi (not part of the public ABI).
//
// Data layout in device memory (one mesh of n triangles at offset `off` in
// the concatenated arrays; a batch concatenates its meshes):
//   keys[2]/vals[2]  u64 sort keys (mesh << 32 | Morton code) / u32 global
//                    triangle index, ping-pong buffers of the radix sort
//   child[2N]        Karras children of internal slot g: >= 0 internal slot,
//                    < 0 leaf -(global sorted position + 1)
//   range[2N]        first, last leaf (global sorted positions) of slot g
//   nbox/lbox[2N]    float4 lo, hi boxes of internal slots / leaves
//   pre/suf[2N]      float4 lo, hi unions of the leaf boxes of each block of
//                    kBoxBlock sorted leaves up to / from each leaf
//   span[N]          internal slots whose leaf range crosses such a block
//                    boundary, {slot, first, last, split} (their boxes come
//                    from pre / suf)
//   nodes[4N]        traversal node per slot = 4 x float4 = 64 B, the two
//                    children's coordinates interleaved in pairs so that one
//                    packed f32x2 operation serves both child boxes:
//                      {c0.lo.x, c1.lo.x, c0.lo.y, c1.lo.y}
//                      {c0.lo.z, c1.lo.z, c0.hi.x, c1.hi.x}
//                      {c0.hi.y, c1.hi.y, c0.hi.z, c1.hi.z}
//                      {ref0, ref1, cnt0, cnt1} as int bit patterns
//                    cnt > 0: leaf of cnt triangles starting at sorted
//                    position ref; cnt == 0: internal slot ref; cnt == -1:
//                    treelet node ref (only inside the treelet copy).
//                    Slot off+n-1 is the root slot (the paper keeps its root
//                    pointer in internalNodes[N_t-1] the same way, Sec. 3.1):
//                    child0 = the Karras root, child1 = empty.
//   nodes4[8N]       4-wide traversal node per slot = 8 x float4 = 128 B: the
//                    slot's grandchildren (a leaf child kept as is), SoA:
//                    {lo.x[4]} {lo.y[4]} {lo.z[4]} {hi.x[4]} {hi.y[4]}
//                    {hi.z[4]} {ref[4]} {cnt[4]}; traversal over these visits
//                    every other level of the binary tree
//   tris[3N]         triangles in leaf order: {v0, orig id}, {v1, -}, {v2, -}
//   treelet[4 S]     breadth-first copy of the top of one mesh's tree
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "rsi.h"

namespace rsi {

constexpr int kMaxLeaf = 8;
constexpr int kTreeletMax = 2048;   // nodes in the breadth-first top treelet
constexpr int kSortThreads = 256;
constexpr int kSortItems = 16;
constexpr int kSortTile = kSortThreads * kSortItems;  // 4096 keys per tile
constexpr int kSortTileMin = kSortThreads * 4;         // 1024 keys per tile (small sorts)
constexpr int kSortBins = 256;
constexpr int kBuildThreads = 256;
constexpr int kBuildChunk = 512;    // triangles per block in bounds / Morton
constexpr int kBoxBlock = 512;      // sorted leaves per block of the bottom-up box pass

// FP32 filter constants (see mt32 below).
constexpr float kFilterK = 0x1p-17f;
constexpr float kFilterEta = 0x1p-100f;
constexpr float kRangeLo = 0x1p-30f;
constexpr float kRangeHi = 0x1p30f;
constexpr float kSlabSlack = 0x1p-18f;
constexpr float kTinyDir = 0x1p-60f;

struct MeshDesc {
    const float* V;
    const int32_t* T;
    int64_t nV;
    int32_t n;     // triangles
    int32_t off;   // offset in concatenated triangle / node arrays
    int32_t blk0;  // first block of this mesh in the bounds / Morton grid
    int32_t nblk;
    int32_t height_axis;  // Morton code: 0 over x, y, z; 1..3 that axis left out
};

struct MeshArgs {
    int32_t M;                // number of meshes
    const MeshDesc* table;    // device table (M > 1)
    const int32_t* blk_mesh;  // block -> mesh (M > 1)
    MeshDesc one;             // inline descriptor (M == 1)
};

__device__ __forceinline__ MeshDesc mesh_of(const MeshArgs& a, int m) {
    return a.M == 1 ? a.one : a.table[m];
}

struct TreeBufs {
    int32_t N;  // total triangles
    int32_t M;  // meshes
    uint64_t* keys[2];
    uint32_t* vals[2];
    uint32_t* hist;
    uint32_t* totals;  // kSortBins digit totals of the current sort pass
    int32_t ntiles;
    int32_t nblk;     // blocks of the bounds / Morton grid
    float* partial;   // 6 * nblk
    float* bounds;    // 6 * M
    float4* rootbox;  // 2 * M: box of each mesh (lo, hi)
    int32_t* child;   // 2N
    int32_t* range;   // 2N
    int4* span;       // N: slots whose leaf range crosses a box-pass block
                      // {slot, first leaf, last leaf, split}
    int32_t* nspan;   // entries of span
    float4* pre;      // 2N: union of the leaf boxes from the box-pass block's first leaf
    float4* suf;      // 2N: union of the leaf boxes to the box-pass block's last leaf
    float4* nbox;     // 2N
    float4* lbox;     // 2N
    float4* nodes;    // 4N
    float4* nodes4;   // 8N: 4-wide records (grandchildren of each slot)
    float4* tris;     // 3N
    float4* treelet;  // 4 * kTreeletMax (single-mesh trees)
    int32_t* treelet_n;
    int32_t* status;  // device status word (rsi_status)
    int32_t leaf_size;
    int32_t height_axis;  // the handle's Morton option (copied into each MeshDesc)
    int32_t top_levels;  // < 0: no treelet
    int32_t sorted;      // which keys/vals buffer holds the sorted result
};

// ---------------------------------------------------------------- helpers
__device__ __forceinline__ float4 ld4(const float4* p) { return __ldg(p); }

__device__ __forceinline__ int f2i(float x) { return __float_as_int(x); }
__device__ __forceinline__ float i2f(int x) { return __int_as_float(x); }

__device__ __forceinline__ float maxabs3(float x, float y, float z) {
    return fmaxf(fmaxf(fabsf(x), fabsf(y)), fabsf(z));
}

__device__ __forceinline__ bool finite3(float x, float y, float z) {
    return isfinite(x) && isfinite(y) && isfinite(z);
}

// 1/x with at most 1 ulp error (PTX rcp.approx.f32, subnormals kept);
// 1/(+-0) = +-inf, 1/(+-inf) = +-0.
__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Packed pairs of floats for the f32x2 instructions (one instruction computes
// the same operation for both children of a node).
__device__ __forceinline__ unsigned long long pk2(float a, float b) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ float2 up2(unsigned long long r) {
    float2 v;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(v.x), "=f"(v.y) : "l"(r));
    return v;
}
__device__ __forceinline__ float lo32(unsigned long long r) {
    float a;
    asm("{\n\t.reg .b32 hi;\n\tmov.b64 {%0, hi}, %1;\n\t}" : "=f"(a) : "l"(r));
    return a;
}

// Per-segment registers of the traversal.  Each endpoint and reciprocal
// coordinate is held once, duplicated in both halves of a packed pair for the
// f32x2 box test; the scalar accessors read the low half, so the register pair
// serves both uses.
struct Seg {
    unsigned long long pax, pay, paz;  // (a_k, a_k): start a, packed for f32x2 arithmetic
    unsigned long long pix, piy, piz;  // (1/d_k, 1/d_k) (IEEE; +-inf for a zero component)
    float dx, dy, dz;  // d = fl(b - a)
    float md;          // max |d_i|
    bool tiny;         // some 0 < |d_i| < 2^-60: boxes tested by overlap instead
    bool fp64only;     // |d| outside the FP32 filter's range: decide in FP64
    __device__ __forceinline__ float ax() const { return lo32(pax); }
    __device__ __forceinline__ float ay() const { return lo32(pay); }
    __device__ __forceinline__ float az() const { return lo32(paz); }
    __device__ __forceinline__ float ix() const { return lo32(pix); }
    __device__ __forceinline__ float iy() const { return lo32(piy); }
    __device__ __forceinline__ float iz() const { return lo32(piz); }
};

__device__ __forceinline__ unsigned long long sub2(unsigned long long a, unsigned long long b) {
    unsigned long long r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ unsigned long long mul2(unsigned long long a, unsigned long long b) {
    unsigned long long r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}

__device__ __forceinline__ bool seg_setup(const float* A, const float* B, int64_t i, Seg& s) {
    const float ax = A[3 * i], ay = A[3 * i + 1], az = A[3 * i + 2];
    const float bx = B[3 * i], by = B[3 * i + 1], bz = B[3 * i + 2];
    if (!(finite3(ax, ay, az) && finite3(bx, by, bz))) return false;
    s.dx = __fsub_rn(bx, ax);
    s.dy = __fsub_rn(by, ay);
    s.dz = __fsub_rn(bz, az);
    // An overflowing difference (|b - a| > FLT_MAX) gives 1/d = 0: that axis
    // then never culls (conservative) and every decision is taken in FP64.
    // The reciprocal may be off by 1 ulp (PTX rcp.approx): the slab test's
    // slack covers it.
    const float ix = rcp_approx(s.dx), iy = rcp_approx(s.dy), iz = rcp_approx(s.dz);
    s.md = maxabs3(s.dx, s.dy, s.dz);
    const float mn = fminf(fminf(s.dx != 0.f ? fabsf(s.dx) : 1.f, s.dy != 0.f ? fabsf(s.dy) : 1.f),
                           s.dz != 0.f ? fabsf(s.dz) : 1.f);
    s.tiny = mn < kTinyDir;
    s.fp64only = !(s.md >= kRangeLo && s.md <= kRangeHi);
    s.pax = pk2(ax, ax);
    s.pay = pk2(ay, ay);
    s.paz = pk2(az, az);
    s.pix = pk2(ix, ix);
    s.piy = pk2(iy, iy);
    s.piz = pk2(iz, iz);
    return true;
}

// Conservative segment / box test.  Per axis the entry parameter uses the
// near face and the exit the far face (chosen by the sign of 1/d), computed
// as (face - a) * (1/d): with d rounded (u), 1/d within 1 ulp (2u) and two
// more roundings, each has relative error <= 5u, so scaling the exit by
// 1 + 2^-18 before `entry <= exit` never rejects a box the exact segment
// a + s d, s in [0, tlim], touches.  A zero direction component gives
// (face - a) * inf = +-inf (correct limit) or NaN when the segment lies in
// the face plane; fmaxf / fminf drop NaN, which is the right answer there.
__device__ __forceinline__ bool slab(const Seg& s, float lx, float ly, float lz, float hx,
                                     float hy, float hz, float tlim, float& tent) {
    if (s.tiny) {
        // box-overlap test of the segment's own box; a + fl(b - a) is within
        // 3u (|a| + |b|) of b, so the box is padded by 2^-21 (|a| + |a + d|)
        tent = 0.f;
        const float bx = s.ax() + s.dx, by = s.ay() + s.dy, bz = s.az() + s.dz;
        const float px = (fabsf(s.ax()) + fabsf(bx)) * 0x1p-21f + 0x1p-140f;
        const float py = (fabsf(s.ay()) + fabsf(by)) * 0x1p-21f + 0x1p-140f;
        const float pz = (fabsf(s.az()) + fabsf(bz)) * 0x1p-21f + 0x1p-140f;
        return !(fmaxf(s.ax(), bx) + px < lx || fminf(s.ax(), bx) - px > hx ||
                 fmaxf(s.ay(), by) + py < ly || fminf(s.ay(), by) - py > hy ||
                 fmaxf(s.az(), bz) + pz < lz || fminf(s.az(), bz) - pz > hz);
    }
    const bool nx = s.ix() < 0.f, ny = s.iy() < 0.f, nz = s.iz() < 0.f;
    const float tnx = (__fsub_rn(nx ? hx : lx, s.ax())) * s.ix();
    const float tfx = (__fsub_rn(nx ? lx : hx, s.ax())) * s.ix();
    const float tny = (__fsub_rn(ny ? hy : ly, s.ay())) * s.iy();
    const float tfy = (__fsub_rn(ny ? ly : hy, s.ay())) * s.iy();
    const float tnz = (__fsub_rn(nz ? hz : lz, s.az())) * s.iz();
    const float tfz = (__fsub_rn(nz ? lz : hz, s.az())) * s.iz();
    const float tn = fmaxf(fmaxf(tnx, tny), fmaxf(tnz, 0.f));
    const float tf = fminf(fminf(tfx, tfy), fminf(tfz, tlim));
    tent = tn;
    return tn <= tf * (1.f + kSlabSlack);
}

// The slab test of both children of a node at once, on the paired node
// layout: per axis the near-face and far-face parameters of the two children
// come from one f32x2 subtraction and one f32x2 multiplication (IEEE RN per
// lane, the same rounding as the scalar test above).  q0..q2 are the node's
// first three 16-byte words.
__device__ __forceinline__ void slab2(const Seg& s, const ulonglong2& q0, const ulonglong2& q1,
                                      const ulonglong2& q2, float tlim, bool& h0, float& t0,
                                      bool& h1, float& t1) {
    const unsigned long long lox = q0.x, loy = q0.y, loz = q1.x;
    const unsigned long long hix = q1.y, hiy = q2.x, hiz = q2.y;
    if (s.tiny) {
        const float2 lx = up2(lox), ly = up2(loy), lz = up2(loz);
        const float2 hx = up2(hix), hy = up2(hiy), hz = up2(hiz);
        h0 = slab(s, lx.x, ly.x, lz.x, hx.x, hy.x, hz.x, tlim, t0);
        h1 = slab(s, lx.y, ly.y, lz.y, hx.y, hy.y, hz.y, tlim, t1);
        return;
    }
    const bool nx = s.ix() < 0.f, ny = s.iy() < 0.f, nz = s.iz() < 0.f;
    const float2 tnx = up2(mul2(sub2(nx ? hix : lox, s.pax), s.pix));
    const float2 tfx = up2(mul2(sub2(nx ? lox : hix, s.pax), s.pix));
    const float2 tny = up2(mul2(sub2(ny ? hiy : loy, s.pay), s.piy));
    const float2 tfy = up2(mul2(sub2(ny ? loy : hiy, s.pay), s.piy));
    const float2 tnz = up2(mul2(sub2(nz ? hiz : loz, s.paz), s.piz));
    const float2 tfz = up2(mul2(sub2(nz ? loz : hiz, s.paz), s.piz));
    const float tn0 = fmaxf(fmaxf(tnx.x, tny.x), fmaxf(tnz.x, 0.f));
    const float tn1 = fmaxf(fmaxf(tnx.y, tny.y), fmaxf(tnz.y, 0.f));
    const float tf0 = fminf(fminf(tfx.x, tfy.x), fminf(tfz.x, tlim));
    const float tf1 = fminf(fminf(tfx.y, tfy.y), fminf(tfz.y, tlim));
    const float2 tf = up2(mul2(pk2(tf0, tf1), pk2(1.f + kSlabSlack, 1.f + kSlabSlack)));
    t0 = tn0;
    t1 = tn1;
    h0 = tn0 <= tf.x;
    h1 = tn1 <= tf.y;
}

// FP32 Moller-Trumbore with a two-stage error filter.
//
// With u = 2^-24 and exact float inputs, every elementary term of a computed
// triple product (det = e1.(d x e2), nU = s0.(d x e2), nV = d.(s0 x e1),
// nT = e2.(s0 x e1)), e.g. s0x d_y e2z, carries at most 8 roundings (the
// three input differences, the product, the cross-product difference, the
// dot product's product and two sums; FMA contraction only removes
// roundings), so |computed - exact| <= gamma_8 M with the componentwise sum
// M = sum_i |x_i| (|y_j| |z_k| + |y_k| |z_j|) <= 6 m_x m_y m_z (m = max_i).
//  - Stage 1 (cheap): B = K m_x m_y m_z + eta, K = 2^-17 (> 6 gamma_8 plus
//    the FP64 definition's own error and the rounding of the bound).
//  - Stage 2, only when stage 1 cannot decide: B = g M~ + eta with M~
//    evaluated from the computed factors (3 + 5 more roundings) and
//    g = 11u (> gamma_8 (1 + gamma_8) plus the FP64 definition's gamma_8 of
//    2^-53).  For long segments over small triangles it is far tighter:
//    |s0| multiplies only the components of d x e2 it meets.
// The derived sums w = det - nU - nV and r = det - nT add 12u of their
// operands' magnitudes (stage 1, folded into K) or their two / one
// roundings (stage 2, 2.01u / 1.01u).  eta = 2^-100 covers absolute errors
// from underflow while every factor's max lies in [2^-30, 2^30] (else the
// FP64 path decides, as it does for a zero or out-of-range value).  A value
// whose computed magnitude clears its bound has the sign of the exact value,
// and so of the FP64 definition's value: certified decisions equal the
// definition's; the rest return 2 and are decided in FP64.  Returns 0 miss,
// 1 hit, 2 undecided; with `want` also (t, u, v) and a bound err on their
// errors against the exact values, (B_x + |x~| B_det) / (|det~| - B_det)
// plus the two roundings of x~ = n_x * fl(1 / |det~|), from the bounds of
// the stage that decided.
__device__ __forceinline__ int mt32(const Seg& s, const float4& A, const float4& B,
                                    const float4& C, bool want, float& t, float& u, float& v,
                                    float& err) {
    const float e1x = B.x - A.x, e1y = B.y - A.y, e1z = B.z - A.z;
    const float e2x = C.x - A.x, e2y = C.y - A.y, e2z = C.z - A.z;
    const float m1 = maxabs3(e1x, e1y, e1z);
    const float m2 = maxabs3(e2x, e2y, e2z);
    // An exactly zero edge makes det exactly zero in FP64 too: never a hit.
    if (m1 == 0.f || m2 == 0.f) return 0;
    const float sx = s.ax() - A.x, sy = s.ay() - A.y, sz = s.az() - A.z;
    const float ms = maxabs3(sx, sy, sz);
    const float mhi = fmaxf(fmaxf(m1, m2), ms);
    const float mlo = fminf(fminf(m1, m2), ms == 0.f ? 1.f : ms);
    if (s.fp64only || mhi > kRangeHi || mlo < kRangeLo) return 2;
    const float px = s.dy * e2z - s.dz * e2y;
    const float py = s.dz * e2x - s.dx * e2z;
    const float pz = s.dx * e2y - s.dy * e2x;
    const float det = e1x * px + e1y * py + e1z * pz;
    const float qx = sy * e1z - sz * e1y;
    const float qy = sz * e1x - sx * e1z;
    const float qz = sx * e1y - sy * e1x;
    float nu = sx * px + sy * py + sz * pz;
    float nv = s.dx * qx + s.dy * qy + s.dz * qz;
    float nt = e2x * qx + e2y * qy + e2z * qz;
    const float adet = fabsf(det);
    if (det < 0.f) {  // used only once a stage has certified the sign of det
        nu = -nu;
        nv = -nv;
        nt = -nt;
    }
    const float w = (adet - nu) - nv;
    const float r = adet - nt;
    float Bdet, BU, BV, BT;
    int res = 2;
    {  // stage 1: max-norm bounds
        const float Pde = s.md * m2, Pse = ms * m1;
        const float Mdet = m1 * Pde, MU = ms * Pde, MV = s.md * Pse, MT = m2 * Pse;
        Bdet = fmaf(kFilterK, Mdet, kFilterEta);
        BU = fmaf(kFilterK, MU, kFilterEta);
        BV = fmaf(kFilterK, MV, kFilterEta);
        BT = fmaf(kFilterK, MT, kFilterEta);
        const float Bw = fmaf(kFilterK, Mdet + MU + MV, kFilterEta);
        const float Br = fmaf(kFilterK, Mdet + MT, kFilterEta);
        if (adet > Bdet) {
            if (nu < -BU || nv < -BV || nt < -BT || w < -Bw || r < -Br) return 0;
            if (nu > BU && nv > BV && nt > BT && w > Bw && r > Br) res = 1;
        }
    }
    if (res == 2) {  // stage 2: componentwise bounds
        const float g = 11.f * 0x1p-24f;
        const float Px = fabsf(s.dy) * fabsf(e2z) + fabsf(s.dz) * fabsf(e2y);
        const float Py = fabsf(s.dz) * fabsf(e2x) + fabsf(s.dx) * fabsf(e2z);
        const float Pz = fabsf(s.dx) * fabsf(e2y) + fabsf(s.dy) * fabsf(e2x);
        const float Qx = fabsf(sy) * fabsf(e1z) + fabsf(sz) * fabsf(e1y);
        const float Qy = fabsf(sz) * fabsf(e1x) + fabsf(sx) * fabsf(e1z);
        const float Qz = fabsf(sx) * fabsf(e1y) + fabsf(sy) * fabsf(e1x);
        Bdet = fmaf(g, fabsf(e1x) * Px + fabsf(e1y) * Py + fabsf(e1z) * Pz, kFilterEta);
        if (!(adet > Bdet)) return 2;
        BU = fmaf(g, fabsf(sx) * Px + fabsf(sy) * Py + fabsf(sz) * Pz, kFilterEta);
        BV = fmaf(g, fabsf(s.dx) * Qx + fabsf(s.dy) * Qy + fabsf(s.dz) * Qz, kFilterEta);
        BT = fmaf(g, fabsf(e2x) * Qx + fabsf(e2y) * Qy + fabsf(e2z) * Qz, kFilterEta);
        const float Bw = fmaf(2.01f * 0x1p-24f, adet + fabsf(nu) + fabsf(nv), Bdet + BU + BV);
        const float Br = fmaf(1.01f * 0x1p-24f, adet + fabsf(nt), Bdet + BT);
        if (nu < -BU || nv < -BV || nt < -BT || w < -Bw || r < -Br) return 0;
        if (!(nu > BU && nv > BV && nt > BT && w > Bw && r > Br)) return 2;
    }
    if (want) {
        const float inv = __frcp_rn(adet);
        t = nt * inv;
        u = nu * inv;
        v = nv * inv;
        const float den = __frcp_rn(adet - Bdet);
        const float eT = fmaf(t, Bdet, BT) * den;
        const float eU = fmaf(u, Bdet, BU) * den;
        const float eV = fmaf(v, Bdet, BV) * den;
        err = fmaxf(fmaxf(eT, eU), eV) * 1.001f + 0x1p-22f;
    }
    return 1;
}

// The FP64 definition (public header) in its exact operation order: no
// contraction, every product / sum rounded where written.  Inputs are the
// float coordinates widened exactly.  Returns hit; t, u, v when hit.
static __device__ __noinline__ int mt64(float ax_, float ay_, float az_, float bx_, float by_,
                                 float bz_, float4 A, float4 B, float4 C, double* tuv) {
    const double ax = ax_, ay = ay_, az = az_;
    const double dx = __dsub_rn((double)bx_, ax), dy = __dsub_rn((double)by_, ay),
                 dz = __dsub_rn((double)bz_, az);
    const double v0x = A.x, v0y = A.y, v0z = A.z;
    const double e1x = __dsub_rn((double)B.x, v0x), e1y = __dsub_rn((double)B.y, v0y),
                 e1z = __dsub_rn((double)B.z, v0z);
    const double e2x = __dsub_rn((double)C.x, v0x), e2y = __dsub_rn((double)C.y, v0y),
                 e2z = __dsub_rn((double)C.z, v0z);
    const double px = __dsub_rn(__dmul_rn(dy, e2z), __dmul_rn(dz, e2y));
    const double py = __dsub_rn(__dmul_rn(dz, e2x), __dmul_rn(dx, e2z));
    const double pz = __dsub_rn(__dmul_rn(dx, e2y), __dmul_rn(dy, e2x));
    double det = __dadd_rn(__dadd_rn(__dmul_rn(e1x, px), __dmul_rn(e1y, py)), __dmul_rn(e1z, pz));
    const double sx = __dsub_rn(ax, v0x), sy = __dsub_rn(ay, v0y), sz = __dsub_rn(az, v0z);
    const double qx = __dsub_rn(__dmul_rn(sy, e1z), __dmul_rn(sz, e1y));
    const double qy = __dsub_rn(__dmul_rn(sz, e1x), __dmul_rn(sx, e1z));
    const double qz = __dsub_rn(__dmul_rn(sx, e1y), __dmul_rn(sy, e1x));
    double nu = __dadd_rn(__dadd_rn(__dmul_rn(sx, px), __dmul_rn(sy, py)), __dmul_rn(sz, pz));
    double nv = __dadd_rn(__dadd_rn(__dmul_rn(dx, qx), __dmul_rn(dy, qy)), __dmul_rn(dz, qz));
    double nt = __dadd_rn(__dadd_rn(__dmul_rn(e2x, qx), __dmul_rn(e2y, qy)), __dmul_rn(e2z, qz));
    if (det < 0.0) {
        det = -det;
        nu = -nu;
        nv = -nv;
        nt = -nt;
    }
    const int hit = (det > 0.0) && (nu >= 0.0) && (nv >= 0.0) && (__dadd_rn(nu, nv) <= det) &&
                    (nt >= 0.0) && (nt <= det);
    if (hit && tuv) {
        tuv[0] = __ddiv_rn(nt, det);
        tuv[1] = __ddiv_rn(nu, det);
        tuv[2] = __ddiv_rn(nv, det);
    }
    return hit;
}

// A tighter rigorous bound on the FP32 (t, u, v) of one (segment,
// triangle) pair, for the nearest crossing's outputs: the same triple
// products as mt32, but the rounding error of each is bounded with the
// componentwise magnitudes sum |x_i| (|y_j| |z_k| + |y_k| |z_j|) and gamma_10
// (every term carries at most 8 roundings, 2 more cover the magnitudes'
// own rounding), instead of the max-norm products and 2^-17 that decisions
// use.  Returns the bound on |t~ - t| and, in euv, the bound on
// max(|u~ - u|, |v~ - v|), with the FP32 values; +inf when det cannot be
// bounded away from zero.
__device__ __forceinline__ float mt32_tight(const Seg& s, const float4& A, const float4& B,
                                           const float4& C, float& t, float& u, float& v,
                                           float& euv) {
    const float e1x = B.x - A.x, e1y = B.y - A.y, e1z = B.z - A.z;
    const float e2x = C.x - A.x, e2y = C.y - A.y, e2z = C.z - A.z;
    const float sx = s.ax() - A.x, sy = s.ay() - A.y, sz = s.az() - A.z;
    const float px = s.dy * e2z - s.dz * e2y, py = s.dz * e2x - s.dx * e2z;
    const float pz = s.dx * e2y - s.dy * e2x;
    const float qx = sy * e1z - sz * e1y, qy = sz * e1x - sx * e1z, qz = sx * e1y - sy * e1x;
    const float det = e1x * px + e1y * py + e1z * pz;
    const float nu = sx * px + sy * py + sz * pz;
    const float nv = s.dx * qx + s.dy * qy + s.dz * qz;
    const float nt = e2x * qx + e2y * qy + e2z * qz;
    // componentwise magnitudes of p and q
    const float Px = fabsf(s.dy) * fabsf(e2z) + fabsf(s.dz) * fabsf(e2y);
    const float Py = fabsf(s.dz) * fabsf(e2x) + fabsf(s.dx) * fabsf(e2z);
    const float Pz = fabsf(s.dx) * fabsf(e2y) + fabsf(s.dy) * fabsf(e2x);
    const float Qx = fabsf(sy) * fabsf(e1z) + fabsf(sz) * fabsf(e1y);
    const float Qy = fabsf(sz) * fabsf(e1x) + fabsf(sx) * fabsf(e1z);
    const float Qz = fabsf(sx) * fabsf(e1y) + fabsf(sy) * fabsf(e1x);
    const float g = 10.f * 0x1p-24f * 1.0001f;
    const float Bd = g * (fabsf(e1x) * Px + fabsf(e1y) * Py + fabsf(e1z) * Pz) + kFilterEta;
    const float Bu = g * (fabsf(sx) * Px + fabsf(sy) * Py + fabsf(sz) * Pz) + kFilterEta;
    const float Bv = g * (fabsf(s.dx) * Qx + fabsf(s.dy) * Qy + fabsf(s.dz) * Qz) + kFilterEta;
    const float Bt = g * (fabsf(e2x) * Qx + fabsf(e2y) * Qy + fabsf(e2z) * Qz) + kFilterEta;
    const float ad = fabsf(det);
    euv = INFINITY;
    if (!(ad > 2.f * Bd) || !isfinite(ad)) return INFINITY;
    const float inv = __frcp_rn(ad);
    const float sg = det < 0.f ? -1.f : 1.f;
    t = sg * nt * inv;
    u = sg * nu * inv;
    v = sg * nv * inv;
    // |x/det~ - x_exact/det_exact| <= (B_x + |x| B_det / |det|) / (|det| - B_det) + rounding
    const float den = __frcp_rn(ad - Bd);
    const float et = fmaf(fabsf(t), Bd, Bt) * den;
    const float eu = fmaf(fabsf(u), Bd, Bu) * den;
    const float ev = fmaf(fabsf(v), Bd, Bv) * den;
    euv = fmaxf(eu, ev) * 1.001f + 0x1p-22f * fmaxf(1.f, fmaxf(fabsf(u), fabsf(v)));
    return et * 1.001f + 0x1p-22f * fmaxf(1.f, fabsf(t));
}

// ---------------------------------------------------------------- double-float
// Unevaluated sums h + l of two floats (about 44 significant bits) built from
// the error-free transformations two-sum (Knuth) and two-product (via FMA),
// for the nearest hit's (t, u, v): FP64 is one to two orders of magnitude
// slower than FP32 on this GPU, and these values need more than FP32 only
// when the segment meets the triangle at a grazing angle.
struct dfl {
    float h, l;
};

__device__ __forceinline__ dfl df_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}

__device__ __forceinline__ dfl df_fast(float a, float b) {  // |a| >= |b|
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ dfl df_add(dfl a, dfl b) {
    dfl s = df_two_sum(a.h, b.h);
    const float e = __fadd_rn(s.l, __fadd_rn(a.l, b.l));
    return df_fast(s.h, e);
}

__device__ __forceinline__ dfl df_neg(dfl a) { return {-a.h, -a.l}; }

__device__ __forceinline__ dfl df_mul(dfl a, dfl b) {
    const float p = __fmul_rn(a.h, b.h);
    float e = __fmaf_rn(a.h, b.h, -p);
    e = __fmaf_rn(a.h, b.l, __fmaf_rn(a.l, b.h, e));
    return df_fast(p, e);
}

// a / b given r ~ 1 / b.h (any 1-ulp approximation): q1 = a.h r, then one
// correction from the exact double-float residual a - b q1.
__device__ __forceinline__ dfl df_div(dfl a, dfl b, float r) {
    const float q1 = __fmul_rn(a.h, r);
    const dfl res = df_add(a, df_neg(df_mul(b, {q1, 0.f})));
    const float q2 = __fmul_rn(res.h, r);
    return df_fast(q1, q2);
}

__device__ __forceinline__ float df_float(dfl a) { return __fadd_rn(a.h, a.l); }

// (t, u, v) of the segment a -> b against triangle (v0, v1, v2) in
// double-float, in the operation order of the definition (differences are
// exact in double-float); t is returned as a double-float pair so that the
// point a + t d can be formed without rounding t to FP32 first.  Only used
// for values, never for decisions.
__device__ __forceinline__ void mt_df(const float* a3, const float* b3, float4 A, float4 B,
                                      float4 C, dfl& t, float& u, float& v) {
    dfl d[3], e1[3], e2[3], s0[3];
    const float v0[3] = {A.x, A.y, A.z}, v1[3] = {B.x, B.y, B.z}, v2[3] = {C.x, C.y, C.z};
    for (int k = 0; k < 3; ++k) {
        d[k] = df_two_sum(b3[k], -a3[k]);
        e1[k] = df_two_sum(v1[k], -v0[k]);
        e2[k] = df_two_sum(v2[k], -v0[k]);
        s0[k] = df_two_sum(a3[k], -v0[k]);
    }
    auto cross = [](const dfl* x, const dfl* y, dfl* r) {
        r[0] = df_add(df_mul(x[1], y[2]), df_neg(df_mul(x[2], y[1])));
        r[1] = df_add(df_mul(x[2], y[0]), df_neg(df_mul(x[0], y[2])));
        r[2] = df_add(df_mul(x[0], y[1]), df_neg(df_mul(x[1], y[0])));
    };
    auto dot = [](const dfl* x, const dfl* y) {
        return df_add(df_add(df_mul(x[0], y[0]), df_mul(x[1], y[1])), df_mul(x[2], y[2]));
    };
    dfl p[3], q[3];
    cross(d, e2, p);
    const dfl det = dot(e1, p);
    cross(s0, e1, q);
    const dfl nu = dot(s0, p), nv = dot(d, q), nt = dot(e2, q);
    const float r = rcp_approx(det.h);
    t = df_div(nt, det, r);
    u = df_float(df_div(nu, det, r));
    v = df_float(df_div(nv, det, r));
}

}  // namespace rsi
