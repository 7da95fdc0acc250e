// Stable LSD radix sort of (key, value) pairs on the device, 8-bit digits,
// used for the triangle Morton keys (a3) and for the coherent segment order.
//
// One pass over digit `shift`:
//   k_sort_hist    per tile of kSortTile keys: digit histogram -> hist[d][tile]
//   k_sort_scan    one block per digit: exclusive scan over the tiles of
//                  hist[d][*] in place, digit total -> totals[d]
//   k_sort_scatter per tile: digit bases (exclusive scan of totals), stable
//                  rank within the tile (each warp owns a contiguous run and
//                  ranks equal digits with __match_any_sync in key order),
//                  scatter to base + tile offset + rank.
// With at most kSortFuseTiles tiles the scan kernel is skipped: every
// scatter block sums the (few) tile histograms of its digit itself.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "rsi_internal.cuh"

namespace rsi {

template <typename K, int ITEMS>
__global__ void __launch_bounds__(kSortThreads) k_sort_hist(const K* __restrict__ keys, int n,
                                                            int shift, uint32_t* __restrict__ hist,
                                                            int ntiles) {
    __shared__ uint32_t h[kSortBins];
    h[threadIdx.x] = 0;
    __syncthreads();
    const int base = blockIdx.x * kSortThreads * ITEMS;
#pragma unroll 4
    for (int it = 0; it < ITEMS; ++it) {
        const int pos = base + it * kSortThreads + threadIdx.x;
        if (pos < n) atomicAdd(&h[(uint32_t)(keys[pos] >> shift) & 0xffu], 1u);
    }
    __syncthreads();
    hist[threadIdx.x * ntiles + blockIdx.x] = h[threadIdx.x];
}

// Block-wide exclusive scan of one value per thread (blockDim.x <= 1024).
__device__ __forceinline__ uint32_t block_scan_u32(uint32_t x, uint32_t* total) {
    __shared__ uint32_t ws[32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t incl = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) ws[w] = incl;
    __syncthreads();
    if (w == 0) {
        const int nw = blockDim.x >> 5;
        uint32_t v = lane < nw ? ws[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += y;
        }
        ws[lane] = v;
    }
    __syncthreads();
    if (total) *total = ws[(blockDim.x >> 5) - 1];
    const uint32_t r = incl - x + (w > 0 ? ws[w - 1] : 0u);
    __syncthreads();
    return r;
}

// One block (256 threads) per digit: exclusive scan of hist[d][0..ntiles).
static __global__ void __launch_bounds__(256) k_sort_scan(uint32_t* __restrict__ hist, int ntiles,
                                                   uint32_t* __restrict__ totals) {
    uint32_t* row = hist + (size_t)blockIdx.x * ntiles;
    const int per = (ntiles + blockDim.x - 1) / blockDim.x;
    const int b = threadIdx.x * per, e = min(ntiles, b + per);
    uint32_t sum = 0;
    for (int q = b; q < e; ++q) sum += row[q];
    uint32_t tot;
    uint32_t run = block_scan_u32(sum, &tot);
    for (int q = b; q < e; ++q) {
        const uint32_t x = row[q];
        row[q] = run;
        run += x;
    }
    if (threadIdx.x == 0) totals[blockIdx.x] = tot;
}

constexpr int kSortFuseTiles = 64;

template <typename K, int ITEMS, bool FUSED>
__global__ void __launch_bounds__(kSortThreads) k_sort_scatter(
    const K* __restrict__ kin, const uint32_t* __restrict__ vin, K* __restrict__ kout,
    uint32_t* __restrict__ vout, int n, int shift, const uint32_t* __restrict__ hist,
    const uint32_t* __restrict__ totals, int ntiles) {
    constexpr int W = kSortThreads / 32;
    __shared__ uint32_t cnt[W][kSortBins];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int q = threadIdx.x; q < W * kSortBins; q += kSortThreads) (&cnt[0][0])[q] = 0;
    // this tile's offset within digit d (FUSED: summed here from the raw tile
    // histograms) and the digit total; kSortThreads == bins, thread = digit
    uint32_t toff, dtot;
    if (FUSED) {
        const uint32_t* row = hist + (size_t)threadIdx.x * ntiles;
        toff = dtot = 0u;
        for (int q = 0; q < ntiles; ++q) {
            const uint32_t x = row[q];
            toff += q < (int)blockIdx.x ? x : 0u;
            dtot += x;
        }
    } else {
        toff = hist[threadIdx.x * ntiles + blockIdx.x];
        dtot = totals[threadIdx.x];
    }
    // digit base = exclusive scan of the digit totals
    const uint32_t dbase = block_scan_u32(dtot, nullptr);
    const int wbase = blockIdx.x * (kSortThreads * ITEMS) + w * (32 * ITEMS);
    const uint32_t lt = (1u << lane) - 1u;
    uint32_t local[ITEMS];
#pragma unroll
    for (int it = 0; it < ITEMS; ++it) {
        const int pos = wbase + it * 32 + lane;
        const bool valid = pos < n;
        const uint32_t d = valid ? ((uint32_t)(kin[pos] >> shift) & 0xffu) : 0x100u;
        const uint32_t peers = __match_any_sync(0xffffffffu, d);
        const uint32_t rank = __popc(peers & lt);
        const uint32_t c = valid ? cnt[w][d] : 0u;
        __syncwarp();
        if (valid && rank == 0) cnt[w][d] = c + __popc(peers);
        __syncwarp();
        local[it] = c + rank;
    }
    __syncthreads();
    {
        const int d = threadIdx.x;
        uint32_t run = dbase + toff;
#pragma unroll
        for (int q = 0; q < W; ++q) {
            const uint32_t x = cnt[q][d];
            cnt[q][d] = run;
            run += x;
        }
    }
    __syncthreads();
#pragma unroll
    for (int it = 0; it < ITEMS; ++it) {
        const int pos = wbase + it * 32 + lane;
        if (pos < n) {
            const K k = kin[pos];
            const uint32_t d = (uint32_t)(k >> shift) & 0xffu;
            const uint32_t o = cnt[w][d] + local[it];
            kout[o] = k;
            vout[o] = vin[pos];
        }
    }
}

// Sort keys[0] / vals[0] (n entries) over the digits at `shifts`; buffers
// keys[1] / vals[1] are ping-pong space; *out receives the index of the
// buffer pair holding the result.  Tiles hold 1024 keys below 2^18 keys (more
// blocks for small sorts), 4096 above.  hist: kSortBins * ceil(n / 1024)
// words, totals: kSortBins words.
template <typename K, int ITEMS>
static cudaError_t radix_sort_tiles(K* keys[2], uint32_t* vals[2], int n, const int* shifts,
                                    int np, uint32_t* hist, uint32_t* totals, cudaStream_t s,
                                    int* out) {
    const int tile = kSortThreads * ITEMS;
    const int ntiles = (n + tile - 1) / tile;
    int cur = 0;
    for (int p = 0; p < np && n > 0; ++p) {
        k_sort_hist<K, ITEMS><<<ntiles, kSortThreads, 0, s>>>(keys[cur], n, shifts[p], hist,
                                                              ntiles);
        if (ntiles <= kSortFuseTiles) {
            k_sort_scatter<K, ITEMS, true><<<ntiles, kSortThreads, 0, s>>>(
                keys[cur], vals[cur], keys[1 - cur], vals[1 - cur], n, shifts[p], hist, totals,
                ntiles);
        } else {
            k_sort_scan<<<kSortBins, 256, 0, s>>>(hist, ntiles, totals);
            k_sort_scatter<K, ITEMS, false><<<ntiles, kSortThreads, 0, s>>>(
                keys[cur], vals[cur], keys[1 - cur], vals[1 - cur], n, shifts[p], hist, totals,
                ntiles);
        }
        cur = 1 - cur;
    }
    *out = cur;
    return cudaGetLastError();
}

template <typename K>
cudaError_t radix_sort(K* keys[2], uint32_t* vals[2], int n, const int* shifts, int np,
                       uint32_t* hist, uint32_t* totals, cudaStream_t s, int* out) {
    if (n < (1 << 18))
        return radix_sort_tiles<K, 4>(keys, vals, n, shifts, np, hist, totals, s, out);
    return radix_sort_tiles<K, kSortItems>(keys, vals, n, shifts, np, hist, totals, s, out);
}

}  // namespace rsi
