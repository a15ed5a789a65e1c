// Key duplication, radix sort and tile ranges (Section II-B; Algorithm 1's
// "load work range").
//
// The sorted order is that of a stable sort of the 64-bit keys
// (tile << 32 | float_bits(depth)) over instances emitted in (Gaussian id,
// row-major tile) order.  It is reached in fewer passes:
//   1. compact the visible splats in id order            (scan, order kept)
//   2. stable LSD radix sort of (depth bits, id)         (4 x 8-bit passes, N_vis)
//   3. exclusive scan of tiles_touched in depth order    -> M, instance offsets
//   4. duplicate: instances in (depth, id, row-major tile) order, full keys
//   5. stable LSD radix sort on the tile bits only       (ceil(log2 T / 8) passes, M)
//   6. ranges by binary search of each tile's first and last key
// Within a tile, step 5 keeps step 4's (depth, id) order, which is exactly
// the tie-broken key order.  All counts stay on the device.
#include "common.cuh"
#include "sort_ws.h"

namespace gs {

namespace {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 1024;   // elements per block in steps 1, 3, 4
constexpr int kRsThreads = 256;
constexpr int kRsIpt = 8;
constexpr int kRsItems = kRsThreads * kRsIpt;  // 2048 keys per radix tile
constexpr int kRsBins = 256;

__device__ __forceinline__ uint32_t splat_tiles(const gs_splat *s, uint32_t g) {
    return reinterpret_cast<const uint4 *>(s + g)[2].w;
}

// --- step 1: order-preserving compaction of visible splats ---------------
__global__ void __launch_bounds__(kScanThreads) count_visible_kernel(const gs_splat *__restrict__ splats, int64_t n,
                                                                     uint32_t *__restrict__ blk) {
    __shared__ uint32_t scratch[33];
    const int64_t base = (int64_t)blockIdx.x * kScanItems;
    uint32_t c = 0;
#pragma unroll
    for (int k = 0; k < kScanItems / kScanThreads; ++k) {
        int64_t i = base + k * kScanThreads + threadIdx.x;
        if (i < n) c += splat_tiles(splats, (uint32_t)i) != 0u;
    }
    uint32_t total;
    block_exclusive_scan(c, scratch, &total);
    if (threadIdx.x == 0) blk[blockIdx.x] = total;
}

// Exclusive scan of nblk block sums in place (single block of 1024 threads);
// the grand total goes to *total.  Values are widened to 64 bits.
__global__ void __launch_bounds__(1024) scan_blocks_kernel(const uint32_t *__restrict__ in, uint64_t *__restrict__ out,
                                                           uint32_t nblk, SortHeader *__restrict__ hdr, int which,
                                                           uint64_t cap) {
    __shared__ uint32_t scratch[33];
    __shared__ uint64_t carry_s;
    if (threadIdx.x == 0) carry_s = 0;
    __syncthreads();
    for (uint32_t b0 = 0; b0 < nblk; b0 += 1024) {
        uint32_t i = b0 + threadIdx.x;
        uint32_t v = i < nblk ? in[i] : 0u;
        uint32_t tot;
        uint32_t ex = block_exclusive_scan(v, scratch, &tot);
        uint64_t carry = carry_s;
        if (i < nblk) out[i] = carry + ex;
        __syncthreads();
        if (threadIdx.x == 0) carry_s = carry + tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        uint64_t total = carry_s;
        if (which == 0) {
            hdr->nvis = (uint32_t)total;
        } else {
            hdr->m_total = total;
            hdr->m_sort = (uint32_t)(total < cap ? total : cap);
            hdr->overflow = total > cap ? 1u : 0u;
        }
    }
}

__global__ void __launch_bounds__(kScanThreads) compact_kernel(const gs_splat *__restrict__ splats, int64_t n,
                                                               const uint64_t *__restrict__ blk_off,
                                                               uint32_t *__restrict__ dkey,
                                                               uint32_t *__restrict__ dval) {
    __shared__ uint32_t scratch[33];
    const int64_t base = (int64_t)blockIdx.x * kScanItems;
    uint32_t out = (uint32_t)blk_off[blockIdx.x];
#pragma unroll
    for (int k = 0; k < kScanItems / kScanThreads; ++k) {
        int64_t i = base + k * kScanThreads + threadIdx.x;
        uint4 w = make_uint4(0, 0, 0, 0);
        if (i < n) w = reinterpret_cast<const uint4 *>(splats + i)[2];
        const uint32_t vis = w.w != 0u;
        uint32_t total;
        uint32_t ex = block_exclusive_scan(vis, scratch, &total);
        if (vis) {
            dkey[out + ex] = w.y;  // FP32 depth bits (positive: uint order = float order)
            dval[out + ex] = (uint32_t)i;
        }
        out += total;
    }
}

// --- generic stable LSD radix pass (reduce-then-scan) ----------------------
template <typename K>
__device__ __forceinline__ uint32_t digit_of(K key, int shift, uint32_t mask) {
    return (uint32_t)(key >> shift) & mask;
}

template <typename K>
__global__ void __launch_bounds__(kRsThreads) radix_upsweep_kernel(const K *__restrict__ keys,
                                                                   const uint32_t *__restrict__ count_ptr,
                                                                   int shift, uint32_t mask,
                                                                   uint32_t *__restrict__ hist, uint32_t ntiles) {
    __shared__ uint32_t h[kRsBins];
    h[threadIdx.x] = 0;
    __syncthreads();
    const uint32_t n = *count_ptr;
    const uint32_t start = blockIdx.x * kRsItems;
    if (start < n) {
#pragma unroll
        for (int k = 0; k < kRsIpt; ++k) {
            uint32_t i = start + k * kRsThreads + threadIdx.x;
            const bool valid = i < n;
            uint32_t d = valid ? digit_of<K>(keys[i], shift, mask) : 0xffffffffu;
            unsigned peers = __match_any_sync(0xffffffffu, d);
            if (valid && (peers & lanemask_lt()) == 0) atomicAdd(&h[d], (uint32_t)__popc(peers));
        }
    }
    __syncthreads();
    hist[threadIdx.x * ntiles + blockIdx.x] = h[threadIdx.x];
}

// One block per digit: exclusive scan of that digit's per-tile counts over
// the active tiles, in place; the digit total goes to dtotal[d].
__global__ void __launch_bounds__(1024) radix_scan_kernel(uint32_t *__restrict__ hist, uint32_t ntiles,
                                                          const uint32_t *__restrict__ count_ptr,
                                                          uint32_t *__restrict__ dtotal) {
    __shared__ uint32_t scratch[33];
    __shared__ uint32_t carry_s;
    const uint32_t d = blockIdx.x;
    const uint32_t n = *count_ptr;
    const uint32_t nt = (n + kRsItems - 1) / kRsItems;
    if (threadIdx.x == 0) carry_s = 0;
    __syncthreads();
    uint32_t *row = hist + (size_t)d * ntiles;
    for (uint32_t b0 = 0; b0 < nt; b0 += 1024) {
        uint32_t i = b0 + threadIdx.x;
        uint32_t v = i < nt ? row[i] : 0u;
        uint32_t tot;
        uint32_t ex = block_exclusive_scan(v, scratch, &tot);
        uint32_t carry = carry_s;
        if (i < nt) row[i] = carry + ex;
        __syncthreads();
        if (threadIdx.x == 0) carry_s = carry + tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) dtotal[d] = carry_s;
}

template <typename K>
__global__ void __launch_bounds__(kRsThreads) radix_downsweep_kernel(
    const K *__restrict__ kin, const uint32_t *__restrict__ vin, K *__restrict__ kout, uint32_t *__restrict__ vout,
    const uint32_t *__restrict__ count_ptr, int shift, uint32_t mask, const uint32_t *__restrict__ hist,
    uint32_t ntiles, const uint32_t *__restrict__ dtotal) {
    __shared__ K s_keys[kRsItems];
    __shared__ uint32_t s_vals[kRsItems];
    __shared__ uint32_t s_wcnt[kRsThreads / 32][kRsBins];
    __shared__ uint32_t s_base[kRsBins];
    __shared__ uint32_t s_dstart[kRsBins];
    __shared__ uint32_t scratch[33];

    const uint32_t n = *count_ptr;
    const uint32_t start = blockIdx.x * kRsItems;
    if (start >= n) return;  // uniform over the block
    const unsigned t = threadIdx.x, lane = lane_id(), warp = t >> 5;

    // global base of each digit for this tile
    uint32_t tot;
    uint32_t dbase = block_exclusive_scan(dtotal[t], scratch, &tot);
    s_base[t] = dbase + hist[(size_t)t * ntiles + blockIdx.x];
#pragma unroll
    for (int w = 0; w < kRsThreads / 32; ++w) s_wcnt[w][t] = 0;
    __syncthreads();

    // stable warp-local ranking; warp w owns elements [w*256, w*256 + 256)
    K key[kRsIpt];
    uint32_t val[kRsIpt], dig[kRsIpt], rank[kRsIpt];
    const unsigned lt = lanemask_lt();
#pragma unroll
    for (int k = 0; k < kRsIpt; ++k) {
        const uint32_t i = start + warp * (kRsIpt * 32) + k * 32 + lane;
        const bool valid = i < n;
        key[k] = valid ? kin[i] : (K)0;
        val[k] = valid ? vin[i] : 0u;
        const uint32_t d = valid ? digit_of<K>(key[k], shift, mask) : kRsBins;
        dig[k] = d;
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        uint32_t old = 0;
        if (valid) old = s_wcnt[warp][d];
        __syncwarp();
        if (valid && (peers & lt) == 0) s_wcnt[warp][d] = old + (uint32_t)__popc(peers);
        __syncwarp();
        rank[k] = old + (uint32_t)__popc(peers & lt);
    }
    __syncthreads();
    // per digit: exclusive scan over warps, and the tile's count of the digit
    uint32_t run = 0;
#pragma unroll
    for (int w = 0; w < kRsThreads / 32; ++w) {
        uint32_t c = s_wcnt[w][t];
        s_wcnt[w][t] = run;
        run += c;
    }
    uint32_t dstart = block_exclusive_scan(run, scratch, &tot);
    s_dstart[t] = dstart;
    __syncthreads();
    // reorder through shared memory so the global writes are coalesced
#pragma unroll
    for (int k = 0; k < kRsIpt; ++k) {
        const uint32_t d = dig[k];
        if (d < kRsBins) {
            const uint32_t pos = s_dstart[d] + s_wcnt[warp][d] + rank[k];
            s_keys[pos] = key[k];
            s_vals[pos] = val[k];
        }
    }
    __syncthreads();
    const uint32_t cnt = min((uint32_t)kRsItems, n - start);
    for (uint32_t j = t; j < cnt; j += kRsThreads) {
        const K kk = s_keys[j];
        const uint32_t d = digit_of<K>(kk, shift, mask);
        const uint32_t gpos = s_base[d] + (j - s_dstart[d]);
        kout[gpos] = kk;
        vout[gpos] = s_vals[j];
    }
}

// --- step 3: tiles_touched in depth order, block sums ----------------------
__global__ void __launch_bounds__(kScanThreads) tile_count_kernel(const gs_splat *__restrict__ splats,
                                                                  const uint32_t *__restrict__ dval,
                                                                  const SortHeader *__restrict__ hdr,
                                                                  uint32_t *__restrict__ tcount,
                                                                  uint32_t *__restrict__ blk) {
    __shared__ uint32_t scratch[33];
    const uint32_t n = hdr->nvis;
    const uint32_t base = blockIdx.x * kScanItems;
    uint32_t c = 0;
    if (base < n) {
#pragma unroll
        for (int k = 0; k < kScanItems / kScanThreads; ++k) {
            uint32_t i = base + k * kScanThreads + threadIdx.x;
            if (i < n) {
                uint32_t tt = splat_tiles(splats, dval[i]);
                tcount[i] = tt;
                c += tt;
            }
        }
    }
    uint32_t total;
    block_exclusive_scan(c, scratch, &total);
    if (threadIdx.x == 0) blk[blockIdx.x] = total;
}

// --- step 4: duplicate, load-balanced within each block ---------------------
__global__ void __launch_bounds__(kScanThreads) duplicate_kernel(const gs_splat *__restrict__ splats,
                                                                 const uint32_t *__restrict__ dval,
                                                                 const uint32_t *__restrict__ tcount,
                                                                 const uint64_t *__restrict__ blk_off,
                                                                 const SortHeader *__restrict__ hdr,
                                                                 int tiles_x, uint64_t m_cap,
                                                                 uint64_t *__restrict__ keys,
                                                                 uint32_t *__restrict__ vals) {
    __shared__ uint32_t s_off[kScanItems + 1];
    __shared__ uint32_t s_rect[kScanItems];    // x0 | y0 << 16
    __shared__ uint32_t s_w[kScanItems];       // rectangle width in tiles
    __shared__ uint32_t s_depth[kScanItems];
    __shared__ uint32_t s_gid[kScanItems];
    __shared__ uint32_t scratch[33];
    const uint32_t n = hdr->nvis;
    const uint32_t base = blockIdx.x * kScanItems;
    if (base >= n) return;
    uint32_t run = 0;
#pragma unroll
    for (int k = 0; k < kScanItems / kScanThreads; ++k) {
        const uint32_t j = k * kScanThreads + threadIdx.x;
        const uint32_t i = base + j;
        uint32_t tt = 0;
        if (i < n) {
            const uint32_t g = dval[i];
            tt = tcount[i];
            const uint4 w2 = reinterpret_cast<const uint4 *>(splats + g)[2];
            const uint4 w3 = reinterpret_cast<const uint4 *>(splats + g)[3];
            s_rect[j] = w3.x;
            s_w[j] = (w3.y & 0xffffu) - (w3.x & 0xffffu);
            s_depth[j] = w2.y;
            s_gid[j] = g;
        }
        uint32_t total;
        const uint32_t ex = block_exclusive_scan(tt, scratch, &total);
        s_off[j] = run + ex;
        run += total;
    }
    if (threadIdx.x == 0) s_off[kScanItems] = run;
    __syncthreads();
    const uint32_t nloc = min((uint32_t)kScanItems, n - base);
    const uint64_t out0 = blk_off[blockIdx.x];
    for (uint32_t q = threadIdx.x; q < run; q += kScanThreads) {
        // element e with s_off[e] <= q < s_off[e + 1] (skips empty ones)
        uint32_t lo = 0, hi = nloc;  // invariant: s_off[lo] <= q < s_off[hi]
        while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) >> 1;
            if (s_off[mid] <= q) lo = mid; else hi = mid;
        }
        const uint32_t local = q - s_off[lo];
        const uint32_t w = s_w[lo];
        const uint32_t r = s_rect[lo];
        const uint32_t ty = (r >> 16) + local / w;
        const uint32_t tx = (r & 0xffffu) + local % w;
        const uint64_t tile = (uint64_t)ty * (uint64_t)tiles_x + tx;
        const uint64_t dst = out0 + q;
        if (dst < m_cap) {
            keys[dst] = (tile << 32) | s_depth[lo];
            vals[dst] = s_gid[lo];
        }
    }
}

// --- step 6: ranges --------------------------------------------------------
__global__ void ranges_kernel(const uint64_t *__restrict__ keys, const SortHeader *__restrict__ hdr,
                              uint32_t num_tiles, uint2 *__restrict__ ranges) {
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= num_tiles) return;
    const uint32_t n = hdr->m_sort;
    auto lower = [&](uint64_t v) {
        uint32_t lo = 0, hi = n;
        while (lo < hi) {
            uint32_t mid = (lo + hi) >> 1;
            if (keys[mid] < v) lo = mid + 1; else hi = mid;
        }
        return lo;
    };
    const uint32_t s = lower((uint64_t)t << 32);
    const uint32_t e = lower((uint64_t)(t + 1) << 32);
    ranges[t] = s < e ? make_uint2(s, e) : make_uint2(0u, 0u);
}

template <typename K>
cudaError_t radix_sort_pass(const K *kin, const uint32_t *vin, K *kout, uint32_t *vout, const uint32_t *count_ptr,
                            uint32_t cap, int shift, int nbits, uint32_t *hist, uint32_t *dtotal, cudaStream_t st) {
    const uint32_t ntiles = (cap + kRsItems - 1) / kRsItems;
    if (ntiles == 0) return cudaSuccess;
    const uint32_t mask = nbits >= 32 ? 0xffffffffu : ((1u << nbits) - 1u);
    radix_upsweep_kernel<K><<<ntiles, kRsThreads, 0, st>>>(kin, count_ptr, shift, mask, hist, ntiles);
    radix_scan_kernel<<<kRsBins, 1024, 0, st>>>(hist, ntiles, count_ptr, dtotal);
    radix_downsweep_kernel<K><<<ntiles, kRsThreads, 0, st>>>(kin, vin, kout, vout, count_ptr, shift, mask, hist,
                                                              ntiles, dtotal);
    return cudaGetLastError();
}

}  // namespace

uint32_t radix_tiles_for(uint64_t count) { return (uint32_t)((count + kRsItems - 1) / kRsItems); }
uint32_t scan_blocks_for(uint64_t count) { return (uint32_t)((count + kScanItems - 1) / kScanItems); }

int tile_bits_for(uint32_t num_tiles) {
    int b = 0;
    while (b < 32 && (1ull << b) < num_tiles) ++b;
    return b;
}

// Steps 1-3 (through M); returns the first launch error.
cudaError_t launch_sort_front(const gs_splat *splats, int64_t n, const SortWs &ws, uint64_t m_cap, cudaStream_t st) {
    cudaMemsetAsync(ws.hdr, 0, sizeof(SortHeader), st);
    if (n == 0) return cudaGetLastError();
    const uint32_t nblk = scan_blocks_for((uint64_t)n);
    count_visible_kernel<<<nblk, kScanThreads, 0, st>>>(splats, n, ws.blk);
    scan_blocks_kernel<<<1, 1024, 0, st>>>(ws.blk, ws.blk_off, nblk, ws.hdr, 0, 0);
    compact_kernel<<<nblk, kScanThreads, 0, st>>>(splats, n, ws.blk_off, ws.dkey[0], ws.dval[0]);
    // depth sort: 4 passes of 8 bits, ping-pong ends back in buffer 0
    for (int p = 0; p < 4; ++p) {
        cudaError_t e = radix_sort_pass<uint32_t>(ws.dkey[p & 1], ws.dval[p & 1], ws.dkey[(p + 1) & 1],
                                                  ws.dval[(p + 1) & 1], &ws.hdr->nvis, (uint32_t)n, 8 * p, 8,
                                                  ws.hist, ws.dtotal, st);
        if (e != cudaSuccess) return e;
    }
    tile_count_kernel<<<nblk, kScanThreads, 0, st>>>(splats, ws.dval[0], ws.hdr, ws.tcount, ws.blk);
    scan_blocks_kernel<<<1, 1024, 0, st>>>(ws.blk, ws.blk_off, nblk, ws.hdr, 1, m_cap);
    return cudaGetLastError();
}

// Steps 4-6.
cudaError_t launch_sort_back(const gs_splat *splats, int64_t n, const SortWs &ws, uint64_t m_cap, int tiles_x,
                             uint32_t num_tiles, uint64_t *keys, uint32_t *vals, uint32_t *ranges, cudaStream_t st) {
    const int tb = tile_bits_for(num_tiles);
    const int passes = (tb + 7) / 8;
    // duplicate into the buffer that makes the last pass land in keys/vals
    uint64_t *k0 = (passes & 1) ? ws.key_alt : keys;
    uint32_t *v0 = (passes & 1) ? ws.val_alt : vals;
    uint64_t *k1 = (passes & 1) ? keys : ws.key_alt;
    uint32_t *v1 = (passes & 1) ? vals : ws.val_alt;
    if (n > 0) {
        const uint32_t nblk = scan_blocks_for((uint64_t)n);
        duplicate_kernel<<<nblk, kScanThreads, 0, st>>>(splats, ws.dval[0], ws.tcount, ws.blk_off, ws.hdr, tiles_x,
                                                         m_cap, k0, v0);
        for (int p = 0; p < passes; ++p) {
            const int nbits = (tb - 8 * p) < 8 ? (tb - 8 * p) : 8;
            const uint64_t *ki = (p & 1) ? k1 : k0;
            const uint32_t *vi = (p & 1) ? v1 : v0;
            uint64_t *ko = (p & 1) ? k0 : k1;
            uint32_t *vo = (p & 1) ? v0 : v1;
            cudaError_t e = radix_sort_pass<uint64_t>(ki, vi, ko, vo, &ws.hdr->m_sort, (uint32_t)m_cap, 32 + 8 * p,
                                                      nbits, ws.hist, ws.dtotal, st);
            if (e != cudaSuccess) return e;
        }
    }
    ranges_kernel<<<(num_tiles + 255) / 256, 256, 0, st>>>(keys, ws.hdr, num_tiles, reinterpret_cast<uint2 *>(ranges));
    return cudaGetLastError();
}

}  // namespace gs
