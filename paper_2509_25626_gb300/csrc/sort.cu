// Key duplication, radix sort and tile ranges (Section II-B; Algorithm 1's
// "load work range").
//
// The sorted order is that of a stable sort of the 64-bit keys
// (tile << 32 | float_bits(depth)) over instances emitted in (Gaussian id,
// row-major tile) order.  It is reached in fewer passes over less data:
//   1. compact   visible splats, id order kept; FP32 depth bits by id; the
//                digit histograms of the depth sort         (one look-back scan)
//   2. depth     stable LSD radix sort of (depth bits, id) over the visible
//                splats, 4 x 8-bit passes                   (one kernel per pass)
//   3. offsets   exclusive scan of tiles_touched in depth order -> M and each
//                splat's first instance                     (one look-back scan)
//   4. dup       instances in (depth, id, row-major tile) order as 32-bit
//                tile ids + ids, balanced by instance; the tile digit histograms
//   5. tiles     stable LSD radix sort on the ceil(log2 T) tile bits, the last
//                pass writing the full 64-bit keys          (one kernel per pass)
//   6. ranges    per tile, binary search of its first and last key
// Within a tile, step 5 keeps step 4's (depth, id) order, which is exactly
// the tie-broken key order.
//
// Radix passes are single-kernel ("onesweep"): every digit's global total is
// known beforehand (steps 1 and 4 count them), and each block learns the
// count of its digit in all earlier blocks by decoupled look-back: it
// publishes its own count, then walks back over its predecessors' published
// counts until one carries an inclusive prefix.  Blocks take their index from
// an atomic counter in launch order, so a block only waits on blocks that
// are already running; every wait is bounded (1 s of %globaltimer), after
// which the block records a timeout in the header and goes on (results are
// then invalid and gs_sort_status reports GS_ERR_TIMEOUT).  All counts stay
// on the device.
#include "common.cuh"
#include "sort_ws.h"

namespace gs {

namespace {

constexpr int kThreads = 256;
constexpr int kIpt = kSortTileItems / kThreads;  // 16 items per thread
constexpr int kBins = 256;

constexpr uint64_t kFlagAgg = 1ull << 62;        // block aggregate published
constexpr uint64_t kFlagPre = 2ull << 62;        // inclusive prefix published
constexpr uint64_t kValMask = (1ull << 62) - 1;
constexpr uint64_t kWaitLimitNs = 1000000000ull;

enum Counter { kCtrCompact = 0, kCtrDepth = 1, kCtrOffsets = 5, kCtrTiles = 6 };

__device__ __forceinline__ uint32_t splat_word(const gs_splat *s, uint32_t g, int w) {
    return reinterpret_cast<const uint32_t *>(s + g)[w];
}

__device__ __forceinline__ uint64_t ld_relaxed(const uint64_t *p) {
    uint64_t v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_relaxed(uint64_t *p, uint64_t v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Waits (bounded) until *p carries a flag.  On timeout -- or once any wait
// of this call has timed out -- records it and returns an empty inclusive
// prefix so the caller's walk ends: a fault costs at most ~1 s per kernel.
__device__ uint64_t wait_flag(const uint64_t *p, SortHeader *hdr) {
    uint64_t v = ld_relaxed(p);
    if (v >> 62) return v;
    volatile uint32_t *timeout = &hdr->timeout;
    const uint64_t t0 = global_ns();
    for (uint32_t it = 1;; ++it) {
        __nanosleep(32);
        v = ld_relaxed(p);
        if (v >> 62) return v;
        if ((it & 63u) == 0u && (*timeout != 0u || global_ns() - t0 > kWaitLimitNs)) {
            atomicExch(&hdr->timeout, 1u);
            return kFlagPre;
        }
    }
}

// Decoupled look-back over `stride`-spaced words: publishes this block's
// aggregate, sums predecessors back to the first inclusive prefix,
// publishes this block's inclusive prefix; returns the exclusive prefix.
// Predecessors are read kWin at a time (independent loads), so a walk over
// many blocks that have only published aggregates costs few round trips.
template <int kWin>
__device__ uint64_t look_back(uint64_t *state, uint32_t block, uint32_t stride, uint64_t local, SortHeader *hdr) {
    uint64_t *mine = state + (size_t)block * stride;
    if (block == 0) {
        st_relaxed(mine, kFlagPre | local);
        return 0;
    }
    st_relaxed(mine, kFlagAgg | local);
    uint64_t excl = 0;
    int64_t p = (int64_t)block - 1;
    bool found = false;
    while (!found) {
        uint64_t v[kWin];
#pragma unroll
        for (int i = 0; i < kWin; ++i) v[i] = (p - i >= 0) ? ld_relaxed(state + (size_t)(p - i) * stride) : 0ull;
#pragma unroll
        for (int i = 0; i < kWin; ++i) {
            if (!found && p - i >= 0) {
                uint64_t x = v[i];
                if ((x >> 62) == 0u) x = wait_flag(state + (size_t)(p - i) * stride, hdr);
                excl += x & kValMask;
                found = (x >> 62) == 2u;
            }
        }
        p -= kWin;
        if (p < 0) found = true;  // block 0 always holds a prefix; defensive end of the walk
    }
    st_relaxed(mine, kFlagPre | (excl + local));
    return excl;
}

// Adds `count` to bin `d` of a shared histogram once per distinct value in
// the warp (every lane must call; d = ~0u means "nothing to add").
__device__ __forceinline__ void warp_hist_add(uint32_t *hist, uint32_t d) {
    const unsigned peers = __match_any_sync(0xffffffffu, d);
    if (d != 0xffffffffu && (peers & lanemask_lt()) == 0) atomicAdd(&hist[d], (uint32_t)__popc(peers));
}

// Exclusive prefix of `blk` for a scan: publish this block's aggregate, then
// sum every predecessor's aggregate with the whole block (coalesced, one
// round trip per 256 predecessors).  No prefix chain is formed, so blocks
// that all start together (the usual case for these small grids) do not
// wait on each other's walks.  Call with every thread; result in every thread.
__device__ uint64_t prefix_from_aggregates(uint64_t *state, uint32_t blk, uint64_t local, SortHeader *hdr,
                                           uint64_t *scratch /* >= 33 */) {
    if (threadIdx.x == 0) st_relaxed(state + blk, kFlagAgg | local);
    uint64_t sum = 0;
#pragma unroll 4
    for (uint32_t p = threadIdx.x; p < blk; p += blockDim.x) {
        uint64_t v = ld_relaxed(state + p);
        if ((v >> 62) == 0u) v = wait_flag(state + p, hdr);
        sum += v & kValMask;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    const unsigned lane = lane_id(), warp = threadIdx.x >> 5;
    if (lane == 0) scratch[warp] = sum;
    __syncthreads();
    uint64_t tot = 0;
    for (unsigned w = 0; w < blockDim.x / 32; ++w) tot += scratch[w];
    __syncthreads();
    return tot;
}

__device__ __forceinline__ uint32_t dynamic_block(uint32_t *ctr, uint32_t *s_slot) {
    if (threadIdx.x == 0) *s_slot = atomicAdd(ctr, 1u);
    __syncthreads();
    return *s_slot;
}

// Block-wide exclusive scan of 64-bit values (blockDim.x == kThreads).
__device__ __forceinline__ uint64_t block_exclusive_scan64(uint64_t v, uint64_t *scratch, uint64_t *total) {
    const unsigned lane = lane_id(), warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    uint64_t inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint64_t t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= (unsigned)o) inc += t;
    }
    if (lane == 31) scratch[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        uint64_t w = lane < nwarps ? scratch[lane] : 0ull;
        uint64_t wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint64_t t = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= (unsigned)o) wi += t;
        }
        if (lane < nwarps) scratch[lane] = wi - w;
        if (lane == 31) scratch[32] = wi;
    }
    __syncthreads();
    const uint64_t res = scratch[warp] + inc - v;
    *total = scratch[32];
    __syncthreads();
    return res;
}

// --- step 1: compaction -----------------------------------------------------
__global__ void __launch_bounds__(kThreads) compact_kernel(const gs_splat *__restrict__ splats, int64_t n, SortWs ws) {
    __shared__ uint32_t s_hist[kThreads / 32][4][kBins];  // per-warp digit histograms, 32 KB
    __shared__ uint32_t scratch[33];
    __shared__ uint64_t scratch64[33];
    __shared__ uint32_t s_slot;
    for (int i = threadIdx.x; i < (kThreads / 32) * 4 * kBins; i += kThreads) (&s_hist[0][0][0])[i] = 0;
    const uint32_t blk = dynamic_block(&ws.hdr->tile_ctr[kCtrCompact], &s_slot);
    const int64_t base = (int64_t)blk * kSortTileItems + (int64_t)threadIdx.x * kIpt;  // 16 consecutive per thread
    uint32_t depth[kIpt], tiles[kIpt];
#pragma unroll
    for (int k = 0; k < kIpt; ++k) {
        const int64_t i = base + k;
        tiles[k] = i < n ? splat_word(splats, (uint32_t)i, rec::kTiles) : 0u;
        depth[k] = i < n ? splat_word(splats, (uint32_t)i, rec::kDepth) : 0u;
    }
    uint32_t vis = 0;  // bit k: element base + k is visible
#pragma unroll
    for (int k = 0; k < kIpt; ++k) vis |= (tiles[k] != 0u ? 1u : 0u) << k;
    uint32_t total;
    const uint32_t ex = block_exclusive_scan((uint32_t)__popc(vis), scratch, &total);
    const uint64_t excl = prefix_from_aggregates(ws.scan_state[0], blk, total, ws.hdr, scratch64);
    uint32_t pos = (uint32_t)excl + ex;
    const unsigned warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < kIpt; ++k) {
        if ((vis >> k) & 1u) {
            const uint32_t d = depth[k], g = (uint32_t)(base + k);
            ws.dkey[0][pos] = d;  // positive float: uint order = float order
            ws.dval[0][pos] = g;
            ws.depthv[g] = d;
            ++pos;
            atomicAdd(&s_hist[warp][0][d & 0xffu], 1u);
            atomicAdd(&s_hist[warp][1][(d >> 8) & 0xffu], 1u);
        }
        // the two high bytes take few distinct values: aggregate them per warp
        warp_hist_add(s_hist[warp][2], ((vis >> k) & 1u) ? ((depth[k] >> 16) & 0xffu) : 0xffffffffu);
        warp_hist_add(s_hist[warp][3], ((vis >> k) & 1u) ? (depth[k] >> 24) : 0xffffffffu);
    }
    if (blk == gridDim.x - 1 && threadIdx.x == 0) ws.hdr->nvis = (uint32_t)(excl + total);
    __syncthreads();
    for (int i = threadIdx.x; i < 4 * kBins; i += kThreads) {
        uint32_t c = 0;
#pragma unroll
        for (int w = 0; w < kThreads / 32; ++w) c += s_hist[w][i / kBins][i % kBins];
        if (c) atomicAdd(&ws.hist_depth[i], c);
    }
}

// --- steps 2 and 5: one stable LSD radix pass -------------------------------
// kFinal: write the full 64-bit key (tile << 32 | depth bits of the value).
template <bool kFinal>
__global__ void __launch_bounds__(kThreads, 3) onesweep_kernel(const uint32_t *__restrict__ kin,
                                                            const uint32_t *__restrict__ vin,
                                                            uint32_t *__restrict__ kout, uint32_t *__restrict__ vout,
                                                            uint64_t *__restrict__ kout64,
                                                            const uint32_t *__restrict__ depthv,
                                                            const uint32_t *__restrict__ count_ptr, int shift,
                                                            const uint32_t *__restrict__ digit_total,
                                                            uint64_t *__restrict__ state, uint32_t *__restrict__ ctr,
                                                            SortHeader *__restrict__ hdr) {
    __shared__ uint32_t s_keys[kSortTileItems];
    __shared__ uint32_t s_vals[kSortTileItems];
    __shared__ uint32_t s_wcnt[kThreads / 32][kBins];
    __shared__ uint32_t s_base[kBins];
    __shared__ uint32_t s_dstart[kBins];
    __shared__ uint32_t scratch[33];
    __shared__ uint32_t s_slot;

    const uint32_t n = *count_ptr;
    const uint32_t nblocks = (n + kSortTileItems - 1) / kSortTileItems;
    const unsigned t = threadIdx.x, lane = lane_id(), warp = t >> 5;
#pragma unroll
    for (int w = 0; w < kThreads / 32; ++w) s_wcnt[w][t] = 0;
    const uint32_t blk = dynamic_block(ctr, &s_slot);  // contains __syncthreads
    if (blk >= nblocks) return;                        // uniform over the block
    const uint32_t start = blk * kSortTileItems;

    // stable warp-local ranking; warp w owns elements [w*512, w*512 + 512)
    uint32_t key[kIpt], rank[kIpt];
    const unsigned lt = lanemask_lt();
    const uint32_t wbase = start + warp * (kIpt * 32) + lane;
#pragma unroll
    for (int k = 0; k < kIpt; ++k) key[k] = (wbase + k * 32 < n) ? kin[wbase + k * 32] : 0u;
#pragma unroll
    for (int k = 0; k < kIpt; ++k) {
        const bool valid = wbase + k * 32 < n;
        const uint32_t d = valid ? ((key[k] >> shift) & 0xffu) : kBins;
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        uint32_t old = 0;
        if (valid) old = s_wcnt[warp][d];
        __syncwarp();
        if (valid && (peers & lt) == 0) s_wcnt[warp][d] = old + (uint32_t)__popc(peers);
        __syncwarp();
        rank[k] = old + (uint32_t)__popc(peers & lt);
    }
    __syncthreads();
    // digit t: prefix over warps, this block's count, and its start in the block
    uint32_t cnt = 0;
#pragma unroll
    for (int w = 0; w < kThreads / 32; ++w) {
        const uint32_t c = s_wcnt[w][t];
        s_wcnt[w][t] = cnt;
        cnt += c;
    }
    uint32_t tot;
    s_dstart[t] = block_exclusive_scan(cnt, scratch, &tot);
    const uint32_t dbase = block_exclusive_scan(digit_total[t], scratch, &tot);
    const uint64_t excl = look_back<8>(state + t, blk, kBins, cnt, hdr);
    s_base[t] = dbase + (uint32_t)excl;
    __syncthreads();
    uint32_t vals[kIpt];
#pragma unroll
    for (int k = 0; k < kIpt; ++k) vals[k] = (wbase + k * 32 < n) ? vin[wbase + k * 32] : 0u;
#pragma unroll
    for (int k = 0; k < kIpt; ++k) {
        if (wbase + k * 32 < n) {
            const uint32_t d = (key[k] >> shift) & 0xffu;
            const uint32_t pos = s_dstart[d] + s_wcnt[warp][d] + rank[k];
            s_keys[pos] = key[k];
            s_vals[pos] = vals[k];
        }
    }
    __syncthreads();
    const uint32_t cnt_blk = min((uint32_t)kSortTileItems, n - start);
    constexpr int kHalf = kIpt / 2;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        uint32_t gp[kHalf], kk[kHalf], vv[kHalf];
#pragma unroll
        for (int k = 0; k < kHalf; ++k) {
            const uint32_t j = t + (h * kHalf + k) * kThreads;
            gp[k] = 0xffffffffu;
            kk[k] = vv[k] = 0u;
            if (j < cnt_blk) {
                kk[k] = s_keys[j];
                vv[k] = s_vals[j];
                const uint32_t d = (kk[k] >> shift) & 0xffu;
                gp[k] = s_base[d] + (j - s_dstart[d]);
            }
        }
        if (kFinal) {
            uint32_t dv[kHalf];
#pragma unroll
            for (int k = 0; k < kHalf; ++k) dv[k] = gp[k] < n ? depthv[vv[k]] : 0u;  // batched gathers
#pragma unroll
            for (int k = 0; k < kHalf; ++k)
                if (gp[k] < n) {  // false only for idle slots (or inconsistent digit totals)
                    kout64[gp[k]] = ((uint64_t)kk[k] << 32) | dv[k];
                    vout[gp[k]] = vv[k];
                }
        } else {
#pragma unroll
            for (int k = 0; k < kHalf; ++k)
                if (gp[k] < n) {
                    kout[gp[k]] = kk[k];
                    vout[gp[k]] = vv[k];
                }
        }
    }
}

// --- step 3: instance offsets in depth order ---------------------------------
__global__ void __launch_bounds__(kThreads) offsets_kernel(const gs_splat *__restrict__ splats, SortWs ws,
                                                           uint64_t m_cap) {
    __shared__ uint64_t scratch[33];
    __shared__ uint32_t s_slot;
    const uint32_t n = ws.hdr->nvis;
    const uint32_t nblocks = (n + kSortTileItems - 1) / kSortTileItems;
    const uint32_t blk = dynamic_block(&ws.hdr->tile_ctr[kCtrOffsets], &s_slot);
    if (blk >= nblocks) return;
    const uint32_t base = blk * kSortTileItems + threadIdx.x * kIpt;
    uint32_t tt[kIpt];
    uint64_t sum = 0;
#pragma unroll
    for (int k = 0; k < kIpt; ++k) {
        const uint32_t i = base + k;
        tt[k] = i < n ? splat_word(splats, ws.dval[0][i], rec::kTiles) : 0u;
        sum += tt[k];
    }
    uint64_t total;
    const uint64_t ex = block_exclusive_scan64(sum, scratch, &total);
    const uint64_t excl = prefix_from_aggregates(ws.scan_state[1], blk, total, ws.hdr, scratch);
    uint64_t pos = excl + ex;
    const uint64_t ndup = (m_cap + kDupItems - 1) / kDupItems;
#pragma unroll
    for (int k = 0; k < kIpt; ++k) {
        const uint32_t i = base + k;
        if (i < n) {
            ws.offs[i] = (uint32_t)(pos < 0xffffffffull ? pos : 0xffffffffull);
            // duplicate blocks whose first instance falls inside this splat's run
            for (uint64_t b = (pos + kDupItems - 1) / kDupItems; b * kDupItems < pos + tt[k] && b <= ndup; ++b)
                ws.dup_start[b] = i;
        }
        pos += tt[k];
    }
    if (blk == nblocks - 1 && threadIdx.x == 0) {
        const uint64_t m = excl + total;
        ws.hdr->m_total = m;
        ws.hdr->m_sort = (uint32_t)(m < m_cap ? m : m_cap);
        ws.hdr->overflow = m > m_cap ? 1u : 0u;
    }
}

// --- step 4: duplicate, balanced by instance ---------------------------------
__global__ void __launch_bounds__(kThreads) duplicate_kernel(const gs_splat *__restrict__ splats, SortWs ws,
                                                             int tiles_x, int passes, uint32_t *__restrict__ okey,
                                                             uint32_t *__restrict__ oval) {
    __shared__ uint32_t s_off[kDupItems + 2];
    __shared__ uint32_t s_rect[kDupItems + 1];  // x0 | y0 << 16
    __shared__ uint32_t s_w[kDupItems + 1];     // rectangle width in tiles
    __shared__ uint32_t s_gid[kDupItems + 1];
    __shared__ uint32_t s_hist[kMaxTilePasses][kBins];
    const uint32_t m = ws.hdr->m_sort, nvis = ws.hdr->nvis;
    const uint64_t m_total = ws.hdr->m_total;
    const uint32_t q0 = blockIdx.x * kDupItems;
    if (q0 >= m) return;  // uniform
    const uint32_t q1 = min(q0 + (uint32_t)kDupItems, m);
    for (int i = threadIdx.x; i < kMaxTilePasses * kBins; i += kThreads) (&s_hist[0][0])[i] = 0;
    // splats from the one holding q0 to the one holding the next block's first
    // instance (at most kDupItems + 1: every splat has >= 1 instance)
    const uint32_t s_lo = ws.dup_start[blockIdx.x];
    const uint32_t s_hi = ((uint64_t)q1 < m_total && q1 == q0 + (uint32_t)kDupItems) ? ws.dup_start[blockIdx.x + 1]
                                                                                      : nvis - 1;
    const uint32_t plo = s_lo, cnt = min(s_hi - s_lo + 1, (uint32_t)kDupItems + 1);
    for (uint32_t j = threadIdx.x; j < cnt; j += kThreads) {
        const uint32_t p = plo + j;
        const uint32_t g = ws.dval[0][p];
        const uint32_t lo = splat_word(splats, g, rec::kRectLo), hi = splat_word(splats, g, rec::kRectHi);
        s_off[j] = ws.offs[p];
        s_rect[j] = lo;
        s_w[j] = (hi & 0xffffu) - (lo & 0xffffu);
        s_gid[j] = g;
    }
    if (threadIdx.x == 0) {
        const uint32_t p = plo + cnt;
        s_off[cnt] = p < nvis ? ws.offs[p] : (uint32_t)(m_total < 0xffffffffull ? m_total : 0xffffffffull);
    }
    __syncthreads();
#pragma unroll 2
    for (int k = 0; k < kDupItems / kThreads; ++k) {
        const uint32_t q = q0 + (uint32_t)(k * kThreads) + threadIdx.x;
        uint32_t tile = 0xffffffffu;
        if (q < q1) {
            uint32_t lo = 0, hi = cnt;  // s_off[lo] <= q < s_off[hi]
            while (hi - lo > 1) {
                const uint32_t mid = (lo + hi) >> 1;
                if (s_off[mid] <= q) lo = mid; else hi = mid;
            }
            const uint32_t local = q - s_off[lo];
            const uint32_t w = s_w[lo], r = s_rect[lo];
            const uint32_t ty = (r >> 16) + local / w;
            const uint32_t tx = (r & 0xffffu) + local % w;
            tile = ty * (uint32_t)tiles_x + tx;
            okey[q] = tile;
            oval[q] = s_gid[lo];
        }
        for (int p = 0; p < passes; ++p)
            warp_hist_add(s_hist[p], tile == 0xffffffffu ? 0xffffffffu : ((tile >> (8 * p)) & 0xffu));
    }
    __syncthreads();
    for (int i = threadIdx.x; i < passes * kBins; i += kThreads) {
        const uint32_t c = (&s_hist[0][0])[i];
        if (c) atomicAdd(&ws.hist_tile[i], c);
    }
}

// --- step 6: ranges ----------------------------------------------------------
__global__ void ranges_kernel(const uint64_t *__restrict__ keys, const SortHeader *__restrict__ hdr,
                              uint32_t num_tiles, uint2 *__restrict__ ranges) {
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= num_tiles) return;
    const uint32_t n = hdr->m_sort;
    auto lower = [&](uint64_t v) {
        uint32_t lo = 0, hi = n;
        while (lo < hi) {
            const uint32_t mid = lo + (hi - lo) / 2;
            if (keys[mid] < v) lo = mid + 1; else hi = mid;
        }
        return lo;
    };
    const uint32_t s = lower((uint64_t)t << 32);
    const uint32_t e = lower((uint64_t)(t + 1) << 32);
    ranges[t] = s < e ? make_uint2(s, e) : make_uint2(0u, 0u);
}

}  // namespace

// Steps 1-3 (through M).
cudaError_t launch_sort_front(const gs_splat *splats, int64_t n, const SortWs &ws, uint64_t m_cap, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(ws.hdr, 0, ws.zero_bytes, st);
    if (e != cudaSuccess || n == 0) return e;
    const uint32_t nb = (uint32_t)sort_blocks_for((uint64_t)n);
    compact_kernel<<<nb, kThreads, 0, st>>>(splats, n, ws);
    for (int p = 0; p < 4; ++p)
        onesweep_kernel<false><<<nb, kThreads, 0, st>>>(ws.dkey[p & 1], ws.dval[p & 1], ws.dkey[(p + 1) & 1],
                                                         ws.dval[(p + 1) & 1], nullptr, nullptr, &ws.hdr->nvis, 8 * p,
                                                         ws.hist_depth + kBins * p, ws.depth_state[p],
                                                         &ws.hdr->tile_ctr[kCtrDepth + p], ws.hdr);
    offsets_kernel<<<nb, kThreads, 0, st>>>(splats, ws, m_cap);
    return cudaGetLastError();
}

// Steps 4-6.  The tile passes ping-pong between the workspace buffer and the
// caller's key buffer (2 x 32 bits per 64-bit slot) so that the last pass
// reads the workspace and writes the caller's keys and values.
cudaError_t launch_sort_back(const gs_splat *splats, int64_t n, const SortWs &ws, uint64_t m_cap, int tiles_x,
                             uint32_t num_tiles, uint64_t *keys, uint32_t *vals, uint32_t *ranges, cudaStream_t st) {
    if (n > 0 && m_cap > 0) {
        const int passes = tile_passes_of(num_tiles);
        uint32_t *scratch_k = reinterpret_cast<uint32_t *>(keys), *scratch_v = scratch_k + m_cap;
        auto buf_k = [&](int k) { return ((passes - 1 - k) % 2 == 0) ? ws.tkey : scratch_k; };
        auto buf_v = [&](int k) { return ((passes - 1 - k) % 2 == 0) ? ws.tval : scratch_v; };
        const uint32_t nd = (uint32_t)((m_cap + kDupItems - 1) / kDupItems);
        duplicate_kernel<<<nd, kThreads, 0, st>>>(splats, ws, tiles_x, passes, buf_k(0), buf_v(0));
        const uint32_t nb = (uint32_t)sort_blocks_for(m_cap);
        for (int p = 0; p < passes; ++p) {
            if (p == passes - 1)
                onesweep_kernel<true><<<nb, kThreads, 0, st>>>(
                    buf_k(p), buf_v(p), nullptr, vals, keys, ws.depthv, &ws.hdr->m_sort, 8 * p,
                    ws.hist_tile + kBins * p, ws.tile_state[p], &ws.hdr->tile_ctr[kCtrTiles + p], ws.hdr);
            else
                onesweep_kernel<false><<<nb, kThreads, 0, st>>>(
                    buf_k(p), buf_v(p), buf_k(p + 1), buf_v(p + 1), nullptr, nullptr, &ws.hdr->m_sort, 8 * p,
                    ws.hist_tile + kBins * p, ws.tile_state[p], &ws.hdr->tile_ctr[kCtrTiles + p], ws.hdr);
        }
    }
    ranges_kernel<<<(num_tiles + 255) / 256, 256, 0, st>>>(keys, ws.hdr, num_tiles, reinterpret_cast<uint2 *>(ranges));
    return cudaGetLastError();
}

}  // namespace gs
