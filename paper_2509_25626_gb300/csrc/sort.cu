// Key duplication, radix sort and tile ranges (Section II-B; Algorithm 1's
// "load work range").
//
// The sorted order is that of a stable sort of the 64-bit keys
// (tile << 32 | float_bits(depth)) over instances emitted in (Gaussian id,
// row-major tile) order.  It is reached in fewer passes over less data:
//   1. compact   visible splats, id order kept; FP32 depth bits and tile
//                rectangles by id; the digit counts of the depth sort and of
//                the tile sort (the latter from rectangle corners alone)
//                                                           (one look-back scan)
//   2. depth     stable LSD radix sort of (depth bits, id) over the visible
//                splats, 4 x 8-bit passes; the last writes each sorted
//                splat's rectangle beside its id            (one kernel per pass)
//   3. offsets   exclusive scan of tiles_touched in depth order -> M and each
//                splat's first instance                     (one look-back scan)
//   4. dup+tile  instances generated in (depth, id, row-major tile) order,
//                balanced by instance, and ranked at once by the first tile
//                digit; then one radix pass per further digit, the last
//                writing the full 64-bit keys
//   5. ranges    per tile, binary search of its first and last key
// The tile passes sort the byte-aligned key ty << 8k | tx (k bytes hold tx),
// which orders like the row-major id ty * tiles_x + tx; within a tile they
// keep step 4's (depth, id) order, which is exactly the tie-broken key order.
//
// Radix passes are single-kernel ("onesweep"): every digit's global total is
// known beforehand (step 1 counts them), and each block learns the count of
// its digit in all earlier blocks by decoupled look-back: it publishes its
// own count, then walks back over its predecessors' published counts until
// one carries an inclusive prefix.  Blocks take their index from an atomic
// counter in launch order, so a block only waits on blocks that are already
// running; every wait is bounded (1 s of %globaltimer), after which the
// block records a timeout in the header and goes on (results are then
// invalid and gs_sort_status reports GS_ERR_TIMEOUT).  All counts stay on
// the device.
#include "common.cuh"
#include "sort_ws.h"

namespace gs {

namespace {

constexpr int kThreads = 256;
constexpr int kIpt = kSortTileItems / kThreads;  // 16 items per thread
// Threads per block of the radix passes over arrays (4096 elements each).
constexpr int kSweepThreads = 256;  // 512 measured slower
#ifndef GS_DEPTH_THREADS
#define GS_DEPTH_THREADS 256
#endif
constexpr int kDepthThreads = GS_DEPTH_THREADS;  // threads per block of the depth passes
// Predecessors read per round trip of the look-back walks (depth passes,
// tile passes).  Every block's live digits walk at once, so wider windows
// mostly add L2 requests: 4 measured faster than 2, 8, 16 and 32.
constexpr int kDepthWin = 4;
constexpr int kTileWin = 4;
constexpr int kBins = 256;

constexpr uint64_t kFlagAgg = 1ull << 62;        // block aggregate published
constexpr uint64_t kFlagPre = 2ull << 62;        // inclusive prefix published
constexpr uint64_t kValMask = (1ull << 62) - 1;
constexpr uint64_t kWaitLimitNs = 1000000000ull;  // default bound on one wait
constexpr uint32_t kWaitMaxPolls = 1u << 26;       // and on its polls (>= 2 s at >= 32 ns each)

enum Counter { kCtrCompact = 0, kCtrDepth = 1, kCtrOffsets = 5, kCtrTiles = 6 };

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
// The bound is the header's wait_limit_ns (0: 1 s) of %globaltimer, and a
// poll count that ends the wait even if the timer stood still.
__device__ uint64_t wait_flag(const uint64_t *p, SortHeader *hdr) {
    uint64_t v = ld_relaxed(p);
    if (v >> 62) return v;
    volatile uint32_t *timeout = &hdr->timeout;
    const uint64_t limit = hdr->wait_limit_ns ? hdr->wait_limit_ns : kWaitLimitNs;
    const uint64_t t0 = global_ns();
    for (uint32_t it = 1;; ++it) {
        __nanosleep(32);
        v = ld_relaxed(p);
        if (v >> 62) return v;
        if ((it & 63u) == 0u && (*timeout != 0u || global_ns() - t0 > limit || it >= kWaitMaxPolls)) {
            atomicExch(&hdr->timeout, 1u);
            return kFlagPre;
        }
    }
}

// Decoupled look-back over `stride`-spaced words, in two steps so that a
// block can publish its aggregate as soon as it is known and walk later.
// publish_aggregate: block 0 publishes its inclusive prefix at once.
__device__ __forceinline__ void publish_aggregate(uint64_t *state, uint32_t block, uint32_t stride, uint64_t local) {
    st_relaxed(state + (size_t)block * stride, (block == 0 ? kFlagPre : kFlagAgg) | local);
}

// walk_back: sums predecessors back to the first inclusive prefix,
// publishes this block's inclusive prefix and returns the exclusive one.
// Predecessors are read kWin at a time (independent loads): while the
// blocks running together have only published aggregates, the inclusive
// prefixes advance by about kWin blocks per round trip, so the window sets
// the pass's block throughput.
template <int kWin>
__device__ uint64_t walk_back(uint64_t *state, uint32_t block, uint32_t stride, uint64_t local, SortHeader *hdr) {
    if (block == 0) return 0;
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
    st_relaxed(state + (size_t)block * stride, kFlagPre | (excl + local));
    return excl;
}

// The lanes of the warp whose valid 8-bit digit equals this lane's: one
// ballot per bit (VOTE runs on the ALU pipes; MATCH goes through the
// shared-memory pipe that the ranking already keeps busy).  Meaningful for
// valid lanes only.
__device__ __forceinline__ unsigned digit_peers(uint32_t d, bool valid) {
    unsigned m = __ballot_sync(0xffffffffu, valid);
#pragma unroll
    for (int b = 0; b < 8; ++b) {
        const bool bit = (d >> b) & 1u;
        const unsigned v = __ballot_sync(0xffffffffu, bit);
        m &= bit ? v : ~v;
    }
    return m;
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

// --- tile digit counts from rectangles ---------------------------------------
// Adds `mult` (mod 2^32: negative counts subtract) to the digit
// (v >> shift) & 255 of every v in [lo, hi), on a 257-entry difference array
// (count[d] = diff[0] + ... + diff[d]).  Coordinates are < 2^16, so a digit
// at shift 8 never wraps.
__device__ __forceinline__ void add_digit_range(uint32_t *diff, uint32_t lo, uint32_t hi, int shift, uint32_t mult) {
    if (hi <= lo || mult == 0u) return;
    if (shift == 0) {
        const uint32_t len = hi - lo, full = len >> 8, rem = len & 0xffu, a = lo & 0xffu;
        if (full) atomicAdd(&diff[0], full * mult);  // every digit, `full` times
        if (rem) {
            atomicAdd(&diff[a], mult);
            if (a + rem <= (uint32_t)kBins) {
                atomicSub(&diff[a + rem], mult);
            } else {
                atomicAdd(&diff[0], mult);
                atomicSub(&diff[a + rem - kBins], mult);
            }
        }
    } else {
        for (uint32_t v = lo >> shift; v <= ((hi - 1u) >> shift); ++v) {
            const uint32_t v0 = v << shift, v1 = (v + 1u) << shift;
            const uint32_t c = (min(hi, v1) - max(lo, v0)) * mult;
            atomicAdd(&diff[v & 0xffu], c);
            atomicSub(&diff[(v & 0xffu) + 1u], c);
        }
    }
}

// The digit counts of the instances of tiles [x0, x1) x [y0, y1), times mult.
__device__ __noinline__ void add_rect_digits(uint32_t (*diff)[kBins + 1], const TileKeyLayout &l, uint32_t x0,
                                                uint32_t x1, uint32_t y0, uint32_t y1, uint32_t mult) {
    if (x1 <= x0 || y1 <= y0) return;
    for (int b = 0; b < l.x_bytes; ++b) add_digit_range(diff[b], x0, x1, 8 * b, (y1 - y0) * mult);
    for (int b = 0; b < l.y_bytes; ++b) add_digit_range(diff[l.x_bytes + b], y0, y1, 8 * b, (x1 - x0) * mult);
}

// --- step 1: compaction -----------------------------------------------------
__global__ void __launch_bounds__(kThreads, 3) compact_kernel(const gs_splat *__restrict__ splats, int64_t n, SortWs ws,
                                                           TileKeyLayout tl) {
    __shared__ uint32_t s_hist[kThreads / 32][4][kBins];  // per-warp depth digit histograms, 32 KB
    __shared__ uint32_t s_tdiff[kMaxTilePasses][kBins + 1];
    __shared__ uint32_t scratch[33];
    __shared__ uint64_t scratch64[33];
    __shared__ uint32_t s_slot;
    for (int i = threadIdx.x; i < (kThreads / 32) * 4 * kBins; i += kThreads) (&s_hist[0][0][0])[i] = 0;
    for (int i = threadIdx.x; i < kMaxTilePasses * (kBins + 1); i += kThreads) (&s_tdiff[0][0])[i] = 0;
    const uint32_t blk = dynamic_block(&ws.hdr->tile_ctr[kCtrCompact], &s_slot);
    // warp w reads elements [w*512, w*512 + 512) of the block, lane-strided, so
    // every load instruction covers 512 contiguous bytes
    const unsigned lane = lane_id(), warp = threadIdx.x >> 5;
    const int64_t wbase = (int64_t)blk * kSortTileItems + (int64_t)warp * (kIpt * 32) + lane;
    // (depth, tiles, rect lo, rect hi): the dense copy after the n records
    const uint4 *__restrict__ sort_in = reinterpret_cast<const uint4 *>(splats + n);
    uint4 r4[kIpt];
#pragma unroll
    for (int k = 0; k < kIpt; ++k) {
        const int64_t i = wbase + k * 32;
        r4[k] = i < n ? __ldg(sort_in + i) : make_uint4(0u, 0u, 0u, 0u);
    }
    // visible elements in element order: per k a ballot over the warp, then
    // warps in order, then blocks in order
    unsigned bal[kIpt];
    uint32_t wcount = 0;
#pragma unroll
    for (int k = 0; k < kIpt; ++k) {
        bal[k] = __ballot_sync(0xffffffffu, r4[k].y != 0u);
        wcount += (uint32_t)__popc(bal[k]);
    }
    uint32_t total;
    const uint32_t wex = block_exclusive_scan(lane == 0 ? wcount : 0u, scratch, &total);
    const uint32_t wexcl = __shfl_sync(0xffffffffu, wex, 0);  // visible elements of the earlier warps
    const uint64_t excl = prefix_from_aggregates(ws.scan_state[0], blk, total, ws.hdr, scratch64);
    uint32_t pos = (uint32_t)excl + wexcl;
    const unsigned lt = lanemask_lt();
    const bool small_grid = tl.x_bytes == 1 && tl.y_bytes <= 1;
#pragma unroll
    for (int k = 0; k < kIpt; ++k) {
        const uint32_t d = r4[k].x;
        const bool vis = (bal[k] >> lane) & 1u;
        if (vis) {
            const uint32_t g = (uint32_t)(wbase + k * 32);
            const uint32_t q = pos + (uint32_t)__popc(bal[k] & lt);
            ws.dkey[0][q] = d;  // positive float: uint order = float order
            ws.dval[0][q] = g;
            ws.depthv[g] = d;
            ws.rectv[g] = make_uint2(r4[k].z, r4[k].w);
            atomicAdd(&s_hist[warp][0][d & 0xffu], 1u);
            atomicAdd(&s_hist[warp][1][(d >> 8) & 0xffu], 1u);
            atomicAdd(&s_hist[warp][2][(d >> 16) & 0xffu], 1u);
            const uint32_t x0 = r4[k].z & 0xffffu, y0 = r4[k].z >> 16, x1 = r4[k].w & 0xffffu, y1 = r4[k].w >> 16;
            if (small_grid) {  // one byte per coordinate: digit = tx, then ty, no wrap
                atomicAdd(&s_tdiff[0][x0], y1 - y0);
                atomicSub(&s_tdiff[0][x1], y1 - y0);
                if (tl.y_bytes) {
                    atomicAdd(&s_tdiff[1][y0], x1 - x0);
                    atomicSub(&s_tdiff[1][y1], x1 - x0);
                }
            } else {
                add_rect_digits(s_tdiff, tl, x0, x1, y0, y1, 1u);
            }
        }
        pos += (uint32_t)__popc(bal[k]);
        // the high byte takes few distinct values (the exponent range): one
        // atomic per distinct value in the warp
        {
            const uint32_t d3 = vis ? (d >> 24) : 0x100u;
            const unsigned pm = __match_any_sync(0xffffffffu, d3);
            if (vis && (pm & lt) == 0u) atomicAdd(&s_hist[warp][3][d3], (uint32_t)__popc(pm));
        }
    }
    if (blk == gridDim.x - 1 && threadIdx.x == 0) ws.hdr->nvis = (uint32_t)(excl + total);
    __syncthreads();
    for (int i = threadIdx.x; i < 4 * kBins; i += kThreads) {
        uint32_t c = 0;
#pragma unroll
        for (int w = 0; w < kThreads / 32; ++w) c += s_hist[w][i / kBins][i % kBins];
        if (c) atomicAdd(&ws.hist_depth[i], c);
    }
    for (int i = threadIdx.x; i < tl.passes * (kBins + 1); i += kThreads) {
        const uint32_t c = (&s_tdiff[0][0])[i];
        if (c) atomicAdd(&ws.hist_tile[i], c);  // differences add mod 2^32
    }
}

// --- steps 2, 4 and 5: stable LSD radix passes -------------------------------
// The ranking and scatter of one block of up to kSortTileItems elements, by
// the 8-bit digit at `shift`.  Warp w holds elements [w*512, w*512 + 512) of
// the block, lane-strided: key[k] is element w*512 + k*32 + lane.
// digit_total: this thread's digit's count over all blocks.  val(k) gives
// element k's value; it is asked for only after the look-back, so a caller
// that loads values from memory keeps them out of registers while ranking.
// kFinal: write the full 64-bit key (row-major tile id << 32 | depth bits of
// the value), the tile id rebuilt from the byte-aligned key.
// NT threads per block, ITEMS elements per block (ITEMS / NT each).
template <int NT, int ITEMS = kSortTileItems>
struct SweepSmemT {
    uint32_t keys[ITEMS];
    uint32_t vals[ITEMS];
    uint32_t wcnt[NT / 32][kBins];
    uint32_t base[kBins];
    uint32_t scratch[33];
};
using SweepSmem = SweepSmemT<kThreads>;

template <bool kFinal, int NT, int WIN, int ITEMS, bool kRect, typename ValFn>
__device__ __forceinline__ void rank_scatter(SweepSmemT<NT, ITEMS> &sm, const uint32_t (&key)[ITEMS / NT], ValFn val,
                                             uint32_t start, uint32_t n, uint32_t blk, int shift,
                                             uint32_t digit_total, uint64_t *__restrict__ state, SortHeader *hdr,
                                             uint32_t *__restrict__ kout, uint32_t *__restrict__ vout,
                                             uint64_t *__restrict__ kout64, const uint32_t *__restrict__ depthv,
                                             int shift_y, uint32_t tiles_x, const uint2 *__restrict__ rect_in,
                                             uint2 *__restrict__ rect_out) {
    constexpr int IPT = ITEMS / NT;
    const unsigned t = threadIdx.x, lane = lane_id(), warp = t >> 5;
    const bool digit_thread = t < (unsigned)kBins;  // thread t < 256 owns digit t
    const unsigned lt = lanemask_lt();
    const uint32_t wbase = start + warp * (IPT * 32) + lane;
    // stable warp-local ranking (sm.wcnt is zero on entry)
    uint32_t rank2[(IPT + 1) / 2];  // ranks (< 2^16: a warp ranks <= 32 IPT elements), two per register
#pragma unroll
    for (int k = 0; k < (IPT + 1) / 2; ++k) rank2[k] = 0u;
#pragma unroll
    for (int k = 0; k < IPT; ++k) {
        const bool valid = wbase + k * 32 < n;
        const uint32_t d = valid ? ((key[k] >> shift) & 0xffu) : kBins;
        const unsigned peers = digit_peers(d, valid);
        uint32_t old = 0;
        if (valid) old = sm.wcnt[warp][d];
        __syncwarp();
        if (valid && (peers & lt) == 0) sm.wcnt[warp][d] = old + (uint32_t)__popc(peers);
        __syncwarp();
        rank2[k / 2] |= (old + (uint32_t)__popc(peers & lt)) << (16 * (k & 1));
    }
    __syncthreads();
    // digit t: prefix over warps, this block's count, and its start in the block
    uint32_t cnt = 0;
    if (digit_thread) {
#pragma unroll
        for (int w = 0; w < NT / 32; ++w) {
            const uint32_t c = sm.wcnt[w][t];
            sm.wcnt[w][t] = cnt;
            cnt += c;
        }
    }
    // a digit that no element of the whole array carries needs no look-back:
    // every block skips its word, and no element asks for its base
    const bool live = digit_thread && digit_total != 0u;
    if (live) publish_aggregate(state + t, blk, kBins, cnt);
    uint32_t tot;
    const uint32_t dst = block_exclusive_scan(cnt, sm.scratch, &tot);
    const uint32_t dbase = block_exclusive_scan(digit_thread ? digit_total : 0u, sm.scratch, &tot);
    if (digit_thread) {  // fold the digit's start in the block into each warp's prefix
#pragma unroll
        for (int w = 0; w < NT / 32; ++w) sm.wcnt[w][t] += dst;
    }
    uint32_t vals[IPT];
#pragma unroll
    for (int k = 0; k < IPT; ++k) vals[k] = val(k);
    __syncthreads();  // the warp prefixes are complete; val() may read shared memory that the scatter below overwrites
    // block-local scatter before the walk: keys, ranks and values leave the
    // registers, which the walk's window then uses
#pragma unroll
    for (int k = 0; k < IPT; ++k) {
        if (wbase + k * 32 < n) {
            const uint32_t d = (key[k] >> shift) & 0xffu;
            const uint32_t pos = sm.wcnt[warp][d] + ((rank2[k / 2] >> (16 * (k & 1))) & 0xffffu);
            sm.keys[pos] = key[k];
            sm.vals[pos] = vals[k];
        }
    }
    const uint32_t cnt_blk = min((uint32_t)ITEMS, n - start);
    // kFinal: the depth bits of each element's value, gathered in block order
    // before the walk so that the gathers' latency overlaps it
    uint32_t dv[kFinal ? IPT : 1];
    if (kFinal) {
        __syncthreads();
#pragma unroll
        for (int k = 0; k < IPT; ++k) {
            const uint32_t j = t + k * NT;
            dv[k] = j < cnt_blk ? depthv[sm.vals[j]] : 0u;
        }
    }
    // base[d]: global position of the block's first digit-d element, less its
    // position in the block (mod 2^32), so that element j goes to base[d] + j
    if (digit_thread) sm.base[t] = dbase + (live ? (uint32_t)walk_back<WIN>(state + t, blk, kBins, cnt, hdr) : 0u) - dst;
    __syncthreads();
    constexpr int kHalf = IPT / 2;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        uint32_t gp[kHalf], kk[kHalf], vv[kHalf];
#pragma unroll
        for (int k = 0; k < kHalf; ++k) {
            const uint32_t j = t + (h * kHalf + k) * NT;
            gp[k] = 0xffffffffu;
            kk[k] = vv[k] = 0u;
            if (j < cnt_blk) {
                kk[k] = sm.keys[j];
                vv[k] = sm.vals[j];
                const uint32_t d = (kk[k] >> shift) & 0xffu;
                gp[k] = sm.base[d] + j;
            }
        }
        if (kFinal) {
#pragma unroll
            for (int k = 0; k < kHalf; ++k)
                if (gp[k] < n) {  // false only for idle slots (or inconsistent digit totals)
                    const uint32_t tile = (kk[k] >> shift_y) * tiles_x + (kk[k] & ((1u << shift_y) - 1u));
                    kout64[gp[k]] = ((uint64_t)tile << 32) | dv[kFinal ? h * kHalf + k : 0];
                    vout[gp[k]] = vv[k];
                }
        } else if (kRect) {  // each value's rectangle instead of its key
            uint2 rc[kHalf];
#pragma unroll
            for (int k = 0; k < kHalf; ++k) rc[k] = gp[k] < n ? rect_in[vv[k]] : make_uint2(0u, 0u);
#pragma unroll
            for (int k = 0; k < kHalf; ++k)
                if (gp[k] < n) {
                    rect_out[gp[k]] = rc[k];
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

// One pass over (key, value) arrays in device memory, ITEMS elements per
// block of NT threads.  diff_hist: the digit totals are given as a
// difference array (the tile passes).
template <bool kFinal, int NT, int WIN, int ITEMS, bool kRect = false>
__global__ void __launch_bounds__(NT, ITEMS / NT <= 8 ? 4 : (NT >= 1024 ? 1 : (NT >= 512 ? 2 : 3))) onesweep_kernel(const uint32_t *__restrict__ kin,
                                                            const uint32_t *__restrict__ vin,
                                                            uint32_t *__restrict__ kout, uint32_t *__restrict__ vout,
                                                            uint64_t *__restrict__ kout64,
                                                            const uint32_t *__restrict__ depthv,
                                                            const uint32_t *__restrict__ count_ptr, int shift,
                                                            const uint32_t *__restrict__ digit_total, bool diff_hist,
                                                            uint64_t *__restrict__ state, uint32_t *__restrict__ ctr,
                                                            SortHeader *__restrict__ hdr, int shift_y,
                                                            uint32_t tiles_x, const uint2 *__restrict__ rect_in = nullptr,
                                                            uint2 *__restrict__ rect_out = nullptr) {
    constexpr int IPT = ITEMS / NT;
    extern __shared__ __align__(16) unsigned char s_dyn[];  // SweepSmemT<NT, ITEMS>, may exceed 48 KB
    SweepSmemT<NT, ITEMS> &sm = *reinterpret_cast<SweepSmemT<NT, ITEMS> *>(s_dyn);
    __shared__ uint32_t s_slot;
    const uint32_t n = *count_ptr;
    const uint32_t nblocks = (n + ITEMS - 1) / ITEMS;
    const unsigned t = threadIdx.x, lane = lane_id(), warp = t >> 5;
    for (int i = (int)t; i < (NT / 32) * kBins; i += NT) (&sm.wcnt[0][0])[i] = 0;
    const uint32_t blk = dynamic_block(ctr, &s_slot);  // contains __syncthreads
    if (blk >= nblocks) return;                        // uniform over the block
    const uint32_t start = blk * ITEMS;
    const uint32_t wbase = start + warp * (IPT * 32) + lane;
    uint32_t key[IPT];
#pragma unroll
    for (int k = 0; k < IPT; ++k) key[k] = (wbase + k * 32 < n) ? kin[wbase + k * 32] : 0u;
    uint32_t dt = t < (unsigned)kBins ? digit_total[t] : 0u;
    if (diff_hist) {  // uniform
        uint32_t tot;
        dt += block_exclusive_scan(dt, sm.scratch, &tot);
    }
    auto val = [&](int k) { return (wbase + k * 32 < n) ? vin[wbase + k * 32] : 0u; };
    rank_scatter<kFinal, NT, WIN, ITEMS, kRect>(sm, key, val, start, n, blk, shift, dt, state, hdr, kout, vout, kout64,
                                              depthv, shift_y, tiles_x, rect_in, rect_out);
}

// --- step 3: instance offsets in depth order -----------------------------------
// Also, if the instances overflow the caller's capacity, takes the dropped
// ones (global index >= m_cap) out of the tile digit counts, so that the
// counts match the instances the tile passes sort.
__global__ void __launch_bounds__(kThreads, 3) offsets_kernel(SortWs ws, uint64_t m_cap, TileKeyLayout tl) {
    __shared__ uint64_t scratch[33];
    __shared__ uint32_t s_slot;
    const uint32_t n = ws.hdr->nvis;
    const uint32_t nblocks = (n + kSortTileItems - 1) / kSortTileItems;
    const uint32_t blk = dynamic_block(&ws.hdr->tile_ctr[kCtrOffsets], &s_slot);
    if (blk >= nblocks) return;
    // warp w holds splats [w*512, w*512 + 512) of the block, lane-strided
    // (coalesced reads of the depth-sorted ids); element order is (k, lane)
    const unsigned lane = lane_id(), warp = threadIdx.x >> 5;
    const uint32_t wbase = blk * kSortTileItems + warp * (kIpt * 32) + lane;
    uint32_t tt[kIpt];
#pragma unroll
    for (int k = 0; k < kIpt; ++k) {
        const uint32_t i = wbase + k * 32;
        const uint2 rc = i < n ? ws.srect[i] : make_uint2(0u, 0u);
        tt[k] = ((rc.y & 0xffffu) - (rc.x & 0xffffu)) * ((rc.y >> 16) - (rc.x >> 16));
    }
    // per k: this lane's exclusive prefix within the warp's 32 elements, and
    // the warp's running total before k
    uint64_t lane_ex[kIpt];
    uint64_t wsum = 0;
#pragma unroll
    for (int k = 0; k < kIpt; ++k) {
        uint64_t inc = tt[k];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint64_t x = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= (unsigned)o) inc += x;
        }
        lane_ex[k] = wsum + inc - tt[k];
        wsum += __shfl_sync(0xffffffffu, inc, 31);
    }
    uint64_t total;
    const uint64_t wex = block_exclusive_scan64(lane == 0 ? wsum : 0ull, scratch, &total);
    const uint64_t wexcl = __shfl_sync(0xffffffffu, wex, 0);  // instances of the earlier warps
    const uint64_t excl = prefix_from_aggregates(ws.scan_state[1], blk, total, ws.hdr, scratch);
    const uint64_t nsweep = (m_cap + kSortTileItems - 1) / kSortTileItems;
#pragma unroll
    for (int k = 0; k < kIpt; ++k) {
        const uint32_t i = wbase + k * 32;
        const uint64_t pos = excl + wexcl + lane_ex[k];
        if (i < n) {
            ws.offs[i] = (uint32_t)(pos < 0xffffffffull ? pos : 0xffffffffull);
            // tile-pass blocks whose first instance falls inside this splat's run
            for (uint64_t b = (pos + kSortTileItems - 1) / kSortTileItems;
                 b * kSortTileItems < pos + tt[k] && b <= nsweep; ++b)
                ws.dup_start[b] = i;
            if (pos + tt[k] > m_cap) {  // overflow: uncount the dropped instances
                const uint2 rc = ws.srect[i];
                const uint32_t x0 = rc.x & 0xffffu, y0 = rc.x >> 16, x1 = rc.y & 0xffffu, y1 = rc.y >> 16;
                const uint32_t kept = pos >= m_cap ? 0u : (uint32_t)(m_cap - pos);
                const uint32_t w = x1 - x0, rows = kept / w, part = kept % w;
                uint32_t(*diff)[kBins + 1] = reinterpret_cast<uint32_t(*)[kBins + 1]>(ws.hist_tile);
                add_rect_digits(diff, tl, x0, x1, y0 + rows + 1u, y1, 0xffffffffu);        // whole rows
                add_rect_digits(diff, tl, x0 + part, x1, y0 + rows, y0 + rows + 1u, 0xffffffffu);  // a partial row
            }
        }
    }
    if (blk == nblocks - 1 && threadIdx.x == 0) {
        const uint64_t m = excl + total;
        ws.hdr->m_total = m;
        ws.hdr->m_sort = (uint32_t)(m < m_cap ? m : m_cap);
        ws.hdr->overflow = m > m_cap ? 1u : 0u;
    }
}

// --- step 4 fused with the first tile pass ------------------------------------
// Block b generates instances [b * 4096, b * 4096 + 4096) in (depth, id,
// row-major tile) order -- each warp finds its instances' splats by a
// running max over the splat starts, not by a search -- and ranks them by
// the low byte of tx straight away, so the instances are written once,
// already partitioned.
struct GenSmem {
    uint32_t off[kSortTileItems + 2];   // first instance of each splat of the block
    uint32_t rect[kSortTileItems + 1];  // x0 | y0 << 16
    uint32_t gid[kSortTileItems + 1];
    uint16_t w[kSortTileItems + 2];     // rectangle width in tiles (< 2^16)
    uint16_t mark[kSortTileItems];      // block-local splat starting at each instance, else 0
};

template <bool kFinal>
__global__ void __launch_bounds__(kThreads, 3) dup_sweep_kernel(SortWs ws, TileKeyLayout tl, uint32_t tiles_x,
                                                             uint32_t *__restrict__ kout, uint32_t *__restrict__ vout,
                                                             uint64_t *__restrict__ kout64) {
    __shared__ union {
        GenSmem gen;
        SweepSmem sweep;
    } sm;
    __shared__ uint32_t s_slot;
    __shared__ uint32_t s_scan[33];
    __shared__ uint32_t s_wmax[kThreads / 32];
    const uint32_t m = ws.hdr->m_sort, nvis = ws.hdr->nvis;
    const uint64_t m_total = ws.hdr->m_total;
    const uint32_t nblocks = (m + kSortTileItems - 1) / kSortTileItems;
    const unsigned t = threadIdx.x, lane = lane_id(), warp = t >> 5;
    const uint32_t blk = dynamic_block(&ws.hdr->tile_ctr[kCtrTiles], &s_slot);  // contains __syncthreads
    if (blk >= nblocks) return;  // uniform
    const uint32_t q0 = blk * kSortTileItems;
    const uint32_t q1 = min(q0 + (uint32_t)kSortTileItems, m);
    // splats from the one holding q0 to the one holding the next block's first
    // instance (at most kSortTileItems + 1: every splat has >= 1 instance)
    const uint32_t s_lo = ws.dup_start[blk];
    const uint32_t s_hi = ((uint64_t)q1 < m_total && q1 == q0 + (uint32_t)kSortTileItems) ? ws.dup_start[blk + 1]
                                                                                           : nvis - 1;
    const uint32_t cnt = min(s_hi - s_lo + 1, (uint32_t)kSortTileItems + 1);
    for (uint32_t p = t; p < kSortTileItems; p += kThreads) sm.gen.mark[p] = 0;
    for (uint32_t j = t; j < cnt; j += kThreads) {
        const uint32_t p = s_lo + j;
        const uint32_t g = ws.dval[0][p];
        const uint2 rc = ws.srect[p];
        sm.gen.off[j] = ws.offs[p];
        sm.gen.rect[j] = rc.x;
        sm.gen.w[j] = (uint16_t)((rc.y & 0xffffu) - (rc.x & 0xffffu));
        sm.gen.gid[j] = g;
    }
    __syncthreads();
    for (uint32_t j = 1 + t; j < cnt; j += kThreads) {
        const uint32_t o = sm.gen.off[j];
        if (o >= q0 && o - q0 < (uint32_t)kSortTileItems) sm.gen.mark[o - q0] = (uint16_t)j;
    }
    __syncthreads();
    // splat of each position = running max of the marks, in the warp layout
    // (position w*512 + k*32 + lane): a warp scan per k, carried across k,
    // then across warps
    const uint32_t pw = warp * (kIpt * 32) + lane;  // this thread's first position
    uint32_t js[kIpt];
    uint32_t carry = 0;
#pragma unroll
    for (int k = 0; k < kIpt; ++k) {
        uint32_t v = sm.gen.mark[pw + k * 32];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t x = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= (unsigned)o) v = max(v, x);
        }
        v = max(v, carry);
        carry = __shfl_sync(0xffffffffu, v, 31);
        js[k] = v;
    }
    if (lane == 0) s_wmax[warp] = carry;
    __syncthreads();
    uint32_t prev = 0;
    for (unsigned w = 0; w < warp; ++w) prev = max(prev, s_wmax[w]);
    uint32_t key[kIpt], val[kIpt];
#pragma unroll
    for (int k = 0; k < kIpt; ++k) {
        const uint32_t p = pw + k * 32;
        key[k] = val[k] = 0u;
        if (q0 + p < q1) {
            const uint32_t j = max(js[k], prev);
            const uint32_t local = q0 + p - sm.gen.off[j];
            const uint32_t w = sm.gen.w[j], r = sm.gen.rect[j];
            // row = local / w by a float estimate and an exact integer correction
            uint32_t row = (uint32_t)((float)local * __frcp_rn((float)w));
            int64_t rem = (int64_t)local - (int64_t)row * w;
            while (rem < 0) { --row; rem += w; }
            while (rem >= (int64_t)w) { ++row; rem -= w; }
            key[k] = (((r >> 16) + row) << tl.shift_y) | ((r & 0xffffu) + (uint32_t)rem);
            val[k] = sm.gen.gid[j];
        }
    }
    // pass-0 digit counts from their difference array
    uint32_t tot;
    const uint32_t diff = ws.hist_tile[t];
    const uint32_t digit_total = block_exclusive_scan(diff, s_scan, &tot) + diff;  // ends with a barrier:
    // generation smem is dead.  Park the values where the sweep's value
    // array lives (read back after its look-back) and free the registers.
#pragma unroll
    for (int k = 0; k < kIpt; ++k) sm.sweep.vals[pw + k * 32] = val[k];
#pragma unroll
    for (int w = 0; w < kThreads / 32; ++w) sm.sweep.wcnt[w][t] = 0;
    __syncthreads();
    rank_scatter<kFinal, kThreads, kTileWin, kSortTileItems, false>(
        sm.sweep, key, [&](int k) { return sm.sweep.vals[pw + k * 32]; }, q0, m, blk, 0, digit_total,
        ws.tile_state[0], ws.hdr, kout, vout, kout64, ws.depthv, tl.shift_y, tiles_x, nullptr, nullptr);
}

// --- step 6: ranges ----------------------------------------------------------
// One warp per tile: each lower-bound search probes 32 keys at once and
// keeps the part of the range between the last probe below the target and
// the first at or above it, so a search over M keys takes ~log33(M) + 1
// dependent round trips (5 at M = 9.4e6) instead of log2(M).
__device__ __forceinline__ uint32_t warp_lower_bound(const uint64_t *__restrict__ keys, uint32_t n, uint64_t v,
                                                     unsigned lane) {
    uint32_t lo = 0, hi = n;  // keys[< lo] < v <= keys[>= hi]
    while (hi - lo > 32u) {
        const uint32_t len = hi - lo;
        const uint32_t p = lo + (uint32_t)(((uint64_t)(lane + 1u) * len) / 33u);  // strictly increasing in lane
        const unsigned below = __ballot_sync(0xffffffffu, keys[p] < v);
        const uint32_t c = (uint32_t)__popc(below);  // probes 0 .. c-1 are below v
        const uint32_t plo = __shfl_sync(0xffffffffu, p, c > 0u ? c - 1u : 0u);
        const uint32_t phi = __shfl_sync(0xffffffffu, p, c < 32u ? c : 31u);
        if (c > 0u) lo = plo + 1u;
        if (c < 32u) hi = phi;
    }
    const bool below = lo + lane < hi && keys[lo + lane] < v;
    return lo + (uint32_t)__popc(__ballot_sync(0xffffffffu, below));
}

__global__ void __launch_bounds__(256) ranges_kernel(const uint64_t *__restrict__ keys,
                                                     const SortHeader *__restrict__ hdr, uint32_t num_tiles,
                                                     uint2 *__restrict__ ranges) {
    const uint32_t t = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;  // warp-uniform
    if (t >= num_tiles) return;
    const unsigned lane = lane_id();
    const uint32_t n = hdr->m_sort;
    const uint32_t s = warp_lower_bound(keys, n, (uint64_t)t << 32, lane);
    const uint32_t e = warp_lower_bound(keys, n, (uint64_t)(t + 1) << 32, lane);
    if (lane == 0) ranges[t] = s < e ? make_uint2(s, e) : make_uint2(0u, 0u);
}

// The failure-detection check: one look-back walk of block 1 whose only
// predecessor (block 0) never publishes, as when a block stalls or dies.
// The walk's bounded wait must give up after wait_limit_ns, record the
// timeout in the header and end the walk.  One thread; the state words are
// zeroed by the host first.
__global__ void lookback_probe_kernel(uint64_t *state, SortHeader *hdr, uint64_t limit_ns) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    hdr->wait_limit_ns = limit_ns;
    walk_back<kTileWin>(state, 1u, 1u, 1ull, hdr);
}

// Launches one radix pass with its shared memory as dynamic shared memory
// (the larger block shapes need more than the 48 KB of static shared
// memory); the opt-in size is set once per instantiation.
template <bool kFinal, int NT, int WIN, int ITEMS, bool kRect = false, typename... Args>
cudaError_t launch_onesweep(uint32_t grid, cudaStream_t st, Args... args) {
    constexpr size_t smem = sizeof(SweepSmemT<NT, ITEMS>);
    static cudaError_t attr = cudaFuncSetAttribute(onesweep_kernel<kFinal, NT, WIN, ITEMS, kRect>,
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (attr != cudaSuccess) return attr;
    onesweep_kernel<kFinal, NT, WIN, ITEMS, kRect><<<grid, NT, smem, st>>>(args...);
    return cudaSuccess;
}

}  // namespace

// Runs lookback_probe_kernel on a zeroed header and two state words of `ws`.
cudaError_t launch_lookback_probe(const SortWs &ws, uint64_t limit_ns, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(ws.hdr, 0, sizeof(SortHeader), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(ws.scan_state[0], 0, 2 * sizeof(uint64_t), st);
    if (e != cudaSuccess) return e;
    lookback_probe_kernel<<<1, 32, 0, st>>>(ws.scan_state[0], ws.hdr, limit_ns);
    return cudaGetLastError();
}

// Steps 1-3 (through M).
cudaError_t launch_sort_front(const gs_splat *splats, int64_t n, const SortWs &ws, uint64_t m_cap, int tiles_x,
                              uint32_t num_tiles, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(ws.hdr, 0, ws.zero_bytes, st);
    if (e != cudaSuccess || n == 0) return e;
    const TileKeyLayout tl = tile_key_layout((uint32_t)tiles_x, num_tiles / (uint32_t)tiles_x);
    const uint32_t nb = (uint32_t)sort_blocks_for((uint64_t)n);
    compact_kernel<<<nb, kThreads, 0, st>>>(splats, n, ws, tl);
    const uint32_t nbd = (uint32_t)depth_blocks_for((uint64_t)n);
    // the last pass writes each sorted splat's rectangle in place of its key
    // (no later step reads the sorted depth bits), so that the offsets and
    // the duplication read rectangles densely instead of gathering them by id
    for (int p = 0; p < 3 && e == cudaSuccess; ++p)
        e = launch_onesweep<false, kDepthThreads, kDepthWin, kDepthItems>(
            nbd, st, (const uint32_t *)ws.dkey[p & 1], (const uint32_t *)ws.dval[p & 1], ws.dkey[(p + 1) & 1],
            ws.dval[(p + 1) & 1], (uint64_t *)nullptr, (const uint32_t *)nullptr, (const uint32_t *)&ws.hdr->nvis,
            8 * p, (const uint32_t *)(ws.hist_depth + kBins * p), false, ws.depth_state[p],
            &ws.hdr->tile_ctr[kCtrDepth + p], ws.hdr, 0, 0u, (const uint2 *)nullptr, (uint2 *)nullptr);
    if (e == cudaSuccess)
        e = launch_onesweep<false, kDepthThreads, kDepthWin, kDepthItems, true>(
            nbd, st, (const uint32_t *)ws.dkey[1], (const uint32_t *)ws.dval[1], (uint32_t *)nullptr, ws.dval[0],
            (uint64_t *)nullptr, (const uint32_t *)nullptr, (const uint32_t *)&ws.hdr->nvis, 24,
            (const uint32_t *)(ws.hist_depth + kBins * 3), false, ws.depth_state[3], &ws.hdr->tile_ctr[kCtrDepth + 3],
            ws.hdr, 0, 0u, (const uint2 *)ws.rectv, ws.srect);
    if (e != cudaSuccess) return e;
    offsets_kernel<<<nb, kThreads, 0, st>>>(ws, m_cap, tl);
    return cudaGetLastError();
}

// Steps 4-6.  The tile passes ping-pong between the workspace buffer and the
// caller's key buffer (2 x 32 bits per 64-bit slot) so that the last pass
// reads the workspace and writes the caller's keys and values.
cudaError_t launch_sort_back(const gs_splat *splats, int64_t n, const SortWs &ws, uint64_t m_cap, int tiles_x,
                             uint32_t num_tiles, uint64_t *keys, uint32_t *vals, uint32_t *ranges, cudaStream_t st) {
    (void)splats;
    if (n > 0 && m_cap > 0) {
        const TileKeyLayout tl = tile_key_layout((uint32_t)tiles_x, num_tiles / (uint32_t)tiles_x);
        const int passes = tl.passes;
        uint32_t *scratch_k = reinterpret_cast<uint32_t *>(keys), *scratch_v = scratch_k + m_cap;
        auto buf_k = [&](int k) { return ((passes - 1 - k) % 2 == 0) ? ws.tkey : scratch_k; };
        auto buf_v = [&](int k) { return ((passes - 1 - k) % 2 == 0) ? ws.tval : scratch_v; };
        const uint32_t nb = (uint32_t)sort_blocks_for(m_cap);
        const uint32_t nbt = (uint32_t)tile_pass_blocks_for(m_cap);
        const uint32_t tx = (uint32_t)tiles_x;
        if (passes == 1)
            dup_sweep_kernel<true><<<nb, kThreads, 0, st>>>(ws, tl, tx, nullptr, vals, keys);
        else
            dup_sweep_kernel<false><<<nb, kThreads, 0, st>>>(ws, tl, tx, buf_k(1), buf_v(1), nullptr);
        for (int p = 1; p < passes; ++p) {
            const uint32_t *hist = ws.hist_tile + (kBins + 1) * p;
            cudaError_t e;
            if (p == passes - 1)
                e = launch_onesweep<true, kSweepThreads, kTileWin, kTilePassItems>(
                    nbt, st, (const uint32_t *)buf_k(p), (const uint32_t *)buf_v(p), (uint32_t *)nullptr, vals, keys,
                    (const uint32_t *)ws.depthv, (const uint32_t *)&ws.hdr->m_sort, 8 * p, hist, true,
                    ws.tile_state[p], &ws.hdr->tile_ctr[kCtrTiles + p], ws.hdr, tl.shift_y, tx,
                    (const uint2 *)nullptr, (uint2 *)nullptr);
            else
                e = launch_onesweep<false, kSweepThreads, kTileWin, kTilePassItems>(
                    nbt, st, (const uint32_t *)buf_k(p), (const uint32_t *)buf_v(p), buf_k(p + 1), buf_v(p + 1),
                    (uint64_t *)nullptr, (const uint32_t *)nullptr, (const uint32_t *)&ws.hdr->m_sort, 8 * p, hist,
                    true, ws.tile_state[p], &ws.hdr->tile_ctr[kCtrTiles + p], ws.hdr, tl.shift_y, tx,
                    (const uint2 *)nullptr, (uint2 *)nullptr);
            if (e != cudaSuccess) return e;
        }
    }
    ranges_kernel<<<(unsigned)(((uint64_t)num_tiles * 32 + 255) / 256), 256, 0, st>>>(
        keys, ws.hdr, num_tiles, reinterpret_cast<uint2 *>(ranges));
    return cudaGetLastError();
}

}  // namespace gs
