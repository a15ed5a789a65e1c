// Layout of the caller-provided gs_sort workspace.
#pragma once

#include <cstddef>
#include <cstdint>

namespace gs {

constexpr int kSortTileItems = 4096;   // elements per block in the look-back scans and tile radix passes
#ifndef GS_DEPTH_ITEMS
#define GS_DEPTH_ITEMS 4096
#endif
constexpr int kDepthItems = GS_DEPTH_ITEMS;  // elements per block in the depth radix passes
constexpr int kTilePassItems = 4096;   // elements per block in the tile passes after the first (2048 measured slower)
constexpr int kMaxTilePasses = 4;      // 8-bit digits of a 32-bit tile id

// Device-side counters of one gs_sort call (first 256 bytes of the workspace).
struct SortHeader {
    uint64_t m_total;      // instances the visible splats produce (may exceed the capacity)
    uint32_t nvis;         // visible splats (tiles_touched > 0)
    uint32_t m_sort;       // min(m_total, m_cap): instances actually written and sorted
    uint32_t overflow;     // 1 if m_total > m_cap
    uint32_t timeout;      // 1 if a bounded look-back wait gave up (results invalid)
    uint32_t tile_ctr[10]; // dynamic block-id counters, one per look-back kernel
    uint64_t wait_limit_ns;  // bound on one look-back wait; 0 = the default (1 s)
    uint32_t reserved[46];
};
static_assert(sizeof(SortHeader) == 256, "header is 256 bytes");

struct SortWs {
    SortHeader *hdr;
    uint64_t *scan_state[2];            // look-back flags of the two scans, [blocks(n)]
    uint64_t *depth_state[4];           // per pass, [depth blocks(n)][256]
    uint64_t *tile_state[kMaxTilePasses];  // per pass, [blocks(m_cap)][256]
    uint32_t *hist_depth;               // [4][256] digit totals
    uint32_t *hist_tile;                // [kMaxTilePasses][257] digit counts as difference arrays
    size_t zero_bytes;                  // bytes from hdr that must be zero at the start of a call
    uint32_t *dkey[2], *dval[2];        // depth sort ping-pong, [n]
    uint32_t *depthv;                   // FP32 depth bits by Gaussian id, [n]
    uint2 *rectv;                       // tile rectangle (lo, hi words) by Gaussian id, [n]
    uint2 *srect;                       // tile rectangle of each depth-sorted splat, [n]
    uint32_t *offs;                     // first instance of each depth-sorted splat, [n]
    uint32_t *dup_start;                // depth-sorted splat holding each tile-pass block's first instance
    uint32_t *tkey, *tval;              // tile sort buffer, [m_cap] each
};

constexpr uint64_t sort_blocks_for(uint64_t count) { return (count + kSortTileItems - 1) / kSortTileItems; }
constexpr uint64_t depth_blocks_for(uint64_t count) { return (count + kDepthItems - 1) / kDepthItems; }
constexpr uint64_t tile_pass_blocks_for(uint64_t count) { return (count + kTilePassItems - 1) / kTilePassItems; }

constexpr int tile_bits_of(uint64_t num_tiles) {
    int b = 0;
    while (b < 32 && (1ull << b) < num_tiles) ++b;
    return b;
}

constexpr int tile_passes_of(uint64_t num_tiles) {
    const int p = (tile_bits_of(num_tiles) + 7) / 8;
    return p < 1 ? 1 : p;
}

// The tile sort orders instances by (ty, tx) through the byte-aligned key
// ty << shift_y | tx (shift_y = 8 x_bytes), so that each radix digit is a
// byte of tx or of ty alone.  A splat's instances then cover a whole range of
// tx in each of its rows, and a whole range of ty: the digit counts of the
// whole rectangle follow from its corners (no per-instance counting).  The
// final pass turns the key back into the row-major tile id ty * tiles_x + tx,
// which orders the same way.
struct TileKeyLayout {
    int x_bytes, y_bytes, passes, shift_y;
};

inline TileKeyLayout tile_key_layout(uint32_t tiles_x, uint32_t tiles_y) {
    auto bytes_for = [](uint32_t count) {  // bytes of the largest coordinate, count - 1
        int b = 0;
        while (b < 4 && count > 1u && ((count - 1u) >> (8 * b)) != 0u) ++b;
        return b;
    };
    TileKeyLayout l;
    l.x_bytes = bytes_for(tiles_x);
    if (l.x_bytes < 1) l.x_bytes = 1;
    l.y_bytes = bytes_for(tiles_y);
    l.passes = l.x_bytes + l.y_bytes;
    l.shift_y = 8 * l.x_bytes;
    return l;
}

// Tile passes the workspace is sized for: the byte-aligned key needs at most
// one pass more than the packed tile id.
constexpr int tile_passes_bound(uint64_t num_tiles) {
    const int p = tile_passes_of(num_tiles) + 1;
    return p < kMaxTilePasses ? p : kMaxTilePasses;
}

// Byte offsets of the workspace regions (256-byte aligned, in this order);
// a constant expression, so that a fixed-size workspace can be checked
// against it at compile time.  kNone marks a tile pass the grid never runs.
struct SortWsOffsets {
    static constexpr size_t kNone = ~(size_t)0;
    size_t hdr = 0, scan_state[2] = {}, depth_state[4] = {}, tile_state[kMaxTilePasses] = {}, hist_depth = 0,
           hist_tile = 0, zero_bytes = 0, dkey[2] = {}, dval[2] = {}, depthv = 0, rectv = 0, srect = 0, offs = 0,
           dup_start = 0, tkey = 0, tval = 0, total = 0;
};

constexpr SortWsOffsets sort_ws_offsets(int64_t n, int64_t m_cap, uint64_t num_tiles) {
    SortWsOffsets o;
    size_t off = 0;
    auto take = [&off](size_t bytes) {
        const size_t at = off;
        off += (bytes + 255) & ~(size_t)255;
        return at;
    };
    const uint64_t nn = (uint64_t)(n > 0 ? n : 0), mc = (uint64_t)(m_cap > 0 ? m_cap : 0);
    const uint64_t bn = sort_blocks_for(nn) + 1, bm = sort_blocks_for(mc) + 1, bd = depth_blocks_for(nn) + 1;
    const uint64_t bt = tile_pass_blocks_for(mc) + 1;
    const int passes = tile_passes_bound(num_tiles);
    o.hdr = take(256);  // sizeof(SortHeader)
    for (int i = 0; i < 2; ++i) o.scan_state[i] = take(8 * bn);
    for (int i = 0; i < 4; ++i) o.depth_state[i] = take(8 * 256 * bd);
    for (int i = 0; i < kMaxTilePasses; ++i)  // pass 0 (fused with duplication) uses 4096-element blocks
        o.tile_state[i] = i < passes ? take(8 * 256 * (i == 0 ? bm : bt)) : SortWsOffsets::kNone;
    o.hist_depth = take(4 * 4 * 256);
    o.hist_tile = take(4 * kMaxTilePasses * 257);
    o.zero_bytes = off;
    for (int i = 0; i < 2; ++i) {
        o.dkey[i] = take(4 * nn);
        o.dval[i] = take(4 * nn);
    }
    o.depthv = take(4 * nn);
    o.rectv = take(8 * nn);
    o.srect = take(8 * nn);
    o.offs = take(4 * nn);
    o.dup_start = take(4 * (sort_blocks_for(mc) + 2));
    o.tkey = take(4 * mc);
    o.tval = take(4 * mc);
    o.total = off;
    return o;
}

// Carves `base` (may be null to only measure) and returns the bytes needed.
inline size_t carve_sort_ws(char *base, int64_t n, int64_t m_cap, uint64_t num_tiles, SortWs *ws) {
    const SortWsOffsets o = sort_ws_offsets(n, m_cap, num_tiles);
    if (ws) {
        auto at = [base](size_t off) -> char * { return base && off != SortWsOffsets::kNone ? base + off : nullptr; };
        SortWs w{};
        w.hdr = reinterpret_cast<SortHeader *>(at(o.hdr));
        for (int i = 0; i < 2; ++i) w.scan_state[i] = reinterpret_cast<uint64_t *>(at(o.scan_state[i]));
        for (int i = 0; i < 4; ++i) w.depth_state[i] = reinterpret_cast<uint64_t *>(at(o.depth_state[i]));
        for (int i = 0; i < kMaxTilePasses; ++i) w.tile_state[i] = reinterpret_cast<uint64_t *>(at(o.tile_state[i]));
        w.hist_depth = reinterpret_cast<uint32_t *>(at(o.hist_depth));
        w.hist_tile = reinterpret_cast<uint32_t *>(at(o.hist_tile));
        w.zero_bytes = o.zero_bytes;
        for (int i = 0; i < 2; ++i) {
            w.dkey[i] = reinterpret_cast<uint32_t *>(at(o.dkey[i]));
            w.dval[i] = reinterpret_cast<uint32_t *>(at(o.dval[i]));
        }
        w.depthv = reinterpret_cast<uint32_t *>(at(o.depthv));
        w.rectv = reinterpret_cast<uint2 *>(at(o.rectv));
        w.srect = reinterpret_cast<uint2 *>(at(o.srect));
        w.offs = reinterpret_cast<uint32_t *>(at(o.offs));
        w.dup_start = reinterpret_cast<uint32_t *>(at(o.dup_start));
        w.tkey = reinterpret_cast<uint32_t *>(at(o.tkey));
        w.tval = reinterpret_cast<uint32_t *>(at(o.tval));
        *ws = w;
    }
    return o.total;
}

}  // namespace gs
