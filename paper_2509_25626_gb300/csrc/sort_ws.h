// Layout of the caller-provided gs_sort workspace.
#pragma once

#include <cstddef>
#include <cstdint>

namespace gs {

constexpr int kSortTileItems = 4096;   // elements per block in the look-back scans and tile radix passes
constexpr int kDepthItems = 4096;      // elements per block in the depth radix passes
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
    uint32_t reserved[48];
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

inline uint64_t sort_blocks_for(uint64_t count) { return (count + kSortTileItems - 1) / kSortTileItems; }
inline uint64_t depth_blocks_for(uint64_t count) { return (count + kDepthItems - 1) / kDepthItems; }
inline uint64_t tile_pass_blocks_for(uint64_t count) { return (count + kTilePassItems - 1) / kTilePassItems; }

inline int tile_bits_of(uint64_t num_tiles) {
    int b = 0;
    while (b < 32 && (1ull << b) < num_tiles) ++b;
    return b;
}

inline int tile_passes_of(uint64_t num_tiles) {
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
inline int tile_passes_bound(uint64_t num_tiles) {
    const int p = tile_passes_of(num_tiles) + 1;
    return p < kMaxTilePasses ? p : kMaxTilePasses;
}

// Carves `base` (may be null to only measure) and returns the bytes needed.
inline size_t carve_sort_ws(char *base, int64_t n, int64_t m_cap, uint64_t num_tiles, SortWs *ws) {
    size_t off = 0;
    auto take = [&](size_t bytes) -> char * {
        char *p = base ? base + off : nullptr;
        off += (bytes + 255) & ~(size_t)255;
        return p;
    };
    const uint64_t nn = (uint64_t)(n > 0 ? n : 0), mc = (uint64_t)(m_cap > 0 ? m_cap : 0);
    const uint64_t bn = sort_blocks_for(nn) + 1, bm = sort_blocks_for(mc) + 1, bd = depth_blocks_for(nn) + 1;
    const uint64_t bt = tile_pass_blocks_for(mc) + 1;
    const int passes = tile_passes_bound(num_tiles);
    SortWs w{};
    w.hdr = reinterpret_cast<SortHeader *>(take(sizeof(SortHeader)));
    for (int i = 0; i < 2; ++i) w.scan_state[i] = reinterpret_cast<uint64_t *>(take(8 * bn));
    for (int i = 0; i < 4; ++i) w.depth_state[i] = reinterpret_cast<uint64_t *>(take(8 * 256 * bd));
    for (int i = 0; i < kMaxTilePasses; ++i)  // pass 0 (fused with duplication) uses 4096-element blocks
        w.tile_state[i] = reinterpret_cast<uint64_t *>(i < passes ? take(8 * 256 * (i == 0 ? bm : bt)) : nullptr);
    w.hist_depth = reinterpret_cast<uint32_t *>(take(4 * 4 * 256));
    w.hist_tile = reinterpret_cast<uint32_t *>(take(4 * kMaxTilePasses * 257));
    w.zero_bytes = off;
    for (int i = 0; i < 2; ++i) {
        w.dkey[i] = reinterpret_cast<uint32_t *>(take(4 * nn));
        w.dval[i] = reinterpret_cast<uint32_t *>(take(4 * nn));
    }
    w.depthv = reinterpret_cast<uint32_t *>(take(4 * nn));
    w.rectv = reinterpret_cast<uint2 *>(take(8 * nn));
    w.srect = reinterpret_cast<uint2 *>(take(8 * nn));
    w.offs = reinterpret_cast<uint32_t *>(take(4 * nn));
    w.dup_start = reinterpret_cast<uint32_t *>(take(4 * (sort_blocks_for(mc) + 2)));
    w.tkey = reinterpret_cast<uint32_t *>(take(4 * mc));
    w.tval = reinterpret_cast<uint32_t *>(take(4 * mc));
    if (ws) *ws = w;
    return off;
}

}  // namespace gs
