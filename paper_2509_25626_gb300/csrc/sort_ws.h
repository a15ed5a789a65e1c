// Layout of the caller-provided gs_sort workspace.
#pragma once

#include <cstddef>
#include <cstdint>

namespace gs {

// Device-side counters of one gs_sort call (first 256 bytes of the workspace).
struct SortHeader {
    uint64_t m_total;   // instances the visible splats produce (may exceed the capacity)
    uint32_t nvis;      // visible splats (tiles_touched > 0)
    uint32_t m_sort;    // min(m_total, m_cap): instances actually written and sorted
    uint32_t overflow;  // 1 if m_total > m_cap
    uint32_t reserved[3];
};

struct SortWs {
    SortHeader *hdr;
    uint32_t *dkey[2], *dval[2];   // depth sort ping-pong, [n]
    uint32_t *tcount;              // tiles_touched in depth order, [n]
    uint32_t *blk;                 // per-block sums, [scan blocks]
    uint64_t *blk_off;             // their exclusive scan, [scan blocks]
    uint64_t *key_alt;             // tile sort ping-pong, [m_cap]
    uint32_t *val_alt;             // [m_cap]
    uint32_t *hist;                // radix histograms, [256][radix tiles]
    uint32_t *dtotal;              // radix digit totals, [256]
};

uint32_t radix_tiles_for(uint64_t count);
uint32_t scan_blocks_for(uint64_t count);

// Carves `base` (may be null to only measure) and returns the bytes needed.
inline size_t carve_sort_ws(char *base, int64_t n, int64_t m_cap, SortWs *ws) {
    size_t off = 0;
    auto take = [&](size_t bytes) -> char * {
        char *p = base ? base + off : nullptr;
        off += (bytes + 255) & ~(size_t)255;
        return p;
    };
    const uint64_t nn = (uint64_t)(n > 0 ? n : 0), mc = (uint64_t)(m_cap > 0 ? m_cap : 0);
    const uint64_t nblk = scan_blocks_for(nn) + 1;
    const uint64_t rt = radix_tiles_for(nn > mc ? nn : mc) + 1;
    SortWs w;
    w.hdr = reinterpret_cast<SortHeader *>(take(256));
    for (int i = 0; i < 2; ++i) {
        w.dkey[i] = reinterpret_cast<uint32_t *>(take(4 * nn));
        w.dval[i] = reinterpret_cast<uint32_t *>(take(4 * nn));
    }
    w.tcount = reinterpret_cast<uint32_t *>(take(4 * nn));
    w.blk = reinterpret_cast<uint32_t *>(take(4 * nblk));
    w.blk_off = reinterpret_cast<uint64_t *>(take(8 * nblk));
    w.key_alt = reinterpret_cast<uint64_t *>(take(8 * mc));
    w.val_alt = reinterpret_cast<uint32_t *>(take(4 * mc));
    w.hist = reinterpret_cast<uint32_t *>(take(4 * 256 * rt));
    w.dtotal = reinterpret_cast<uint32_t *>(take(4 * 256));
    if (ws) *ws = w;
    return off;
}

}  // namespace gs
