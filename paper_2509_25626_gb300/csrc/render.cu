// Per-tile front-to-back alpha blending (Section II-B (2), Algorithm 1,
// Eq. 1 with the kernel's alpha and the Appendix B per-pixel rules).
//
// One 128-thread block per 16x16 tile.  Each warp owns an 8x8 pixel block
// and each lane two horizontally adjacent pixels, which share every term
// that depends only on the row (dy, v, the w01 dy product).  Per round the
// block stages up to 256 of the tile's splats in shared memory (two gathers
// per thread) and marks, per warp, the splats whose alpha >= 1/255 region
// can reach that warp's 8x8 block (quarter_mask: the bounding box
// gs_splat.cull_hx/hy, and a slanted band along the first row of the
// inverse-covariance factor); each warp then walks only its marked splats,
// front to back.  A splat left out has alpha < 1/255 at every pixel of the
// block, so the per-pixel result, n_contrib (a list position) and the
// stopping point are unchanged.
//
// Exits are block-uniform (__syncthreads_and at the round boundary) and
// warp-uniform inside a round, so no thread leaves while others still reach
// a barrier, and a pixel that stopped stays stopped across rounds.
#include "common.cuh"

namespace gs {

namespace {

constexpr int kThreads = 128;  // 4 warps, 2x2 blocks of 8x8 pixels
constexpr int kBatch = 256;    // splats staged per round
constexpr int kWarps = kThreads / 32;

struct __align__(16) StagedA { float x, y, w00, w01; };
struct __align__(16) StagedB { float w11, lg2o, r, g; };

struct Pixel {
    float T, c0, c1, c2;
    float id;       // inverse depth accumulated like a colour channel (kDepth only)
    uint32_t last;  // 1-based list position of the last blended splat
    uint32_t stop;  // list position of the splat that stopped the pixel, 0 if none
    bool done;
};

// keep: alpha >= 1/255 (decided by the caller on log2 alpha); iz = 1 / depth
template <bool kDepth>
__device__ __forceinline__ void blend(Pixel &p, bool keep, float alpha, float r, float g, float b, float iz,
                                      uint32_t idx) {
    if (p.done || !keep) return;
    const float w = alpha * p.T;  // this splat's weight
    const float Tn = p.T - w;     // T (1 - alpha)
    if (Tn < kTStop) {  // stop without blending this splat
        p.done = true;
        p.stop = idx;
        return;
    }
    p.c0 = fmaf(r, w, p.c0);
    p.c1 = fmaf(g, w, p.c1);
    p.c2 = fmaf(b, w, p.c2);
    if (kDepth) p.id = fmaf(iz, w, p.id);
    p.T = Tn;
    p.last = idx;
}

// kDepth: also write, per pixel, the inverse depth blended like a colour
// channel (no background term): sum of alpha T / depth over the blended
// splats, the optional output of the paper's kernels (Appendix B).
// kCount: also write, per pixel, how many splats were evaluated before the
// pixel stopped (the stopping one included; the whole list if it never
// stopped) -- the work measure of the paper's workload characterisation
// (Table III) -- and, if tile_cycles is set, the SM clock cycles the block
// spent on the tile (the per-block load-balance measure of Section IV-C).
// Both follow from state the loop keeps anyway, so the loop is the same in
// both instantiations.
struct RenderSmem {
    StagedA a[kBatch];
    StagedB b[kBatch];
    float c[kBatch];
    uint8_t mask[kBatch];
    uint8_t list[kWarps][kBatch];
    float iz[kBatch];  // 1 / depth (kDepth only)
};

// Where this thread's two pixels sit in a tile, and the tile's corner.
struct TileGeom {
    int tile, px, py;
    float pxf, pyf, tx0, ty0;
    bool in0, in1;
};

__device__ __forceinline__ TileGeom tile_geom(int tile, int width, int height) {
    TileGeom g;
    const int tiles_x = (width + kTile - 1) / kTile;
    const int tx = tile % tiles_x, ty = tile / tiles_x;
    const unsigned lane = lane_id(), warp = threadIdx.x >> 5;
    const int bx0 = tx * kTile + (int)(warp & 1u) * 8, by0 = ty * kTile + (int)(warp >> 1) * 8;
    g.tile = tile;
    g.px = bx0 + 2 * (int)(lane & 3u);
    g.py = by0 + (int)(lane >> 2);
    g.pxf = (float)g.px;
    g.pyf = (float)g.py;
    g.in0 = g.px < width && g.py < height;
    g.in1 = g.px + 1 < width && g.py < height;
    g.tx0 = (float)(tx * kTile);
    g.ty0 = (float)(ty * kTile);
    return g;
}

// Walks list entries [from, to) of a tile whose list starts at `begin`
// (list positions are counted from `begin`, 1-based), front to back, in
// rounds of kBatch staged splats, updating the two pixels' states; stops
// early once every pixel of the block is done, or after max_rounds rounds.
// Returns the first entry not walked (`to` if the walk reached the end or
// every pixel is done).  Every thread must call it; it begins each round
// with a block-wide barrier.
// The job's splat and value pointers are read where a round stages its
// batch, not held in registers across the walk: the batch kernels keep the
// job in shared memory, the single-image kernel in its parameters.
// kBudget: max_rounds is honoured (the split render's budgeted walk); the
// other walks compile without the round count.
// kContrib: the contribution-aware walk (the Seele-style variant): before
// blending a round, each warp -- a group of 32 lanes, 8x8 pixels -- builds
// by warp votes the mask of the splats whose alpha reaches 1/255 at one of
// its still-live pixels (the exact per-pixel test, on log2 alpha) and then
// blends only those.  Every other splat would be a no-op for every pixel
// of the group, so images, n_contrib and the stopping points are those of
// the plain walk, bit for bit.
template <bool kDepth, bool kBudget = false, bool kContrib = false>
__device__ __forceinline__ uint32_t walk_tile(RenderSmem &sm, const gs_render_job &job, uint32_t begin, uint32_t from,
                                              uint32_t to, uint32_t max_rounds, const TileGeom &g, Pixel &p0,
                                              Pixel &p1) {
    StagedA *s_a = sm.a;
    StagedB *s_b = sm.b;
    float *s_c = sm.c;
    uint8_t *s_mask = sm.mask;
    uint8_t(*s_list)[kBatch] = sm.list;
    const unsigned lane = lane_id(), warp = threadIdx.x >> 5;
    const unsigned lt = lanemask_lt();
    const float pxf = g.pxf, pyf = g.pyf;
    uint32_t rounds = 0;
    uint32_t base = from;
    for (; base < to; base += kBatch) {
        // every thread has finished the previous round; stop if all pixels are done
        if (__syncthreads_and(p0.done && p1.done)) return to;
        if (kBudget && rounds++ == max_rounds) return base;  // uniform: every thread counts the same rounds
        const gs_splat *__restrict__ splats = job.splats;
        const uint32_t *__restrict__ vals = job.vals;
#pragma unroll
        for (int r = 0; r < kBatch / kThreads; ++r) {
            const int k = (int)threadIdx.x + r * kThreads;
            const uint32_t i = base + (uint32_t)k;
            uint32_t m = 0;
            if (i < to) {
                // read-only path: the batch kernel takes these pointers from memory
                const float4 *src = reinterpret_cast<const float4 *>(splats + __ldg(vals + i));
                const float4 a = __ldg(src), b = __ldg(src + 1), c = __ldg(src + 2);
                s_a[k] = StagedA{a.x, a.y, a.z, a.w};
                s_b[k] = StagedB{b.x, b.y, b.z, b.w};
                s_c[k] = c.x;
                if (kDepth) sm.iz[k] = __frcp_rn(__ldg(reinterpret_cast<const float *>(src + 3)));
                m = quarter_mask(a, b, c, g.tx0, g.ty0);
            }
            s_mask[k] = (uint8_t)m;
        }
        __syncthreads();

        // this warp's splats, in list order
        uint32_t cnt = 0;
#pragma unroll
        for (int c = 0; c < kBatch / 32; ++c) {
            const uint32_t bit = (s_mask[c * 32 + lane] >> warp) & 1u;
            const unsigned bal = __ballot_sync(0xffffffffu, bit);
            if (bit) s_list[warp][cnt + __popc(bal & lt)] = (uint8_t)(c * 32 + lane);
            cnt += __popc(bal);
        }
        __syncwarp();

        if (kContrib) {
            // the group's contribution mask, compacted in place (an entry is
            // written only at or before the one being read)
            uint32_t kept = 0;
            for (uint32_t q = 0; q < cnt; ++q) {
                const uint32_t j = s_list[warp][q];
                const StagedA sa = s_a[j];
                const StagedB sb = s_b[j];
                const float dy = sa.y - pyf;
                const float dx = sa.x - pxf;
                const float u0 = fmaf(sa.w00, dx, sa.w01 * dy);
                const float u1 = u0 - sa.w00;
                const float v = sb.w11 * dy;
                const float vv = fmaf(-v, v, sb.lg2o);
                const bool reach = (!p0.done && fmaf(-u0, u0, vv) >= -kLog2_255) ||
                                   (!p1.done && fmaf(-u1, u1, vv) >= -kLog2_255);
                if (__any_sync(0xffffffffu, reach)) {
                    if (lane == 0) s_list[warp][kept] = (uint8_t)j;
                    ++kept;
                }
            }
            __syncwarp();
            cnt = kept;
        }

        const uint32_t pos0 = base - begin + 1;  // list position of staged splat 0
        // the warp votes on stopping once per kVote splats (4 and 64 measured
        // slower than 16; a stopped pixel's blend is a no-op in between)
        constexpr uint32_t kVote = 16;
        for (uint32_t qv = 0; qv < cnt; qv += kVote) {
            if (__all_sync(0xffffffffu, p0.done && p1.done)) break;  // warp-uniform
            const uint32_t qe = min(cnt, qv + kVote);
#pragma unroll 4
            for (uint32_t q = qv; q < qe; ++q) {
                const uint32_t j = s_list[warp][q];
                const StagedA sa = s_a[j];
                const StagedB sb = s_b[j];
                const float dy = sa.y - pyf;
                const float dx = sa.x - pxf;
                const float t = sa.w01 * dy;
                const float u0 = fmaf(sa.w00, dx, t);
                const float u1 = u0 - sa.w00;  // dx - 1 for the right-hand pixel
                const float v = sb.w11 * dy;
                const float vv = fmaf(-v, v, sb.lg2o);
                const float e0 = fmaf(-u0, u0, vv), e1 = fmaf(-u1, u1, vv);  // log2 alpha before the clamp
                // alpha >= 1/255 <=> log2 alpha >= -log2 255: decided before the exp
                const bool k0 = e0 >= -kLog2_255, k1 = e1 >= -kLog2_255;
                if (k0 || k1) {
                    const float b = s_c[j];
                    const float iz = kDepth ? sm.iz[j] : 0.f;
                    blend<kDepth>(p0, k0, fminf(kAlphaMax, ex2_approx(e0)), sb.r, sb.g, b, iz, pos0 + j);
                    blend<kDepth>(p1, k1, fminf(kAlphaMax, ex2_approx(e1)), sb.r, sb.g, b, iz, pos0 + j);
                }
            }
        }
    }
    return to;
}

// Writes a finished tile's pixels (out = C + T bg, final T, n_contrib, and
// the optional outputs), then ends with a block-wide barrier so the shared
// memory may be reused for the next tile.
template <bool kCount, bool kDepth>
__device__ __forceinline__ void store_tile(const gs_render_job &job, const TileGeom &g, const Pixel &p0,
                                           const Pixel &p1, uint32_t len, float *__restrict__ invdepth,
                                           uint32_t *__restrict__ n_eval) {
    const int width = job.width;
    const size_t plane = (size_t)width * job.height;
    float *__restrict__ out_color = job.out_color;
    const float bg_r = job.bg[0], bg_g = job.bg[1], bg_b = job.bg[2];
    if (g.in0) {
        const size_t pix = (size_t)g.py * width + g.px;
        out_color[pix] = fmaf(p0.T, bg_r, p0.c0);
        out_color[plane + pix] = fmaf(p0.T, bg_g, p0.c1);
        out_color[2 * plane + pix] = fmaf(p0.T, bg_b, p0.c2);
        job.final_T[pix] = p0.T;
        job.n_contrib[pix] = p0.last;
        if (kCount) n_eval[pix] = p0.stop ? p0.stop : len;
        if (kDepth) invdepth[pix] = p0.id;
    }
    if (g.in1) {
        const size_t pix = (size_t)g.py * width + g.px + 1;
        out_color[pix] = fmaf(p1.T, bg_r, p1.c0);
        out_color[plane + pix] = fmaf(p1.T, bg_g, p1.c1);
        out_color[2 * plane + pix] = fmaf(p1.T, bg_b, p1.c2);
        job.final_T[pix] = p1.T;
        job.n_contrib[pix] = p1.last;
        if (kCount) n_eval[pix] = p1.stop ? p1.stop : len;
        if (kDepth) invdepth[pix] = p1.id;
    }
    __syncthreads();  // shared memory free for the next tile
}

// Renders one tile with the whole block.  Every thread must call it; it
// begins and ends with block-wide barriers, so the shared memory may be
// reused for the next tile.  The job's pointers and sizes are read where
// they are used, not held in registers: the batch kernel keeps its job in
// shared memory, the single-image kernel in its parameters.
template <bool kCount, bool kDepth, bool kContrib = false>
__device__ __forceinline__ void render_tile(RenderSmem &sm, const gs_render_job &job, const uint2 range, int tile,
                                            float *__restrict__ invdepth, uint32_t *__restrict__ n_eval,
                                            uint32_t *__restrict__ tile_cycles) {
    long long t_start = 0;
    if (kCount) t_start = clock64();
    const TileGeom g = tile_geom(tile, job.width, job.height);
    Pixel p0{1.f, 0.f, 0.f, 0.f, 0.f, 0u, 0u, !g.in0};
    Pixel p1{1.f, 0.f, 0.f, 0.f, 0.f, 0u, 0u, !g.in1};
    walk_tile<kDepth, false, kContrib>(sm, job, range.x, range.x, range.y, 0xffffffffu, g, p0, p1);
    store_tile<kCount, kDepth>(job, g, p0, p1, range.y - range.x, invdepth, n_eval);
    if (kCount && tile_cycles != nullptr && threadIdx.x == 0) {
        const long long dt = clock64() - t_start;
        tile_cycles[tile] = dt < 0 ? 0u : (dt > 0xffffffffll ? 0xffffffffu : (uint32_t)dt);
    }
}

template <bool kCount, bool kDepth, bool kContrib = false>
__global__ void __launch_bounds__(kThreads, (kCount || kDepth) ? 10 : 12) render_kernel(const gs_splat *__restrict__ splats,
                                                          const uint32_t *__restrict__ vals,
                                                          const uint2 *__restrict__ ranges, int width, int height,
                                                          float bg_r, float bg_g, float bg_b,
                                                          float *__restrict__ out_color,
                                                          float *__restrict__ final_T,
                                                          uint32_t *__restrict__ n_contrib,
                                                          float *__restrict__ invdepth,
                                                          uint32_t *__restrict__ n_eval,
                                                          uint32_t *__restrict__ tile_cycles) {
    __shared__ RenderSmem sm;
    gs_render_job job;
    job.splats = splats;
    job.vals = vals;
    job.ranges = nullptr;
    job.out_color = out_color;
    job.final_T = final_T;
    job.n_contrib = n_contrib;
    job.width = width;
    job.height = height;
    job.bg[0] = bg_r;
    job.bg[1] = bg_g;
    job.bg[2] = bg_b;
    job.tile_begin = 0;
    render_tile<kCount, kDepth, kContrib>(sm, job, ranges[blockIdx.x], blockIdx.x, invdepth, n_eval, tile_cycles);
}

// --- heavy tiles split across blocks -----------------------------------------
// A queued tile: job, tile, its list's first entry, the first entry not yet
// walked, and the end of its list.
struct SplitEntry {
    uint32_t job, tile, begin, pos, end, pad[3];
};
static_assert(sizeof(SplitEntry) == 32, "split entry layout");

// Views of the split render's workspace (the caller's memory).
struct SplitLayout {
    uint32_t *n_entries;   // tiles queued by the budgeted walk (may exceed cap)
    uint32_t *chunk_ctr;   // work counter of the chunk walks
    uint32_t *n_heavy;     // long-list tiles found by classify_kernel (may exceed heavy_cap)
    uint32_t *heavy;       // [heavy_cap] their work-item numbers
    uint32_t heavy_cap, heavy_len;
    SplitEntry *entries;   // [cap]
    float4 *state;         // [cap][256] (c0, c1, c2, T) after the budgeted walk
    uint32_t *state_last;  // [cap][256] last blended position | done << 31
    float4 *part;          // [cap][K][256] chunk partials (c0, c1, c2, T from 1)
    uint32_t *part_last;   // [cap][K][256] last blended position | stopped << 31
    uint32_t cap, K;
};

constexpr uint32_t kDoneBit = 1u << 31;

// The chunks of an entry: K windows of `chunk` splats (whole batches) after
// the budgeted walk's stopping point; the list beyond them, if any, is
// walked by the merge itself.  Every chunk is walked in full from T = 1, so
// chunks past the point where a pixel would stop are wasted work: the
// window bounds that waste, instead of chunking the whole remainder (lists
// of the slab tiles reach 10^5 splats while their pixels stop within ~10^4).
__device__ __forceinline__ uint32_t split_chunk_size(const SplitEntry &, uint32_t, uint32_t chunk) { return chunk; }

__device__ __forceinline__ void pixel_save(float4 *st, uint32_t *last, const Pixel &p, bool stopped_flag) {
    *st = make_float4(p.c0, p.c1, p.c2, p.T);
    *last = p.last | (stopped_flag ? kDoneBit : 0u);
}

// Copies job `j` of the batch into shared memory (threads < the job's words).
__device__ __forceinline__ void fetch_job(gs_render_job *dst, const gs_render_batch_desc *desc, uint32_t j) {
    constexpr int kJobWords = (int)(sizeof(gs_render_job) / 4);
    if (threadIdx.x < (unsigned)kJobWords)
        reinterpret_cast<uint32_t *>(dst)[threadIdx.x] = reinterpret_cast<const uint32_t *>(&desc->jobs[j])[threadIdx.x];
}

// Loads the batch's job table into shared memory when it has at most
// kJobsCached jobs; returns whether it did.
constexpr int kJobsCached = 64;  // job tables up to this size live in shared memory

__device__ __forceinline__ bool cache_jobs(gs_render_job *s_jobs, const gs_render_batch_desc *desc, int n_jobs) {
    constexpr int kJobWords = (int)(sizeof(gs_render_job) / 4);
    const bool cached = n_jobs <= kJobsCached;  // uniform
    if (cached)
        for (int i = threadIdx.x; i < n_jobs * kJobWords; i += blockDim.x)
            reinterpret_cast<uint32_t *>(s_jobs)[i] = reinterpret_cast<const uint32_t *>(desc->jobs)[i];
    return cached;
}

// The job holding work item w: the last job with tile_begin <= w.
__device__ __forceinline__ int job_of(const gs_render_job *s_jobs, bool cached, const gs_render_batch_desc *desc,
                                      int n_jobs, uint32_t w) {
    int lo = 0, hi = n_jobs;
    if (cached) {
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (s_jobs[mid].tile_begin <= w) lo = mid; else hi = mid;
        }
    } else {
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (desc->jobs[mid].tile_begin <= w) lo = mid; else hi = mid;
        }
    }
    return lo;
}

__device__ __forceinline__ uint32_t list_length(const gs_render_job &job, uint32_t w) {
    const uint2 r = reinterpret_cast<const uint2 *>(job.ranges)[w - job.tile_begin];
    return r.y - r.x;
}

// Queues the work items (job, tile) whose list holds at least heavy_len
// splats, so that the batch render starts them first: a long list costs
// the most when a block picks it up near the end of the launch.
__global__ void __launch_bounds__(256) classify_kernel(const gs_render_batch_desc *__restrict__ desc, SplitLayout sl) {
    __shared__ gs_render_job s_jobs[kJobsCached];
    const int n_jobs = desc->n_jobs;
    const uint32_t total = desc->total_tiles;
    const bool cached = cache_jobs(s_jobs, desc, n_jobs);
    __syncthreads();
    for (uint32_t w = blockIdx.x * blockDim.x + threadIdx.x; w < total; w += gridDim.x * blockDim.x) {
        const int j = job_of(s_jobs, cached, desc, n_jobs, w);
        const uint32_t len = list_length(cached ? s_jobs[j] : desc->jobs[j], w);
        if (len >= sl.heavy_len) {
            const uint32_t slot = atomicAdd(sl.n_heavy, 1u);
            if (slot < sl.heavy_cap) sl.heavy[slot] = w;
        }
    }
}

// Persistent render of many jobs (requests): blocks pull work items -- one
// (job, tile) each, numbered through the jobs' tile_begin prefix -- from an
// atomic counter until all are taken.  Each block asks for its next item
// when it starts the current one, so the atomic's round trip overlaps the
// blend, and keeps the job table (up to 64 jobs) in shared memory, so
// finding an item's job costs no global round trip.  The job table and its
// counts live in device memory, so one captured launch serves any batch.
// Held to the register count of render_kernel so as many blocks stay
// resident per SM.
// kSplit: a tile still live after budget_rounds rounds of its list is not
// finished here: its pixels' state and the rest of its list go to the split
// workspace (while it has room) for the chunk walks and the merge below.
// kHeavy: the items classify_kernel queued come first (item i < n_heavy
// is queued tile heavy[i]), then every tile in order, skipping the queued
// ones; if the queue overflowed it is ignored and the order is the plain one.
#ifndef GS_BATCH_MIN_BLOCKS
#define GS_BATCH_MIN_BLOCKS 10
#endif
template <bool kSplit, bool kHeavy>
__global__ void __launch_bounds__(kThreads, GS_BATCH_MIN_BLOCKS) render_batch_kernel(
    const gs_render_batch_desc *__restrict__ desc, uint32_t *__restrict__ counter, SplitLayout sl,
    uint32_t budget_rounds) {
    constexpr int kJobWords = (int)(sizeof(gs_render_job) / 4);
    static_assert(sizeof(gs_render_job) % 4 == 0 && kJobWords <= kThreads, "job copy");
    __shared__ RenderSmem sm;
    __shared__ gs_render_job s_jobs[kJobsCached];
    // the loop's state lives here, not in registers across the tile walk
    __shared__ uint32_t s_w, s_next, s_slot, s_nh, s_total;
    __shared__ int s_njobs;
    if (threadIdx.x == 0) {
        uint32_t nh = 0;
        if (kHeavy) {
            nh = *sl.n_heavy;
            if (nh > sl.heavy_cap) nh = 0;
        }
        s_nh = nh;
        s_total = desc->total_tiles + nh;
        s_njobs = desc->n_jobs;
        s_w = atomicAdd(counter, 1u);
    }
    cache_jobs(s_jobs, desc, desc->n_jobs);
    __syncthreads();
    for (;;) {
        const uint32_t item = s_w;
        if (item >= s_total) break;  // uniform
        if (threadIdx.x == 0) s_next = atomicAdd(counter, 1u);  // read after this tile
        const int n_jobs = s_njobs;
        const bool cached = n_jobs <= kJobsCached;
        const uint32_t nh = kHeavy ? s_nh : 0u;
        const uint32_t w = (kHeavy && item < nh) ? __ldg(sl.heavy + item) : item - nh;
        int lo = job_of(s_jobs, cached, desc, n_jobs, w);
        const bool skip = kHeavy && nh > 0 && item >= nh &&
                          list_length(cached ? s_jobs[lo] : desc->jobs[lo], w) >= sl.heavy_len;
        if (!skip) {  // uniform; a skipped item was queued and rendered first
            const uint32_t jidx = (uint32_t)lo;
            if (!cached) {
                // the previous tile ended with a barrier, so slot 0 is free
                fetch_job(&s_jobs[0], desc, jidx);
                __syncthreads();
                lo = 0;
            }
            const gs_render_job &job = s_jobs[lo];
            const int tile = (int)(w - job.tile_begin);
            const uint2 range = reinterpret_cast<const uint2 *>(job.ranges)[tile];
            if (!kSplit) {
                render_tile<false, false>(sm, job, range, tile, nullptr, nullptr, nullptr);
            } else {
                const TileGeom g = tile_geom(tile, job.width, job.height);
                Pixel p0{1.f, 0.f, 0.f, 0.f, 0.f, 0u, 0u, !g.in0};
                Pixel p1{1.f, 0.f, 0.f, 0.f, 0.f, 0u, 0u, !g.in1};
                uint32_t at = walk_tile<false, true>(sm, job, range.x, range.x, range.y, budget_rounds, g, p0, p1);
                bool queued = false;
                if (at < range.y) {  // uniform: the budget ran out with live pixels
                    if (threadIdx.x == 0) s_slot = atomicAdd(sl.n_entries, 1u);
                    __syncthreads();
                    const uint32_t slot = s_slot;
                    if (slot < sl.cap) {
                        queued = true;
                        if (threadIdx.x == 0)
                            sl.entries[slot] = SplitEntry{jidx, (uint32_t)tile, range.x, at, range.y, {0u, 0u, 0u}};
                        const size_t px = (size_t)slot * kTilePixels + 2 * threadIdx.x;
                        pixel_save(sl.state + px, sl.state_last + px, p0, p0.done);
                        pixel_save(sl.state + px + 1, sl.state_last + px + 1, p1, p1.done);
                    } else {
                        walk_tile<false>(sm, job, range.x, at, range.y, 0xffffffffu, g, p0, p1);
                    }
                }
                if (!queued)
                    store_tile<false, false>(job, g, p0, p1, 0u, nullptr, nullptr);
                else
                    __syncthreads();  // as store_tile: shared memory free for the next tile
            }
        } else {
            __syncthreads();  // s_next is written before it is read
        }
        // the tile ended with a barrier: nobody reads s_w any more
        if (threadIdx.x == 0) s_w = s_next;
        __syncthreads();
    }
}

// The chunk walks of the queued tiles: blocks pull (entry, chunk) items from
// the workspace's counter; each walks its chunk of the list front to back
// from T = 1 (with the per-pixel stop on that local T) and records the
// partial colour, transmittance, last blended position and whether the
// pixel stopped.
__global__ void __launch_bounds__(kThreads, 10) split_chunk_kernel(const gs_render_batch_desc *__restrict__ desc,
                                                               SplitLayout sl, uint32_t chunk) {
    __shared__ RenderSmem sm;
    __shared__ gs_render_job s_job;
    __shared__ SplitEntry s_e;
    __shared__ uint32_t s_w;
    const uint32_t n = min(*sl.n_entries, sl.cap);
    const uint32_t total = n * sl.K;
    for (;;) {
        if (threadIdx.x == 0) s_w = atomicAdd(sl.chunk_ctr, 1u);
        __syncthreads();
        const uint32_t w = s_w;
        if (w >= total) break;  // uniform
        const uint32_t e = w / sl.K, c = w % sl.K;
        if (threadIdx.x == 0) s_e = sl.entries[e];
        __syncthreads();
        const SplitEntry ent = s_e;
        const uint32_t csz = split_chunk_size(ent, sl.K, chunk);
        const uint32_t s0 = ent.pos + c * csz;
        if (s0 < ent.end) {  // uniform
            fetch_job(&s_job, desc, ent.job);
            __syncthreads();
            const TileGeom g = tile_geom((int)ent.tile, s_job.width, s_job.height);
            Pixel p0{1.f, 0.f, 0.f, 0.f, 0.f, 0u, 0u, !g.in0};
            Pixel p1{1.f, 0.f, 0.f, 0.f, 0.f, 0u, 0u, !g.in1};
            walk_tile<false>(sm, s_job, ent.begin, s0, min(ent.end, s0 + csz), 0xffffffffu, g, p0, p1);
            const size_t px = ((size_t)e * sl.K + c) * kTilePixels + 2 * threadIdx.x;
            pixel_save(sl.part + px, sl.part_last + px, p0, p0.stop != 0u);
            pixel_save(sl.part + px + 1, sl.part_last + px + 1, p1, p1.stop != 0u);
        }
        __syncthreads();  // s_w, s_e and s_job are rewritten by the next item
    }
}

// Folds chunk partial (c, T_k, last_k) into a pixel's running state, or
// reports that the absolute transmittance crosses the stop inside the chunk.
__device__ __forceinline__ bool merge_chunk(Pixel &p, const float4 part, uint32_t plast) {
    if (p.done) return false;
    if ((plast & kDoneBit) || p.T * part.w < kTStop) return true;
    p.c0 = fmaf(p.T, part.x, p.c0);
    p.c1 = fmaf(p.T, part.y, p.c1);
    p.c2 = fmaf(p.T, part.z, p.c2);
    p.T *= part.w;
    if (plast) p.last = plast;
    return false;
}

// The merge of each queued tile: its pixels' state after the budgeted walk,
// then the chunks in list order (merge_chunk); a chunk inside which some
// pixel's absolute transmittance crosses the stop is walked again by the
// block for those pixels, from their true incoming state, so they stop
// where the single walk stops.  Writes the tile's outputs.
__global__ void __launch_bounds__(kThreads, 10) split_merge_kernel(const gs_render_batch_desc *__restrict__ desc,
                                                               SplitLayout sl, uint32_t chunk) {
    __shared__ RenderSmem sm;
    __shared__ gs_render_job s_job;
    __shared__ SplitEntry s_e;
    const uint32_t n = min(*sl.n_entries, sl.cap);
    for (uint32_t e = blockIdx.x; e < n; e += gridDim.x) {
        if (threadIdx.x == 0) s_e = sl.entries[e];
        __syncthreads();
        const SplitEntry ent = s_e;
        fetch_job(&s_job, desc, ent.job);
        __syncthreads();
        const TileGeom g = tile_geom((int)ent.tile, s_job.width, s_job.height);
        const size_t px = (size_t)e * kTilePixels + 2 * threadIdx.x;
        Pixel p0, p1;
        {
            const float4 a = sl.state[px], b = sl.state[px + 1];
            const uint32_t la = sl.state_last[px], lb = sl.state_last[px + 1];
            p0 = Pixel{a.w, a.x, a.y, a.z, 0.f, la & ~kDoneBit, 0u, (la & kDoneBit) != 0u};
            p1 = Pixel{b.w, b.x, b.y, b.z, 0.f, lb & ~kDoneBit, 0u, (lb & kDoneBit) != 0u};
        }
        const uint32_t csz = split_chunk_size(ent, sl.K, chunk);
        for (uint32_t c = 0; c < sl.K; ++c) {
            const uint32_t s0 = ent.pos + c * csz;
            if (s0 >= ent.end) break;  // uniform
            const size_t pp = ((size_t)e * sl.K + c) * kTilePixels + 2 * threadIdx.x;
            const bool x0 = merge_chunk(p0, sl.part[pp], sl.part_last[pp]);
            const bool x1 = merge_chunk(p1, sl.part[pp + 1], sl.part_last[pp + 1]);
            if (__syncthreads_or(x0 || x1)) {
                // walk the chunk again for the pixels that stop inside it
                const bool hold0 = !p0.done && !x0, hold1 = !p1.done && !x1;
                if (hold0) p0.done = true;
                if (hold1) p1.done = true;
                walk_tile<false>(sm, s_job, ent.begin, s0, min(ent.end, s0 + csz), 0xffffffffu, g, p0, p1);
                if (hold0) p0.done = false;
                if (hold1) p1.done = false;
            }
        }
        // the list beyond the chunked window, from the merged state (exact)
        const uint64_t window_end = (uint64_t)ent.pos + (uint64_t)sl.K * csz;
        if (window_end < ent.end)
            walk_tile<false>(sm, s_job, ent.begin, (uint32_t)window_end, ent.end, 0xffffffffu, g, p0, p1);
        store_tile<false, false>(s_job, g, p0, p1, 0u, nullptr, nullptr);
    }
}

}  // namespace

cudaError_t launch_render_contrib(const gs_splat *splats, const uint32_t *vals, const uint32_t *ranges,
                                  const CamParams &cam, const float bg[3], float *out_color, float *final_T,
                                  uint32_t *n_contrib, cudaStream_t stream) {
    const int num_tiles = cam.tiles_x * cam.tiles_y;
    render_kernel<false, false, true><<<num_tiles, kThreads, 0, stream>>>(
        splats, vals, reinterpret_cast<const uint2 *>(ranges), cam.width, cam.height, bg[0], bg[1], bg[2], out_color,
        final_T, n_contrib, nullptr, nullptr, nullptr);
    return cudaGetLastError();
}

cudaError_t launch_render(const gs_splat *splats, const uint32_t *vals, const uint32_t *ranges, const CamParams &cam,
                          const float bg[3], float *out_color, float *final_T, uint32_t *n_contrib, float *invdepth,
                          uint32_t *n_eval, uint32_t *tile_cycles, cudaStream_t stream) {
    const int num_tiles = cam.tiles_x * cam.tiles_y;
    const uint2 *rg = reinterpret_cast<const uint2 *>(ranges);
#define GS_RENDER_LAUNCH(C, D)                                                                                      \
    render_kernel<C, D><<<num_tiles, kThreads, 0, stream>>>(splats, vals, rg, cam.width, cam.height, bg[0], bg[1], \
                                                            bg[2], out_color, final_T, n_contrib, invdepth, n_eval, \
                                                            tile_cycles)
    if (n_eval && invdepth)
        GS_RENDER_LAUNCH(true, true);
    else if (n_eval)
        GS_RENDER_LAUNCH(true, false);
    else if (invdepth)
        GS_RENDER_LAUNCH(false, true);
    else
        GS_RENDER_LAUNCH(false, false);
#undef GS_RENDER_LAUNCH
    return cudaGetLastError();
}

// One full wave of the device for the batch kernels; looked up on the first
// call per device (make that call outside stream capture) and cached.
static cudaError_t batch_wave(int *grid) {
    static int wave[64] = {0};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (wave[dev] == 0) {
        int sms = 0, per_sm = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, render_batch_kernel<true, true>, kThreads, 0);
        wave[dev] = (sms > 0 ? sms : 1) * (per_sm > 0 ? per_sm : 1);
    }
    *grid = wave[dev];
    return cudaSuccess;
}

cudaError_t launch_render_batch(const gs_render_batch_desc *desc, uint32_t *counter, int grid, cudaStream_t stream) {
    cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(uint32_t), stream);
    if (e != cudaSuccess) return e;
    if (grid <= 0 && (e = batch_wave(&grid)) != cudaSuccess) return e;
    render_batch_kernel<false, false><<<grid, kThreads, 0, stream>>>(desc, counter, SplitLayout{}, 0xffffffffu);
    return cudaGetLastError();
}

// Workspace of the balanced render: a 256-byte header (split-queue count,
// chunk counter, long-list count), the long-list queue, the split queue,
// the pixel states and the chunk partials.
static size_t carve_balance_ws(char *base, const gs_balance_params &p, SplitLayout *out) {
    size_t off = 0;
    auto take = [&](size_t bytes) -> char * {
        char *q = base ? base + off : nullptr;
        off += (bytes + 255) & ~(size_t)255;
        return q;
    };
    const uint32_t cap = (uint32_t)(p.budget > 0 ? p.max_split_tiles : 0), K = (uint32_t)p.max_chunks;
    const uint32_t hcap = (uint32_t)(p.heavy_len > 0 ? p.max_heavy_tiles : 0);
    SplitLayout l{};
    char *hdr = take(256);
    l.n_entries = reinterpret_cast<uint32_t *>(hdr);
    l.chunk_ctr = hdr ? reinterpret_cast<uint32_t *>(hdr + 4) : nullptr;
    l.n_heavy = hdr ? reinterpret_cast<uint32_t *>(hdr + 8) : nullptr;
    l.heavy = reinterpret_cast<uint32_t *>(take(sizeof(uint32_t) * (size_t)hcap));
    l.heavy_cap = hcap;
    l.heavy_len = (uint32_t)(p.heavy_len > 0 ? p.heavy_len : 0);
    l.entries = reinterpret_cast<SplitEntry *>(take(sizeof(SplitEntry) * (size_t)cap));
    l.state = reinterpret_cast<float4 *>(take(sizeof(float4) * kTilePixels * (size_t)cap));
    l.state_last = reinterpret_cast<uint32_t *>(take(sizeof(uint32_t) * kTilePixels * (size_t)cap));
    l.part = reinterpret_cast<float4 *>(take(sizeof(float4) * kTilePixels * (size_t)cap * K));
    l.part_last = reinterpret_cast<uint32_t *>(take(sizeof(uint32_t) * kTilePixels * (size_t)cap * K));
    l.cap = cap;
    l.K = K;
    if (out) *out = l;
    return off;
}

size_t balance_ws_bytes(const gs_balance_params &p) { return carve_balance_ws(nullptr, p, nullptr); }

cudaError_t launch_render_batch_balanced(const gs_render_batch_desc *desc, uint32_t *counter,
                                         const gs_balance_params &p, void *workspace, int grid,
                                         cudaStream_t stream) {
    SplitLayout sl;
    carve_balance_ws(static_cast<char *>(workspace), p, &sl);
    cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(uint32_t), stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(sl.n_entries, 0, 16, stream);  // queue counts, chunk counter
    if (e != cudaSuccess) return e;
    if (grid <= 0 && (e = batch_wave(&grid)) != cudaSuccess) return e;
    const bool heavy = p.heavy_len > 0 && p.max_heavy_tiles > 0, split = p.budget > 0 && p.max_split_tiles > 0;
    const uint32_t rounds = split ? ((uint32_t)p.budget + kBatch - 1) / kBatch : 0xffffffffu;
    const uint32_t chunk = ((uint32_t)p.chunk + kBatch - 1) / kBatch * kBatch;
    if (heavy) classify_kernel<<<grid, 256, 0, stream>>>(desc, sl);
    if (heavy && split)
        render_batch_kernel<true, true><<<grid, kThreads, 0, stream>>>(desc, counter, sl, rounds);
    else if (heavy)
        render_batch_kernel<false, true><<<grid, kThreads, 0, stream>>>(desc, counter, sl, rounds);
    else if (split)
        render_batch_kernel<true, false><<<grid, kThreads, 0, stream>>>(desc, counter, sl, rounds);
    else
        render_batch_kernel<false, false><<<grid, kThreads, 0, stream>>>(desc, counter, sl, rounds);
    if (split) {
        split_chunk_kernel<<<grid, kThreads, 0, stream>>>(desc, sl, chunk);
        split_merge_kernel<<<grid, kThreads, 0, stream>>>(desc, sl, chunk);
    }
    return cudaGetLastError();
}

}  // namespace gs
