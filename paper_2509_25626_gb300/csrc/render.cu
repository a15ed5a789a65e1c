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

// Renders one tile with the whole block.  Every thread must call it; it
// begins and ends with block-wide barriers, so the shared memory may be
// reused for the next tile.  The job's pointers and sizes are read where
// they are used, not held in registers: the batch kernel keeps its job in
// shared memory, the single-image kernel in its parameters.
template <bool kCount, bool kDepth>
__device__ __forceinline__ void render_tile(RenderSmem &sm, const gs_render_job &job, const uint2 range, int tile,
                                            float *__restrict__ invdepth, uint32_t *__restrict__ n_eval,
                                            uint32_t *__restrict__ tile_cycles) {
    long long t_start = 0;
    if (kCount) t_start = clock64();
    const int width = job.width, tiles_x = (width + kTile - 1) / kTile;
    StagedA *s_a = sm.a;
    StagedB *s_b = sm.b;
    float *s_c = sm.c;
    uint8_t *s_mask = sm.mask;
    uint8_t(*s_list)[kBatch] = sm.list;

    const int tx = tile % tiles_x, ty = tile / tiles_x;
    const unsigned lane = lane_id(), warp = threadIdx.x >> 5;
    const int bx0 = tx * kTile + (int)(warp & 1u) * 8, by0 = ty * kTile + (int)(warp >> 1) * 8;
    const int px = bx0 + 2 * (int)(lane & 3u), py = by0 + (int)(lane >> 2);
    const float pxf = (float)px, pyf = (float)py;
    const bool in0 = px < width && py < job.height, in1 = px + 1 < width && py < job.height;
    Pixel p0{1.f, 0.f, 0.f, 0.f, 0.f, 0u, 0u, !in0};
    Pixel p1{1.f, 0.f, 0.f, 0.f, 0.f, 0u, 0u, !in1};

    // corners of the tile, for the per-warp culling masks
    const float tx0 = (float)(tx * kTile), ty0 = (float)(ty * kTile);
    const unsigned lt = lanemask_lt();

    for (uint32_t base = range.x; base < range.y; base += kBatch) {
        // every thread has finished the previous round; stop if all pixels are done
        if (__syncthreads_and(p0.done && p1.done)) break;
#pragma unroll
        for (int r = 0; r < kBatch / kThreads; ++r) {
            const int k = (int)threadIdx.x + r * kThreads;
            const uint32_t i = base + (uint32_t)k;
            uint32_t m = 0;
            if (i < range.y) {
                // read-only path: the batch kernel takes these pointers from memory
                const float4 *src = reinterpret_cast<const float4 *>(job.splats + __ldg(job.vals + i));
                const float4 a = __ldg(src), b = __ldg(src + 1), c = __ldg(src + 2);
                s_a[k] = StagedA{a.x, a.y, a.z, a.w};
                s_b[k] = StagedB{b.x, b.y, b.z, b.w};
                s_c[k] = c.x;
                if (kDepth) sm.iz[k] = __frcp_rn(__ldg(reinterpret_cast<const float *>(src + 3)));
                m = quarter_mask(a, b, c, tx0, ty0);
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

        const uint32_t pos0 = base - range.x + 1;  // list position of staged splat 0
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

    const size_t plane = (size_t)width * job.height;
    const uint32_t len = range.y - range.x;
    float *__restrict__ out_color = job.out_color;
    const float bg_r = job.bg[0], bg_g = job.bg[1], bg_b = job.bg[2];
    if (in0) {
        const size_t pix = (size_t)py * width + px;
        out_color[pix] = fmaf(p0.T, bg_r, p0.c0);
        out_color[plane + pix] = fmaf(p0.T, bg_g, p0.c1);
        out_color[2 * plane + pix] = fmaf(p0.T, bg_b, p0.c2);
        job.final_T[pix] = p0.T;
        job.n_contrib[pix] = p0.last;
        if (kCount) n_eval[pix] = p0.stop ? p0.stop : len;
        if (kDepth) invdepth[pix] = p0.id;
    }
    if (in1) {
        const size_t pix = (size_t)py * width + px + 1;
        out_color[pix] = fmaf(p1.T, bg_r, p1.c0);
        out_color[plane + pix] = fmaf(p1.T, bg_g, p1.c1);
        out_color[2 * plane + pix] = fmaf(p1.T, bg_b, p1.c2);
        job.final_T[pix] = p1.T;
        job.n_contrib[pix] = p1.last;
        if (kCount) n_eval[pix] = p1.stop ? p1.stop : len;
        if (kDepth) invdepth[pix] = p1.id;
    }
    __syncthreads();  // shared memory free for the next tile
    if (kCount && tile_cycles != nullptr && threadIdx.x == 0) {
        const long long dt = clock64() - t_start;
        tile_cycles[tile] = dt < 0 ? 0u : (dt > 0xffffffffll ? 0xffffffffu : (uint32_t)dt);
    }
}

template <bool kCount, bool kDepth>
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
    render_tile<kCount, kDepth>(sm, job, ranges[blockIdx.x], blockIdx.x, invdepth, n_eval, tile_cycles);
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
__global__ void __launch_bounds__(kThreads, 10) render_batch_kernel(const gs_render_batch_desc *__restrict__ desc,
                                                                uint32_t *__restrict__ counter) {
    constexpr int kJobsCached = 64;  // job tables up to this size live in shared memory
    constexpr int kJobWords = (int)(sizeof(gs_render_job) / 4);
    static_assert(sizeof(gs_render_job) % 4 == 0 && kJobWords <= kThreads, "job copy");
    __shared__ RenderSmem sm;
    __shared__ gs_render_job s_jobs[kJobsCached];
    __shared__ uint32_t s_w;
    const int n_jobs = desc->n_jobs;
    const uint32_t total = desc->total_tiles;
    const bool cached = n_jobs <= kJobsCached;  // uniform
    if (cached)
        for (int i = threadIdx.x; i < n_jobs * kJobWords; i += kThreads)
            reinterpret_cast<uint32_t *>(s_jobs)[i] = reinterpret_cast<const uint32_t *>(desc->jobs)[i];
    if (threadIdx.x == 0) s_w = atomicAdd(counter, 1u);
    __syncthreads();
    for (uint32_t w = s_w; w < total;) {
        uint32_t next = 0;
        if (threadIdx.x == 0) next = atomicAdd(counter, 1u);
        int lo = 0, hi = n_jobs;  // last job with tile_begin <= w
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
            // the previous tile ended with a barrier, so slot 0 is free
            if (threadIdx.x < kJobWords)
                reinterpret_cast<uint32_t *>(&s_jobs[0])[threadIdx.x] =
                    reinterpret_cast<const uint32_t *>(&desc->jobs[lo])[threadIdx.x];
            __syncthreads();
            lo = 0;
        }
        const gs_render_job &job = s_jobs[lo];
        const int tile = (int)(w - job.tile_begin);
        render_tile<false, false>(sm, job, reinterpret_cast<const uint2 *>(job.ranges)[tile], tile, nullptr, nullptr,
                                  nullptr);
        // render_tile ended with a barrier: nobody reads s_w any more
        if (threadIdx.x == 0) s_w = next;
        __syncthreads();
        w = s_w;
    }
}

}  // namespace

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

cudaError_t launch_render_batch(const gs_render_batch_desc *desc, uint32_t *counter, int grid, cudaStream_t stream) {
    cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(uint32_t), stream);
    if (e != cudaSuccess) return e;
    if (grid <= 0) {
        // one full wave; looked up on the first call per device (make that
        // call outside stream capture) and cached
        static int wave[64] = {0};
        int dev = 0;
        e = cudaGetDevice(&dev);
        if (e != cudaSuccess) return e;
        if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
        if (wave[dev] == 0) {
            int sms = 0, per_sm = 0;
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, render_batch_kernel, kThreads, 0);
            wave[dev] = (sms > 0 ? sms : 1) * (per_sm > 0 ? per_sm : 1);
        }
        grid = wave[dev];
    }
    render_batch_kernel<<<grid, kThreads, 0, stream>>>(desc, counter);
    return cudaGetLastError();
}

}  // namespace gs
