// Per-tile front-to-back alpha blending (Section II-B (2), Algorithm 1,
// Eq. 1 with the kernel's alpha and the Appendix B per-pixel rules).
//
// One 256-thread block per 16x16 tile, one pixel per thread.  The tile's
// splats are staged in shared memory in batches of 256 (each thread gathers
// one record), then every thread walks the batch front to back.  Exits are
// block-uniform (__syncthreads_and at the batch boundary), so no thread
// leaves while others still reach a barrier, and a pixel that stopped stays
// stopped across batches.
#include "common.cuh"

namespace gs {

namespace {

constexpr int kBatch = 256;

struct __align__(16) StagedA { float x, y, w00, w01; };
struct __align__(16) StagedB { float w11, lg2o, r, g; };

// kCount: also write, per pixel, how many splats were evaluated before the
// pixel stopped (the stopping one included) -- the work measure of the
// paper's workload characterisation (Table III).
template <bool kCount>
__global__ void __launch_bounds__(kTilePixels) render_kernel(const gs_splat *__restrict__ splats,
                                                             const uint32_t *__restrict__ vals,
                                                             const uint2 *__restrict__ ranges, int width, int height,
                                                             int tiles_x, float bg_r, float bg_g, float bg_b,
                                                             float *__restrict__ out_color,
                                                             float *__restrict__ final_T,
                                                             uint32_t *__restrict__ n_contrib,
                                                             uint32_t *__restrict__ n_eval) {
    __shared__ StagedA s_a[kBatch];
    __shared__ StagedB s_b[kBatch];
    __shared__ float s_c[kBatch];

    const int tile = blockIdx.x;
    const int tx = tile % tiles_x, ty = tile / tiles_x;
    const int px = tx * kTile + (threadIdx.x & (kTile - 1));
    const int py = ty * kTile + (threadIdx.x >> 4);
    const bool inside = px < width && py < height;
    const float pxf = (float)px, pyf = (float)py;

    const uint2 range = ranges[tile];
    float T = 1.0f, C0 = 0.f, C1 = 0.f, C2 = 0.f;
    uint32_t last = 0, evals = 0;
    bool done = !inside;

    for (uint32_t base = range.x; base < range.y; base += kBatch) {
        // every thread has finished the previous batch; stop if all pixels are done
        if (__syncthreads_and(done)) break;
        const uint32_t i = base + threadIdx.x;
        if (i < range.y) {
            const float4 *rec = reinterpret_cast<const float4 *>(splats + vals[i]);
            const float4 a = rec[0], b = rec[1], c = rec[2];
            s_a[threadIdx.x] = StagedA{a.x, a.y, a.z, a.w};
            s_b[threadIdx.x] = StagedB{b.x, b.y, b.z, b.w};
            s_c[threadIdx.x] = c.x;
        }
        __syncthreads();
        const int cnt = (int)min((uint32_t)kBatch, range.y - base);
        if (!done) {
            for (int j = 0; j < cnt; ++j) {
                if (kCount) ++evals;
                const StagedA sa = s_a[j];
                const StagedB sb = s_b[j];
                const float dx = sa.x - pxf, dy = sa.y - pyf;
                const float u = fmaf(sa.w00, dx, sa.w01 * dy);
                const float v = sb.w11 * dy;
                const float arg = fmaf(-u, u, fmaf(-v, v, sb.lg2o));
                const float alpha = fminf(kAlphaMax, ex2_approx(arg));
                if (alpha < kAlphaMin) continue;
                const float Tn = T * (1.0f - alpha);
                if (Tn < kTStop) {
                    done = true;
                    break;
                }
                const float w = alpha * T;
                C0 = fmaf(sb.r, w, C0);
                C1 = fmaf(sb.g, w, C1);
                C2 = fmaf(s_c[j], w, C2);
                T = Tn;
                last = base - range.x + j + 1;
            }
        }
    }
    if (inside) {
        const size_t pix = (size_t)py * width + px;
        const size_t plane = (size_t)width * height;
        out_color[pix] = fmaf(T, bg_r, C0);
        out_color[plane + pix] = fmaf(T, bg_g, C1);
        out_color[2 * plane + pix] = fmaf(T, bg_b, C2);
        final_T[pix] = T;
        n_contrib[pix] = last;
        if (kCount) n_eval[pix] = evals;
    }
}

}  // namespace

cudaError_t launch_render(const gs_splat *splats, const uint32_t *vals, const uint32_t *ranges, const CamParams &cam,
                          const float bg[3], float *out_color, float *final_T, uint32_t *n_contrib,
                          uint32_t *n_eval, cudaStream_t stream) {
    const int num_tiles = cam.tiles_x * cam.tiles_y;
    if (n_eval)
        render_kernel<true><<<num_tiles, kTilePixels, 0, stream>>>(
            splats, vals, reinterpret_cast<const uint2 *>(ranges), cam.width, cam.height, cam.tiles_x, bg[0], bg[1],
            bg[2], out_color, final_T, n_contrib, n_eval);
    else
        render_kernel<false><<<num_tiles, kTilePixels, 0, stream>>>(
            splats, vals, reinterpret_cast<const uint2 *>(ranges), cam.width, cam.height, cam.tiles_x, bg[0], bg[1],
            bg[2], out_color, final_T, n_contrib, nullptr);
    return cudaGetLastError();
}

}  // namespace gs
