// Backward of the forward pass: gradients of a loss L(image) with respect to
// the scene parameters, given dL/d(image).
//
// render_backward_kernel: per 16x16 tile (same block shape, pixel mapping
// and alpha >= 1/255 culling as the forward render), each pixel walks its
// list back to front from its n_contrib (the last splat it blended),
// recovering the transmittance in front of each blended splat from final_T
// by T_before = T_after / (1 - alpha), and the colour accumulated behind it
// by A <- alpha c + (1 - alpha) A (starting from the background).  With
// C = sum_i c_i alpha_i T_i + T_final bg (Eq. 1):
//     dL/dc_i     = alpha_i T_i dL/dC
//     dL/dalpha_i = T_i (c_i - A_i) . dL/dC
// and alpha = min(0.99, o exp(power)), power = -(a dx^2 + c dy^2)/2 - b dx dy.
// Per splat the gradients with respect to its pixel-space mean, conic
// (a, b, c), opacity and colour are summed over the warp (shuffles), over
// the block (shared atomics) and then into global memory (one atomic per
// value per block).  No per-pixel or per-splat state is stored by the
// forward beyond final_T and n_contrib.
//
// preprocess_backward_kernel: per Gaussian, the chain rule through the
// forward's preprocessing: conic -> Sigma' (dSigma' = -Q G Q), Sigma' =
// A A^T + 0.3 I with A = J W R S, the EWA Jacobian's dependence on the
// view-space mean (with the frustum clamp), the projection of the mean, the
// SH colour (clamped channels pass no gradient) and its viewing direction,
// and the sigmoid of the opacity.
#include "common.cuh"

namespace gs {

namespace {

constexpr int kThreads = 128;
constexpr int kBatch = 128;
constexpr int kWarps = kThreads / 32;
constexpr int kNGrad = 9;  // x, y, a, b, c, opacity, r, g, b
constexpr float kLn2 = 0.6931471805599453f;

struct __align__(16) StagedA { float x, y, w00, w01; };
struct __align__(16) StagedB { float w11, lg2o, r, g; };

// Sums 8 per-lane values over the warp with 7 shuffles instead of 8 x 5: at
// each of the offsets 16, 8, 4 a lane keeps one half of its values (the
// upper half if its offset bit is set), adds its partner's copy of that half
// and passes the other half on; offsets 2 and 1 finish.  On return v[0] is
// the warp sum of value 4 b4 + 2 b3 + b2 (b_i = bit i of the lane), that is
// of value lane >> 2, the same in the four lanes of each group.
__device__ __forceinline__ float warp_sum8(float (&v)[8], unsigned lane) {
#pragma unroll
    for (int n = 8, off = 16; n > 1; n >>= 1, off >>= 1) {
        const bool hi = (lane & (unsigned)off) != 0u;
#pragma unroll
        for (int i = 0; i < n / 2; ++i) {
            const float send = hi ? v[i] : v[i + n / 2];
            const float keep = hi ? v[i + n / 2] : v[i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, off);
        }
    }
    v[0] += __shfl_xor_sync(0xffffffffu, v[0], 2);
    return v[0] + __shfl_xor_sync(0xffffffffu, v[0], 1);
}

__device__ __forceinline__ float warp_sum(float x) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) x += __shfl_xor_sync(0xffffffffu, x, off);
    return x;
}

struct PixelBack {
    float T;        // transmittance behind the current splat (starts at final_T)
    float A0, A1, A2;  // colour accumulated behind the current splat
    float g0, g1, g2;  // dL/dC of this pixel
    uint32_t last;  // n_contrib
};

// One pixel's contribution for one splat at list position `pos`; adds to g[9].
// arg = log2 alpha before the clamp, computed exactly as the forward does,
// so the skip decision (taken on it, as in the forward) is the forward's.
// inv_o = 1 / opacity.
__device__ __forceinline__ void back_pixel(PixelBack &p, uint32_t pos, float u, float v, float dx, float dy,
                                           float arg, float w00, float w01, float w11, float r, float g, float b,
                                           float inv_o, float *acc) {
    if (pos > p.last) return;
    if (!(arg >= -kLog2_255)) return;  // alpha < 1/255: skipped by the forward
    const float raw = ex2_approx(arg);
    const float alpha = fminf(kAlphaMax, raw);
    const float om = 1.0f - alpha;  // >= 0.01
    const float Tb = __fdividef(p.T, om);  // transmittance in front of this splat
    const float wgt = alpha * Tb;
    acc[6] = fmaf(wgt, p.g0, acc[6]);
    acc[7] = fmaf(wgt, p.g1, acc[7]);
    acc[8] = fmaf(wgt, p.g2, acc[8]);
    const float dL_dalpha = Tb * ((r - p.A0) * p.g0 + (g - p.A1) * p.g1 + (b - p.A2) * p.g2);
    p.A0 = fmaf(alpha, r - p.A0, p.A0);
    p.A1 = fmaf(alpha, g - p.A1, p.A1);
    p.A2 = fmaf(alpha, b - p.A2, p.A2);
    p.T = Tb;
    if (raw > kAlphaMax) return;  // clamped: alpha does not depend on o or power
    // alpha = o G, G = exp(power): dL/do = dL/dalpha G, dL/dpower = dL/dalpha alpha
    acc[5] = fmaf(dL_dalpha, raw * inv_o, acc[5]);
    const float gp = dL_dalpha * alpha;
    // Q d = 2 ln2 W^T (u, v): d power / d mean = -Q d
    const float qx = 2.0f * kLn2 * (w00 * u), qy = 2.0f * kLn2 * fmaf(w01, u, w11 * v);
    acc[0] = fmaf(-gp, qx, acc[0]);
    acc[1] = fmaf(-gp, qy, acc[1]);
    acc[2] = fmaf(-0.5f * gp, dx * dx, acc[2]);
    acc[3] = fmaf(-gp, dx * dy, acc[3]);
    acc[4] = fmaf(-0.5f * gp, dy * dy, acc[4]);
}

__global__ void __launch_bounds__(kThreads) render_backward_kernel(
    const gs_splat *__restrict__ splats, const uint32_t *__restrict__ vals, const uint2 *__restrict__ ranges,
    int width, int height, int tiles_x, float bg_r, float bg_g, float bg_b, const float *__restrict__ final_T,
    const uint32_t *__restrict__ n_contrib, const float *__restrict__ dL_dcolor, float *__restrict__ dsplat) {
    __shared__ StagedA s_a[kBatch];
    __shared__ StagedB s_b[kBatch];
    __shared__ float s_c[kBatch];
    __shared__ float s_o[kBatch];
    __shared__ uint32_t s_gid[kBatch];
    __shared__ uint8_t s_mask[kBatch];
    __shared__ uint8_t s_list[kWarps][kBatch];
    __shared__ float s_grad[kBatch][kNGrad];
    __shared__ uint32_t s_maxlast;

    const int tile = blockIdx.x;
    const int tx = tile % tiles_x, ty = tile / tiles_x;
    const unsigned lane = lane_id(), warp = threadIdx.x >> 5;
    const int bx0 = tx * kTile + (int)(warp & 1u) * 8, by0 = ty * kTile + (int)(warp >> 1) * 8;
    const int px = bx0 + 2 * (int)(lane & 3u), py = by0 + (int)(lane >> 2);
    const float pxf = (float)px, pyf = (float)py;
    const bool in0 = px < width && py < height, in1 = px + 1 < width && py < height;
    const size_t plane = (size_t)width * height;
    PixelBack p0{1.f, bg_r, bg_g, bg_b, 0.f, 0.f, 0.f, 0u}, p1 = p0;
    if (in0) {
        const size_t pix = (size_t)py * width + px;
        p0.T = final_T[pix];
        p0.last = n_contrib[pix];
        p0.g0 = dL_dcolor[pix];
        p0.g1 = dL_dcolor[plane + pix];
        p0.g2 = dL_dcolor[2 * plane + pix];
    }
    if (in1) {
        const size_t pix = (size_t)py * width + px + 1;
        p1.T = final_T[pix];
        p1.last = n_contrib[pix];
        p1.g0 = dL_dcolor[pix];
        p1.g1 = dL_dcolor[plane + pix];
        p1.g2 = dL_dcolor[2 * plane + pix];
    }
    if (threadIdx.x == 0) s_maxlast = 0;
    __syncthreads();
    atomicMax(&s_maxlast, max(p0.last, p1.last));
    __syncthreads();
    const uint2 range = ranges[tile];
    const uint32_t max_last = min(s_maxlast, range.y - range.x);  // n_contrib never exceeds the list
    const uint32_t wlast = __reduce_max_sync(0xffffffffu, max(p0.last, p1.last));
    const float tx0 = (float)(tx * kTile), ty0 = (float)(ty * kTile);
    const unsigned lt = lanemask_lt();

    // rounds over list positions (start, end], from the back
    for (int64_t end = max_last; end > 0; end -= kBatch) {
        const uint32_t start = (uint32_t)(end > kBatch ? end - kBatch : 0);
        const uint32_t cnt = (uint32_t)end - start;
        __syncthreads();  // previous round's shared data fully consumed
        for (int k = threadIdx.x; k < kBatch * kNGrad; k += kThreads) (&s_grad[0][0])[k] = 0.f;
        {
            const int k = threadIdx.x;
            uint32_t m = 0;
            if ((uint32_t)k < cnt) {
                const uint32_t gid = vals[range.x + start + k];
                const float4 *src = reinterpret_cast<const float4 *>(splats + gid);
                const float4 a = src[0], b = src[1], c = src[2];
                s_a[k] = StagedA{a.x, a.y, a.z, a.w};
                s_b[k] = StagedB{b.x, b.y, b.z, b.w};
                s_c[k] = c.x;
                s_o[k] = ex2_approx(-b.y);  // 1 / opacity
                s_gid[k] = gid;
                m = quarter_mask(a, b, c, tx0, ty0);
            }
            s_mask[k] = (uint8_t)m;
        }
        __syncthreads();
        uint32_t wcnt = 0;
#pragma unroll
        for (int c = 0; c < kBatch / 32; ++c) {
            const uint32_t bit = (s_mask[c * 32 + lane] >> warp) & 1u;
            const unsigned bal = __ballot_sync(0xffffffffu, bit);
            if (bit) s_list[warp][wcnt + __popc(bal & lt)] = (uint8_t)(c * 32 + lane);
            wcnt += __popc(bal);
        }
        __syncwarp();
#pragma unroll 4
        for (int q = (int)wcnt - 1; q >= 0; --q) {
            const uint32_t j = s_list[warp][q];
            const uint32_t pos = start + j + 1;
            if (pos > wlast) continue;  // warp-uniform: no pixel of this warp reached it
            const StagedA sa = s_a[j];
            const StagedB sb = s_b[j];
            const float b = s_c[j], inv_o = s_o[j];
            const float dy = sa.y - pyf;
            const float dx0 = sa.x - pxf, dx1 = dx0 - 1.0f;
            const float t = sa.w01 * dy;
            const float u0 = fmaf(sa.w00, dx0, t);
            const float u1 = u0 - sa.w00;
            const float v = sb.w11 * dy;
            const float vv = fmaf(-v, v, sb.lg2o);
            float acc[kNGrad];
#pragma unroll
            for (int k = 0; k < kNGrad; ++k) acc[k] = 0.f;
            back_pixel(p0, pos, u0, v, dx0, dy, fmaf(-u0, u0, vv), sa.w00, sa.w01, sb.w11, sb.r, sb.g, b, inv_o, acc);
            back_pixel(p1, pos, u1, v, dx1, dy, fmaf(-u1, u1, vv), sa.w00, sa.w01, sb.w11, sb.r, sb.g, b, inv_o, acc);
            const bool any = acc[6] != 0.f || acc[7] != 0.f || acc[8] != 0.f || acc[5] != 0.f || acc[0] != 0.f;
            if (__any_sync(0xffffffffu, any)) {
                // values 0-7 by halving (lane group lane >> 2 holds value lane >> 2),
                // value 8 by a plain butterfly; one shared atomic per value
                float v8[8];
#pragma unroll
                for (int k = 0; k < 8; ++k) v8[k] = acc[k];
                const float sum = warp_sum8(v8, lane);
                const float sum8 = warp_sum(acc[8]);
                const bool first = (lane & 3u) == 0u;
                if (first || lane == 1u) atomicAdd(&s_grad[j][first ? lane >> 2 : 8u], first ? sum : sum8);
            }
        }
        __syncthreads();
        for (int k = threadIdx.x; k < (int)cnt * kNGrad; k += kThreads) {
            const float g = (&s_grad[0][0])[k];
            if (g != 0.f) atomicAdd(&dsplat[(size_t)s_gid[k / kNGrad] * 12 + (k % kNGrad)], g);
        }
    }
}

// SH constants (Condon-Shortley phase), as in the forward.
constexpr float kSH0 = 0.28209479177387814f;
constexpr float kSH1 = 0.4886025119029199f;
constexpr float kSH2a = 1.0925484305920792f;
constexpr float kSH2b = 0.31539156525252005f;
constexpr float kSH2c = 0.5462742152960396f;
constexpr float kSH3a = 0.5900435899266435f;
constexpr float kSH3b = 2.890611442640554f;
constexpr float kSH3c = 0.4570457994644658f;
constexpr float kSH3d = 0.3731763325901154f;
constexpr float kSH3e = 1.445305721320277f;

constexpr int kPreBackThreads = 128;
constexpr int kShStride = 49;  // 48 floats + 1: rows start in different banks

// A visible Gaussian's inputs to the backward, loaded before its SH
// coefficients are staged so that both sets of loads are in flight at once.
struct GaussIn {
    float G[9];  // dL/d(x, y, conic a, b, c, opacity, r, g, b)
    float m[3], ls[3], logit;
    float4 q;
};

__device__ __forceinline__ GaussIn load_gauss_in(const float *__restrict__ means, const float *__restrict__ log_scales,
                                                 const float4 *__restrict__ quats, const float *__restrict__ logits,
                                                 const float *__restrict__ dsplat, int64_t gi) {
    GaussIn in;
    const float *G = dsplat + 12 * gi;
#pragma unroll
    for (int k = 0; k < 9; ++k) in.G[k] = G[k];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        in.m[k] = means[3 * gi + k];
        in.ls[k] = log_scales[3 * gi + k];
    }
    in.q = quats[gi];
    in.logit = logits[gi];
    return in;
}

__device__ __forceinline__ void preprocess_backward_one(const GaussIn &in, float *shg, int64_t gi, int sh_degree,
                                                        const CamParams &cam, uint32_t tiles,
                                                        float *__restrict__ dmeans, float *__restrict__ dlog_scales,
                                                        float *__restrict__ dquats, float *__restrict__ dlogits);

// 6 blocks per SM (80 registers): with the inputs held across the SH
// staging the kernel would take 92 registers and 5 blocks, measured slower.
#ifndef GS_PREBACK_MIN_BLOCKS
#define GS_PREBACK_MIN_BLOCKS 6
#endif
#define GS_PREBACK_BOUNDS __launch_bounds__(kPreBackThreads, GS_PREBACK_MIN_BLOCKS)
__global__ void GS_PREBACK_BOUNDS preprocess_backward_kernel(
    const float *__restrict__ means, const float *__restrict__ log_scales, const float4 *__restrict__ quats,
    const float *__restrict__ logits, const float *__restrict__ sh, int64_t n, int sh_degree, CamParams cam,
    const gs_splat *__restrict__ splats, const float *__restrict__ dsplat, float *__restrict__ dmeans,
    float *__restrict__ dlog_scales, float *__restrict__ dquats, float *__restrict__ dlogits,
    float *__restrict__ dsh) {
    // The block's SH coefficients pass through shared memory both ways, so
    // global loads and stores are coalesced (one thread's 48 floats span 192
    // bytes); a thread reads its own row and overwrites it with its gradient.
    __shared__ float s_sh[kPreBackThreads][kShStride];
    __shared__ uint32_t s_tiles[kPreBackThreads];
    const int64_t g0 = (int64_t)blockIdx.x * kPreBackThreads;
    const int nb = (int)min((int64_t)kPreBackThreads, n - g0);  // Gaussians of this block
    // visibility first, from the dense copy of the sort inputs (16 bytes per
    // Gaussian, not a word of each 64-byte record): a culled Gaussian's SH
    // coefficients are never read (its gradients are zeros)
    const uint4 *sort_in = reinterpret_cast<const uint4 *>(splats + n);
    if ((int)threadIdx.x < nb) s_tiles[threadIdx.x] = __ldg(&sort_in[g0 + threadIdx.x].y);
    __syncthreads();
    const int64_t gi = g0 + threadIdx.x;
    GaussIn in{};
    if (gi < n && s_tiles[threadIdx.x]) in = load_gauss_in(means, log_scales, quats, logits, dsplat, gi);
    // full blocks with 16-byte aligned SH arrays move them as float4, all 12
    // loads of a thread in flight at once
    const bool vec = nb == kPreBackThreads &&
                     ((reinterpret_cast<uintptr_t>(sh) | reinterpret_cast<uintptr_t>(dsh)) & 15u) == 0u;
    if (vec) {
        const float4 *src = reinterpret_cast<const float4 *>(sh + g0 * 48);
        float4 v[12];
#pragma unroll
        for (int r = 0; r < 12; ++r) {
            const int f4 = (int)threadIdx.x + r * kPreBackThreads;
            v[r] = s_tiles[(4 * f4) / 48] ? __ldg(src + f4) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int r = 0; r < 12; ++r) {
            const int f = 4 * ((int)threadIdx.x + r * kPreBackThreads), row = f / 48, col = f % 48;
            s_sh[row][col] = v[r].x;
            s_sh[row][col + 1] = v[r].y;
            s_sh[row][col + 2] = v[r].z;
            s_sh[row][col + 3] = v[r].w;
        }
    } else {
        for (int f = threadIdx.x; f < nb * 48; f += kPreBackThreads)
            s_sh[f / 48][f % 48] = s_tiles[f / 48] ? sh[g0 * 48 + f] : 0.f;
    }
    __syncthreads();
    if (gi < n)
        preprocess_backward_one(in, s_sh[threadIdx.x], gi, sh_degree, cam, s_tiles[threadIdx.x], dmeans, dlog_scales,
                                dquats, dlogits);
    __syncthreads();
    if (vec) {
        float4 *dst = reinterpret_cast<float4 *>(dsh + g0 * 48);
#pragma unroll
        for (int r = 0; r < 12; ++r) {
            const int f4 = (int)threadIdx.x + r * kPreBackThreads, f = 4 * f4, row = f / 48, col = f % 48;
            dst[f4] = make_float4(s_sh[row][col], s_sh[row][col + 1], s_sh[row][col + 2], s_sh[row][col + 3]);
        }
    } else {
        for (int f = threadIdx.x; f < nb * 48; f += kPreBackThreads) dsh[g0 * 48 + f] = s_sh[f / 48][f % 48];
    }
}

// The real SH basis function k (degree <= 3, Condon-Shortley phase, k =
// l^2 + l + m) at the unit direction (x, y, z), and its gradient with
// respect to the direction, in Cartesian form; xx, yy, zz are the squares.
// k is a constant after unrolling, so only one branch survives (the basis
// values are not kept in arrays, which put them in local memory).
__device__ __forceinline__ void sh_term(int k, float x, float y, float z, float xx, float yy, float zz, float &Y,
                                        float &gx, float &gy, float &gz) {
    gx = gy = gz = 0.f;
    switch (k) {
        case 0: Y = kSH0; break;
        case 1: Y = -kSH1 * y; gy = -kSH1; break;
        case 2: Y = kSH1 * z; gz = kSH1; break;
        case 3: Y = -kSH1 * x; gx = -kSH1; break;
        case 4: Y = kSH2a * x * y; gx = kSH2a * y; gy = kSH2a * x; break;
        case 5: Y = -kSH2a * y * z; gy = -kSH2a * z; gz = -kSH2a * y; break;
        case 6: Y = kSH2b * (2.f * zz - xx - yy); gx = -2.f * kSH2b * x; gy = -2.f * kSH2b * y; gz = 4.f * kSH2b * z; break;
        case 7: Y = -kSH2a * x * z; gx = -kSH2a * z; gz = -kSH2a * x; break;
        case 8: Y = kSH2c * (xx - yy); gx = 2.f * kSH2c * x; gy = -2.f * kSH2c * y; break;
        case 9: Y = -kSH3a * y * (3.f * xx - yy); gx = -6.f * kSH3a * x * y; gy = -3.f * kSH3a * (xx - yy); break;
        case 10: Y = kSH3b * x * y * z; gx = kSH3b * y * z; gy = kSH3b * x * z; gz = kSH3b * x * y; break;
        case 11:
            Y = -kSH3c * y * (4.f * zz - xx - yy);
            gx = 2.f * kSH3c * x * y;
            gy = -kSH3c * (4.f * zz - xx - 3.f * yy);
            gz = -8.f * kSH3c * y * z;
            break;
        case 12:
            Y = kSH3d * z * (2.f * zz - 3.f * xx - 3.f * yy);
            gx = -6.f * kSH3d * x * z;
            gy = -6.f * kSH3d * y * z;
            gz = kSH3d * (6.f * zz - 3.f * xx - 3.f * yy);
            break;
        case 13:
            Y = -kSH3c * x * (4.f * zz - xx - yy);
            gx = -kSH3c * (4.f * zz - 3.f * xx - yy);
            gy = 2.f * kSH3c * x * y;
            gz = -8.f * kSH3c * x * z;
            break;
        case 14: Y = kSH3e * z * (xx - yy); gx = 2.f * kSH3e * x * z; gy = -2.f * kSH3e * y * z; gz = kSH3e * (xx - yy); break;
        default: Y = -kSH3a * x * (xx - 3.f * yy); gx = -3.f * kSH3a * (xx - yy); gy = 6.f * kSH3a * x * y; break;
    }
}

// One Gaussian of preprocess_backward_kernel; shg: its 48 SH coefficients,
// replaced by their gradients on return.
__device__ __forceinline__ void preprocess_backward_one(const GaussIn &in, float *shg, int64_t gi, int sh_degree,
                                                        const CamParams &cam, uint32_t tiles,
                                                        float *__restrict__ dmeans, float *__restrict__ dlog_scales,
                                                        float *__restrict__ dquats, float *__restrict__ dlogits) {
    float *dm = dmeans + 3 * gi;
    float *dls = dlog_scales + 3 * gi;
    float *dq = dquats + 4 * gi;
    float *dshg = shg;
    if (tiles == 0u) {  // culled: appears in no list
        for (int k = 0; k < 3; ++k) dm[k] = dls[k] = 0.f;
        for (int k = 0; k < 4; ++k) dq[k] = 0.f;
        dlogits[gi] = 0.f;
        for (int k = 0; k < 48; ++k) dshg[k] = 0.f;
        return;
    }
    const float *G = in.G;
    const float gx = G[0], gy = G[1], ga = G[2], gb = G[3], gc = G[4], gop = G[5];
    float grgb[3] = {G[6], G[7], G[8]};
    const float mx = in.m[0], my = in.m[1], mz = in.m[2];
    const float *V = cam.V;
    const float z = fmaf(V[10], mz, fmaf(V[9], my, fmaf(V[8], mx, V[11])));
    const float tx = fmaf(V[2], mz, fmaf(V[1], my, fmaf(V[0], mx, V[3])));
    const float ty = fmaf(V[6], mz, fmaf(V[5], my, fmaf(V[4], mx, V[7])));

    // forward recomputation
    const float4 q4 = in.q;
    const float qinv = 1.0f / sqrtf(q4.x * q4.x + q4.y * q4.y + q4.z * q4.z + q4.w * q4.w);
    const float qw = q4.x * qinv, qx = q4.y * qinv, qy = q4.z * qinv, qz = q4.w * qinv;
    const float s[3] = {expf(in.ls[0]), expf(in.ls[1]), expf(in.ls[2])};
    const float R[3][3] = {
        {1.f - 2.f * (qy * qy + qz * qz), 2.f * (qx * qy - qw * qz), 2.f * (qx * qz + qw * qy)},
        {2.f * (qx * qy + qw * qz), 1.f - 2.f * (qx * qx + qz * qz), 2.f * (qy * qz - qw * qx)},
        {2.f * (qx * qz - qw * qy), 2.f * (qy * qz + qw * qx), 1.f - 2.f * (qx * qx + qy * qy)},
    };
    float M[3][3];
    for (int i = 0; i < 3; ++i)
        for (int k = 0; k < 3; ++k) M[i][k] = R[i][k] * s[k];
    const float inv_z = 1.0f / z;
    const float limx = kFrustumSlack * cam.tan_fovx, limy = kFrustumSlack * cam.tan_fovy;
    const float rx = tx * inv_z, ry = ty * inv_z;
    const bool clx = fabsf(rx) > limx, cly = fabsf(ry) > limy;
    const float txc = fminf(limx, fmaxf(-limx, rx)) * z;
    const float tyc = fminf(limy, fmaxf(-limy, ry)) * z;
    const float J00 = cam.fx * inv_z, J02 = -cam.fx * txc * inv_z * inv_z;
    const float J11 = cam.fy * inv_z, J12 = -cam.fy * tyc * inv_z * inv_z;
    float T0[3], T1[3];
    for (int j = 0; j < 3; ++j) {
        T0[j] = fmaf(J00, V[j], J02 * V[8 + j]);
        T1[j] = fmaf(J11, V[4 + j], J12 * V[8 + j]);
    }
    float A0[3], A1[3];
    for (int k = 0; k < 3; ++k) {
        A0[k] = fmaf(T0[0], M[0][k], fmaf(T0[1], M[1][k], T0[2] * M[2][k]));
        A1[k] = fmaf(T1[0], M[0][k], fmaf(T1[1], M[1][k], T1[2] * M[2][k]));
    }
    const float s00 = fmaf(A0[0], A0[0], fmaf(A0[1], A0[1], A0[2] * A0[2])) + kDilation;
    const float s11 = fmaf(A1[0], A1[0], fmaf(A1[1], A1[1], A1[2] * A1[2])) + kDilation;
    const float s01 = fmaf(A0[0], A1[0], fmaf(A0[1], A1[1], A0[2] * A1[2]));
    const float det = s00 * s11 - s01 * s01;
    const float Qa = s11 / det, Qb = -s01 / det, Qc = s00 / det;

    // conic -> Sigma': P = -Q G Q, G = [[ga, gb/2], [gb/2, gc]]
    const float G01 = 0.5f * gb;
    const float QG00 = Qa * ga + Qb * G01, QG01 = Qa * G01 + Qb * gc;
    const float QG10 = Qb * ga + Qc * G01, QG11 = Qb * G01 + Qc * gc;
    const float P00 = -(QG00 * Qa + QG01 * Qb), P01 = -(QG00 * Qb + QG01 * Qc), P11 = -(QG10 * Qb + QG11 * Qc);
    // Sigma' = A A^T + 0.3 I: dA = 2 P A
    float dA0[3], dA1[3];
    for (int k = 0; k < 3; ++k) {
        dA0[k] = 2.f * (P00 * A0[k] + P01 * A1[k]);
        dA1[k] = 2.f * (P01 * A0[k] + P11 * A1[k]);
    }
    // A = T M
    float dT0[3], dT1[3], dM[3][3];
    for (int j = 0; j < 3; ++j) {
        dT0[j] = dA0[0] * M[j][0] + dA0[1] * M[j][1] + dA0[2] * M[j][2];
        dT1[j] = dA1[0] * M[j][0] + dA1[1] * M[j][1] + dA1[2] * M[j][2];
        for (int k = 0; k < 3; ++k) dM[j][k] = T0[j] * dA0[k] + T1[j] * dA1[k];
    }
    // M = R diag(s)
    float dR[3][3];
    for (int k = 0; k < 3; ++k) {
        float ds = 0.f;
        for (int j = 0; j < 3; ++j) {
            ds = fmaf(dM[j][k], R[j][k], ds);
            dR[j][k] = dM[j][k] * s[k];
        }
        dls[k] = ds * s[k];
    }
    // R(q^) -> q^ (derivatives of the rotation matrix entries)
    const float dqw = 2.f * (-qz * dR[0][1] + qy * dR[0][2] + qz * dR[1][0] - qx * dR[1][2] - qy * dR[2][0] +
                             qx * dR[2][1]);
    const float dqx = 2.f * (qy * dR[0][1] + qz * dR[0][2] + qy * dR[1][0] - 2.f * qx * dR[1][1] - qw * dR[1][2] +
                             qz * dR[2][0] + qw * dR[2][1] - 2.f * qx * dR[2][2]);
    const float dqy = 2.f * (-2.f * qy * dR[0][0] + qx * dR[0][1] + qw * dR[0][2] + qx * dR[1][0] + qz * dR[1][2] -
                             qw * dR[2][0] + qz * dR[2][1] - 2.f * qy * dR[2][2]);
    const float dqz = 2.f * (-2.f * qz * dR[0][0] - qw * dR[0][1] + qx * dR[0][2] + qw * dR[1][0] -
                             2.f * qz * dR[1][1] + qy * dR[1][2] + qx * dR[2][0] + qy * dR[2][1]);
    // normalisation q^ = q / |q|
    const float dot = dqw * qw + dqx * qx + dqy * qy + dqz * qz;
    dq[0] = (dqw - dot * qw) * qinv;
    dq[1] = (dqx - dot * qx) * qinv;
    dq[2] = (dqy - dot * qy) * qinv;
    dq[3] = (dqz - dot * qz) * qinv;

    // T = J W
    float dJ00 = 0.f, dJ02 = 0.f, dJ11 = 0.f, dJ12 = 0.f;
    for (int j = 0; j < 3; ++j) {
        dJ00 = fmaf(dT0[j], V[j], dJ00);
        dJ02 = fmaf(dT0[j], V[8 + j], dJ02);
        dJ11 = fmaf(dT1[j], V[4 + j], dJ11);
        dJ12 = fmaf(dT1[j], V[8 + j], dJ12);
    }
    // J(t), with the frustum clamp: J02 = -fx c_x / z with c_x = clamp(tx / z)
    float dtx = 0.f, dty = 0.f, dtz = 0.f;
    const float iz2 = inv_z * inv_z;
    dtz += dJ00 * (-cam.fx * iz2) + dJ11 * (-cam.fy * iz2);
    if (!clx) {
        dtx += dJ02 * (-cam.fx * iz2);
        dtz += dJ02 * (2.f * cam.fx * tx * iz2 * inv_z);
    } else {
        dtz += dJ02 * (-J02 * inv_z);
    }
    if (!cly) {
        dty += dJ12 * (-cam.fy * iz2);
        dtz += dJ12 * (2.f * cam.fy * ty * iz2 * inv_z);
    } else {
        dtz += dJ12 * (-J12 * inv_z);
    }
    // pixel mean
    dtx += gx * cam.fx * inv_z;
    dty += gy * cam.fy * inv_z;
    dtz -= (gx * cam.fx * tx + gy * cam.fy * ty) * iz2;
    // t = W m + t0
    float gm[3];
    for (int c = 0; c < 3; ++c) gm[c] = V[c] * dtx + V[4 + c] * dty + V[8 + c] * dtz;

    // colour
    float dx = mx - cam.campos[0], dy = my - cam.campos[1], dz = mz - cam.campos[2];
    const float inv_len = 1.0f / sqrtf(dx * dx + dy * dy + dz * dz);
    const float x = dx * inv_len, y = dy * inv_len, zz_ = dz * inv_len;
    const float xx = x * x, yy = y * y, zz = zz_ * zz_;
    const int ncoef = (sh_degree + 1) * (sh_degree + 1);
    // clamped channels (raw < 0) pass no gradient
    float raw[3] = {0.5f, 0.5f, 0.5f};
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        float Yk, gxk, gyk, gzk;
        sh_term(k, x, y, zz_, xx, yy, zz, Yk, gxk, gyk, gzk);
        if (k < ncoef)
            for (int ch = 0; ch < 3; ++ch) raw[ch] = fmaf(shg[3 * k + ch], Yk, raw[ch]);
    }
    for (int ch = 0; ch < 3; ++ch)
        if (raw[ch] < 0.f) grgb[ch] = 0.f;
    float gdx = 0.f, gdy = 0.f, gdz = 0.f;
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        float Yk, gxk, gyk, gzk;
        sh_term(k, x, y, zz_, xx, yy, zz, Yk, gxk, gyk, gzk);
        const bool on = k < ncoef;
        float gY = 0.f;
        for (int ch = 0; ch < 3; ++ch) {
            gY = fmaf(grgb[ch], on ? shg[3 * k + ch] : 0.f, gY);  // read before the gradient overwrites it
            dshg[3 * k + ch] = on ? grgb[ch] * Yk : 0.f;
        }
        gdx = fmaf(gY, gxk, gdx);
        gdy = fmaf(gY, gyk, gdy);
        gdz = fmaf(gY, gzk, gdz);
    }
    // dir = v / |v|: remove the radial part
    const float radial = gdx * x + gdy * y + gdz * zz_;
    gm[0] += (gdx - radial * x) * inv_len;
    gm[1] += (gdy - radial * y) * inv_len;
    gm[2] += (gdz - radial * zz_) * inv_len;
    for (int c = 0; c < 3; ++c) dm[c] = gm[c];

    // opacity = sigmoid(logit)
    const float o = 1.0f / (1.0f + expf(-in.logit));
    dlogits[gi] = gop * o * (1.0f - o);
}

}  // namespace

// Per-splat 2D gradients: dsplat [n][12] zeroed, then accumulated per tile.
cudaError_t launch_render_backward_splats(int64_t n, const CamParams &cam, const gs_splat *splats,
                                          const uint32_t *vals, const uint32_t *ranges, const float bg[3],
                                          const float *final_T, const uint32_t *n_contrib, const float *dL_dcolor,
                                          float *dsplat, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(dsplat, 0, sizeof(float) * 12 * (size_t)(n > 0 ? n : 1), st);
    if (e != cudaSuccess) return e;
    const int num_tiles = cam.tiles_x * cam.tiles_y;
    render_backward_kernel<<<num_tiles, kThreads, 0, st>>>(splats, vals, reinterpret_cast<const uint2 *>(ranges),
                                                            cam.width, cam.height, cam.tiles_x, bg[0], bg[1], bg[2],
                                                            final_T, n_contrib, dL_dcolor, dsplat);
    return cudaGetLastError();
}

// The chain rule from the per-splat gradients to the scene parameters.
cudaError_t launch_preprocess_backward(const gs_scene &s, const CamParams &cam, const gs_splat *splats,
                                       const float *dsplat, const gs_scene_grads &g, cudaStream_t st) {
    if (s.n > 0)
        preprocess_backward_kernel<<<(unsigned)((s.n + kPreBackThreads - 1) / kPreBackThreads), kPreBackThreads, 0, st>>>(
            s.means, s.log_scales, reinterpret_cast<const float4 *>(s.quats), s.opacity_logits, s.sh, s.n,
            s.sh_degree, cam, splats, dsplat, g.dmeans, g.dlog_scales, g.dquats, g.dopacity_logits, g.dsh);
    return cudaGetLastError();
}

cudaError_t launch_render_backward(const gs_scene &s, const CamParams &cam, const gs_splat *splats,
                                   const uint32_t *vals, const uint32_t *ranges, const float bg[3],
                                   const float *final_T, const uint32_t *n_contrib, const float *dL_dcolor,
                                   float *dsplat, const gs_scene_grads &g, cudaStream_t st) {
    cudaError_t e = launch_render_backward_splats(s.n, cam, splats, vals, ranges, bg, final_T, n_contrib, dL_dcolor,
                                                  dsplat, st);
    if (e != cudaSuccess) return e;
    return launch_preprocess_backward(s, cam, splats, dsplat, g, st);
}

}  // namespace gs
