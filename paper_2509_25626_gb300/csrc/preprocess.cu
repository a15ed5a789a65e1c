// Per-Gaussian preprocessing (Section II-B (1)): cull, EWA projection to a
// 2D splat, 3-sigma radius and tile rectangle, degree-3 SH colour.
//
// One thread per Gaussian; the kernel is bound by HBM (236 B read, 64 B
// written per Gaussian).  Numerics that differ from a literal transcription
// of the 3DGS formulas, chosen for FP32 accuracy:
//   * Sigma' = A A^T + 0.3 I with A = J W R S (2x3), and det(Sigma') from the
//     Cauchy-Binet sum of squared 2x2 minors of A plus 0.3 tr(A A^T) + 0.09:
//     every term is positive, so very thin splats keep an accurate inverse.
//   * mid^2 - det is formed as ((s00 - s11)/2)^2 + s01^2 (the same quantity
//     without cancellation).
//   * The inverse covariance is stored as an upper-triangular factor (see
//     gs_splat), so the render evaluates the exponent as a sum of two squares.
#include "common.cuh"

namespace gs {

namespace {

// Real SH normalisation constants (Condon-Shortley phase), l <= 3.
constexpr float kSH0 = 0.28209479177387814f;   // 1 / (2 sqrt(pi))
constexpr float kSH1 = 0.4886025119029199f;    // sqrt(3 / (4 pi))
constexpr float kSH2a = 1.0925484305920792f;   // sqrt(15 / pi) / 2
constexpr float kSH2b = 0.31539156525252005f;  // sqrt(5 / pi) / 4
constexpr float kSH2c = 0.5462742152960396f;   // sqrt(15 / pi) / 4
constexpr float kSH3a = 0.5900435899266435f;   // sqrt(35 / (2 pi)) / 4
constexpr float kSH3b = 2.890611442640554f;    // sqrt(105 / pi) / 2
constexpr float kSH3c = 0.4570457994644658f;   // sqrt(21 / (2 pi)) / 4
constexpr float kSH3d = 0.3731763325901154f;   // sqrt(7 / pi) / 4
constexpr float kSH3e = 1.445305721320277f;    // sqrt(105 / pi) / 4

// a*b - c*d with one rounding error in total (Kahan's fma formulation).
__device__ __forceinline__ float diff_of_products(float a, float b, float c, float d) {
    float cd = c * d;
    float err = fmaf(-c, d, cd);
    float dop = fmaf(a, b, -cd);
    return dop + err;
}

// A culled Gaussian appears in no tile list, so nothing reads its first 32
// bytes: only the radius, the empty cull box and the sort inputs are written.
__device__ __forceinline__ void write_culled(gs_splat *out, uint4 *sort_in, float depth) {
    float4 *o = reinterpret_cast<float4 *>(out);
    o[2] = make_float4(0.f, -1.f, -1.f, 0.f);     // b, cull box empty, radius = 0
    o[3] = make_float4(depth, 0.f, 0.f, 0.f);     // depth, tiles = 0, rect 0
    *sort_in = make_uint4(__float_as_uint(depth), 0u, 0u, 0u);
}

// The projection of Gaussian g (one thread).
__device__ __forceinline__ void preprocess_one(const int64_t g, const float *__restrict__ means,
                                               const float *__restrict__ log_scales, const float4 *__restrict__ quats,
                                               const float *__restrict__ logits, const float4 *__restrict__ sh,
                                               int sh_degree, const CamParams &cam, gs_splat *__restrict__ out,
                                               uint4 *__restrict__ sort_in) {
    // the rotation, scales and opacity of a Gaussian that survives the
    // near-plane test are needed next: start them towards L2 with the mean
    asm volatile("prefetch.global.L2 [%0];" ::"l"(quats + g));
    asm volatile("prefetch.global.L2 [%0];" ::"l"(log_scales + 3 * g));
    asm volatile("prefetch.global.L2 [%0];" ::"l"(logits + g));
    const float mx = means[3 * g], my = means[3 * g + 1], mz = means[3 * g + 2];
    const float *V = cam.V;

    // Depth in the exact form the sort key is defined with.
    const float z = fmaf(V[10], mz, fmaf(V[9], my, fmaf(V[8], mx, V[11])));
    if (!(z > kNearZ)) {
        write_culled(out + g, sort_in + g, z);
        return;
    }
    const float tx = fmaf(V[2], mz, fmaf(V[1], my, fmaf(V[0], mx, V[3])));
    const float ty = fmaf(V[6], mz, fmaf(V[5], my, fmaf(V[4], mx, V[7])));
    const float s0 = expf(log_scales[3 * g]), s1 = expf(log_scales[3 * g + 1]), s2 = expf(log_scales[3 * g + 2]);

    // Early, conservative frustum cull from the mean and the largest scale:
    // lambda_max(Sigma') <= trace(T T^T) max(s)^2 + 0.3 with T = J W (the
    // Frobenius norm bounds the spectral one), and the radius test below adds
    // at most sqrt(0.1) to lambda, so a Gaussian whose mean lies farther than
    // that bound outside the image has an empty rectangle.
    // Survivors are likely visible: start fetching their SH into L2 now, so
    // the loads after the covariance arithmetic find it there.
    {
        const float iz = 1.0f / z;
        const float lx = kFrustumSlack * cam.tan_fovx, ly = kFrustumSlack * cam.tan_fovy;
        const float cx_ = fminf(lx, fmaxf(-lx, tx * iz)), cy_ = fminf(ly, fmaxf(-ly, ty * iz));
        const float fxz = cam.fx * iz, fyz = cam.fy * iz;
        const float smax = fmaxf(s0, fmaxf(s1, s2));
        float tr = 0.f;  // |T row 0|^2 + |T row 1|^2, rows fx/z (W0 - cx W2), fy/z (W1 - cy W2)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const float a = fxz * fmaf(-cx_, V[8 + j], V[j]), b = fyz * fmaf(-cy_, V[8 + j], V[4 + j]);
            tr = fmaf(a, a, fmaf(b, b, tr));
        }
        const float r_ub = 3.0f * sqrtf(fmaf(tr, smax * smax, kDilation + 0.3163f)) * 1.01f + 2.0f;
        const float px_ = fmaf(cam.fx, tx * iz, cam.cx), py_ = fmaf(cam.fy, ty * iz, cam.cy);
        const float wimg = (float)(cam.tiles_x * kTile), himg = (float)(cam.tiles_y * kTile);
        if (px_ + r_ub < 0.f || py_ + r_ub < 0.f || px_ - r_ub > wimg || py_ - r_ub > himg) {
            write_culled(out + g, sort_in + g, z);
            return;
        }
        const char *shp = reinterpret_cast<const char *>(sh + 12 * g);
        asm volatile("prefetch.global.L2 [%0];" ::"l"(shp));
        asm volatile("prefetch.global.L2 [%0];" ::"l"(shp + 64));
        asm volatile("prefetch.global.L2 [%0];" ::"l"(shp + 128));
    }

    // R(q) S: rotation from the normalised quaternion, columns scaled.
    float4 q = quats[g];
    const float qinv = 1.0f / sqrtf(q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w);
    const float qw = q.x * qinv, qx = q.y * qinv, qy = q.z * qinv, qz = q.w * qinv;
    float M[3][3];
    M[0][0] = (1.f - 2.f * (qy * qy + qz * qz)) * s0;
    M[0][1] = 2.f * (qx * qy - qw * qz) * s1;
    M[0][2] = 2.f * (qx * qz + qw * qy) * s2;
    M[1][0] = 2.f * (qx * qy + qw * qz) * s0;
    M[1][1] = (1.f - 2.f * (qx * qx + qz * qz)) * s1;
    M[1][2] = 2.f * (qy * qz - qw * qx) * s2;
    M[2][0] = 2.f * (qx * qz - qw * qy) * s0;
    M[2][1] = 2.f * (qy * qz + qw * qx) * s1;
    M[2][2] = (1.f - 2.f * (qx * qx + qy * qy)) * s2;

    // EWA Jacobian at the frustum-clamped mean, times the view rotation W.
    const float inv_z = 1.0f / z;
    const float limx = kFrustumSlack * cam.tan_fovx, limy = kFrustumSlack * cam.tan_fovy;
    const float txc = fminf(limx, fmaxf(-limx, tx * inv_z)) * z;
    const float tyc = fminf(limy, fmaxf(-limy, ty * inv_z)) * z;
    const float j00 = cam.fx * inv_z, j02 = -cam.fx * txc * inv_z * inv_z;
    const float j11 = cam.fy * inv_z, j12 = -cam.fy * tyc * inv_z * inv_z;
    float T0[3], T1[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        T0[j] = fmaf(j00, V[j], j02 * V[8 + j]);
        T1[j] = fmaf(j11, V[4 + j], j12 * V[8 + j]);
    }
    // A = (J W) (R S), 2 x 3
    float A0[3], A1[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        A0[k] = fmaf(T0[0], M[0][k], fmaf(T0[1], M[1][k], T0[2] * M[2][k]));
        A1[k] = fmaf(T1[0], M[0][k], fmaf(T1[1], M[1][k], T1[2] * M[2][k]));
    }
    const float aa = fmaf(A0[0], A0[0], fmaf(A0[1], A0[1], A0[2] * A0[2]));
    const float bb = fmaf(A1[0], A1[0], fmaf(A1[1], A1[1], A1[2] * A1[2]));
    const float s01 = fmaf(A0[0], A1[0], fmaf(A0[1], A1[1], A0[2] * A1[2]));
    const float s00 = aa + kDilation, s11 = bb + kDilation;
    const float m01 = diff_of_products(A0[0], A1[1], A0[1], A1[0]);
    const float m02 = diff_of_products(A0[0], A1[2], A0[2], A1[0]);
    const float m12 = diff_of_products(A0[1], A1[2], A0[2], A1[1]);
    const float det = fmaf(m01, m01, fmaf(m02, m02, m12 * m12)) + fmaf(kDilation, aa + bb, kDilation * kDilation);

    const float half_diff = 0.5f * (aa - bb);
    const float disc = fmaf(half_diff, half_diff, s01 * s01);
    const float lambda = 0.5f * (s00 + s11) + sqrtf(fmaxf(kLambdaFloor, disc));
    const float radius = ceilf(3.0f * sqrtf(lambda));

    const float x = fmaf(cam.fx, tx * inv_z, cam.cx);
    const float y = fmaf(cam.fy, ty * inv_z, cam.cy);
    const float inv_tile = 1.0f / kTile;
    const float gx = (float)cam.tiles_x, gy = (float)cam.tiles_y;
    const float fx0 = fminf(gx, fmaxf(0.f, floorf((x - radius) * inv_tile)));
    const float fy0 = fminf(gy, fmaxf(0.f, floorf((y - radius) * inv_tile)));
    const float fx1 = fminf(gx, fmaxf(0.f, floorf((x + radius + (kTile - 1)) * inv_tile)));
    const float fy1 = fminf(gy, fmaxf(0.f, floorf((y + radius + (kTile - 1)) * inv_tile)));
    const uint32_t x0 = (uint32_t)fx0, y0 = (uint32_t)fy0, x1 = (uint32_t)fx1, y1 = (uint32_t)fy1;
    const uint32_t tiles = (x1 - x0) * (y1 - y0);
    if (tiles == 0u) {
        write_culled(out + g, sort_in + g, z);
        return;
    }

    // Upper-triangular factor of Sigma'^-1 (scaled by sqrt(log2(e)/2)).
    const float inv_s11 = 1.0f / s11;
    const float w00 = kWhiten * sqrtf(s11 / det);
    const float w01 = -w00 * s01 * inv_s11;
    const float w11 = kWhiten * sqrtf(inv_s11);

    // Colour: SH bands along the direction from the camera centre.
    float dx = mx - cam.campos[0], dy = my - cam.campos[1], dz = mz - cam.campos[2];
    const float dinv = 1.0f / sqrtf(dx * dx + dy * dy + dz * dz);
    dx *= dinv;
    dy *= dinv;
    dz *= dinv;
    float Y[16];
    Y[0] = kSH0;
    const float xx = dx * dx, yy = dy * dy, zz = dz * dz;
    Y[1] = -kSH1 * dy;
    Y[2] = kSH1 * dz;
    Y[3] = -kSH1 * dx;
    Y[4] = kSH2a * dx * dy;
    Y[5] = -kSH2a * dy * dz;
    Y[6] = kSH2b * (2.f * zz - xx - yy);
    Y[7] = -kSH2a * dx * dz;
    Y[8] = kSH2c * (xx - yy);
    Y[9] = -kSH3a * dy * (3.f * xx - yy);
    Y[10] = kSH3b * dx * dy * dz;
    Y[11] = -kSH3c * dy * (4.f * zz - xx - yy);
    Y[12] = kSH3d * dz * (2.f * zz - 3.f * xx - 3.f * yy);
    Y[13] = -kSH3c * dx * (4.f * zz - xx - yy);
    Y[14] = kSH3e * dz * (xx - yy);
    Y[15] = -kSH3a * dx * (xx - 3.f * yy);
    const int ncoef = (sh_degree + 1) * (sh_degree + 1);
#pragma unroll
    for (int k = 1; k < 16; ++k)
        if (k >= ncoef) Y[k] = 0.f;
    float c[48];
    const float4 *shg = sh + 12 * g;
#pragma unroll
    for (int j = 0; j < 12; ++j) {
        float4 v = __ldg(shg + j);
        c[4 * j] = v.x;
        c[4 * j + 1] = v.y;
        c[4 * j + 2] = v.z;
        c[4 * j + 3] = v.w;
    }
    float rgb[3];
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) {
        float acc = 0.f;
#pragma unroll
        for (int k = 0; k < 16; ++k) acc = fmaf(c[3 * k + ch], Y[k], acc);
        rgb[ch] = fmaxf(acc + 0.5f, 0.f);
    }

    const float logit = logits[g];
    const float e = expf(-logit);
    const float log2_opacity = -log1pf(e) * kLog2e;

    // Bounding box of the alpha >= 1/255 ellipse |W d|^2 <= rho:
    // half-extents sqrt(rho Sigma'_xx) / k and sqrt(rho Sigma'_yy) / k.
    const float rho = log2_opacity + kLog2_255;
    float hx = -1.f, hy = -1.f;
    if (rho > 0.f) {
        hx = sqrtf(rho * s00) * (1.0f / kWhiten);
        hy = sqrtf(rho * s11) * (1.0f / kWhiten);
        hx = fmaf(hx, kCullRel, hx) + kCullAbs;
        hy = fmaf(hy, kCullRel, hy) + kCullAbs;
    }

    float4 *o = reinterpret_cast<float4 *>(out + g);
    o[0] = make_float4(x, y, w00, w01);
    o[1] = make_float4(w11, log2_opacity, rgb[0], rgb[1]);
    o[2] = make_float4(rgb[2], hx, hy, __int_as_float((int)radius));
    const uint4 si = make_uint4(__float_as_uint(z), tiles, x0 | (y0 << 16), x1 | (y1 << 16));
    o[3] = make_float4(__uint_as_float(si.x), __uint_as_float(si.y), __uint_as_float(si.z), __uint_as_float(si.w));
    sort_in[g] = si;  // the dense copy gs_sort reads
}

__global__ void __launch_bounds__(256) preprocess_kernel(const float *__restrict__ means,
                                                         const float *__restrict__ log_scales,
                                                         const float4 *__restrict__ quats,
                                                         const float *__restrict__ logits,
                                                         const float4 *__restrict__ sh, int64_t n, int sh_degree,
                                                         CamParams cam, gs_splat *__restrict__ out,
                                                         uint4 *__restrict__ sort_in) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n) return;
    preprocess_one(g, means, log_scales, quats, logits, sh, sh_degree, cam, out, sort_in);
}

// The same with the camera read from device memory, so that a captured CUDA
// graph can be replayed for a new pose by rewriting that memory.
__global__ void __launch_bounds__(256) preprocess_camdev_kernel(const float *__restrict__ means,
                                                                const float *__restrict__ log_scales,
                                                                const float4 *__restrict__ quats,
                                                                const float *__restrict__ logits,
                                                                const float4 *__restrict__ sh, int64_t n,
                                                                int sh_degree, const CamParams *__restrict__ camp,
                                                                gs_splat *__restrict__ out,
                                                                uint4 *__restrict__ sort_in) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n) return;
    const CamParams cam = *camp;
    preprocess_one(g, means, log_scales, quats, logits, sh, sh_degree, cam, out, sort_in);
}

}  // namespace

cudaError_t launch_preprocess(const gs_scene &s, const CamParams &cam, gs_splat *out, cudaStream_t stream) {
    if (s.n == 0) return cudaSuccess;
    const int threads = 256;
    const int64_t blocks = (s.n + threads - 1) / threads;
    preprocess_kernel<<<(unsigned)blocks, threads, 0, stream>>>(
        s.means, s.log_scales, reinterpret_cast<const float4 *>(s.quats), s.opacity_logits,
        reinterpret_cast<const float4 *>(s.sh), s.n, s.sh_degree, cam, out, reinterpret_cast<uint4 *>(out + s.n));
    return cudaGetLastError();
}

cudaError_t launch_preprocess_camdev(const gs_scene &s, const CamParams *cam_dev, gs_splat *out, cudaStream_t stream) {
    if (s.n == 0) return cudaSuccess;
    const int threads = 256;
    const int64_t blocks = (s.n + threads - 1) / threads;
    preprocess_camdev_kernel<<<(unsigned)blocks, threads, 0, stream>>>(
        s.means, s.log_scales, reinterpret_cast<const float4 *>(s.quats), s.opacity_logits,
        reinterpret_cast<const float4 *>(s.sh), s.n, s.sh_degree, cam_dev, out, reinterpret_cast<uint4 *>(out + s.n));
    return cudaGetLastError();
}

}  // namespace gs
