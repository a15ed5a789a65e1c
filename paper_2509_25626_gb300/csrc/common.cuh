// Internal definitions shared by the CUDA translation units of libgs.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "gs.h"

namespace gs {

constexpr int kTile = GS_TILE;
constexpr int kTilePixels = kTile * kTile;

// Per-pixel blend rules printed by the paper's render kernels (Appendix B).
constexpr float kAlphaMax = 0.99f;
constexpr float kAlphaMin = 1.0f / 255.0f;
constexpr float kTStop = 1e-4f;

// Projection constants of the 3DGS preprocess the paper builds on.
constexpr float kNearZ = 0.2f;          // near-plane cull
constexpr float kDilation = 0.3f;       // low-pass added to the 2D covariance
constexpr float kFrustumSlack = 1.3f;   // Jacobian evaluated inside 1.3 tan(fov)
constexpr float kLambdaFloor = 0.1f;    // floor under the eigenvalue discriminant

constexpr float kLog2e = 1.4426950408889634f;
// sqrt(log2(e) / 2): folds the -1/2 of the Gaussian exponent and the change
// of base to 2 into the inverse-covariance factor.
constexpr float kWhiten = 0.8493218002880191f;

// Word offsets inside a gs_splat record (16 x 4 bytes).
namespace rec {
enum : int {
    kX = 0, kY = 1, kW00 = 2, kW01 = 3, kW11 = 4, kLog2O = 5, kR = 6, kG = 7, kB = 8, kHx = 9, kHy = 10,
    kRadius = 11, kDepth = 12, kTiles = 13, kRectLo = 14, kRectHi = 15,
};
}  // namespace rec

// Culling box slack: relative and absolute widening of the alpha >= 1/255
// bounding box (FP32 rounding of the render's exponent is ~1e-5 of it).
constexpr float kCullRel = 1.0f / 1024.0f;
constexpr float kCullAbs = 1.0f / 64.0f;
// log2(255): alpha >= 1/255  <=>  log2_opacity - (u^2 + v^2) >= -log2(255)
constexpr float kLog2_255 = 7.994353436858858f;

// Which 8x8 quarters of the 16x16 tile whose top-left pixel is (tx0, ty0) a
// splat's alpha >= 1/255 region can reach, from the first three vectors of
// its record: a = (x, y, w00, w01), b = (w11, ...), c = (..., hx, hy, ...).
// Bit 2 qy + qx stands for the quarter of pixels [tx0 + 8 qx, +7] x
// [ty0 + 8 qy, +7].  A quarter is ruled out by either of two separating
// tests, each necessary for alpha >= 1/255 at one of its pixel centres:
//  - the bounding box [x - hx, x + hx] x [y - hy, y + hy] misses it;
//  - the band |u| <= R misses it, where u = w00 dx + w01 dy is the first
//    component of W d (the render keeps a splat iff u^2 + v^2 <= R^2 =
//    log2 o + log2 255, so |u| <= R).  u is affine in the pixel, so over a
//    quarter it spans u(centre) +- 3.5 (|w00| + |w01|).
// R is taken as hy w11 + 1/64 >= sqrt(log2 o + log2 255)(1 + 2^-10) + 1/64
// (hy carries the box slack), a margin that covers the FP32 rounding of u
// here and in the render (|w| <= ~1.6 after the 0.3 dilation and |d| within
// a few thousand pixels put it near 1e-3).  The band removes the quarters
// the box keeps only because the ellipse is thin and slanted.
__host__ __device__ __forceinline__ uint32_t quarter_mask(const float4 a, const float4 b, const float4 c,
                                                          float tx0, float ty0) {
    if (!(c.y >= 0.f)) return 0u;  // alpha < 1/255 everywhere (empty box)
    // coordinates relative to the tile's first pixel (the slack in hx, hy
    // and R covers the rounding of these differences)
    const float x = a.x - tx0, y = a.y - ty0;
    const float xlo = x - c.y, xhi = x + c.y, ylo = y - c.z, yhi = y + c.z;
    const uint32_t mx0 = (xhi >= 0.f) & (xlo <= 7.f);
    const uint32_t mx1 = (xhi >= 8.f) & (xlo <= 15.f);
    const uint32_t my0 = (yhi >= 0.f) & (ylo <= 7.f);
    const uint32_t my1 = (yhi >= 8.f) & (ylo <= 15.f);
    const uint32_t box = (mx0 & my0) | ((mx1 & my0) << 1) | ((mx0 & my1) << 2) | ((mx1 & my1) << 3);
    // u at the quarter centres (3.5 + 8 qx, 3.5 + 8 qy)
    const float u00 = fmaf(a.z, x - 3.5f, a.w * (y - 3.5f));
    const float u10 = fmaf(-8.f, a.z, u00), u01 = fmaf(-8.f, a.w, u00), u11 = fmaf(-8.f, a.w, u10);
    const float L = fmaf(c.z, b.x, 1.0f / 64.0f) + 3.5f * (fabsf(a.z) + fabsf(a.w));
    const uint32_t band = (uint32_t)(fabsf(u00) <= L) | ((uint32_t)(fabsf(u10) <= L) << 1) |
                          ((uint32_t)(fabsf(u01) <= L) << 2) | ((uint32_t)(fabsf(u11) <= L) << 3);
    return box & band;
}

// Camera as the kernels see it (kernel parameter, passed by value).
struct CamParams {
    float V[12];          // rows 0..2 of the world->camera matrix
    float fx, fy, cx, cy;
    float tan_fovx, tan_fovy;
    float campos[3];      // camera centre in world space
    int width, height, tiles_x, tiles_y;
};

// Host-side conversion; the camera centre -R^T t is formed in double.
inline CamParams make_cam_params(const gs_camera &c) {
    CamParams p;
    for (int i = 0; i < 12; ++i) p.V[i] = c.viewmat[i];
    p.fx = c.fx;
    p.fy = c.fy;
    p.cx = c.cx;
    p.cy = c.cy;
    p.tan_fovx = c.tan_fovx;
    p.tan_fovy = c.tan_fovy;
    for (int i = 0; i < 3; ++i) {
        double acc = 0.0;
        for (int j = 0; j < 3; ++j) acc -= (double)c.viewmat[4 * j + i] * (double)c.viewmat[4 * j + 3];
        p.campos[i] = (float)acc;
    }
    p.width = c.width;
    p.height = c.height;
    p.tiles_x = (c.width + kTile - 1) / kTile;
    p.tiles_y = (c.height + kTile - 1) / kTile;
    return p;
}

__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31u; }

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Block-wide exclusive scan of one uint32 per thread (blockDim.x a multiple
// of 32, at most 1024).  `scratch` holds >= 33 words.  Returns the exclusive
// prefix; *total receives the block sum.  Contains __syncthreads().
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t *scratch, uint32_t *total) {
    const unsigned lane = lane_id(), warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    uint32_t inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= (unsigned)o) inc += t;
    }
    if (lane == 31) scratch[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = lane < nwarps ? scratch[lane] : 0u;
        uint32_t wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t t = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= (unsigned)o) wi += t;
        }
        if (lane < nwarps) scratch[lane] = wi - w;
        if (lane == 31) scratch[32] = wi;
    }
    __syncthreads();
    uint32_t res = scratch[warp] + inc - v;
    *total = scratch[32];
    __syncthreads();
    return res;
}

// Records the first CUDA error of a launch sequence.
void set_cuda_error(cudaError_t e);

}  // namespace gs
