"""The render's per-warp culling test (quarter_mask in csrc/common.cuh), run
on the CPU: for random splats -- thin and slanted ones in particular -- a
quarter of the tile that quarter_mask leaves out must hold no pixel at which
the render's own FP32 arithmetic keeps the splat (alpha >= 1/255), or the
culling would change the image.  The driver compiles the header's function
for the host with nvcc and restates the render's per-pixel decision (the
same FP32 operations in the same order) and the preprocess's record fields;
no GPU."""

import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "..", "paper_2509_25626_gb300", "csrc")
INCLUDE = os.path.join(HERE, "..", "include")

DRIVER = r"""
#include <cmath>
#include <cstdio>
#include <random>
#include "common.cuh"
using namespace gs;

// Record fields of a splat with 2D covariance (s00, s01, s11), as the
// preprocess writes them (upper-triangular factor of the inverse, the
// alpha >= 1/255 box with its slack).
static void make_record(float x, float y, float s00, float s01, float s11, float lg2o, float4 &a, float4 &b,
                        float4 &c) {
    const float det = s00 * s11 - s01 * s01;
    const float inv_s11 = 1.0f / s11;
    const float w00 = kWhiten * sqrtf(s11 / det);
    const float w01 = -w00 * s01 * inv_s11;
    const float w11 = kWhiten * sqrtf(inv_s11);
    const float rho = lg2o + kLog2_255;
    float hx = -1.f, hy = -1.f;
    if (rho > 0.f) {
        hx = sqrtf(rho * s00) * (1.0f / kWhiten);
        hy = sqrtf(rho * s11) * (1.0f / kWhiten);
        hx = fmaf(hx, kCullRel, hx) + kCullAbs;
        hy = fmaf(hy, kCullRel, hy) + kCullAbs;
    }
    a = make_float4(x, y, w00, w01);
    b = make_float4(w11, lg2o, 0.f, 0.f);
    c = make_float4(0.f, hx, hy, 0.f);
}

// The render's decision for pixel (px, py): pixels are evaluated in pairs
// (px even, px + 1), the second as u - w00.
static bool keeps(const float4 &a, const float4 &b, int px, int py) {
    const int p0 = px & ~1;
    const float dy = a.y - (float)py;
    const float t = a.w * dy;
    float u = fmaf(a.z, a.x - (float)p0, t);
    if (px != p0) u = u - a.z;
    const float v = b.x * dy;
    const float vv = fmaf(-v, v, b.y);
    const float e = fmaf(-u, u, vv);
    return e >= -kLog2_255;
}

int main() {
    std::mt19937_64 rng(12345);
    std::uniform_real_distribution<float> U(0.f, 1.f);
    long long missed = 0, band_culled = 0, box_kept = 0, reached = 0;
    const int tiles[][2] = {{0, 0}, {50, 33}, {99, 66}, {240, 135}};
    for (int it = 0; it < 300000; ++it) {
        const int tx = tiles[it & 3][0], ty = tiles[it & 3][1];
        const float tx0 = (float)(tx * kTile), ty0 = (float)(ty * kTile);
        // long axis 0.6..60 px, aspect up to 100, any angle; dilation floor 0.3
        const float sl = 0.6f * powf(100.f, U(rng));
        const float ss = fmaxf(0.55f, sl / (1.f + 99.f * U(rng)));
        const float th = 6.2831853f * U(rng), cs = cosf(th), sn = sinf(th);
        const float s00 = sl * sl * cs * cs + ss * ss * sn * sn + 0.3f;
        const float s11 = sl * sl * sn * sn + ss * ss * cs * cs + 0.3f;
        const float s01 = (sl * sl - ss * ss) * cs * sn;
        const float reach = 3.5f * sl + 8.f;
        const float x = tx0 + 8.f + (2.f * U(rng) - 1.f) * reach, y = ty0 + 8.f + (2.f * U(rng) - 1.f) * reach;
        const float lg2o = -kLog2_255 * 0.999f * U(rng);
        float4 a, b, c;
        make_record(x, y, s00, s01, s11, lg2o, a, b, c);
        const unsigned m = quarter_mask(a, b, c, tx0, ty0);
        for (int q = 0; q < 4; ++q) {
            const int qx = q & 1, qy = q >> 1;
            bool any = false;
            for (int j = 0; j < 8 && !any; ++j)
                for (int i = 0; i < 8 && !any; ++i)
                    any = keeps(a, b, tx * kTile + 8 * qx + i, ty * kTile + 8 * qy + j);
            reached += any;
            if (any && !((m >> q) & 1u)) {
                if (missed < 5) std::printf("missed: x %.3f y %.3f w %g %g %g lg2o %g quarter %d\n", a.x, a.y, a.z,
                                            a.w, b.x, b.y, q);
                ++missed;
            }
            // the box alone: does it keep the quarter that the band removes?
            const float xl = a.x - c.y - tx0, xh = a.x + c.y - tx0, yl = a.y - c.z - ty0, yh = a.y + c.z - ty0;
            const bool box = c.y >= 0.f && xh >= 8.f * qx && xl <= 8.f * qx + 7.f && yh >= 8.f * qy &&
                             yl <= 8.f * qy + 7.f;
            box_kept += box;
            band_culled += box && !((m >> q) & 1u);
        }
    }
    std::printf("reached %lld box %lld band_culled %lld missed %lld\n", reached, box_kept, band_culled, missed);
    std::printf("%s\n", missed == 0 && band_culled > 0 && reached > 0 ? "OK" : "FAIL");
    return missed == 0 && band_culled > 0 ? 0 : 1;
}
"""


def test_quarter_mask_never_drops_a_kept_pixel(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("no nvcc")
    src = tmp_path / "qm.cu"
    src.write_text(DRIVER)
    exe = tmp_path / "qm"
    subprocess.run([nvcc, "-std=c++17", "-O2", f"-I{CSRC}", f"-I{INCLUDE}", str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    print(out.stdout)
    assert out.returncode == 0 and out.stdout.strip().endswith("OK"), out.stdout


# Plausible mistakes in the mask, each of which must make the check above
# fail (so the check can see them): a band half-width without the w01 term,
# the wrong sign of a quarter-centre step, quarter centres off by half a
# pixel.
MUTANTS = {
    "no_w01_half_width": ("3.5f * (fabsf(a.z) + fabsf(a.w))", "3.5f * fabsf(a.z)"),
    "sign_of_w01_step": ("u01 = fmaf(-8.f, a.w, u00)", "u01 = fmaf(8.f, a.w, u00)"),
    "centre_shift": ("x - 3.5f", "x - 4.0f"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_quarter_mask_check_catches_mutants(tmp_path, name):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("no nvcc")
    old, new = MUTANTS[name]
    with open(os.path.join(CSRC, "common.cuh")) as f:
        text = f.read()
    assert text.count(old) == 1, name
    mdir = tmp_path / "mut"
    mdir.mkdir()
    (mdir / "common.cuh").write_text(text.replace(old, new))
    src = tmp_path / "qm.cu"
    src.write_text(DRIVER)
    exe = tmp_path / "qm"
    subprocess.run([nvcc, "-std=c++17", "-O2", f"-I{mdir}", f"-I{CSRC}", f"-I{INCLUDE}", str(src), "-o", str(exe)],
                   check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert out.returncode != 0 and "missed 0" not in out.stdout, out.stdout
