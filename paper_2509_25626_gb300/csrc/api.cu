// C ABI entry points (include/gs.h): argument checks, then launches.
#include <cmath>
#include <cstdio>
#include <cstring>

#include <nvtx3/nvToolsExt.h>

#include "common.cuh"
#include "sort_ws.h"

#ifndef GS_BUILT_ARCH
#define GS_BUILT_ARCH 0
#endif

namespace gs {

// One NVTX range per compute entry point, named after it, so that a
// timeline tool shows the library's calls; nearly free without a tool.
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

cudaError_t launch_preprocess(const gs_scene &s, const CamParams &cam, gs_splat *out, cudaStream_t stream);
cudaError_t launch_preprocess_camdev(const gs_scene &s, const CamParams *cam_dev, gs_splat *out, cudaStream_t stream);
cudaError_t launch_sort_front(const gs_splat *splats, int64_t n, const SortWs &ws, uint64_t m_cap, int tiles_x,
                              uint32_t num_tiles, cudaStream_t st);
cudaError_t launch_sort_back(const gs_splat *splats, int64_t n, const SortWs &ws, uint64_t m_cap, int tiles_x,
                             uint32_t num_tiles, uint64_t *keys, uint32_t *vals, uint32_t *ranges, cudaStream_t st);
cudaError_t launch_render_backward(const gs_scene &s, const CamParams &cam, const gs_splat *splats,
                                   const uint32_t *vals, const uint32_t *ranges, const float bg[3],
                                   const float *final_T, const uint32_t *n_contrib, const float *dL_dcolor,
                                   float *dsplat, const gs_scene_grads &g, cudaStream_t st);
cudaError_t launch_render_backward_splats(int64_t n, const CamParams &cam, const gs_splat *splats,
                                          const uint32_t *vals, const uint32_t *ranges, const float bg[3],
                                          const float *final_T, const uint32_t *n_contrib, const float *dL_dcolor,
                                          float *dsplat, cudaStream_t st);
cudaError_t launch_preprocess_backward(const gs_scene &s, const CamParams &cam, const gs_splat *splats,
                                       const float *dsplat, const gs_scene_grads &g, cudaStream_t st);
cudaError_t launch_lookback_probe(const SortWs &ws, uint64_t limit_ns, cudaStream_t st);
cudaError_t launch_render_batch(const gs_render_batch_desc *desc, uint32_t *counter, int grid, cudaStream_t stream);
size_t balance_ws_bytes(const gs_balance_params &p);
cudaError_t launch_render_batch_balanced(const gs_render_batch_desc *desc, uint32_t *counter,
                                         const gs_balance_params &p, void *workspace, int grid,
                                         cudaStream_t stream);
cudaError_t launch_render(const gs_splat *splats, const uint32_t *vals, const uint32_t *ranges, const CamParams &cam,
                          const float bg[3], float *out_color, float *final_T, uint32_t *n_contrib, float *invdepth,
                          uint32_t *n_eval, uint32_t *tile_cycles, cudaStream_t stream);
cudaError_t launch_render_contrib(const gs_splat *splats, const uint32_t *vals, const uint32_t *ranges,
                                  const CamParams &cam, const float bg[3], float *out_color, float *final_T,
                                  uint32_t *n_contrib, cudaStream_t stream);

static_assert(sizeof(gs_splat) == 64 && sizeof(gs_sort_input) == 16, "splat buffer layout");

static thread_local char g_cuda_err[256] = "no CUDA error recorded";

void set_cuda_error(cudaError_t e) {
    std::snprintf(g_cuda_err, sizeof(g_cuda_err), "%s: %s", cudaGetErrorName(e), cudaGetErrorString(e));
}

}  // namespace gs

using namespace gs;

namespace {

bool aligned(const void *p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

bool camera_ok(const gs_camera *c) {
    if (!c) return false;
    if (c->width < 1 || c->height < 1 || c->width > 65535 * kTile || c->height > 65535 * kTile) return false;
    const float f[] = {c->fx, c->fy, c->cx, c->cy, c->tan_fovx, c->tan_fovy};
    for (float v : f)
        if (!std::isfinite(v)) return false;
    for (int i = 0; i < 16; ++i)
        if (!std::isfinite(c->viewmat[i])) return false;
    return c->fx > 0.f && c->fy > 0.f && c->tan_fovx > 0.f && c->tan_fovy > 0.f;
}

uint64_t tiles_of(const gs_camera *c) {
    return (uint64_t)((c->width + kTile - 1) / kTile) * (uint64_t)((c->height + kTile - 1) / kTile);
}

int cuda_status(cudaError_t e) {
    if (e == cudaSuccess) return GS_OK;
    set_cuda_error(e);
    return GS_ERR_CUDA;
}

}  // namespace

extern "C" {

int gs_preprocess(const gs_scene *scene, const gs_camera *cam, gs_splat *splats, void *stream) {
    gs::NvtxRange nvtx_range("gs_preprocess");
    if (!scene || !camera_ok(cam)) return GS_ERR_INVALID_ARG;
    if (scene->n < 0 || scene->n > (int64_t)UINT32_MAX || scene->sh_degree < 0 || scene->sh_degree > 3)
        return GS_ERR_INVALID_ARG;
    if (scene->n > 0) {
        const void *ptrs[] = {scene->means, scene->log_scales, scene->quats, scene->opacity_logits, scene->sh, splats};
        for (const void *p : ptrs)
            if (!p || !aligned(p, 16)) return GS_ERR_INVALID_ARG;
    }
    return cuda_status(launch_preprocess(*scene, make_cam_params(*cam), splats, (cudaStream_t)stream));
}

size_t gs_camera_block_bytes(void) { return sizeof(CamParams); }

int gs_camera_block(const gs_camera *cam, void *block) {
    if (!camera_ok(cam) || !block) return GS_ERR_INVALID_ARG;
    const CamParams p = make_cam_params(*cam);
    std::memcpy(block, &p, sizeof(p));
    return GS_OK;
}

int gs_preprocess_camblock(const gs_scene *scene, const void *camera_block, gs_splat *splats, void *stream) {
    gs::NvtxRange nvtx_range("gs_preprocess_camblock");
    if (!scene || !camera_block || !aligned(camera_block, 16)) return GS_ERR_INVALID_ARG;
    if (scene->n < 0 || scene->n > (int64_t)UINT32_MAX || scene->sh_degree < 0 || scene->sh_degree > 3)
        return GS_ERR_INVALID_ARG;
    if (scene->n > 0) {
        const void *ptrs[] = {scene->means, scene->log_scales, scene->quats, scene->opacity_logits, scene->sh, splats};
        for (const void *p : ptrs)
            if (!p || !aligned(p, 16)) return GS_ERR_INVALID_ARG;
    }
    return cuda_status(launch_preprocess_camdev(*scene, static_cast<const CamParams *>(camera_block), splats,
                                                (cudaStream_t)stream));
}

size_t gs_sort_workspace_bytes(int64_t n, int64_t m_cap, int32_t num_tiles) {
    return carve_sort_ws(nullptr, n, m_cap, (uint64_t)(num_tiles > 0 ? num_tiles : 1), nullptr);
}

int gs_sort(const gs_splat *splats, int64_t n, const gs_camera *cam, uint64_t *keys, uint32_t *vals, int64_t m_cap,
            uint32_t *ranges, void *workspace, size_t workspace_bytes, int64_t *m_out, void *stream) {
    gs::NvtxRange nvtx_range("gs_sort");
    if (!camera_ok(cam) || n < 0 || n > (int64_t)UINT32_MAX || m_cap < 0 || m_cap > (int64_t)UINT32_MAX)
        return GS_ERR_INVALID_ARG;
    const uint64_t num_tiles = tiles_of(cam);
    if (num_tiles > (uint64_t)UINT32_MAX) return GS_ERR_INVALID_ARG;
    if (!ranges || !aligned(ranges, 8) || !workspace || !aligned(workspace, 256)) return GS_ERR_INVALID_ARG;
    if (n > 0 && (!splats || !aligned(splats, 16))) return GS_ERR_INVALID_ARG;
    if (m_cap > 0 && (!keys || !vals || !aligned(keys, 16) || !aligned(vals, 16))) return GS_ERR_INVALID_ARG;
    if (workspace_bytes < carve_sort_ws(nullptr, n, m_cap, num_tiles, nullptr)) return GS_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    SortWs ws;
    carve_sort_ws(static_cast<char *>(workspace), n, m_cap, num_tiles, &ws);
    const int tiles_x = (cam->width + kTile - 1) / kTile;
    cudaError_t e = launch_sort_front(splats, n, ws, (uint64_t)m_cap, tiles_x, (uint32_t)num_tiles, st);
    if (e != cudaSuccess) return cuda_status(e);
    if (m_out) {
        SortHeader h;
        e = cudaMemcpyAsync(&h, ws.hdr, sizeof(h), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return cuda_status(e);
        *m_out = (int64_t)h.m_total;
        if (h.timeout) return GS_ERR_TIMEOUT;
        if (h.m_total > (uint64_t)m_cap) return GS_ERR_CAPACITY;
    }
    return cuda_status(launch_sort_back(splats, n, ws, (uint64_t)m_cap, tiles_x, (uint32_t)num_tiles, keys, vals,
                                        ranges, st));
}

int gs_sort_status(const void *workspace, int64_t *m_out, void *stream) {
    if (!workspace || !aligned(workspace, 256) || !m_out) return GS_ERR_INVALID_ARG;
    SortHeader h;
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaMemcpyAsync(&h, workspace, sizeof(h), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_status(e);
    *m_out = (int64_t)h.m_total;
    if (h.timeout) return GS_ERR_TIMEOUT;
    return h.overflow ? GS_ERR_CAPACITY : GS_OK;
}

int gs_check_wait_timeout(void *workspace, size_t workspace_bytes, uint64_t limit_ns, void *stream) {
    gs::NvtxRange nvtx_range("gs_check_wait_timeout");
    if (!workspace || !aligned(workspace, 256) || limit_ns == 0 || limit_ns > 1000000000ull) return GS_ERR_INVALID_ARG;
    if (workspace_bytes < carve_sort_ws(nullptr, 1, 1, 1, nullptr)) return GS_ERR_INVALID_ARG;
    SortWs ws;
    carve_sort_ws(static_cast<char *>(workspace), 1, 1, 1, &ws);
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = launch_lookback_probe(ws, limit_ns, st);
    SortHeader h;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, ws.hdr, sizeof(h), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_status(e);
    return h.timeout ? GS_ERR_TIMEOUT : GS_OK;
}

static int render_common(const gs_splat *splats, const uint32_t *vals, const uint32_t *ranges, const gs_camera *cam,
                         const float bg[3], float *out_color, float *final_T, uint32_t *n_contrib,
                         float *invdepth, uint32_t *n_eval, uint32_t *tile_cycles, void *stream) {
    if (!camera_ok(cam) || !bg || !ranges || !aligned(ranges, 8)) return GS_ERR_INVALID_ARG;
    if (tiles_of(cam) > (uint64_t)INT32_MAX) return GS_ERR_INVALID_ARG;
    if (!out_color || !final_T || !n_contrib || !aligned(out_color, 4) || !aligned(final_T, 4) ||
        !aligned(n_contrib, 4))
        return GS_ERR_INVALID_ARG;
    if (!splats || !aligned(splats, 16) || !vals || !aligned(vals, 4)) return GS_ERR_INVALID_ARG;
    for (int i = 0; i < 3; ++i)
        if (!std::isfinite(bg[i])) return GS_ERR_INVALID_ARG;
    return cuda_status(launch_render(splats, vals, ranges, make_cam_params(*cam), bg, out_color, final_T, n_contrib,
                                     invdepth, n_eval, tile_cycles, (cudaStream_t)stream));
}

int gs_render(const gs_splat *splats, const uint32_t *vals, const uint32_t *ranges, const gs_camera *cam,
              const float bg[3], float *out_color, float *final_T, uint32_t *n_contrib, void *stream) {
    gs::NvtxRange nvtx_range("gs_render");
    return render_common(splats, vals, ranges, cam, bg, out_color, final_T, n_contrib, nullptr, nullptr, nullptr,
                         stream);
}

int gs_render_contrib(const gs_splat *splats, const uint32_t *vals, const uint32_t *ranges, const gs_camera *cam,
                      const float bg[3], float *out_color, float *final_T, uint32_t *n_contrib, void *stream) {
    gs::NvtxRange nvtx_range("gs_render_contrib");
    // the argument checks of gs_render (a launch-free call with no outputs
    // would not be reached: outputs are required)
    if (!camera_ok(cam) || !bg || !ranges || !aligned(ranges, 8)) return GS_ERR_INVALID_ARG;
    if (tiles_of(cam) > (uint64_t)INT32_MAX) return GS_ERR_INVALID_ARG;
    if (!out_color || !final_T || !n_contrib || !aligned(out_color, 4) || !aligned(final_T, 4) ||
        !aligned(n_contrib, 4))
        return GS_ERR_INVALID_ARG;
    if (!splats || !aligned(splats, 16) || !vals || !aligned(vals, 4)) return GS_ERR_INVALID_ARG;
    for (int i = 0; i < 3; ++i)
        if (!std::isfinite(bg[i])) return GS_ERR_INVALID_ARG;
    return cuda_status(launch_render_contrib(splats, vals, ranges, make_cam_params(*cam), bg, out_color, final_T,
                                             n_contrib, (cudaStream_t)stream));
}

int gs_render_workload(const gs_splat *splats, const uint32_t *vals, const uint32_t *ranges, const gs_camera *cam,
                       const float bg[3], float *out_color, float *final_T, uint32_t *n_contrib, uint32_t *n_eval,
                       uint32_t *tile_cycles, void *stream) {
    gs::NvtxRange nvtx_range("gs_render_workload");
    if (!n_eval || !aligned(n_eval, 4) || (tile_cycles && !aligned(tile_cycles, 4))) return GS_ERR_INVALID_ARG;
    return render_common(splats, vals, ranges, cam, bg, out_color, final_T, n_contrib, nullptr, n_eval, tile_cycles,
                         stream);
}

int gs_render_ex(const gs_splat *splats, const uint32_t *vals, const uint32_t *ranges, const gs_camera *cam,
                 const float bg[3], float *out_color, float *final_T, uint32_t *n_contrib, float *invdepth,
                 uint32_t *n_eval, uint32_t *tile_cycles, void *stream) {
    gs::NvtxRange nvtx_range("gs_render_ex");
    if ((invdepth && !aligned(invdepth, 4)) || (n_eval && !aligned(n_eval, 4)) ||
        (tile_cycles && (!n_eval || !aligned(tile_cycles, 4))))
        return GS_ERR_INVALID_ARG;
    return render_common(splats, vals, ranges, cam, bg, out_color, final_T, n_contrib, invdepth, n_eval, tile_cycles,
                         stream);
}

int gs_render_batch(const gs_render_batch_desc *desc, uint32_t *counter, int32_t grid, void *stream) {
    gs::NvtxRange nvtx_range("gs_render_batch");
    if (!desc || !aligned(desc, 8) || !counter || !aligned(counter, 4) || grid < 0) return GS_ERR_INVALID_ARG;
    return cuda_status(launch_render_batch(desc, counter, grid, (cudaStream_t)stream));
}

static bool balance_params_ok(const gs_balance_params *p) {
    if (!p) return false;
    if (p->heavy_len < 0 || p->max_heavy_tiles < 0 || p->budget < 0 || p->max_split_tiles < 0) return false;
    if (p->budget > 0 && (p->max_chunks < 1 || p->max_chunks > 64 || p->chunk < 1)) return false;
    return true;
}

size_t gs_render_balance_workspace_bytes(const gs_balance_params *params) {
    if (!balance_params_ok(params)) return 0;
    return balance_ws_bytes(*params);
}

int gs_render_batch_balanced(const gs_render_batch_desc *desc, uint32_t *counter, const gs_balance_params *params,
                             void *workspace, size_t workspace_bytes, int32_t grid, void *stream) {
    gs::NvtxRange nvtx_range("gs_render_batch_balanced");
    if (!desc || !aligned(desc, 8) || !counter || !aligned(counter, 4) || grid < 0) return GS_ERR_INVALID_ARG;
    if (!balance_params_ok(params)) return GS_ERR_INVALID_ARG;
    if (!workspace || !aligned(workspace, 256) || workspace_bytes < balance_ws_bytes(*params))
        return GS_ERR_INVALID_ARG;
    return cuda_status(launch_render_batch_balanced(desc, counter, *params, workspace, grid, (cudaStream_t)stream));
}

int gs_frame(const gs_scene *scene, const gs_camera *cam, gs_splat *splats, uint64_t *keys, uint32_t *vals,
             int64_t m_cap, uint32_t *ranges, void *workspace, size_t workspace_bytes, const float bg[3],
             float *out_color, float *final_T, uint32_t *n_contrib, void *stream) {
    gs::NvtxRange nvtx_range("gs_frame");
    if (!scene) return GS_ERR_INVALID_ARG;
    int code = gs_preprocess(scene, cam, splats, stream);
    if (code != GS_OK) return code;
    code = gs_sort(splats, scene->n, cam, keys, vals, m_cap, ranges, workspace, workspace_bytes, nullptr, stream);
    if (code != GS_OK) return code;
    return gs_render(splats, vals, ranges, cam, bg, out_color, final_T, n_contrib, stream);
}

size_t gs_splat_buffer_bytes(int64_t n) { return (size_t)(n > 0 ? n : 0) * (sizeof(gs_splat) + sizeof(gs_sort_input)); }

size_t gs_backward_workspace_bytes(int64_t n) { return (size_t)(n > 0 ? n : 1) * 12 * sizeof(float); }

int gs_render_backward_splats(const gs_camera *cam, const gs_splat *splats, int64_t n, const uint32_t *vals,
                              const uint32_t *ranges, const float bg[3], const float *final_T,
                              const uint32_t *n_contrib, const float *dL_dcolor, float *dsplat, void *stream) {
    gs::NvtxRange nvtx_range("gs_render_backward_splats");
    if (!camera_ok(cam) || !bg || n < 0 || n > (int64_t)UINT32_MAX) return GS_ERR_INVALID_ARG;
    if (tiles_of(cam) > (uint64_t)INT32_MAX) return GS_ERR_INVALID_ARG;
    if (!ranges || !aligned(ranges, 8) || !final_T || !n_contrib || !dL_dcolor || !aligned(final_T, 4) ||
        !aligned(n_contrib, 4) || !aligned(dL_dcolor, 4) || !dsplat || !aligned(dsplat, 16))
        return GS_ERR_INVALID_ARG;
    if (n > 0 && (!splats || !aligned(splats, 16) || !vals)) return GS_ERR_INVALID_ARG;
    for (int i = 0; i < 3; ++i)
        if (!std::isfinite(bg[i])) return GS_ERR_INVALID_ARG;
    return cuda_status(launch_render_backward_splats(n, make_cam_params(*cam), splats, vals, ranges, bg, final_T,
                                                     n_contrib, dL_dcolor, dsplat, (cudaStream_t)stream));
}

int gs_preprocess_backward(const gs_scene *scene, const gs_camera *cam, const gs_splat *splats, const float *dsplat,
                           const gs_scene_grads *grads, void *stream) {
    gs::NvtxRange nvtx_range("gs_preprocess_backward");
    if (!scene || !camera_ok(cam) || !grads) return GS_ERR_INVALID_ARG;
    if (scene->n < 0 || scene->n > (int64_t)UINT32_MAX || scene->sh_degree < 0 || scene->sh_degree > 3)
        return GS_ERR_INVALID_ARG;
    if (scene->n > 0) {
        const void *ptrs[] = {scene->means, scene->log_scales, scene->quats, scene->opacity_logits, scene->sh,
                              splats, dsplat, grads->dmeans, grads->dlog_scales, grads->dquats,
                              grads->dopacity_logits, grads->dsh};
        for (const void *p : ptrs)
            if (!p || !aligned(p, 4)) return GS_ERR_INVALID_ARG;
        if (!aligned(scene->quats, 16) || !aligned(splats, 16)) return GS_ERR_INVALID_ARG;
    }
    return cuda_status(launch_preprocess_backward(*scene, make_cam_params(*cam), splats, dsplat, *grads,
                                                  (cudaStream_t)stream));
}

int gs_render_backward(const gs_scene *scene, const gs_camera *cam, const gs_splat *splats, const uint32_t *vals,
                       const uint32_t *ranges, const float bg[3], const float *final_T, const uint32_t *n_contrib,
                       const float *dL_dcolor, void *workspace, size_t workspace_bytes,
                       const gs_scene_grads *grads, void *stream) {
    gs::NvtxRange nvtx_range("gs_render_backward");
    if (!scene || !camera_ok(cam) || !grads || !bg) return GS_ERR_INVALID_ARG;
    if (scene->n < 0 || scene->n > (int64_t)UINT32_MAX || scene->sh_degree < 0 || scene->sh_degree > 3)
        return GS_ERR_INVALID_ARG;
    if (tiles_of(cam) > (uint64_t)INT32_MAX) return GS_ERR_INVALID_ARG;
    if (!ranges || !aligned(ranges, 8) || !final_T || !n_contrib || !dL_dcolor || !aligned(final_T, 4) ||
        !aligned(n_contrib, 4) || !aligned(dL_dcolor, 4))
        return GS_ERR_INVALID_ARG;
    if (!workspace || !aligned(workspace, 16) || workspace_bytes < gs_backward_workspace_bytes(scene->n))
        return GS_ERR_INVALID_ARG;
    if (scene->n > 0) {
        const void *ptrs[] = {scene->means, scene->log_scales, scene->quats, scene->opacity_logits, scene->sh,
                              splats, grads->dmeans, grads->dlog_scales, grads->dquats, grads->dopacity_logits,
                              grads->dsh};
        for (const void *p : ptrs)
            if (!p || !aligned(p, 4)) return GS_ERR_INVALID_ARG;
        if (!aligned(scene->quats, 16) || !aligned(splats, 16) || !vals) return GS_ERR_INVALID_ARG;
    }
    for (int i = 0; i < 3; ++i)
        if (!std::isfinite(bg[i])) return GS_ERR_INVALID_ARG;
    return cuda_status(launch_render_backward(*scene, make_cam_params(*cam), splats, vals, ranges, bg, final_T,
                                              n_contrib, dL_dcolor, static_cast<float *>(workspace), *grads,
                                              (cudaStream_t)stream));
}

const char *gs_strerror(int code) {
    switch (code) {
        case GS_OK: return "ok";
        case GS_ERR_INVALID_ARG: return "invalid argument (null or misaligned pointer, bad size or camera)";
        case GS_ERR_CAPACITY: return "tile instances exceed the key buffer capacity";
        case GS_ERR_CUDA: return g_cuda_err;
        case GS_ERR_TIMEOUT: return "bounded device wait timed out";
        case GS_ERR_TOO_LARGE: return "size exceeds the fixed scratch of gs_sort_static";
        default: return "unknown gs error code";
    }
}

const char *gs_last_cuda_error(void) { return g_cuda_err; }

int gs_version(void) { return 1; }

int gs_built_arch(void) { return GS_BUILT_ARCH; }

}  // extern "C"
