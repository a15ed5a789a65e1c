/*
 * gs.h -- C ABI of the GB300 (sm_103a) 3D Gaussian splatting hot path.
 *
 * The forward pass follows the pipeline of Section II-B of "LLM-Powered Code
 * Analysis and Optimization for Gaussian Splatting Kernels" (arXiv
 * 2509.25626): (1) preprocessing -- cull, project each 3D Gaussian to a 2D
 * splat with colour and depth, replicate it for every 16x16 pixel tile it
 * touches, sort the replicas by depth within each tile; (2) alpha blending --
 * per-tile ranges, then one thread block per tile blends its splats front to
 * back (Eq. 1, Algorithm 1).
 *
 *   gs_preprocess   per-Gaussian projection, colour, radius, tile rectangle
 *   gs_sort         key duplication, radix sort, per-tile ranges
 *   gs_render       per-tile front-to-back alpha blending
 *
 * Conventions shared by every call:
 *   - Every pointer argument named as device memory must point to memory of
 *     the current CUDA device.  The caller owns every buffer and the stream;
 *     the library allocates nothing and keeps no state between calls.
 *   - `stream` is a cudaStream_t passed as void*; NULL means the legacy
 *     default stream.  Calls only enqueue work (no host synchronisation)
 *     unless stated otherwise.
 *   - Return value: GS_OK (0) or a negative GS_ERR_* code.  Argument checks
 *     happen before any launch; a launch failure returns GS_ERR_CUDA and
 *     gs_last_cuda_error() names the CUDA error.  No C++ exception crosses
 *     this boundary.
 *   - Pixel (px, py) has its centre at integer coordinates; images are
 *     row-major, channel-major for colour ([3][H][W]).
 */
#ifndef GS_H_
#define GS_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GS_TILE 16 /* tile edge in pixels (Section II-B: default 16 x 16) */

enum {
    GS_OK = 0,
    GS_ERR_INVALID_ARG = -1, /* null/misaligned pointer, bad size or camera */
    GS_ERR_CAPACITY = -2,    /* more tile instances than the key buffers hold */
    GS_ERR_CUDA = -3,        /* a CUDA launch or runtime call failed */
    GS_ERR_TIMEOUT = -4,     /* a bounded device-side wait gave up */
    GS_ERR_TOO_LARGE = -5,   /* size beyond gs_sort_static's fixed scratch */
};

/* Pinhole camera, OpenCV axes (x right, y down, z forward).  Host memory. */
typedef struct gs_camera {
    float viewmat[16];   /* world -> camera, row-major 4x4; last row 0 0 0 1 */
    float fx, fy;        /* focal lengths in pixels */
    float cx, cy;        /* principal point in pixels */
    int32_t width;       /* image size in pixels, 1 .. 65535 * 16 */
    int32_t height;
    float tan_fovx;      /* tan(half field of view); the EWA Jacobian is */
    float tan_fovy;      /* evaluated inside 1.3 x these (3DGS frustum slack) */
} gs_camera;

/* Scene parameters: float32 structure-of-arrays in device memory, each array
 * 16-byte aligned.  n may be 0. */
typedef struct gs_scene {
    const float *means;          /* [n][3] world-space centres */
    const float *log_scales;     /* [n][3] log standard deviations per axis */
    const float *quats;          /* [n][4] rotation (w, x, y, z), any norm > 0 */
    const float *opacity_logits; /* [n] opacity = sigmoid(logit) */
    const float *sh;             /* [n][16][3] SH coefficients, RGB-minor */
    int64_t n;
    int32_t sh_degree;           /* 0 .. 3 bands used (the array is always 16) */
    int32_t reserved;
} gs_scene;

/* One projected Gaussian ("splat"), written by gs_preprocess: 64 bytes.
 * The 2D covariance Sigma' = J W Sigma W^T J^T + 0.3 I is stored through an
 * upper-triangular factor of its inverse, scaled so that for d = (x, y) - p
 *     -0.5 d^T Sigma'^-1 d * log2(e) = -(u*u + v*v),
 *     u = w00 dx + w01 dy,   v = w11 dy,
 * and alpha = min(0.99, 2^(log2_opacity - u*u - v*v)).
 * cull_hx / cull_hy bound the region where alpha can reach 1/255: outside
 * |dx| <= cull_hx, |dy| <= cull_hy the splat is skipped for every pixel (the
 * bound is the ellipse's bounding box, widened by 2^-10 relative + 1/64
 * pixel to absorb FP32 rounding); both are negative if alpha < 1/255
 * everywhere.  A culled Gaussian has radius = 0, tiles_touched = 0, an
 * empty rectangle, negative cull_hx / cull_hy and its depth; gs_preprocess
 * leaves its other fields (x .. g) unwritten, since it is in no tile list. */
typedef struct gs_splat {
    float x, y;               /* pixel-space mean */
    float w00, w01, w11;      /* inverse-covariance factor (see above) */
    float log2_opacity;       /* log2(sigmoid(logit)) */
    float r, g, b;            /* SH colour + 0.5, clamped at 0 */
    float cull_hx, cull_hy;   /* half-extents of the alpha >= 1/255 region */
    int32_t radius;           /* ceil(3 sqrt(lambda_max(Sigma'))) pixels */
    float depth;              /* view-space z, FP32; its bits form the sort key */
    uint32_t tiles_touched;   /* (x1 - x0) (y1 - y0) */
    uint32_t rect_lo;         /* x0 | y0 << 16, tile rectangle, inclusive */
    uint32_t rect_hi;         /* x1 | y1 << 16, exclusive */
} gs_splat;

/* The sort's inputs of one splat, 16 bytes: the last four words of its
 * record, repeated.  gs_preprocess writes them a second time, densely, after
 * the n records of the splat buffer, so that gs_sort reads 16 bytes per
 * Gaussian instead of a 64-byte record (DRAM moves whole 64-byte
 * granules). */
typedef struct gs_sort_input {
    uint32_t depth_bits;    /* float bits of gs_splat.depth */
    uint32_t tiles_touched;
    uint32_t rect_lo, rect_hi;
} gs_sort_input;

/* Bytes of a splat buffer for n Gaussians: n gs_splat records followed by n
 * gs_sort_input vectors (80 n bytes). */
size_t gs_splat_buffer_bytes(int64_t n);

/* Section II-B (1), projection step.  One thread per Gaussian:
 *   z = V.[m, 1] (FP32, fmaf(V22, mz, fmaf(V21, my, fmaf(V20, mx, V23))));
 *   cull if z <= 0.2;
 *   Sigma = R(q) diag(exp(2 s)) R(q)^T;  J at the mean clamped to 1.3 tan(fov);
 *   Sigma' = J W Sigma W^T J^T + 0.3 I;
 *   radius = ceil(3 sqrt(lambda_max)), lambda_max = mid + sqrt(max(0.1, mid^2 - det));
 *   rect = [floor((p - r) / 16), floor((p + r + 15) / 16)) clamped to the grid; cull if empty;
 *   colour = max(sum_lm c_lm Y_lm(dir) + 0.5, 0), dir from the camera centre to the mean.
 * scene: device arrays; cam: host struct; splats: device splat buffer of
 * gs_splat_buffer_bytes(n) bytes, 16-byte aligned: [n] records, then [n]
 * gs_sort_input.  Errors: GS_ERR_INVALID_ARG, GS_ERR_CUDA. */
int gs_preprocess(const gs_scene *scene, const gs_camera *cam, gs_splat *splats, void *stream);

/* Cameras in device memory.  gs_preprocess takes the camera as kernel
 * parameters, which a captured CUDA graph freezes; a server that replays one
 * captured preprocess + sort per (scene, resolution) for every request
 * instead keeps the camera in device memory and rewrites it before each
 * replay (e.g. by a host-to-device copy captured in the same graph).
 * gs_camera_block writes the kernels' form of `cam` (host, 16-byte
 * aligned, gs_camera_block_bytes() bytes; the camera centre -R^T t is
 * formed in double) into host memory `block`; gs_preprocess_camblock is
 * gs_preprocess with that block read from device memory (16-byte aligned)
 * when the kernel runs.  The block holds the image size: the gs_sort and
 * gs_render calls of the same frame must use a camera of that size.
 * Errors: GS_ERR_INVALID_ARG, GS_ERR_CUDA. */
size_t gs_camera_block_bytes(void);
int gs_camera_block(const gs_camera *cam, void *block);
int gs_preprocess_camblock(const gs_scene *scene, const void *camera_block, gs_splat *splats, void *stream);

/* Bytes of device workspace gs_sort needs for n Gaussians, m_cap tile
 * instances and num_tiles = ceil(W/16) * ceil(H/16) tiles (the workspace
 * must be 256-byte aligned).  gs_sort also uses the key buffer (8 bytes per
 * instance) as scratch until its last pass. */
size_t gs_sort_workspace_bytes(int64_t n, int64_t m_cap, int32_t num_tiles);

/* Section II-B: replicate every visible splat for each tile of its
 * rectangle with key (tile_id << 32 | float_bits(depth)), tile_id =
 * ty * ceil(W/16) + tx, value = Gaussian id; sort stably by key (ties keep
 * ascending id); ranges[t] = [start, end) of tile t's instances in the sorted
 * list, [0, 0) for an empty tile (Algorithm 1, "load work range").
 *
 * splats: device splat buffer from gs_preprocess with the same camera
 * (gs_sort reads its gs_sort_input part, after the n records).
 * keys, vals: device, capacity m_cap each (8- and 4-byte elements, 16-byte
 * aligned); on return the first M entries hold the sorted instances.
 * ranges: device, [num_tiles][2] uint32.
 * workspace: device, gs_sort_workspace_bytes(n, m_cap, num_tiles) bytes.
 * m_out: HOST pointer or NULL.  If non-NULL the call synchronises the stream
 * once to read M, stores it, and returns GS_ERR_CAPACITY (having written
 * nothing else) when M > m_cap, GS_ERR_TIMEOUT if a bounded wait gave up.  If NULL the call never synchronises: M
 * stays on the device, an overflow is recorded there, only the first m_cap
 * instances are sorted, and gs_sort_status() reports it later.
 * Errors: GS_ERR_INVALID_ARG, GS_ERR_CAPACITY, GS_ERR_CUDA. */
int gs_sort(const gs_splat *splats, int64_t n, const gs_camera *cam, uint64_t *keys, uint32_t *vals,
            int64_t m_cap, uint32_t *ranges, void *workspace, size_t workspace_bytes, int64_t *m_out,
            void *stream);

/* Read back the device-side instance count and overflow flag of the last
 * gs_sort that used `workspace` (synchronises `stream`).  m_out: host, the
 * true M (which may exceed m_cap).  Returns GS_OK, GS_ERR_CAPACITY, or
 * GS_ERR_TIMEOUT if one of the sort's bounded inter-block waits gave up
 * (the output is then invalid; it does not happen when blocks progress). */
int gs_sort_status(const void *workspace, int64_t *m_out, void *stream);

/* Section II-B (2), Algorithm 1, Eq. 1: one 16x16 thread block per tile walks
 * ranges[tile] of the sorted values front to back; per pixel p and splat g:
 *   alpha = min(0.99, o_g exp(-0.5 d^T Sigma'^-1 d)), d = (x_g, y_g) - p;
 *   skip if alpha < 1/255; stop (without blending g) once T (1 - alpha) < 1e-4;
 *   C += rgb_g alpha T; T *= 1 - alpha.
 * Writes out_color[c][py][px] = C_c + T bg_c, final_T[py][px] = T and
 * n_contrib[py][px] = 1-based list position of the last blended splat.
 * splats, vals, ranges: device inputs from gs_preprocess / gs_sort; bg: host
 * float[3]; out_color [3][H][W], final_T [H][W], n_contrib [H][W]: device,
 * 4-byte elements.  Errors: GS_ERR_INVALID_ARG, GS_ERR_CUDA. */
int gs_render(const gs_splat *splats, const uint32_t *vals, const uint32_t *ranges, const gs_camera *cam,
              const float bg[3], float *out_color, float *final_T, uint32_t *n_contrib, void *stream);

/* gs_render with contribution-aware rasterization, the algorithmic change of
 * the Seele renderer the paper's case study optimises (Section III): per
 * staged batch, each group of 32 lanes (one warp, 8x8 pixels) first builds,
 * by warp votes, the mask of the splats whose alpha reaches 1/255 at one of
 * the group's still-live pixels, then blends only those; the mask is the
 * exact per-pixel test, so images, final_T and n_contrib equal gs_render's
 * bit for bit.  Arguments and errors as gs_render. */
int gs_render_contrib(const gs_splat *splats, const uint32_t *vals, const uint32_t *ranges, const gs_camera *cam,
                      const float bg[3], float *out_color, float *final_T, uint32_t *n_contrib, void *stream);

/* Gradients of a loss with respect to the scene parameters (device, each
 * [n]-major like gs_scene, written -- not accumulated -- by the call). */
typedef struct gs_scene_grads {
    float *dmeans;          /* [n][3] */
    float *dlog_scales;     /* [n][3] */
    float *dquats;          /* [n][4] */
    float *dopacity_logits; /* [n] */
    float *dsh;             /* [n][16][3]; bands above sh_degree get 0 */
} gs_scene_grads;

/* Bytes of device workspace gs_render_backward needs for n Gaussians.  On
 * return the workspace holds, per Gaussian, the gradient with respect to its
 * 2D splat: float [n][12] = dL/d(x, y, conic a, b, c, opacity, r, g, b)
 * and 3 unused floats (power = -(a dx^2 + c dy^2)/2 - b dx dy). */
size_t gs_backward_workspace_bytes(int64_t n);

/* Backward of gs_preprocess + gs_render for the same scene, camera and
 * background, given dL_dcolor [3][H][W] (device): Eq. 1 differentiated per
 * pixel back to front from n_contrib, the transmittance in front of each
 * blended splat recovered from final_T as T_after / (1 - alpha) (no
 * per-splat state is kept by the forward), then the chain rule through the
 * preprocessing of Section II-B (1).  Piecewise: skipped splats, the 0.99
 * clamp and clamped colour channels pass no gradient; the tile lists and the
 * sort are constant.  splats, vals, ranges, final_T, n_contrib: the forward's
 * outputs.  workspace: gs_backward_workspace_bytes(n) bytes, 16-byte aligned.
 * Equivalent to gs_render_backward_splats into the workspace, then
 * gs_preprocess_backward.  Errors: GS_ERR_INVALID_ARG, GS_ERR_CUDA. */
int gs_render_backward(const gs_scene *scene, const gs_camera *cam, const gs_splat *splats, const uint32_t *vals,
                       const uint32_t *ranges, const float bg[3], const float *final_T, const uint32_t *n_contrib,
                       const float *dL_dcolor, void *workspace, size_t workspace_bytes,
                       const gs_scene_grads *grads, void *stream);

/* The first half of gs_render_backward: the per-splat 2D gradients alone
 * (Eq. 1 differentiated per pixel, as above).  dsplat: float [n][12]
 * (device, 16-byte aligned), zeroed by the call and filled with
 * dL/d(x, y, conic a, b, c, opacity, r, g, b) per Gaussian (3 floats
 * unused); Gaussians in no list get zeros.  The pixel-space mean gradient is
 * what densification heuristics read.  Other arguments as for
 * gs_render_backward, n = the scene's Gaussian count.
 * Errors: GS_ERR_INVALID_ARG, GS_ERR_CUDA. */
int gs_render_backward_splats(const gs_camera *cam, const gs_splat *splats, int64_t n, const uint32_t *vals,
                              const uint32_t *ranges, const float bg[3], const float *final_T,
                              const uint32_t *n_contrib, const float *dL_dcolor, float *dsplat, void *stream);

/* The second half of gs_render_backward: the chain rule from the per-splat
 * gradients dsplat (gs_render_backward_splats' output, float [n][12],
 * device) through the preprocessing of Section II-B (1) to the scene
 * parameters.  splats: gs_preprocess's output for the same scene and camera.
 * Every gradient array is written in full (zeros for culled Gaussians).
 * Errors: GS_ERR_INVALID_ARG, GS_ERR_CUDA. */
int gs_preprocess_backward(const gs_scene *scene, const gs_camera *cam, const gs_splat *splats, const float *dsplat,
                           const gs_scene_grads *grads, void *stream);

/* gs_render plus, per pixel, the number of splats evaluated before the
 * pixel stopped (the stopping splat included; all of the tile's splats if it
 * never stopped): n_eval [H][W] uint32, device.  Its sum over the image is
 * the "Gaussian-pixel evaluations" work count, the per-thread workload
 * measure of the paper's Table III.  tile_cycles (device uint32
 * [tiles_y][tiles_x], or NULL): SM clock cycles the block spent on each
 * tile, from its first instruction to its last store (saturated at
 * 2^32 - 1) -- the per-block load-balance measure of Section IV-C.
 * Slightly slower than gs_render; meant for workload characterisation, not
 * for the hot path.  Errors: as gs_render. */
int gs_render_workload(const gs_splat *splats, const uint32_t *vals, const uint32_t *ranges, const gs_camera *cam,
                       const float bg[3], float *out_color, float *final_T, uint32_t *n_contrib, uint32_t *n_eval,
                       uint32_t *tile_cycles, void *stream);

/* One forward frame: gs_preprocess, gs_sort (m_out = NULL: no host
 * synchronisation; an overflow of m_cap is recorded in the workspace and
 * read with gs_sort_status) and gs_render, enqueued on `stream` in one call.
 * Arguments and errors as those calls. */
int gs_frame(const gs_scene *scene, const gs_camera *cam, gs_splat *splats, uint64_t *keys, uint32_t *vals,
             int64_t m_cap, uint32_t *ranges, void *workspace, size_t workspace_bytes, const float bg[3],
             float *out_color, float *final_T, uint32_t *n_contrib, void *stream);

/* gs_render with optional outputs, each NULL to skip (the same per-pixel
 * blend, so out_color, final_T and n_contrib equal gs_render's bit for bit):
 *   invdepth [H][W] float: the inverse depth blended like a colour channel,
 *     without background -- sum over the blended splats of
 *     alpha T / depth (the optional output of the paper's render kernels,
 *     Appendix B listings);
 *   n_eval, tile_cycles: as gs_render_workload (tile_cycles needs n_eval).
 * Device buffers, 4-byte aligned.  Errors: as gs_render. */
int gs_render_ex(const gs_splat *splats, const uint32_t *vals, const uint32_t *ranges, const gs_camera *cam,
                 const float bg[3], float *out_color, float *final_T, uint32_t *n_contrib, float *invdepth,
                 uint32_t *n_eval, uint32_t *tile_cycles, void *stream);

/* gs_sort without a caller-provided workspace, for callers that cannot
 * allocate device memory: code running inside another framework's memory
 * pool, a plugin that is handed only its input and output buffers, or a
 * service that reserves all device memory up front.  The paper has no
 * counterpart; this is a deployment convenience.
 *
 * Same arguments, results and errors as gs_sort minus the workspace.  The
 * scratch is a fixed 42 MiB array inside the library (the workspace gs_sort
 * needs at the largest accepted n and m_cap, for any tile grid), which every
 * GPU that loads the library holds until the process exits; it bounds the
 * sizes:
 * n <= GS_SORT_STATIC_MAX_GAUSSIANS and m_cap <= GS_SORT_STATIC_MAX_INSTANCES,
 * else GS_ERR_TOO_LARGE (checked before any GPU work).  The call allocates
 * nothing.  The first call on each device looks up the array's device
 * address (cudaGetSymbolAddress, with that device current) and caches it:
 * make that first call before any stream capture (a lookup that fails is
 * not cached, so a later call outside capture retries it).  All calls share the
 * array; each call clears the counters that must start at zero, but calls
 * whose work overlaps on the GPU (other streams, other host threads) race on
 * it, so serialise them.  With m_out NULL an overflow cannot be read back
 * (the counters live in the shared array): pass m_out unless m_cap bounds M. */
#define GS_SORT_STATIC_MAX_GAUSSIANS (1 << 19)
#define GS_SORT_STATIC_MAX_INSTANCES (1 << 21)
int gs_sort_static(const gs_splat *splats, int64_t n, const gs_camera *cam, uint64_t *keys, uint32_t *vals,
                   int64_t m_cap, uint32_t *ranges, int64_t *m_out, void *stream);

/* One request of a batched render: the inputs and outputs of a gs_render
 * call (all device pointers) plus its first work item.  72 bytes. */
typedef struct gs_render_job {
    const gs_splat *splats;
    const uint32_t *vals;
    const uint32_t *ranges;
    float *out_color;       /* [3][height][width] */
    float *final_T;         /* [height][width] */
    uint32_t *n_contrib;    /* [height][width] */
    int32_t width, height;
    float bg[3];
    uint32_t tile_begin;    /* sum of the tile counts of the jobs before it */
} gs_render_job;

/* A batch, in device memory: jobs[0 .. n_jobs) sorted by tile_begin, and
 * total_tiles = the sum of all their tile counts. */
typedef struct gs_render_batch_desc {
    int32_t n_jobs;
    uint32_t total_tiles;
    uint64_t reserved;
    gs_render_job jobs[1];  /* n_jobs entries follow */
} gs_render_batch_desc;

/* gs_render for many requests in one persistent launch: blocks take (job,
 * tile) work items from `counter` (device uint32, reset by the call) and run
 * exactly gs_render's per-tile blend on each, so every job's outputs equal a
 * gs_render call with the same inputs, bit for bit.  The batch is read from
 * device memory, so the call (a memset and one kernel) can be captured once
 * in a CUDA graph and replayed for any batch after rewriting `desc`.
 * grid: blocks to launch, 0 = one full wave of the device (looked up on the
 * first such call per device; make that call before any stream capture).
 * The caller must keep jobs' buffers alive until the launch completes.
 * Errors: GS_ERR_INVALID_ARG, GS_ERR_CUDA. */
int gs_render_batch(const gs_render_batch_desc *desc, uint32_t *counter, int32_t grid, void *stream);

/* Failure-detection check of the sort's bounded waits (the paper has no
 * counterpart).  gs_sort's radix passes and scans learn earlier blocks'
 * counts by decoupled look-back; a block whose predecessor never publishes
 * (it stalled or died) must not spin forever.  This call runs one look-back
 * walk of block 1 whose predecessor, block 0, never runs, with its wait
 * bounded by limit_ns nanoseconds (1 .. 1e9; gs_sort itself uses 1 s),
 * synchronises `stream`, and returns GS_ERR_TIMEOUT when the wait gave up
 * as it must (GS_OK would mean it found a flag nobody wrote).  workspace:
 * device, 256-byte aligned, >= gs_sort_workspace_bytes(1, 1, 1) bytes; its
 * header then records the timeout exactly as a failed gs_sort would, so
 * gs_sort_status on it returns GS_ERR_TIMEOUT too.  The context stays
 * usable.  Errors: GS_ERR_INVALID_ARG, GS_ERR_CUDA. */
int gs_check_wait_timeout(void *workspace, size_t workspace_bytes, uint64_t limit_ns, void *stream);

/* Settings of gs_render_batch_balanced. */
typedef struct gs_balance_params {
    int32_t heavy_len;       /* tiles whose list holds >= heavy_len splats start first; 0 = off */
    int32_t max_heavy_tiles; /* capacity of that queue; if more tiles qualify, the plain order is kept */
    int32_t budget;          /* splats walked before a still-live tile is split; 0 = never split */
    int32_t max_split_tiles; /* capacity of the split queue; further tiles are walked whole */
    int32_t max_chunks;      /* chunks walked per split tile, 1 .. 64 (with budget > 0) */
    int32_t chunk;           /* splats per chunk, >= 1, rounded up to 256 (with budget > 0) */
} gs_balance_params;

/* Bytes of device workspace gs_render_batch_balanced needs (256-byte
 * aligned); 0 if the parameters are invalid. */
size_t gs_render_balance_workspace_bytes(const gs_balance_params *params);

/* gs_render_batch with the inter-block load imbalance of heavy tiles
 * (Section IV-C, Table III; the list splitting of Balanced-3DGS, Section
 * II-A) evened out, in up to four launches enqueued on `stream`:
 *   0. (heavy_len > 0) the (job, tile) items whose list holds at least
 *      heavy_len splats are queued; the persistent render takes them first,
 *      so a long list is not picked up at the end of the launch;
 *   1. the persistent batch render, except that (budget > 0) a block that
 *      has walked `budget` splats of a tile's list while some pixel is still
 *      live saves the pixels' state (C, T, last blended position) and queues
 *      the rest of the list instead of walking it;
 *   2. (budget > 0) the next max_chunks chunks of `chunk` splats of each
 *      queued list walked in parallel from T = 1 into per-chunk partial (C,
 *      T, last, stopped);
 *   3. (budget > 0) per queued tile, the chunks combined front to back:
 *      C += T C_k, T *= T_k, while T T_k >= 1e-4 and chunk k did not stop;
 *      the chunk where the absolute transmittance crosses 1e-4 is walked
 *      again from the true incoming (C, T), so each pixel stops exactly
 *      where one walk of the whole list stops; the list beyond the chunks,
 *      if a pixel still needs it, is walked there too.
 * Without splitting every job's outputs equal gs_render's bit for bit (only
 * the order of the tiles changes); split tiles equal it up to the FP32
 * rounding of the regrouped products (the same decisions off the
 * thresholds).  desc, counter, grid: as gs_render_batch.  workspace:
 * gs_render_balance_workspace_bytes(params) bytes, 256-byte aligned.
 * Errors: GS_ERR_INVALID_ARG, GS_ERR_CUDA. */
int gs_render_batch_balanced(const gs_render_batch_desc *desc, uint32_t *counter, const gs_balance_params *params,
                             void *workspace, size_t workspace_bytes, int32_t grid, void *stream);

/* Text for a GS_* code, or the CUDA error string of the last GS_ERR_CUDA. */
const char *gs_strerror(int code);
const char *gs_last_cuda_error(void);

/* Library version and the compute capability it was built for (e.g. 103). */
int gs_version(void);
int gs_built_arch(void);

#ifdef __cplusplus
}
#endif

#endif /* GS_H_ */
