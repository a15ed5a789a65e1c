// gs_sort_static: gs_sort for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc or any allocating routine: code that
// runs inside another framework's allocator-managed region, a plugin handed
// only its input and output buffers, or a process whose memory pool is
// reserved up front.  This entry point runs exactly gs_sort's kernels, but
// takes its scratch from a fixed array compiled into the library instead of
// a caller-provided workspace.
//
// The array is a file-scope __device__ variable, so every GPU that loads
// the library holds it (42 MiB: the workspace gs_sort needs at the largest
// accepted n and m_cap, for any tile grid) until the process exits.  Host
// code cannot use the array's name as a device address, so the first call
// on each device resolves the address with cudaGetSymbolAddress (with that
// device current) and caches it; make that first call before any stream
// capture.  A failed lookup is not cached: the next call tries again.
// All calls share the one array: the part that must start at zero (the
// counters header) is cleared by every call, and calls whose work overlaps
// on the GPU (concurrent streams, or several host threads) race on it.
#include <mutex>

#include "common.cuh"
#include "sort_ws.h"

namespace gs {

cudaError_t launch_sort_front(const gs_splat *splats, int64_t n, const SortWs &ws, uint64_t m_cap, int tiles_x,
                              uint32_t num_tiles, cudaStream_t st);
cudaError_t launch_sort_back(const gs_splat *splats, int64_t n, const SortWs &ws, uint64_t m_cap, int tiles_x,
                             uint32_t num_tiles, uint64_t *keys, uint32_t *vals, uint32_t *ranges, cudaStream_t st);
void set_cuda_error(cudaError_t e);

namespace {

// The workspace at the largest accepted sizes; the tile grid only changes
// how many tile passes are laid out, and 2^32 tiles takes the most.
constexpr size_t kStaticBound =
    sort_ws_offsets(GS_SORT_STATIC_MAX_GAUSSIANS, GS_SORT_STATIC_MAX_INSTANCES, 1ull << 32).total;
constexpr size_t kStaticScratchBytes = (size_t)42 << 20;  // the size stated in gs.h
static_assert(kStaticScratchBytes >= kStaticBound, "static scratch below the workspace bound");
constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned char g_sort_scratch[kStaticScratchBytes];

std::mutex g_scratch_mutex;
void *g_scratch_ptr[kMaxDevices] = {};  // device address per device, once looked up

bool aligned(const void *p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

}  // namespace
}  // namespace gs

using namespace gs;

extern "C" int gs_sort_static(const gs_splat *splats, int64_t n, const gs_camera *cam, uint64_t *keys,
                              uint32_t *vals, int64_t m_cap, uint32_t *ranges, int64_t *m_out, void *stream) {
    if (n > GS_SORT_STATIC_MAX_GAUSSIANS || m_cap > GS_SORT_STATIC_MAX_INSTANCES) return GS_ERR_TOO_LARGE;
    if (!cam || n < 0 || m_cap < 0 || cam->width < 1 || cam->height < 1 || cam->width > 65535 * kTile ||
        cam->height > 65535 * kTile)
        return GS_ERR_INVALID_ARG;
    if (!ranges || !aligned(ranges, 8)) return GS_ERR_INVALID_ARG;
    if (n > 0 && (!splats || !aligned(splats, 16))) return GS_ERR_INVALID_ARG;
    if (m_cap > 0 && (!keys || !vals || !aligned(keys, 16) || !aligned(vals, 16))) return GS_ERR_INVALID_ARG;
    const uint64_t tiles_x = (uint64_t)((cam->width + kTile - 1) / kTile);
    const uint64_t num_tiles = tiles_x * (uint64_t)((cam->height + kTile - 1) / kTile);
    if (carve_sort_ws(nullptr, n, m_cap, num_tiles, nullptr) > kStaticScratchBytes) return GS_ERR_TOO_LARGE;

    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        set_cuda_error(e);
        return GS_ERR_CUDA;
    }
    if (dev < 0 || dev >= kMaxDevices) return GS_ERR_INVALID_ARG;
    void *scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_scratch_mutex);
        if (!g_scratch_ptr[dev]) {  // only a successful lookup is kept
            void *p = nullptr;
            e = cudaGetSymbolAddress(&p, g_sort_scratch);
            if (e != cudaSuccess || !p) {
                set_cuda_error(e != cudaSuccess ? e : cudaErrorInvalidSymbol);
                return GS_ERR_CUDA;
            }
            g_scratch_ptr[dev] = p;
        }
        scratch = g_scratch_ptr[dev];
    }

    cudaStream_t st = (cudaStream_t)stream;
    SortWs ws;
    carve_sort_ws(static_cast<char *>(scratch), n, m_cap, num_tiles, &ws);
    e = launch_sort_front(splats, n, ws, (uint64_t)m_cap, (int)tiles_x, (uint32_t)num_tiles, st);
    if (e == cudaSuccess && m_out) {
        SortHeader h;
        e = cudaMemcpyAsync(&h, ws.hdr, sizeof(h), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e == cudaSuccess) {
            *m_out = (int64_t)h.m_total;
            if (h.timeout) return GS_ERR_TIMEOUT;
            if (h.m_total > (uint64_t)m_cap) return GS_ERR_CAPACITY;
        }
    }
    if (e == cudaSuccess)
        e = launch_sort_back(splats, n, ws, (uint64_t)m_cap, (int)tiles_x, (uint32_t)num_tiles, keys, vals, ranges,
                             st);
    if (e != cudaSuccess) {
        set_cuda_error(e);
        return GS_ERR_CUDA;
    }
    return GS_OK;
}
