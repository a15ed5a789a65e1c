"""GB300 (sm_103a) CUDA implementation of the 3D Gaussian splatting forward
hot path: preprocess -> duplicate keys -> radix sort -> tile ranges ->
per-tile alpha blending, behind the C ABI in include/gs.h (libgs.so).
"""

from ._lib import GS_ERR_CAPACITY, GS_ERR_CUDA, GS_ERR_INVALID_ARG, GS_ERR_TOO_LARGE, GS_OK, SPLAT_DTYPE, GsError  # noqa: F401
from .api import (  # noqa: F401
    BalanceParams,
    BatchJob,
    RenderBatch,
    balance_workspace,
    Renderer,
    FramePipeline,
    RasterizeGaussians,
    rasterize,
    render_backward,
    render_backward_splats,
    preprocess_backward,
    SceneTensors,
    camera_struct,
    num_tiles,
    preprocess,
    render,
    render_contrib,
    render_workload,
    render_invdepth,
    sort,
    sort_static,
    sort_status,
    sort_workspace_bytes,
    splat_buffer,
)
