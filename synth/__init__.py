"""Seeded synthetic inputs for the Gaussian-splatting hot path.

This package draws scenes (Gaussian parameters) and pinhole cameras with
numpy.  It holds none of the renderer's arithmetic: no projection, no
covariance, no colour, no blending.  Both the FP64 CPU oracle (through the
tests and the CPU-baseline leg of the benchmark) and the CUDA path consume the
arrays it returns, so neither side depends on the other for its inputs.
"""

from .scenes import (  # noqa: F401
    Camera,
    Scene,
    CONFIGS,
    pinhole_camera,
    orbit_camera,
    uniform_box_scene,
    clustered_scene,
    slab_scene,
    tiny_scene,
    needle_scene,
    concat_scenes,
    subset_scene,
)
