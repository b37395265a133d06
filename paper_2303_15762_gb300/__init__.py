"""GB300-native backward path tracing of generalized rays (arXiv 2303.15762).

The compute path is libgr.so (hand-written CUDA for sm_103a, C ABI in
include/gr.h); this package is its thin binding (``_native``), the seeded input
generators (``scenegen``) and the build script (``build``).  The binding is
loaded lazily so that importing the input generators needs neither torch nor a
GPU.
"""
from . import scenegen  # noqa: F401

_NATIVE_NAMES = ("Scene", "Frame", "render", "render_image", "make_opts", "GrError", "lib_handle",
                 "FLAG_NEE", "FLAG_RR", "FLAG_NO_RENORM", "FLAG_WIDE_BVH", "FLAG_HERO", "FLAG_ANISO", "FLAG_FP32_NODES", "pack_views", "current_stream", "debug_rng",
                 "render_multi", "measure_fp32_peak", "debug_order_table", "debug_footprint",
                 "aperture_backward_2d", "aperture_backward_3d", "accum_floats",
                 "render_scratch_bytes")


def load():
    """Load libgr.so (raises if it is missing or no CUDA device is present)."""
    from . import _native
    return _native.lib_handle()


def __getattr__(name):
    if name in _NATIVE_NAMES:
        from . import _native
        return getattr(_native, name)
    raise AttributeError(name)
