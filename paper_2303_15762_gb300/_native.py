"""ctypes binding of libgr.so (include/gr.h): argument marshalling only.

Every step of rendering runs in the library's CUDA kernels; this module packs
the scene generator's arrays into the C structs, passes PyTorch's current CUDA
stream, and unpacks results.  There is no CPU fallback: without a CUDA device
or without the built library every call raises.
"""
import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libgr.so")

GR_OK, GR_E_INVALID, GR_E_OOM, GR_E_CUDA, GR_E_TIMEOUT, GR_E_BUSY = range(6)
FLAG_NEE, FLAG_RR, FLAG_NO_RENORM, FLAG_WIDE_BVH, FLAG_HERO, FLAG_ANISO, FLAG_FP32_NODES = 1, 2, 4, 8, 16, 32, 64
TABLE_DTYPES = {"f32": 0, "f16": 1, "bf16": 2}

EXPORTED = ["gr_scene_create", "gr_scene_destroy", "gr_frame_create", "gr_frame_wrap", "gr_frame_reset", "gr_frame_release",
            "gr_render", "gr_readback", "gr_frame_stats", "gr_scene_bvh", "gr_debug_rng", "gr_render_static", "gr_render_multi",
            "gr_last_error", "gr_abi_version", "gr_measure_fp32_peak", "gr_debug_order_table",
            "gr_debug_footprint", "gr_aperture_backward_2d", "gr_scene_bytes", "gr_frame_bytes",
            "gr_render_scratch_bytes", "gr_aperture_backward_3d"]


class GrError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("gr status %d: %s" % (status, msg))
        self.status = status


class gr_material(ctypes.Structure):
    _fields_ = [("type", ctypes.c_int32), ("fresnel", ctypes.c_int32), ("n_re", ctypes.c_float),
                ("n_im", ctypes.c_float), ("period_um", ctypes.c_float), ("height_um", ctypes.c_float),
                ("gdir", ctypes.c_float * 3), ("sigma_h_um", ctypes.c_float), ("corr_len_um", ctypes.c_float),
                ("Le", ctypes.c_float), ("coh_len_um", ctypes.c_float), ("cauchy_b_um2", ctypes.c_float),
                ("reserved", ctypes.c_float * 2)]


class gr_light(ctypes.Structure):
    _fields_ = [("type", ctypes.c_int32), ("dir", ctypes.c_float * 3), ("E", ctypes.c_float),
                ("coh_len_um", ctypes.c_float), ("reserved", ctypes.c_float * 2)]


class gr_scene_desc(ctypes.Structure):
    _fields_ = [("n_tris", ctypes.c_int32), ("verts", ctypes.c_void_p), ("tri_mat", ctypes.c_void_p),
                ("n_mats", ctypes.c_int32), ("mats", ctypes.c_void_p), ("n_lights", ctypes.c_int32),
                ("lights", ctypes.c_void_p)]


class gr_view_desc(ctypes.Structure):
    _fields_ = [("eye", ctypes.c_float * 3), ("look_at", ctypes.c_float * 3), ("up", ctypes.c_float * 3),
                ("vfov_deg", ctypes.c_float), ("width", ctypes.c_int32), ("height", ctypes.c_int32),
                ("p_pix_um", ctypes.c_float), ("f_beta", ctypes.c_float), ("lambda_min_um", ctypes.c_float),
                ("lambda_max_um", ctypes.c_float), ("n_bins", ctypes.c_int32), ("n_stokes", ctypes.c_int32),
                ("max_depth", ctypes.c_int32), ("spp", ctypes.c_int32), ("first_sample", ctypes.c_int32),
                ("view_index", ctypes.c_int32), ("scene_index", ctypes.c_int32), ("ortho", ctypes.c_int32),
                ("ortho_half_m", ctypes.c_float)]


class gr_render_opts(ctypes.Structure):
    _fields_ = [("seed", ctypes.c_uint32), ("flags", ctypes.c_int32), ("table_dtype", ctypes.c_int32),
                ("pool_size", ctypes.c_int32), ("block", ctypes.c_int32), ("use_graph", ctypes.c_int32),
                ("max_iterations", ctypes.c_int32), ("profile", ctypes.c_int32),
                ("regen_threshold_pct", ctypes.c_int32)]


class gr_stats(ctypes.Structure):
    _fields_ = [("samples", ctypes.c_int64), ("segments", ctypes.c_int64), ("shadow_rays", ctypes.c_int64),
                ("refine64_hits", ctypes.c_int64), ("refine64_lobes", ctypes.c_int64),
                ("iterations", ctypes.c_int64), ("kernel_launches", ctypes.c_int64),
                ("node_visits", ctypes.c_int64), ("tri_tests", ctypes.c_int64),
                ("kernel_ms", ctypes.c_double * 4), ("kernel_count", ctypes.c_int64 * 4)]


_lib = None


def lib_handle(require_gpu=True):
    """Load libgr.so.  With require_gpu (the default for every compute call)
    a CUDA device must be present."""
    global _lib
    if require_gpu:
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("libgr needs a CUDA device; there is no CPU fallback")
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("libgr.so is not built (run __graft_entry__.build() or "
                           "python -m paper_2303_15762_gb300.build)")
    L = ctypes.CDLL(LIB_PATH)
    P, I32 = ctypes.c_void_p, ctypes.c_int32
    L.gr_scene_create.argtypes = [P, P, P]
    L.gr_scene_destroy.argtypes = [P]
    L.gr_frame_create.argtypes = [P, I32, P, P]
    L.gr_frame_wrap.argtypes = [P, I32, P, P, P]
    L.gr_frame_reset.argtypes = [P, P]
    L.gr_frame_release.argtypes = [P]
    L.gr_render.argtypes = [P, I32, P, I32, P, P, P]
    L.gr_readback.argtypes = [P, I32, P, ctypes.c_size_t, I32, P]
    L.gr_frame_stats.argtypes = [P, P, P]
    L.gr_scene_bvh.argtypes = [P, P, P, P, P]
    U32 = ctypes.c_uint32
    L.gr_debug_rng.argtypes = [U32, U32, U32, U32, I32, I32, I32, P, P]
    L.gr_render_static.argtypes = [P, I32, P, I32, P, P, P]
    L.gr_render_multi.argtypes = [P, I32, P, I32, P, P, P, P]
    L.gr_scene_bytes.argtypes = [P, P]
    L.gr_frame_bytes.argtypes = [P, P]
    L.gr_render_scratch_bytes.argtypes = [P, I32, P, I32, P, P]
    L.gr_last_error.restype = ctypes.c_char_p
    L.gr_abi_version.restype = I32
    for name in EXPORTED:
        if name not in ("gr_last_error", "gr_abi_version"):
            getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


def _check(status):
    if status != GR_OK:
        raise GrError(status, _lib.gr_last_error().decode(errors="replace"))


def current_stream():
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def pack_view(v):
    d = gr_view_desc()
    d.eye[:] = v["eye"]
    d.look_at[:] = v["look_at"]
    d.up[:] = v["up"]
    d.vfov_deg = v["vfov_deg"]
    d.width, d.height = v["width"], v["height"]
    d.p_pix_um, d.f_beta = v["p_pix_um"], v["f_beta"]
    d.lambda_min_um, d.lambda_max_um = v["lambda_min_um"], v["lambda_max_um"]
    d.n_bins, d.n_stokes, d.max_depth = v["n_bins"], v["n_stokes"], v["max_depth"]
    d.spp, d.first_sample = v["spp"], v.get("first_sample", 0)
    d.view_index, d.scene_index = v.get("view_index", 0), v.get("scene_index", 0)
    d.ortho, d.ortho_half_m = v.get("ortho", 0), v.get("ortho_half_m", 0.0)
    return d


def pack_views(views):
    arr = (gr_view_desc * len(views))()
    for i, v in enumerate(views):
        arr[i] = pack_view(v)
    return arr


def _pack_materials(rows):
    rows = np.asarray(rows, dtype=np.float32).reshape(-1, 16)
    arr = (gr_material * max(1, len(rows)))()
    for i, r in enumerate(rows):
        m = arr[i]
        m.type, m.fresnel = int(r[0]), int(r[1])
        m.n_re, m.n_im, m.period_um, m.height_um = float(r[2]), float(r[3]), float(r[4]), float(r[5])
        m.gdir[:] = [float(x) for x in r[6:9]]
        m.sigma_h_um, m.corr_len_um, m.Le, m.coh_len_um = float(r[9]), float(r[10]), float(r[11]), float(r[12])
        m.cauchy_b_um2 = float(r[13])
    return arr, len(rows)


def _pack_lights(rows):
    rows = np.asarray(rows, dtype=np.float32).reshape(-1, 8)
    arr = (gr_light * max(1, len(rows)))()
    for i, r in enumerate(rows):
        L = arr[i]
        L.type = int(r[0])
        L.dir[:] = [float(x) for x in r[1:4]]
        L.E, L.coh_len_um = float(r[4]), float(r[5])
    return arr, len(rows)


class Scene:
    """Device copy of a scene (triangles, materials, lights) with its BVH."""

    def __init__(self, scene, stream=None):
        L = lib_handle()
        self._h = ctypes.c_void_p()
        verts = np.ascontiguousarray(scene["verts"], dtype=np.float32).reshape(-1, 9)
        tri_mat = np.ascontiguousarray(scene["tri_mat"], dtype=np.int32)
        mats, n_mats = _pack_materials(scene["mats"])
        lights, n_lights = _pack_lights(scene["lights"])
        desc = gr_scene_desc(len(tri_mat), _ptr(verts), _ptr(tri_mat), n_mats,
                             ctypes.cast(mats, ctypes.c_void_p), n_lights, ctypes.cast(lights, ctypes.c_void_p))
        self.n_tris = len(tri_mat)
        self.host_bytes = verts.nbytes + tri_mat.nbytes + n_mats * 64 + n_lights * 32
        _check(L.gr_scene_create(ctypes.byref(desc), stream or current_stream(), ctypes.byref(self._h)))

    @property
    def handle(self):
        return self._h

    def device_bytes(self):
        """Device bytes the scene holds (gr_scene_bytes)."""
        b = ctypes.c_size_t()
        _check(_lib.gr_scene_bytes(self._h, ctypes.byref(b)))
        return b.value

    def bvh(self):
        n = ctypes.c_int32()
        _check(_lib.gr_scene_bvh(self._h, ctypes.byref(n), None, None, None))
        n = n.value
        keys = np.zeros(max(n, 1), dtype=np.uint64)
        ch = np.zeros((max(n - 1, 1), 2), dtype=np.int32)
        bx = np.zeros((max(n - 1, 1), 12), dtype=np.float32)
        _check(_lib.gr_scene_bvh(self._h, ctypes.byref(ctypes.c_int32()), _ptr(keys), _ptr(ch), _ptr(bx)))
        return keys[:n], ch[: max(n - 1, 0)], bx[: max(n - 1, 0)]

    def close(self):
        if self._h:
            _lib.gr_scene_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def accum_floats(views):
    """Floats of a frame's accumulators: 2 * sum of W * H * n_bins * n_stokes."""
    return 2 * sum(int(v["width"]) * int(v["height"]) * int(v["n_bins"]) * int(v["n_stokes"]) for v in views)


class Frame:
    """Resident per-view accumulators (sum + Kahan compensation).

    accum: None for library-owned accumulators (gr_frame_create), or a
    contiguous float32 CUDA tensor of accum_floats(views) elements that the
    library adds into (gr_frame_wrap; sums view after view as [bin][y][x]
    [stokes], then compensations).  The tensor is kept referenced while the
    frame lives."""

    def __init__(self, views, stream=None, accum=None):
        L = lib_handle()
        self.views = [dict(v) for v in views]
        self._h = ctypes.c_void_p()
        arr = pack_views(self.views)
        self.accum = accum
        if accum is None:
            _check(L.gr_frame_create(arr, len(self.views), stream or current_stream(), ctypes.byref(self._h)))
        else:
            import torch
            if not (accum.is_cuda and accum.dtype == torch.float32 and accum.is_contiguous()
                    and accum.numel() >= accum_floats(self.views)):
                raise ValueError("accum must be a contiguous float32 CUDA tensor of at least %d elements"
                                 % accum_floats(self.views))
            _check(L.gr_frame_wrap(arr, len(self.views), ctypes.c_void_p(accum.data_ptr()),
                                   stream or current_stream(), ctypes.byref(self._h)))

    @property
    def handle(self):
        return self._h

    def reset(self, stream=None):
        _check(_lib.gr_frame_reset(self._h, stream or current_stream()))

    def device_bytes(self):
        """Device bytes the frame holds now (gr_frame_bytes)."""
        b = ctypes.c_size_t()
        _check(_lib.gr_frame_bytes(self._h, ctypes.byref(b)))
        return b.value

    def readback(self, view=0, out=None, stream=None):
        """Mean image float32 [H][W][n_bins][n_stokes]: a numpy array (host),
        or written into `out` if it is a CUDA torch tensor."""
        v = self.views[view]
        shape = (v["height"], v["width"], v["n_bins"], v["n_stokes"])
        if out is not None:
            assert out.is_cuda and out.is_contiguous() and out.numel() >= int(np.prod(shape))
            _check(_lib.gr_readback(self._h, view, ctypes.c_void_p(out.data_ptr()), out.numel() * 4, 1,
                                    stream or current_stream()))
            return out
        host = np.empty(shape, dtype=np.float32)
        _check(_lib.gr_readback(self._h, view, _ptr(host), host.nbytes, 0, stream or current_stream()))
        return host

    def stats(self, stream=None):
        s = gr_stats()
        _check(_lib.gr_frame_stats(self._h, stream or current_stream(), ctypes.byref(s)))
        out = {k: getattr(s, k) for k, _ in gr_stats._fields_}
        out["kernel_ms"] = list(s.kernel_ms)
        out["kernel_count"] = list(s.kernel_count)
        return out

    def close(self):
        if self._h:
            _lib.gr_frame_release(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def make_opts(seed=1, flags=0, table_dtype="f32", pool_size=0, block=0, use_graph=False, max_iterations=0,
              profile=False, regen_threshold_pct=0):
    o = gr_render_opts()
    o.seed = int(seed) & 0xFFFFFFFF
    o.flags = int(flags)
    o.table_dtype = TABLE_DTYPES[table_dtype] if isinstance(table_dtype, str) else int(table_dtype)
    o.pool_size, o.block = int(pool_size), int(block)
    o.use_graph = int(bool(use_graph))
    o.max_iterations = int(max_iterations)
    o.profile = int(bool(profile))
    o.regen_threshold_pct = int(regen_threshold_pct)
    return o


def render(scenes, views, frame, stream=None, **opts):
    """Enqueue the samples of every view into `frame` (asynchronous)."""
    L = lib_handle()
    sc = (ctypes.c_void_p * len(scenes))(*[s.handle.value for s in scenes])
    arr = pack_views(views)
    o = make_opts(**opts)
    _check(L.gr_render(sc, len(scenes), arr, len(views), ctypes.byref(o), frame.handle, stream or current_stream()))


def render_multi(scenes, views, frames, frame_view, stream=None, **opts):
    """One render over views accumulating into different frames
    (continuous batching): view i adds into frames[i]'s view frame_view[i]."""
    L = lib_handle()
    sc = (ctypes.c_void_p * len(scenes))(*[s.handle.value for s in scenes])
    arr = pack_views(views)
    fr = (ctypes.c_void_p * len(frames))(*[f.handle.value for f in frames])
    fv = (ctypes.c_int32 * len(frame_view))(*[int(x) for x in frame_view])
    o = make_opts(**opts)
    _check(L.gr_render_multi(sc, len(scenes), arr, len(views), ctypes.byref(o), fr, fv, stream or current_stream()))


def render_scratch_bytes(scenes, views, **opts):
    """Device scratch bytes a render of these views would hold
    (gr_render_scratch_bytes)."""
    L = lib_handle()
    sc = (ctypes.c_void_p * len(scenes))(*[s.handle.value for s in scenes])
    arr = pack_views(views)
    o = make_opts(**opts)
    b = ctypes.c_size_t()
    _check(L.gr_render_scratch_bytes(sc, len(scenes), arr, len(views), ctypes.byref(o), ctypes.byref(b)))
    return b.value


def debug_rng(seed, view_index, pixel, sample, segment, call, n, stream=None):
    """Raw device Philox words [n][4] for samples sample..sample+n-1."""
    L = lib_handle()
    out = np.zeros((n, 4), dtype=np.uint32)
    _check(L.gr_debug_rng(seed & 0xFFFFFFFF, view_index, pixel, sample, segment, call, n, _ptr(out),
                          stream or current_stream()))
    return out


def render_image(scene, view, **opts):
    """Convenience: one scene dict + one view dict -> mean image (numpy)."""
    s = Scene(scene)
    f = Frame([view])
    try:
        render([s], [dict(view, scene_index=0)], f, **opts)
        return f.readback(0)
    finally:
        f.close()
        s.close()


def measure_fp32_peak():
    """FP32 FMA throughput of the current device (include/gr_measure.h):
    returns (TFLOP/s, best launch ms)."""
    L = lib_handle()
    tf, ms = ctypes.c_double(), ctypes.c_double()
    _check(L.gr_measure_fp32_peak(current_stream(), ctypes.byref(tf), ctypes.byref(ms)))
    return tf.value, ms.value


_TABLE_CODES = {"f32": 0, "f16": 1, "bf16": 2}


def debug_order_table(height_um, lambda_um, jmax, table_dtype="f32"):
    """Grating order weights a_j = J_j(pi h / lambda)^2, j = 0..jmax, as the
    render stores them in `table_dtype`, decoded to float32 (gr_debug_order_table)."""
    L = lib_handle()
    fn = L.gr_debug_order_table
    fn.argtypes = [ctypes.c_float, ctypes.c_double, ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p]
    out = np.zeros(int(jmax) + 1, dtype=np.float32)
    _check(fn(float(height_um), float(lambda_um), int(jmax), _TABLE_CODES[table_dtype], _ptr(out), current_stream()))
    return out


def debug_footprint(quads):
    """The path's FP32 footprint update (gr_debug_footprint): quads [n][4] =
    (beta^2 um^2, rho, t m, kw 1/um) -> [n][2] = (beta^2, rho)."""
    L = lib_handle()
    fn = L.gr_debug_footprint
    fn.argtypes = [ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    q = np.ascontiguousarray(quads, dtype=np.float32).reshape(-1, 4)
    out = np.zeros((q.shape[0], 2), dtype=np.float32)
    _check(fn(q.shape[0], _ptr(q), _ptr(out), current_stream()))
    return out


def aperture_backward_3d(x0, x_ap, w_ap, beta, z, k, reach, dt, rho_cut=2.5):
    """Footprint-resolved generalized rays through a plane aperture in a 3D
    world (gr_aperture_backward_3d): x0 [n][2] detector element centres, x_ap
    [m][2] aperture samples with weights w_ap [m]; returns (intensity per
    detector element, kernel ms)."""
    L = lib_handle()
    fn = L.gr_aperture_backward_3d
    D = ctypes.c_double
    fn.argtypes = [ctypes.c_int32, ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, D, D, D, D, D,
                   D, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    x0 = np.ascontiguousarray(x0, dtype=np.float64).reshape(-1, 2)
    xa = np.ascontiguousarray(x_ap, dtype=np.float64).reshape(-1, 2)
    wa = np.ascontiguousarray(w_ap, dtype=np.float64).reshape(-1)
    out = np.zeros(len(x0), dtype=np.float64)
    ms = ctypes.c_float()
    _check(fn(len(x0), _ptr(x0), len(xa), _ptr(xa), _ptr(wa), beta, z, k, reach, dt, rho_cut, _ptr(out),
              ctypes.byref(ms), current_stream()))
    return out, ms.value


def aperture_backward_2d(x0, x_ap, w_ap, beta, z, k, reach, dtheta, rho_cut=2.5):
    """Footprint-resolved generalized rays through a 1D aperture
    (gr_aperture_backward_2d): returns (intensity per detector element,
    kernel ms)."""
    L = lib_handle()
    fn = L.gr_aperture_backward_2d
    D = ctypes.c_double
    fn.argtypes = [ctypes.c_int32, ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, D, D, D, D, D,
                   D, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    x0 = np.ascontiguousarray(x0, dtype=np.float64)
    xa = np.ascontiguousarray(x_ap, dtype=np.float64)
    wa = np.ascontiguousarray(w_ap, dtype=np.float64)
    out = np.zeros(len(x0), dtype=np.float64)
    ms = ctypes.c_float()
    _check(fn(len(x0), _ptr(x0), len(xa), _ptr(xa), _ptr(wa), beta, z, k, reach, dtheta, rho_cut, _ptr(out),
              ctypes.byref(ms), current_stream()))
    return out, ms.value
