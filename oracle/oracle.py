"""ctypes access to the FP64 CPU oracle (``gr_oracle.cpp``).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and ``bench.py`` (its ``cpu_baseline`` leg and ``--impl reference`` arm).  The
product package never imports this module, and this module imports nothing from
the product package: both sides receive the same plain input arrays from the
seeded scene generator and marshal them independently.

Input layouts (plain arrays written by the scene generator):
  material row float32[16]: 0 type (0 absorber, 1 grating, 2 rough, 3 mirror,
      4 emitter, 5 dielectric), 1 fresnel (0 unit, 1 conductor), 2 n_re,
      3 n_im, 4 period_um, 5 height_um (peak to peak), 6-8 grating direction,
      9 sigma_h_um, 10 corr_len_um, 11 Le, 12 coh_len_um, 13 cauchy_b_um2
      (dielectric index n_re + cauchy_b_um2 / lambda^2), 14-15 unused
  light row float32[8]: 0 type (0 distant, 1 constant environment),
      1-3 direction toward the source, 4 E, 5 coh_len_um, 6-7 unused
"""
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRCS = [os.path.join(_HERE, "gr_oracle.cpp"), os.path.join(_HERE, "lbvh_ref.cpp")]
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")

FLAG_NEE = 1
FLAG_RR = 2
FLAG_NO_RENORM = 4
FLAG_HERO = 16
FLAG_ANISO = 32

_lib = None


def build(force=False):
    """Compile the oracle shared library (plain g++, no CUDA)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and all(os.path.getmtime(_LIB_PATH) >= os.path.getmtime(f) for f in _SRCS)):
        return _LIB_PATH
    tmp = _LIB_PATH + ".tmp%d" % os.getpid()
    cmd = ["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-pthread",
           "-ffp-contract=off", "-o", tmp] + _SRCS
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def build_cmd_popen():
    """Start the oracle compile in the background (used by the package build)."""
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _LIB_PATH + ".tmp%d" % os.getpid()
    cmd = ["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-pthread",
           "-ffp-contract=off", "-o", tmp] + _SRCS
    return subprocess.Popen(cmd), tmp, _LIB_PATH


def lib():
    global _lib
    if _lib is not None:
        return _lib
    build()
    L = ctypes.CDLL(_LIB_PATH)
    D, I, P, U32, L_ = ctypes.c_double, ctypes.c_int, ctypes.c_void_p, ctypes.c_uint32, ctypes.c_long
    L.oracle_philox4x32_10.argtypes = [P, P, P]
    L.oracle_bessel_j.argtypes = [I, D]
    L.oracle_bessel_j.restype = D
    L.oracle_vmf.argtypes = [P, P, D]
    L.oracle_vmf.restype = D
    L.oracle_vmf_sample.argtypes = [P, D, D, D, P]
    L.oracle_onb.argtypes = [P, P, P]
    L.oracle_propagate.argtypes = [D, D, D, P]
    L.oracle_grating_lobes.argtypes = [P, P, P, D, I, I, P, P, P]
    L.oracle_grating_lobes.restype = I
    L.oracle_rough_density.argtypes = [D, D, D, D, D]
    L.oracle_rough_density.restype = D
    L.oracle_fresnel_mueller.argtypes = [D, D, D, P, P]
    L.oracle_stokes_rotation.argtypes = [D, P]
    L.oracle_scene_create.argtypes = [I, P, P, I, P, I, P]
    L.oracle_scene_create.restype = P
    L.oracle_scene_destroy.argtypes = [P]
    L.oracle_closest_hit.argtypes = [P, P, P, I, I, P, P]
    L.oracle_closest_hit.restype = I
    L.oracle_trace_sample.argtypes = [P, P, U32, I, I, I, L_, P]
    L.oracle_render.argtypes = [P, P, U32, I, I, I, I, I, I, P, P]
    L.oracle_render.restype = L_
    L.oracle_lbvh_build.argtypes = [I, P, P, P, P]
    L.oracle_lbvh_build.restype = I
    L.oracle_fresnel_dielectric.argtypes = [D, D, P]
    L.oracle_refract.argtypes = [P, P, D, D, P]
    L.oracle_refract.restype = I
    L.oracle_aniso_propagate.argtypes = [P, D, P]
    L.oracle_aniso_interaction.argtypes = [P, P, P, P, P, P, P]
    L.oracle_aniso_emitter.argtypes = [P, P, P, D, D, P, D, D, P]
    L.oracle_work_counters.argtypes = [P]
    L.oracle_work_reset.argtypes = []
    _lib = L
    return L


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _d3(v):
    return np.ascontiguousarray(np.asarray(v, dtype=np.float64).reshape(3))


# ------------------------------------------------------------------ traversal work
def work_reset():
    """Zero the oracle's traversal-work counters."""
    lib().oracle_work_reset()


def work_counters():
    """Closest-hit queries, internal node visits and ray-triangle tests of the
    oracle's SAH reference tree since the last reset."""
    o = np.zeros(3, dtype=np.int64)
    lib().oracle_work_counters(_p(o))
    return {"queries": int(o[0]), "node_visits": int(o[1]), "tri_tests": int(o[2])}


# ------------------------------------------------------------------ primitives
def philox4x32_10(ctr, key):
    c = np.ascontiguousarray(np.asarray(ctr, dtype=np.uint32).reshape(4))
    k = np.ascontiguousarray(np.asarray(key, dtype=np.uint32).reshape(2))
    o = np.zeros(4, dtype=np.uint32)
    lib().oracle_philox4x32_10(_p(c), _p(k), _p(o))
    return o


def bessel_j(n, x):
    return lib().oracle_bessel_j(int(n), float(x))


def vmf(w, mu, kappa):
    return lib().oracle_vmf(_p(_d3(w)), _p(_d3(mu)), float(kappa))


def vmf_sample(mu, kappa, u0, u1):
    o = np.zeros(3)
    lib().oracle_vmf_sample(_p(_d3(mu)), float(kappa), float(u0), float(u1), _p(o))
    return o


def onb(n):
    e1 = np.zeros(3)
    e2 = np.zeros(3)
    lib().oracle_onb(_p(_d3(n)), _p(e1), _p(e2))
    return e1, e2


def propagate(beta2, rho, zbar):
    o = np.zeros(2)
    lib().oracle_propagate(float(beta2), float(rho), float(zbar), _p(o))
    return o[0], o[1]


def _k6(K):
    K = np.asarray(K, dtype=np.complex128)
    return np.ascontiguousarray([K[0, 0].real, K[0, 0].imag, K[0, 1].real, K[0, 1].imag, K[1, 1].real, K[1, 1].imag])


def _kmat(o):
    a, b, c = o[0] + 1j * o[1], o[2] + 1j * o[3], o[4] + 1j * o[5]
    return np.array([[a, b], [b, c]])


def aniso_propagate(K, zbar):
    """Anisotropic footprint K = A^-1 (complex symmetric 2x2, um^2) after free
    propagation by zbar = z / |k| (um)."""
    o = np.zeros(6)
    lib().oracle_aniso_propagate(_p(_k6(K)), float(zbar), _p(o))
    return _kmat(o)


def aniso_interaction(K, f_in, d_in, f_out, d_out, n):
    """K mapped from the incident frame (f_in, d_in x f_in) to the outgoing
    frame (f_out, d_out x f_out) through a surface of normal n."""
    o = np.zeros(6)
    lib().oracle_aniso_interaction(_p(_k6(K)), _p(_d3(f_in)), _p(_d3(d_in)), _p(_d3(f_out)), _p(_d3(d_out)),
                                   _p(_d3(n)), _p(o))
    return _kmat(o)


def aniso_emitter(K, xf, d, k, s2, ne, z0, z1):
    """Footprint point (x1, x2 in um, frame onb(d)), its direction shift (m1,
    m2) and the emitter lobe value (unit exitance, point covered) for the
    standard normal pair (z0, z1)."""
    o = np.zeros(6)
    lib().oracle_aniso_emitter(_p(_k6(K)), _p(_d3(xf)), _p(_d3(d)), float(k), float(s2), _p(_d3(ne)), float(z0),
                               float(z1), _p(o))
    return o[:2].copy(), o[2:4].copy(), float(o[4])


def fresnel_dielectric(cos_i, n_rel):
    """Smooth dielectric interface: dict of Rs, Rp, Ts, Tp (power), R, T
    (unpolarised), cos_t and tir."""
    o = np.zeros(8)
    lib().oracle_fresnel_dielectric(float(cos_i), float(n_rel), _p(o))
    return dict(Rs=o[0], Rp=o[1], Ts=o[2], Tp=o[3], R=o[4], T=o[5], cos_t=o[6], tir=bool(o[7]))


def refract(d, n, eta_a, eta_b):
    """Refracted unit direction from index eta_a into eta_b, or None under
    total internal reflection."""
    o = np.zeros(3)
    ok = lib().oracle_refract(_p(_d3(d)), _p(_d3(n)), float(eta_a), float(eta_b), _p(o))
    return o if ok else None


def grating_lobes(mat_row, d_in, n, lambda_um, renorm=True, cap=128):
    m = np.ascontiguousarray(np.asarray(mat_row, dtype=np.float32).reshape(16))
    orders = np.zeros(cap, dtype=np.int32)
    w = np.zeros(cap)
    dirs = np.zeros((cap, 3))
    cnt = lib().oracle_grating_lobes(_p(m), _p(_d3(d_in)), _p(_d3(n)), float(lambda_um),
                                     int(bool(renorm)), cap, _p(orders), _p(w), _p(dirs))
    cnt = min(cnt, cap)
    return orders[:cnt].copy(), w[:cnt].copy(), dirs[:cnt].copy()


def rough_density(g, k, ell, dx, dy):
    return lib().oracle_rough_density(float(g), float(k), float(ell), float(dx), float(dy))


def fresnel_mueller(cos_i, n_re, n_im):
    m = np.zeros(16)
    r = np.zeros(4)
    lib().oracle_fresnel_mueller(float(cos_i), float(n_re), float(n_im), _p(m), _p(r))
    return m.reshape(4, 4), complex(r[0], r[1]), complex(r[2], r[3])


def stokes_rotation(phi):
    m = np.zeros(16)
    lib().oracle_stokes_rotation(float(phi), _p(m))
    return m.reshape(4, 4)


def lbvh_build(verts):
    """CPU LBVH of float32 triangles [n][3][3]: (sorted keys, child refs, child boxes)."""
    v = np.ascontiguousarray(np.asarray(verts, dtype=np.float32).reshape(-1, 9))
    n = len(v)
    keys = np.zeros(max(n, 1), dtype=np.uint64)
    ch = np.zeros((max(n - 1, 1), 2), dtype=np.int32)
    bx = np.zeros((max(n - 1, 1), 12), dtype=np.float32)
    lib().oracle_lbvh_build(n, _p(v), _p(keys), _p(ch), _p(bx))
    return keys[:n], ch[: max(n - 1, 0)], bx[: max(n - 1, 0)]


# ------------------------------------------------------------------ scenes
def view_vector(view):
    """Pack a view dict (scene generator format) into the oracle's double[24]."""
    v = np.zeros(24, dtype=np.float64)
    v[0:3] = view["eye"]
    v[3:6] = view["look_at"]
    v[6:9] = view["up"]
    v[9] = view["vfov_deg"]
    v[10] = view["width"]
    v[11] = view["height"]
    v[12] = view["p_pix_um"]
    v[13] = view["f_beta"]
    v[14] = view["lambda_min_um"]
    v[15] = view["lambda_max_um"]
    v[16] = view["n_bins"]
    v[17] = view["n_stokes"]
    v[18] = view["max_depth"]
    v[19] = view["spp"]
    v[20] = view.get("first_sample", 0)
    v[21] = view.get("view_index", 0)
    v[22] = view.get("ortho", 0)
    v[23] = view.get("ortho_half_m", 0.0)
    return v


class Scene:
    """Oracle-side copy of a scene (FP64 triangles, median-split BVH)."""

    def __init__(self, scene):
        self.verts = np.ascontiguousarray(scene["verts"], dtype=np.float32).reshape(-1, 9)
        self.tri_mat = np.ascontiguousarray(scene["tri_mat"], dtype=np.int32)
        self.mats = np.ascontiguousarray(scene["mats"], dtype=np.float32).reshape(-1, 16)
        self.lights = np.ascontiguousarray(scene["lights"], dtype=np.float32).reshape(-1, 8)
        self._h = lib().oracle_scene_create(len(self.tri_mat), _p(self.verts), _p(self.tri_mat),
                                            len(self.mats), _p(self.mats),
                                            len(self.lights), _p(self.lights))

    def close(self):
        if self._h:
            lib().oracle_scene_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def closest_hit(self, o, d, exclude=-1, use_bvh=True):
        t = ctypes.c_double()
        prim = ctypes.c_int()
        lib().oracle_closest_hit(self._h, _p(_d3(o)), _p(_d3(d)), int(exclude), int(bool(use_bvh)),
                                 ctypes.byref(t), ctypes.byref(prim))
        return t.value, prim.value

    def trace_sample(self, view, seed, flags, px, py, sample):
        v = view_vector(view)
        o = np.zeros(16)
        lib().oracle_trace_sample(self._h, _p(v), int(seed) & 0xFFFFFFFF, int(flags), int(px), int(py),
                                  int(sample), _p(o))
        ns = int(view["n_stokes"])
        if flags & FLAG_HERO:  # [class bin][Stokes]
            return o.reshape(4, 4)[:, :ns].copy()
        return o[:ns].copy()

    def render(self, view, seed, flags, crop=None, n_threads=None, want_var=False):
        """Mean image [h][w][n_bins][n_stokes] over the crop (x0, y0, x1, y1)."""
        W, H = int(view["width"]), int(view["height"])
        x0, y0, x1, y1 = crop if crop is not None else (0, 0, W, H)
        nb, ns = int(view["n_bins"]), int(view["n_stokes"])
        mean = np.zeros((y1 - y0, x1 - x0, nb, ns))
        var = np.zeros_like(mean) if want_var else None
        if n_threads is None:
            n_threads = os.cpu_count() or 1
        v = view_vector(view)
        n = lib().oracle_render(self._h, _p(v), int(seed) & 0xFFFFFFFF, int(flags), x0, y0, x1, y1,
                                int(n_threads), _p(mean), _p(var) if want_var else None)
        if n == -1:
            raise ValueError("hero-wavelength MIS needs n_bins to be a multiple of 4")
        if n == -2:
            raise ValueError("hero-wavelength MIS and anisotropic footprints are not combined")
        return (mean, var) if want_var else mean
