"""System-level pins of the FP64 oracle: white furnace, closed-form pixel
expectations by deterministic quadrature, measurement identities, unbiasedness
of next-event estimation with MIS, and its BVH against an exhaustive scan."""
import math

import numpy as np
import pytest
from scipy import special

from paper_2303_15762_gb300 import scenegen as sg

F32 = lambda x: float(np.float32(x))  # noqa: E731  (material/light rows are float32)


def _furnace_scene(kind, n_stokes=1, two_planes=False):
    if kind == "grating":
        m = sg.material(sg.MAT_GRATING, period_um=1.1, height_um=0.3, gdir=(0.6, 0.8, 0))
    elif kind == "mirror":
        m = sg.material(sg.MAT_MIRROR)
    else:
        m = sg.material(sg.MAT_ROUGH, sigma_h_um=0.08, corr_len_um=4.0)
    tris = [sg._quad((0, 0, 0), (0.05, 0, 0), (0, 0.05, 0))]
    if two_planes:
        tris.append(sg._quad((0, 0, 0.01), (0, 0.05, 0), (0.05, 0, 0)))
    T = np.concatenate(tris)
    return sg._scene(T, [0] * len(T), [m], [sg.env_light(1.0)])


@pytest.mark.parametrize("kind", ["grating", "mirror"])
@pytest.mark.parametrize("two_planes", [False, True])
@pytest.mark.parametrize("n_stokes", [1, 4])
def test_white_furnace_exact(oracle, kind, two_planes, n_stokes):
    """Unit environment, unit-reflectance lobes, renormalised grating orders:
    every sample equals exactly 1 (S0), and stays unpolarised."""
    sc = oracle.Scene(_furnace_scene(kind, n_stokes, two_planes))
    v = sg.view(eye=(0.02, -0.01, 0.3) if not two_planes else (0.3, 0.0, 0.005), look_at=(0, 0, 0.005),
                up=(0, 1, 0) if not two_planes else (0, 0, 1), vfov_deg=20, width=16, height=16,
                n_bins=5, n_stokes=n_stokes, max_depth=200, spp=5)
    for px in range(0, 16, 3):
        for py in range(0, 16, 3):
            for s in range(5):
                c = sc.trace_sample(v, 7, oracle.FLAG_NEE, px, py, s)
                assert abs(c[0] - 1.0) < 1e-12
                if n_stokes == 4:
                    assert np.all(np.abs(c[1:]) < 1e-12)


def test_white_furnace_rough_zero_or_one(oracle):
    """Rough lobe without renormalisation: a sample is 1 unless its diffuse
    direction came out evanescent (then 0)."""
    sc = oracle.Scene(_furnace_scene("rough"))
    v = sg.view(eye=(0.0, -0.15, 0.1), look_at=(0, 0, 0), vfov_deg=20, width=8, height=8, n_bins=4,
                max_depth=4, spp=8)
    vals = [sc.trace_sample(v, 3, 0, px, py, s)[0] for px in range(8) for py in range(8) for s in range(8)]
    assert set(np.round(vals, 12)) <= {0.0, 1.0}
    assert np.mean(vals) > 0.5


def _gl_nodes(n):
    x, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * (x + 1), 0.5 * w


def _grating_pixel_expectation(px, py, b, view, scene):
    """E_jitter[ sum_j a_j vMF(d_j; w_L, kappa) ] for the planar grating
    workload, by 32x32 Gauss-Legendre quadrature over the pixel (no MC)."""
    W, H = view["width"], view["height"]
    nb = view["n_bins"]
    lam = view["lambda_min_um"] + b * (view["lambda_max_um"] - view["lambda_min_um"]) / (nb - 1)
    k = 2 * math.pi / lam
    beta0 = view["f_beta"] * view["p_pix_um"]
    kappa = 2 * beta0 ** 2 * k ** 2  # 1 / s_ray^2 with s_ray^2 = 1/(2 beta0^2 k^2)
    row = scene["mats"][0]
    period, h = float(row[4]), float(row[5])
    mu = scene["lights"][0][1:4].astype(np.float64)
    mu /= np.linalg.norm(mu)
    th = math.tan(math.radians(view["vfov_deg"]) / 2)
    xs, ws = _gl_nodes(32)
    U0, U1 = np.meshgrid(xs, xs, indexing="ij")
    Wt = np.outer(ws, ws)
    sx = (2 * (px + U0) / W - 1) * th * (W / H)
    sy = (1 - 2 * (py + U1) / H) * th
    d = np.stack([sx, sy, -np.ones_like(sx)], -1)
    d /= np.linalg.norm(d, axis=-1, keepdims=True)
    x = math.pi * h / lam
    total = np.zeros_like(sx)
    vals = np.zeros_like(sx)
    for j in range(-40, 41):
        tx = d[..., 0] + j * lam / period
        ty = d[..., 1]
        tt = tx * tx + ty * ty
        prop = tt < 1
        a = special.jv(j, x) ** 2
        dj = np.stack([tx, ty, np.sqrt(np.clip(1 - tt, 0, None))], -1)
        dd = dj - mu
        vm = kappa / (2 * math.pi * (-math.expm1(-2 * kappa))) * np.exp(-0.5 * kappa * (dd * dd).sum(-1))
        total += np.where(prop, a, 0.0)
        vals += np.where(prop, a * vm, 0.0)
    return float((Wt * vals / total).sum())


def test_grating_workload_matches_quadrature(oracle):
    """The MC oracle's pixel means agree with the deterministic quadrature of
    their expectation within 4 standard errors (pins sampling, RNG use, bin
    stratification and accumulation)."""
    scene = sg.grating_scene()
    sc = oracle.Scene(scene)
    view = sg.grating_view(spp=16 * 256)
    pix = [(5, 5), (20, 31), (31, 31), (40, 22), (44, 31), (50, 40), (60, 60), (33, 10), (27, 45)]
    n_checked = 0
    for px, py in pix:
        mean, var = sc.render(view, 1, 0, crop=(px, py, px + 1, py + 1), want_var=True)
        for b in range(16):
            q = _grating_pixel_expectation(px, py, b, view, scene)
            se = math.sqrt(max(var[0, 0, b, 0], 0.0) / 256)
            assert abs(mean[0, 0, b, 0] - q) <= 4 * se + 1e-9 * (1 + abs(q)), (px, py, b, mean[0, 0, b, 0], q, se)
            n_checked += q > 1e-3
    assert n_checked > 10  # the +1 order actually lands in some of these pixels


def test_measurement_lobe_width_from_overlap_integral(oracle):
    """Eq. measurement_operator for a plane-wave source: the overlap
    |int psi_s psi*_{beta,rho}|^2 (brute-force quadrature of Eq. def_gen_ray,
    one transverse axis) is a Gaussian in the wavevector offset whose variance
    must equal the oracle's angular variance s_ray^2 |k|^2 = (1+rho^2)/(2 beta^2)."""
    for beta, rho in [(1.0, 0.0), (3.0, 0.0), (2.0, 1.5), (5.0, 7.0)]:
        x = np.linspace(-12 * beta * (1 + rho), 12 * beta * (1 + rho), 20001)
        psi = (1 / (math.pi * beta ** 2)) ** 0.25 * np.exp(-(1 - 1j * rho) * x ** 2 / (2 * beta ** 2))
        dks = np.linspace(-2.5, 2.5, 11) * math.sqrt((1 + rho ** 2) / (2 * beta ** 2))
        I = np.array([abs(np.trapezoid(np.exp(1j * dk * x) * np.conj(psi), x)) ** 2 for dk in dks])
        # fit log I = c - dk^2 / (2 var)
        A = np.stack([np.ones_like(dks), -dks ** 2 / 2], 1)
        c, inv_var = np.linalg.lstsq(A, np.log(I), rcond=None)[0]
        var_fit = 1 / inv_var
        assert abs(var_fit - (1 + rho ** 2) / (2 * beta ** 2)) < 1e-6 * var_fit
    # the oracle's direct view of a distant source uses exactly that width:
    # a one-pixel camera of negligible field of view looks along d
    lam = 0.5
    k = 2 * math.pi / lam
    beta0 = 1.0
    var_fit_unit = (1.0 / (2 * beta0 ** 2)) / k ** 2
    scene = sg._scene(np.zeros((0, 3, 3)), [], [sg.material(sg.MAT_ABSORBER)],
                      [sg.light(sg.LIGHT_DISTANT, (0.0, 0.0, -1.0), 2.0, 0.0)])
    sc = oracle.Scene(scene)
    for ang in [0.0, 0.02, 0.05, 0.09]:
        d = np.array([math.sin(ang), 0.0, -math.cos(ang)])
        v = sg.view(eye=(0, 0, 0), look_at=tuple(d), vfov_deg=1e-6, width=1, height=1, p_pix_um=2.0,
                    f_beta=0.5, lambda_min_um=lam, lambda_max_um=lam, n_bins=1, spp=1, max_depth=0)
        val = sc.trace_sample(v, 11, 0, 0, 0, 0)[0]
        kappa = 1 / var_fit_unit
        expect = 2.0 * kappa / (2 * math.pi * (-math.expm1(-2 * kappa))) * math.exp(-kappa * (1 - math.cos(ang)))
        assert abs(val - expect) <= 1e-6 * expect + 1e-300, (ang, val, expect)


def test_emitter_footprint_measurement_matches_marginal(oracle):
    """Footprint-sampled emitter measurement over an emitter much larger than
    the footprint reproduces the closed-form k-marginal (variances add):
    E_x[vMF(d + mu(x); n_e, 1/(s_c^2 + s_src^2))] = vMF(d; n_e, 1/(s_ray^2 + s_src^2))."""
    lc = 20.0
    em = sg.material(sg.MAT_EMITTER, Le=1.0, coh_len_um=lc)
    tris = sg._quad((0, 0, -3.0), (40.0, 0, 0), (0, 40.0, 0))  # normal +z, faces the camera
    scene = sg._scene(tris, [0, 0], [em], np.zeros((0, 8)))
    sc = oracle.Scene(scene)
    lam = 0.55
    v = sg.view(eye=(0, 0, 0), look_at=(0.0, 0.0, -1), vfov_deg=12, width=5, height=5, lambda_min_um=lam,
                lambda_max_um=lam, n_bins=1, spp=40000, max_depth=0)
    k = 2 * math.pi / lam
    beta0 = v["f_beta"] * v["p_pix_um"]
    s_ray2 = 1 / (2 * beta0 ** 2 * k ** 2)
    s_src2 = (lam / F32(lc)) ** 2
    kappa = 1 / (s_ray2 + s_src2)
    for px, py in [(2, 2), (4, 1)]:
        mean, var = sc.render(v, 5, 0, crop=(px, py, px + 1, py + 1), want_var=True)
        # expectation over the pixel jitter of the closed-form marginal
        th = math.tan(math.radians(6))
        xs, ws = _gl_nodes(24)
        acc = 0.0
        for a, wa in zip(xs, ws):
            for b, wb in zip(xs, ws):
                d = np.array([(2 * (px + a) / 5 - 1) * th, (1 - 2 * (py + b) / 5) * th, -1.0])
                d /= np.linalg.norm(d)
                acc += wa * wb * oracle.vmf(-d, np.array([0, 0, 1.0]), kappa)
        se = math.sqrt(var[0, 0, 0, 0] / 40000)
        assert abs(mean[0, 0, 0, 0] - acc) < 4 * se + 2e-3 * acc, (mean[0, 0, 0, 0], acc, se)


def _nee_scene():
    ground = sg.material(sg.MAT_ROUGH, sigma_h_um=0.4, corr_len_um=1.2)
    em = sg.material(sg.MAT_EMITTER, Le=1.0, coh_len_um=1.5)
    tris = np.concatenate([sg._quad((0, 0, 0), (0, 0, 1.0), (1.0, 0, 0)),      # normal +y
                           sg._quad((0.1, 0.8, 0.0), (0.35, 0, 0), (0, 0, 0.35))])  # faces -y
    return sg._scene(tris, [0, 0, 1, 1], [ground, em], np.zeros((0, 8)))


def test_nee_mis_unbiased(oracle):
    """Next-event estimation with power-heuristic MIS estimates the same pixel
    expectation as pure lobe sampling (FLAG_NEE on vs off)."""
    sc = oracle.Scene(_nee_scene())
    v = sg.view(eye=(0, 0.6, 1.6), look_at=(0, 0, 0), vfov_deg=30, width=8, height=8, lambda_min_um=0.45,
                lambda_max_um=0.65, n_bins=2, max_depth=2, spp=30000)
    for px, py in [(3, 5), (4, 6), (2, 7)]:
        m1, v1 = sc.render(v, 9, oracle.FLAG_NEE, crop=(px, py, px + 1, py + 1), want_var=True)
        m0, v0 = sc.render(v, 10, 0, crop=(px, py, px + 1, py + 1), want_var=True)
        for b in range(2):
            se = math.sqrt(v1[0, 0, b, 0] / 15000 + v0[0, 0, b, 0] / 15000)
            assert m1[0, 0, b, 0] > 0
            assert abs(m1[0, 0, b, 0] - m0[0, 0, b, 0]) < 4 * se, (px, py, b, m1[0, 0, b, 0], m0[0, 0, b, 0], se)
            # NEE reduces the variance in this lit configuration
            assert v1[0, 0, b, 0] < v0[0, 0, b, 0]


def test_rough_sampler_matches_density(oracle):
    """One rough bounce under a distant source: the MC mean equals the
    quadrature of the (separately pinned) lobe density times the measurement
    lobe, integrated over tangential direction cosines."""
    sigma, ell, lam = 0.06, 6.0, 0.5
    m = sg.material(sg.MAT_ROUGH, sigma_h_um=sigma, corr_len_um=ell)
    tris = sg._quad((0, 0, 0), (1.0, 0, 0), (0, 1.0, 0))
    Ldir = np.array([0.25, 0.1, 1.0])
    scene = sg._scene(tris, [0, 0], [m], [sg.light(sg.LIGHT_DISTANT, Ldir, 1.0, 8.0)])
    sc = oracle.Scene(scene)
    v = sg.view(eye=(-0.05, -0.02, 0.2), look_at=(0.05, 0.02, 0), vfov_deg=0.001, width=1, height=1,
                lambda_min_um=lam, lambda_max_um=lam, n_bins=1, max_depth=1, spp=200000)
    mean, var = sc.render(v, 4, 0, want_var=True)
    # deterministic expectation (the pixel is a single direction at this FOV)
    d = np.array([0.1, 0.04, -0.2])
    d /= np.linalg.norm(d)
    n = np.array([0, 0, 1.0])
    k = 2 * math.pi / lam
    cos_i = -d @ n
    g = (2 * k * F32(sigma) * cos_i) ** 2
    mu = np.asarray(scene["lights"][0][1:4], np.float64)
    mu /= np.linalg.norm(mu)
    s_ray2 = 1 / (2 * (v["f_beta"] * v["p_pix_um"]) ** 2 * k ** 2)
    kappa = 1 / (s_ray2 + (lam / F32(8.0)) ** 2)
    t_m = d[:2]
    # specular part
    spec = math.exp(-g) * oracle.vmf(np.array([d[0], d[1], -d[2]]), mu, kappa)
    e1, e2 = oracle.onb(n)
    R = 0.6
    N = 601
    xs = np.linspace(-R, R, N)
    acc = 0.0
    h = xs[1] - xs[0]
    for a in xs:
        for b in xs:
            delta = a * e1 + b * e2
            t = np.array([t_m[0], t_m[1], 0]) + delta
            tt = t @ t
            if tt >= 1:
                continue
            dout = t + math.sqrt(1 - tt) * n
            acc += oracle.rough_density(g, k, F32(ell), a, b) * oracle.vmf(dout, mu, kappa)
    expect = spec + acc * h * h
    se = math.sqrt(var[0, 0, 0, 0] / 200000)
    assert abs(mean[0, 0, 0, 0] - expect) < 4 * se + 2e-3 * expect, (mean[0, 0, 0, 0], expect, se)


def test_stokes_s0_equals_scalar_single_bounce(oracle):
    """One Fresnel reflection of unpolarised light: the Stokes S0 equals the
    scalar (unpolarised reflectance) result sample by sample, and the output
    stays physical (S0 >= |S1..S3|)."""
    m = sg.material(sg.MAT_MIRROR, fresnel=1, n_re=0.3, n_im=3.2)
    tris = sg._quad((0, 0, 0), (0.05, 0, 0), (0, 0.05, 0))
    scene = sg._scene(tris, [0, 0], [m], [sg.light(sg.LIGHT_DISTANT, (0.2, 0.1, 1.0), 1.0, 30.0)])
    sc = oracle.Scene(scene)
    v1 = sg.view(eye=(-0.03, -0.01, 0.2), look_at=(0, 0, 0), vfov_deg=20, width=8, height=8, n_bins=4, spp=4)
    v4 = dict(v1, n_stokes=4)
    for px in range(8):
        for s in range(4):
            a = sc.trace_sample(v1, 2, 0, px, 3, s)
            b = sc.trace_sample(v4, 2, 0, px, 3, s)
            assert abs(a[0] - b[0]) <= 1e-12 * max(1.0, abs(a[0]))
            assert b[0] >= np.linalg.norm(b[1:]) - 1e-12


def test_render_accumulation_is_in_sample_order(oracle):
    """A render over [0, 2n) equals the count-weighted combination of renders
    over [0, n) and [n, 2n) (same per-sample stream), and is deterministic."""
    scene = sg.grating_scene()
    sc = oracle.Scene(scene)
    v = sg.grating_view(spp=64)
    a = sc.render(v, 1, 0, crop=(20, 20, 28, 24))
    b = sc.render(v, 1, 0, crop=(20, 20, 28, 24))
    assert np.array_equal(a, b)
    h1 = sc.render(dict(v, spp=32), 1, 0, crop=(20, 20, 28, 24))
    h2 = sc.render(dict(v, spp=32, first_sample=32), 1, 0, crop=(20, 20, 28, 24))
    np.testing.assert_allclose(a, 0.5 * (h1 + h2), rtol=1e-12, atol=1e-14)


def test_bvh_matches_exhaustive_scan(oracle):
    """The oracle's BVH returns exactly the exhaustive scan's closest hit."""
    scene = sg.procedural_scene(seed=11, n_objects=6, target_tris=6000, n_emitters=2)
    sc = oracle.Scene(scene)
    rng = np.random.default_rng(12)
    n = 20000
    hits = 0
    for i in range(n):
        o = rng.uniform([-2, -0.2, -2], [2, 1.5, 2])
        d = rng.standard_normal(3)
        d /= np.linalg.norm(d)
        a = sc.closest_hit(o, d, exclude=-1, use_bvh=True)
        b = sc.closest_hit(o, d, exclude=-1, use_bvh=False)
        assert a == b, (i, a, b)
        hits += a[1] >= 0
    assert hits > n // 5
