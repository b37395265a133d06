"""Pins of the oracle's anisotropic generalized rays (beta and rho as 2x2
matrices, Sec. 3.1 and Eq. def_gen_ray; the general form is in a supplemental
that is not available, so the model is derived from the Gaussian field).
The state is K = A^-1 of the transverse field exp(-x^T A x / 2):
- free propagation K + i zbar I is checked against the paraxial transfer
  function applied to a sampled field by FFT;
- the scalar ray reduces to Eq. K_free_space_propagation;
- the interaction map is checked against the anamorphic factors that the
  differentials of the grating equation and of Snell's law give, against the
  projected-area ratio, and for mirrors against orthogonality;
- a scene whose interactions are all mirror reflections renders exactly as
  the scalar model does."""
import math

import numpy as np
import pytest

from paper_2303_15762_gb300 import scenegen as sg


def _field(K, x, y):
    A = np.linalg.inv(K)
    return np.exp(-0.5 * (A[0, 0] * x * x + 2 * A[0, 1] * x * y + A[1, 1] * y * y))


@pytest.mark.parametrize("zbar", [0.5, 3.0, 12.0])
def test_propagation_is_the_paraxial_transfer_function(oracle, zbar):
    """A sampled anisotropic Gaussian field propagated by the transfer
    function exp(-i zbar |q|^2 / 2) (numpy FFT) equals the Gaussian of
    K + i zbar I up to its amplitude sqrt(det K / det K')."""
    K = np.array([[4.0 + 1.0j, 1.2 - 0.6j], [1.2 - 0.6j, 2.5 + 2.0j]])
    n, L = 512, 120.0
    x1 = (np.arange(n) - n // 2) * (L / n)
    X, Y = np.meshgrid(x1, x1, indexing="ij")
    psi = _field(K, X, Y)
    q = 2 * np.pi * np.fft.fftfreq(n, d=L / n)
    QX, QY = np.meshgrid(q, q, indexing="ij")
    out = np.fft.ifft2(np.fft.fft2(psi) * np.exp(-0.5j * zbar * (QX ** 2 + QY ** 2)))
    K2 = oracle.aniso_propagate(K, zbar)
    model = np.sqrt(np.linalg.det(K) / np.linalg.det(K2)) * _field(K2, X, Y)
    inner = (np.abs(X) < 15) & (np.abs(Y) < 15)
    err = np.max(np.abs(out[inner] - model[inner])) / np.max(np.abs(model))
    assert err < 1e-9, err


def test_scalar_ray_reduces_to_free_space_update(oracle):
    rng = np.random.default_rng(1)
    for _ in range(50):
        b2 = float(np.exp(rng.uniform(-2, 8)))
        rho = float(rng.uniform(0, 50))
        zbar = float(np.exp(rng.uniform(-3, 8)))
        K = b2 / (1 - 1j * rho) * np.eye(2)
        K2 = oracle.aniso_propagate(K, zbar)
        a = 1.0 / K2[0, 0]  # (1 - i rho') / beta'^2
        b2n, rn = oracle.propagate(b2, rho, zbar)
        assert abs(1.0 / a.real - b2n) <= 1e-12 * b2n
        assert abs(-a.imag / a.real - rn) <= 1e-12 * max(1.0, rn)
        assert abs(K2[0, 1]) == 0.0 and K2[0, 0] == K2[1, 1]


def _in_plane(theta):
    """Unit direction in the x-z plane travelling toward the surface z = 0
    (normal +z) at angle theta from the normal."""
    return np.array([math.sin(theta), 0.0, -math.cos(theta)])


def _out_plane(theta):
    return np.array([math.sin(theta), 0.0, math.cos(theta)])


@pytest.mark.parametrize("theta_i_deg,order,period_um,lam_um", [(20.0, 1, 1.6, 0.5), (60.0, -1, 1.2, 0.45),
                                                                 (5.0, 2, 3.0, 0.7), (75.0, -2, 2.0, 0.4)])
def test_grating_map_follows_the_grating_equation(oracle, theta_i_deg, order, period_um, lam_um):
    """Differentiating sin(theta_o) = sin(theta_i) + j lambda / Lambda gives
    cos(theta_o) d theta_o = cos(theta_i) d theta_i: the in-plane angular
    spread scales by cos(theta_i) / cos(theta_o), the in-plane width of a
    waist by the inverse, and the out-of-plane axis is unchanged."""
    ti = math.radians(theta_i_deg)
    so = math.sin(ti) + order * lam_um / period_um
    assert abs(so) < 1
    to = math.asin(so)
    b2 = 3.0
    K = b2 * np.eye(2)
    y = np.array([0.0, 1.0, 0.0])
    K2 = oracle.aniso_interaction(K, y, _in_plane(ti), y, _out_plane(to), [0, 0, 1])
    m = math.cos(to) / math.cos(ti)
    # frame axis 0 = y (out of plane), axis 1 = d x y (in plane)
    assert abs(K2[0, 0] - b2) < 1e-12
    assert abs(K2[1, 1] - b2 * m * m) < 1e-12 * b2
    assert abs(K2[0, 1]) < 1e-12
    # the wavevector spread Re(K)^-1 / 2 follows the differential relation
    assert abs(0.5 / K2[1, 1].real - (0.5 / b2) / (m * m)) < 1e-12


@pytest.mark.parametrize("theta_i_deg,eta_i,eta_t", [(30.0, 1.0, 1.5), (40.0, 1.5, 1.0), (70.0, 1.0, 2.4)])
def test_refraction_map_follows_snell(oracle, theta_i_deg, eta_i, eta_t):
    """eta_i sin(theta_i) = eta_t sin(theta_t) differentiates to eta_t
    cos(theta_t) d theta_t = eta_i cos(theta_i) d theta_i: the transverse
    wavevector spread in the plane scales by cos(theta_i) / cos(theta_t) and
    the width by the inverse."""
    ti = math.radians(theta_i_deg)
    tt = math.asin(eta_i * math.sin(ti) / eta_t)
    K = np.array([[2.0 + 0.3j, 0.0], [0.0, 5.0 - 1.0j]])
    y = np.array([0.0, 1.0, 0.0])
    d_t = np.array([math.sin(tt), 0.0, -math.cos(tt)])  # continues through z = 0
    K2 = oracle.aniso_interaction(K, y, _in_plane(ti), y, d_t, [0, 0, 1])
    m = math.cos(tt) / math.cos(ti)
    assert abs(K2[0, 0] - K[0, 0]) < 1e-12
    assert abs(K2[1, 1] - K[1, 1] * m * m) < 1e-12 * abs(K[1, 1])


def test_mirror_map_is_orthogonal_and_area_ratio(oracle):
    """Mirror reflection maps the footprint by a rotation (eigenvalues kept;
    an isotropic ray stays isotropic); for any pair of directions |det W|
    = |d_out . n| / |d_in . n| (the projected-area ratio), seen through
    det K_out = det(W)^2 det K."""
    rng = np.random.default_rng(3)
    for _ in range(40):
        n = rng.standard_normal(3)
        n /= np.linalg.norm(n)
        d = rng.standard_normal(3)
        d /= np.linalg.norm(d)
        if d @ n > -0.05:
            d = d - 2 * (d @ n) * n if d @ n > 0.05 else -n
        f = np.cross(d, rng.standard_normal(3))
        f /= np.linalg.norm(f)
        K = np.array([[3.0 + 1j, 0.7 - 0.2j], [0.7 - 0.2j, 1.5 + 0.5j]])
        r = d - 2 * (d @ n) * n
        g = np.cross(r, rng.standard_normal(3))
        g /= np.linalg.norm(g)
        Km = oracle.aniso_interaction(K, f, d, g, r, n)
        ev = np.sort_complex(np.linalg.eigvals(K))
        evm = np.sort_complex(np.linalg.eigvals(Km))
        assert np.max(np.abs(ev - evm)) < 1e-10
        iso = oracle.aniso_interaction(2.0 * np.eye(2), f, d, g, r, n)
        assert np.max(np.abs(iso - 2.0 * np.eye(2))) < 1e-12
        # any outgoing direction on the same side as r
        o = r + 0.6 * rng.standard_normal(3)
        o /= np.linalg.norm(o)
        if o @ n < 0.05:
            continue
        h = np.cross(o, rng.standard_normal(3))
        h /= np.linalg.norm(h)
        Ko = oracle.aniso_interaction(K, f, d, h, o, n)
        ratio2 = (abs(o @ n) / abs(d @ n)) ** 2
        assert abs(np.linalg.det(Ko) - ratio2 * np.linalg.det(K)) < 1e-10 * abs(ratio2 * np.linalg.det(K))


def _mirror_scene():
    """A tilted mirror reflecting an emitter and a distant source, plus a
    constant environment: every interaction is a mirror reflection."""
    mats = [sg.material(sg.MAT_MIRROR, fresnel=1, n_re=0.3, n_im=3.5),
            sg.material(sg.MAT_EMITTER, Le=1.0, coh_len_um=3.0)]
    tris = np.concatenate([sg._quad((0, 0, 0), (0, 0, 0.5), (0.5, 0, 0)),
                           sg._quad((0.0, 0.29, -0.52), (0.15, 0, 0), (0, 0.131, 0.0729))])
    lights = [sg.light(sg.LIGHT_DISTANT, (0.05, 0.5, -0.86), 1.0, 20.0), sg.light(sg.LIGHT_ENV, (0, 0, 1), 0.1, 0.0)]
    return sg._scene(tris, [0, 0, 1, 1], mats, np.asarray(lights, dtype=np.float32))


def _view(**kw):
    base = dict(eye=(0.0, 0.25, 0.45), look_at=(0.0, 0.0, 0.0), up=(0, 1, 0), vfov_deg=40.0, width=12, height=10,
                n_bins=4, n_stokes=1, max_depth=4, spp=16)
    base.update(kw)
    return sg.view(**base)


@pytest.mark.parametrize("ns", [1, 4])
def test_mirror_scene_equals_scalar_model(oracle, ns):
    """Mirror reflections keep an isotropic ray isotropic, and the
    anisotropic measurements reduce to the scalar ones: the image equals the
    scalar model's to rounding."""
    scene = _mirror_scene()
    v = _view(n_stokes=ns)
    O = oracle.Scene(scene)
    a = O.render(v, 3, oracle.FLAG_ANISO | oracle.FLAG_NEE)
    b = O.render(v, 3, oracle.FLAG_NEE)
    assert np.max(b) > 1e-3
    assert np.max(np.abs(a - b)) <= 1e-10 * np.max(np.abs(b))


def test_grating_scene_differs_from_scalar_model(oracle):
    """Grating orders leave at other angles: the footprint becomes
    anisotropic and the measured lobes change."""
    scene = sg.grating_scene()
    v = sg.grating_view(width=16, height=16, spp=16, n_bins=4)
    O = oracle.Scene(scene)
    a = O.render(v, 2, oracle.FLAG_ANISO)
    b = O.render(v, 2, 0)
    assert np.isfinite(a).all()
    rel = np.linalg.norm(a - b) / np.linalg.norm(b)
    print("anisotropic vs scalar on the planar grating: rel diff", rel)
    assert rel > 1e-3


def test_hero_and_aniso_not_combined(oracle):
    with pytest.raises(ValueError):
        oracle.Scene(_mirror_scene()).render(_view(), 1, oracle.FLAG_ANISO | oracle.FLAG_HERO)


def _frame(d):
    d = np.asarray(d, float) / np.linalg.norm(d)
    f = np.cross(d, [0.3, 0.9, 0.1])
    return d, f / np.linalg.norm(f)


def test_emitter_footprint_marginal_is_the_wavevector_marginal(oracle):
    """Averaged over the footprint point (Gauss-Hermite quadrature), the
    emitter lobe seen through the conditional direction (mean -Im(A) x / k,
    covariance Re(A) / (2 k^2)) is the lobe of the wavevector marginal
    Re(K)^-1 / (2 k^2): the Wigner decomposition of the Gaussian field.  A
    wrong footprint covariance, shift magnitude or residual fails it."""
    d, xf = _frame([0.1, -0.2, -1.0])
    k = 2 * np.pi / 0.5
    K = np.array([[30.0 + 200.0j, 8.0 - 60.0j], [8.0 - 60.0j, 12.0 + 150.0j]])  # um^2, propagated
    s2 = 1e-4
    e1, e2 = oracle.onb(d)
    # the marginal covariance in the frame onb(d)
    u2 = np.cross(d, xf)
    R = np.array([[e1 @ xf, e1 @ u2], [e2 @ xf, e2 @ u2]])
    Ke = R @ K @ R.T
    Cm = 0.5 * np.linalg.inv(Ke.real) / k ** 2 + s2 * np.eye(2)
    z, w = np.polynomial.hermite_e.hermegauss(60)
    w = w / w.sum()
    for off in ([0.0, 0.0], [0.01, -0.004], [-0.006, 0.012]):
        ne = -(d + off[0] * e1 + off[1] * e2)
        ne /= np.linalg.norm(ne)
        mean = 0.0
        for i in range(len(z)):
            for j in range(len(z)):
                mean += w[i] * w[j] * oracle.aniso_emitter(K, xf, d, k, s2, ne, z[i], z[j])[2]
        # Gaussian in the tangent plane (small angles)
        delta = np.array([(-ne - d) @ e1, (-ne - d) @ e2])
        ref = np.exp(-0.5 * delta @ np.linalg.solve(Cm, delta)) / (2 * np.pi * np.sqrt(np.linalg.det(Cm)))
        assert abs(mean - ref) < 2e-3 * ref, (off, mean, ref)


def test_far_field_shift_is_geometric(oracle):
    """Far from the waist (zbar >> K), the direction at footprint point x is
    the geometric x / z (um / um), whatever the waist's anisotropy."""
    d, xf = _frame([0.0, 0.0, -1.0])
    k = 2 * np.pi / 0.6
    K0 = np.array([[2.0, 0.7], [0.7, 5.0]])
    zbar = 1e6
    K = oracle.aniso_propagate(K0, zbar)
    for z0, z1 in ((1.0, 0.0), (0.0, -1.3), (0.8, 0.5)):
        x, m, _ = oracle.aniso_emitter(K, xf, d, k, 0.0, -d, z0, z1)
        g = x / (zbar * k)
        assert np.linalg.norm(m - g) <= 1e-5 * np.linalg.norm(g)


def test_footprint_point_covariance_is_the_spatial_marginal(oracle):
    """The footprint point's covariance (Gauss-Hermite moments over the
    standard normal pair) equals Re(A)^-1 / 2 with A = K^-1, K rotated into
    the frame onb(d), computed here with numpy: a wrong Cholesky factor,
    frame rotation or transposition fails it."""
    d, xf = _frame([0.3, -0.4, -0.8])
    k = 2 * np.pi / 0.55
    K = np.array([[25.0 + 90.0j, -6.0 + 40.0j], [-6.0 + 40.0j, 9.0 + 120.0j]])
    e1, e2 = oracle.onb(d)
    u2 = np.cross(d, xf)
    R = np.array([[e1 @ xf, e1 @ u2], [e2 @ xf, e2 @ u2]])
    A = np.linalg.inv(R @ K @ R.T)
    sigma = 0.5 * np.linalg.inv(A.real)
    z, w = np.polynomial.hermite_e.hermegauss(12)
    w = w / w.sum()
    cov = np.zeros((2, 2))
    mean = np.zeros(2)
    for i in range(len(z)):
        for j in range(len(z)):
            x, _, _ = oracle.aniso_emitter(K, xf, d, k, 0.0, -d, z[i], z[j])
            cov += w[i] * w[j] * np.outer(x, x)
            mean += w[i] * w[j] * x
    assert np.max(np.abs(mean)) < 1e-12 * np.sqrt(np.max(np.abs(sigma)))
    assert np.max(np.abs(cov - sigma)) < 1e-10 * np.max(np.abs(sigma))
