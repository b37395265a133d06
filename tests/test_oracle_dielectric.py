"""Pins of the oracle's dielectric interface (Eq. K_reflection_refraction with
refraction): Fresnel reflectance and transmittance against the textbook angle
forms of the Fresnel equations, energy conservation per polarisation,
Brewster's angle, total internal reflection, Snell's law and reversibility,
and a white furnace through a glass slab."""
import math

import numpy as np
import pytest

from paper_2303_15762_gb300 import scenegen as sg

N_RELS = [1.5, 1 / 1.5, 2.4, 1 / 2.4, 1.33]


def _angle_forms(ti, n_rel):
    """Fresnel power coefficients in angle form (Hecht, Optics, Sec. 4.6):
    Rs = sin^2(ti-tt)/sin^2(ti+tt), Rp = tan^2(ti-tt)/tan^2(ti+tt),
    Ts = sin 2ti sin 2tt / sin^2(ti+tt), Tp = Ts / cos^2(ti-tt)."""
    tt = math.asin(math.sin(ti) / n_rel)
    Rs = math.sin(ti - tt) ** 2 / math.sin(ti + tt) ** 2
    Rp = math.tan(ti - tt) ** 2 / math.tan(ti + tt) ** 2
    Ts = math.sin(2 * ti) * math.sin(2 * tt) / math.sin(ti + tt) ** 2
    Tp = Ts / math.cos(ti - tt) ** 2
    return Rs, Rp, Ts, Tp


@pytest.mark.parametrize("n_rel", N_RELS)
def test_fresnel_against_angle_forms_and_energy(oracle, n_rel):
    crit = math.asin(n_rel) if n_rel < 1 else math.pi / 2
    for ti in np.linspace(0.02, min(crit, math.pi / 2) - 0.02, 25):
        got = oracle.fresnel_dielectric(math.cos(ti), n_rel)
        Rs, Rp, Ts, Tp = _angle_forms(ti, n_rel)
        for a, b in ((got["Rs"], Rs), (got["Rp"], Rp), (got["Ts"], Ts), (got["Tp"], Tp)):
            assert abs(a - b) < 1e-12, (n_rel, ti, a, b)
        assert abs(got["Rs"] + got["Ts"] - 1) < 1e-13 and abs(got["Rp"] + got["Tp"] - 1) < 1e-13
        assert abs(got["R"] + got["T"] - 1) < 1e-13
        assert not got["tir"]


@pytest.mark.parametrize("n_rel", N_RELS)
def test_normal_incidence_and_brewster(oracle, n_rel):
    got = oracle.fresnel_dielectric(1.0, n_rel)
    r0 = ((n_rel - 1) / (n_rel + 1)) ** 2
    assert abs(got["Rs"] - r0) < 1e-15 and abs(got["Rp"] - r0) < 1e-15
    tb = math.atan(n_rel)  # Brewster: the reflected p component vanishes
    assert oracle.fresnel_dielectric(math.cos(tb), n_rel)["Rp"] < 1e-28


@pytest.mark.parametrize("n_rel", [1 / 1.5, 1 / 2.4, 1 / 1.33])
def test_total_internal_reflection(oracle, n_rel):
    crit = math.asin(n_rel)
    below = oracle.fresnel_dielectric(math.cos(crit - 1e-3), n_rel)
    assert not below["tir"] and below["T"] > 0
    for ti in np.linspace(crit + 1e-6, math.pi / 2 - 1e-3, 17):
        got = oracle.fresnel_dielectric(math.cos(ti), n_rel)
        assert got["tir"] and got["T"] == 0.0
        # |r_s| = |r_p| = 1 past the critical angle
        assert abs(got["Rs"] - 1) < 1e-14 and abs(got["Rp"] - 1) < 1e-14


def test_snell_coplanarity_and_reversibility(oracle):
    rng = np.random.default_rng(7)
    for _ in range(300):
        n = rng.standard_normal(3)
        n /= np.linalg.norm(n)
        d = rng.standard_normal(3)
        d /= np.linalg.norm(d)
        if abs(d @ n) < 1e-3:
            continue
        ea, eb = (1.0, 1.5) if rng.uniform() < 0.5 else (1.5, 1.0)
        t = oracle.refract(d, n, ea, eb)
        nf = n if d @ n < 0 else -n
        sin_i = np.linalg.norm(np.cross(d, nf))
        if ea * sin_i >= eb:
            assert t is None  # total internal reflection
            continue
        assert abs(np.linalg.norm(t) - 1) < 1e-14
        # Snell: eta_a sin(theta_i) = eta_b sin(theta_t); same side of the plane
        assert abs(ea * sin_i - eb * np.linalg.norm(np.cross(t, nf))) < 1e-13
        assert abs(np.dot(np.cross(d, nf), t)) < 1e-13  # in the plane of incidence
        assert t @ nf < 0  # continues through the interface
        back = oracle.refract(-t, n, eb, ea)
        assert np.max(np.abs(back + d)) < 1e-13  # light paths are reversible


@pytest.mark.parametrize("cauchy_b", [0.0, 0.0042])
def test_white_furnace_through_glass_slab(oracle, cauchy_b):
    """A closed glass slab in a constant unit environment with the lobe chosen
    by reflectance: every escaping path carries exactly 1 (the (eta_a/eta_b)^2
    radiance factors of entering and leaving cancel), so every pixel is 1."""
    scene = sg.dielectric_scene(cauchy_b_um2=cauchy_b, with_ground=False, emitter=False, distant=False, env=1.0)
    view = sg.dielectric_view(width=12, height=10, spp=16, n_bins=4, n_stokes=1, max_depth=64)
    img = oracle.Scene(scene).render(view, 3, 0)
    assert np.max(np.abs(img - 1.0)) < 1e-12


def test_slab_transmits_less_than_one_and_disperses(oracle):
    """Through the slab (no environment, a distant source and an emitter over a
    rough ground) the image differs across wavelength bins once the index
    depends on lambda, and not without dispersion except through the
    wavelength-dependent lobes; a sanity check that refraction changes paths."""
    view = sg.dielectric_view(width=16, height=12, spp=8, n_bins=4, n_stokes=1, max_depth=6)
    a = oracle.Scene(sg.dielectric_scene(cauchy_b_um2=0.0)).render(view, 5, oracle.FLAG_NEE)
    b = oracle.Scene(sg.dielectric_scene(cauchy_b_um2=0.0042)).render(view, 5, oracle.FLAG_NEE)
    assert np.isfinite(a).all() and np.isfinite(b).all()
    assert np.abs(a - b).max() > 0  # dispersion moves refracted paths
    assert a.max() > 0


@pytest.mark.parametrize("cauchy_b", [0.0, 0.0042])
def test_camera_inside_glass_sees_eta_squared(oracle, cauchy_b):
    """Radiance compression across an interface (L / eta^2 is invariant along a
    ray): a camera inside a glass cube in a constant unit environment sees
    eta(lambda)^2 in every pixel.  With a 30 degree field of view every camera
    ray keeps |d_z| > cos(theta_c), so no path is trapped by total internal
    reflection, and each leaves through a face with the factor eta^2 (a
    missing or inverted radiance factor would give 1 or 1/eta^2)."""
    n_re = 1.5
    box = sg._box((0.0, 0.0, 0.0), (0.2, 0.2, 0.2))
    scene = sg._scene(box, [0] * len(box), [sg.material(sg.MAT_DIELECTRIC, n_re=n_re, cauchy_b_um2=cauchy_b)],
                      [sg.light(sg.LIGHT_ENV, (0, 0, 1), 1.0, 0.0)])
    view = sg.view(eye=(0.0, 0.0, 0.0), look_at=(0.0, 0.0, -1.0), up=(0, 1, 0), vfov_deg=30.0, width=10, height=10,
                   n_bins=4, n_stokes=1, max_depth=64, spp=16)
    img = oracle.Scene(scene).render(view, 2, 0)
    lmin, lmax = view["lambda_min_um"], view["lambda_max_um"]  # float32-rounded
    for b in range(4):
        lam = lmin + b * (lmax - lmin) / 3
        eta = float(np.float32(n_re)) + float(np.float32(cauchy_b)) / lam ** 2
        assert np.max(np.abs(img[:, :, b, 0] - eta * eta)) < 1e-11, (b, img[:, :, b, 0].min(), eta * eta)
