"""Pins of the oracle's hero-wavelength spectral MIS (Sec. 7.2; Wilkie et al.
2014): with the flag a path's bin is the hero of a class of four bins, an
escape is measured at all four wavelengths and weighted by the balance
heuristic over their path densities, and emitter contributions stay with the
hero.  Pinned by a mirror furnace (exactly 1 in every bin), by the plain
estimator wherever every path is hero-only (dispersive glass; one sample per
class), by agreement with the plain estimator's means, and by a lower error
at equal sample count where no decision is dispersive."""
import numpy as np
import pytest

from paper_2303_15762_gb300 import scenegen as sg


def _view(**kw):
    base = dict(eye=(0.0, 0.25, 0.45), look_at=(0.0, 0.0, 0.0), up=(0, 1, 0), vfov_deg=40.0, width=6, height=5,
                n_bins=8, n_stokes=1, max_depth=4, spp=64)
    base.update(kw)
    return sg.view(**base)


def _rough_grating_scene(env=0.3):
    """Rough conductor ground and a grating tile under a distant source and a
    constant environment."""
    mats = [sg.material(sg.MAT_ROUGH, fresnel=1, n_re=0.3, n_im=3.5, sigma_h_um=0.12, corr_len_um=3.0),
            sg.material(sg.MAT_GRATING, fresnel=1, n_re=0.3, n_im=3.5, period_um=1.8, height_um=0.2,
                        gdir=(1, 0, 0))]
    tris = np.concatenate([sg._quad((0, 0, 0), (0, 0, 0.5), (0.5, 0, 0)),
                           sg._quad((0.05, 0.02, -0.05), (0, 0, 0.06), (0.06, 0, 0))])
    # the source lies near the mirror direction of the central camera ray
    lights = [sg.light(sg.LIGHT_DISTANT, (0.05, 0.5, -0.86), 1.0, 20.0), sg.light(sg.LIGHT_ENV, (0, 0, 1), env, 0.0)]
    return sg._scene(tris, [0, 0, 1, 1], mats, np.asarray(lights, dtype=np.float32))


def test_mirror_furnace_every_bin_exactly_one(oracle):
    """Mirror and environment only: no decision depends on the wavelength, so
    the class weights sum to one per path and every bin is exactly 1."""
    mats = [sg.material(sg.MAT_MIRROR)]
    tris = sg._quad((0, 0, 0), (0, 0, 0.2), (0.2, 0, 0))
    scene = sg._scene(tris, [0, 0], mats, [sg.light(sg.LIGHT_ENV, (0, 0, 1), 1.0, 0.0)])
    img = oracle.Scene(scene).render(_view(spp=40), 3, oracle.FLAG_HERO)
    assert np.max(np.abs(img - 1.0)) < 1e-12


@pytest.mark.parametrize("first", [0, 5])
def test_single_sample_per_class_equals_plain(oracle, first):
    """With one sample per class (spp = 2 < 8 bins) a class holds no
    companion samples, so hero MIS is the plain estimator."""
    scene = _rough_grating_scene()
    v = _view(spp=2, first_sample=first)
    O = oracle.Scene(scene)
    a = O.render(v, 7, oracle.FLAG_HERO | oracle.FLAG_NEE)
    b = O.render(v, 7, oracle.FLAG_NEE)
    assert np.max(np.abs(a - b)) <= 1e-12 * max(1.0, np.max(np.abs(b)))


def test_paths_through_dispersive_glass_are_hero_only(oracle):
    """A camera inside dispersive glass: every path crosses a dispersive
    interface, no other wavelength could make it, and hero MIS gives the
    plain estimator's image."""
    box = sg._box((0.0, 0.0, 0.0), (0.2, 0.2, 0.2))
    scene = sg._scene(box, [0] * len(box), [sg.material(sg.MAT_DIELECTRIC, n_re=1.5, cauchy_b_um2=0.0042)],
                      [sg.light(sg.LIGHT_DISTANT, (0.1, 0.2, 1.0), 1.0, 30.0)])
    v = sg.view(eye=(0.0, 0.0, 0.0), look_at=(0.0, 0.0, -1.0), up=(0, 1, 0), vfov_deg=30.0, width=6, height=6,
                n_bins=8, n_stokes=1, max_depth=16, spp=32)
    O = oracle.Scene(scene)
    a = O.render(v, 2, oracle.FLAG_HERO)
    b = O.render(v, 2, 0)
    assert np.max(np.abs(a - b)) <= 1e-12 * max(1.0, np.max(np.abs(b)))


def test_unbiased_against_plain_estimator(oracle):
    """Rough ground, a grating tile, a distant source and an environment:
    at high sample counts the two estimators' bin means agree within their
    Monte Carlo errors."""
    scene = _rough_grating_scene()
    v = _view(width=3, height=2, spp=8192)
    O = oracle.Scene(scene)
    mp, vp = O.render(v, 11, 0, want_var=True)
    mh = O.render(v, 12, oracle.FLAG_HERO)
    n_per_bin = v["spp"] // v["n_bins"]
    se = np.sqrt(np.maximum(vp, 0.0) / n_per_bin)
    # hero's error is below plain's; allow five of plain's standard errors each way
    assert np.all(np.abs(mh - mp) <= 5.0 * np.sqrt(2.0) * se + 1e-9)


def test_lower_error_at_equal_samples(oracle):
    """Where no decision is dispersive (rough ground under a distant source),
    each path informs four bins: at 16 samples per pixel the hero estimator's
    error against a high-sample reference is clearly below the plain one's."""
    mats = [sg.material(sg.MAT_ROUGH, fresnel=1, n_re=0.3, n_im=3.5, sigma_h_um=0.15, corr_len_um=1.5)]
    tris = sg._quad((0, 0, 0), (0, 0, 0.5), (0.5, 0, 0))
    scene = sg._scene(tris, [0, 0], mats, [sg.light(sg.LIGHT_DISTANT, (0.05, 0.5, -0.86), 1.0, 20.0)])
    v = _view(width=8, height=6, spp=16)
    O = oracle.Scene(scene)
    ref = O.render(dict(v, spp=4096), 99, 0)
    ep = np.sqrt(np.mean((O.render(v, 5, 0) - ref) ** 2))
    eh = np.sqrt(np.mean((O.render(v, 5, oracle.FLAG_HERO) - ref) ** 2))
    print("rms error plain %.4g hero %.4g (reference rms %.4g)" % (ep, eh, np.sqrt(np.mean(ref ** 2))))
    assert np.sqrt(np.mean(ref ** 2)) > 1e-3  # a lit image
    assert eh < 0.8 * ep


def test_bins_not_multiple_of_four_rejected(oracle):
    with pytest.raises(ValueError):
        oracle.Scene(_rough_grating_scene()).render(_view(n_bins=6), 1, oracle.FLAG_HERO)


def _emitter_scene():
    """Rough ground and a grating tile lit only by a partially coherent
    emissive quad in the mirror direction of the camera, facing them, so
    that every contribution is an emitter hit or a next-event estimate."""
    mats = [sg.material(sg.MAT_ROUGH, fresnel=1, n_re=0.3, n_im=3.5, sigma_h_um=0.15, corr_len_um=1.5),
            sg.material(sg.MAT_GRATING, fresnel=1, n_re=0.3, n_im=3.5, period_um=1.8, height_um=0.2,
                        gdir=(1, 0, 0)),
            sg.material(sg.MAT_EMITTER, Le=1.0, coh_len_um=3.0)]
    # the emitter faces the ground patch the camera sees (normal (0, -0.486, 0.874))
    tris = np.concatenate([sg._quad((0, 0, 0), (0, 0, 0.5), (0.5, 0, 0)),
                           sg._quad((0.05, 0.02, -0.05), (0, 0, 0.06), (0.06, 0, 0)),
                           sg._quad((0.0, 0.29, -0.52), (0.15, 0, 0), (0, 0.131, 0.0729))])
    return sg._scene(tris, [0, 0, 1, 1, 2, 2], mats, np.zeros((0, 8), dtype=np.float32))


@pytest.mark.parametrize("nee", [False, True])
def test_emitters_single_sample_per_class_equals_plain(oracle, nee):
    """One sample per class: the joint power heuristic over (wavelength,
    technique) is the plain estimator's power heuristic between lobe and
    emitter sampling, and every weight of a class without companion samples
    is the plain one."""
    scene = _emitter_scene()
    v = _view(spp=2, first_sample=3)
    O = oracle.Scene(scene)
    f = oracle.FLAG_NEE if nee else 0
    a = O.render(v, 7, oracle.FLAG_HERO | f)
    b = O.render(v, 7, f)
    assert np.max(b) > 0
    assert np.max(np.abs(a - b)) <= 1e-12 * max(1.0, np.max(np.abs(b)))


@pytest.mark.parametrize("nee", [False, True])
def test_emitters_unbiased_against_plain_estimator(oracle, nee):
    """Emitter hits (and next-event estimates) shared across the class: the
    bin means agree with the plain estimator's within Monte Carlo error, so
    the weights of every path sum to one over the techniques that make it."""
    scene = _emitter_scene()
    v = _view(width=3, height=2, spp=8192)
    O = oracle.Scene(scene)
    f = oracle.FLAG_NEE if nee else 0
    mp, vp = O.render(v, 21, f, want_var=True)
    mh = O.render(v, 22, oracle.FLAG_HERO | f)
    se = np.sqrt(np.maximum(vp, 0.0) / (v["spp"] // v["n_bins"]))
    assert np.max(mp) > 1e-3
    assert np.all(np.abs(mh - mp) <= 5.0 * np.sqrt(2.0) * se + 1e-9)


def test_emitters_lower_error_at_equal_samples(oracle):
    """With next-event estimation, each connection informs four bins: at 16
    samples per pixel the hero estimator's error is clearly below the plain
    one's."""
    scene = _emitter_scene()
    v = _view(width=8, height=6, spp=16)
    O = oracle.Scene(scene)
    ref = O.render(dict(v, spp=4096), 99, oracle.FLAG_NEE)
    ep = np.sqrt(np.mean((O.render(v, 5, oracle.FLAG_NEE) - ref) ** 2))
    eh = np.sqrt(np.mean((O.render(v, 5, oracle.FLAG_HERO | oracle.FLAG_NEE) - ref) ** 2))
    print("emitters: rms error plain %.4g hero %.4g (reference rms %.4g)" % (ep, eh, np.sqrt(np.mean(ref ** 2))))
    assert np.sqrt(np.mean(ref ** 2)) > 1e-3
    assert eh < 0.8 * ep


def test_member_footprints_follow_from_the_heros():
    """The kernels do not carry a footprint per class member: they derive it
    from the hero's rho.  Free propagation (Eq. K_free_space_propagation, the
    oracle's `propagate`) chained over a path's segments, at each class
    wavelength from the same camera footprint (beta0^2, 0), gives rho_g =
    rho_hero lambda_g / lambda_hero and beta_g^2 = beta0^2 (1 + rho_g^2) to
    FP64 rounding, for any segment lengths and media (zbar = z lambda /
    (2 pi eta))."""
    from oracle import oracle as orc
    rng = np.random.default_rng(7)
    for _ in range(20):
        beta0 = rng.uniform(0.5, 30.0)
        lam = np.sort(rng.uniform(0.4, 0.7, 4))
        hero = int(rng.integers(4))
        segs = [(rng.uniform(1e-4, 2.0), rng.choice([1.0, 1.33, 1.5])) for _ in range(int(rng.integers(1, 6)))]
        fp = []
        for lg in lam:
            b2, r = beta0 * beta0, 0.0
            for t_m, eta in segs:
                b2, r = orc.propagate(b2, r, t_m * 1e6 * lg / (2 * np.pi * eta))
            fp.append((b2, r))
        rho_h = fp[hero][1]
        for g in range(4):
            rho_g = rho_h * lam[g] / lam[hero]
            assert fp[g][1] == pytest.approx(rho_g, rel=1e-12)
            assert fp[g][0] == pytest.approx(beta0 * beta0 * (1.0 + rho_g * rho_g), rel=1e-12)
