"""Anisotropic generalized rays on the GPU (GR_FLAG_ANISO; beta and rho as
2x2 matrices, Sec. 3.1) against the FP64 oracle with the same flag, on the
same seeded inputs: the complex footprint K is propagated exactly, mapped
through every interaction by the surface's anamorphic projection, and the
sources are measured with its anisotropic Gaussians.  Tolerance: relative L2
<= 1e-3, as for the scalar model."""
import numpy as np
import pytest

from paper_2303_15762_gb300 import scenegen as sg

from _parity import ELEM_TOL, assert_parity, elem_err

pytestmark = pytest.mark.gpu
TOL = 1e-3


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-300))


def _view(**kw):
    base = dict(eye=(0.0, 0.25, 0.45), look_at=(0.0, 0.0, 0.0), up=(0, 1, 0), vfov_deg=40.0, width=24, height=20,
                n_bins=8, n_stokes=1, max_depth=4, spp=32)
    base.update(kw)
    return sg.view(**base)


def _emitter_scene():
    """Rough ground and a grating tile lit by a partially coherent emissive
    quad in the mirror direction of the camera, plus a distant source and a
    constant environment."""
    mats = [sg.material(sg.MAT_ROUGH, fresnel=1, n_re=0.3, n_im=3.5, sigma_h_um=0.15, corr_len_um=1.5),
            sg.material(sg.MAT_GRATING, fresnel=1, n_re=0.3, n_im=3.5, period_um=1.8, height_um=0.2,
                        gdir=(1, 0, 0)),
            sg.material(sg.MAT_EMITTER, Le=1.0, coh_len_um=3.0)]
    tris = np.concatenate([sg._quad((0, 0, 0), (0, 0, 0.5), (0.5, 0, 0)),
                           sg._quad((0.05, 0.02, -0.05), (0, 0, 0.06), (0.06, 0, 0)),
                           sg._quad((0.0, 0.29, -0.52), (0.15, 0, 0), (0, 0.131, 0.0729))])
    lights = [sg.light(sg.LIGHT_DISTANT, (0.05, 0.5, -0.86), 1.0, 20.0), sg.light(sg.LIGHT_ENV, (0, 0, 1), 0.05, 0.0)]
    return sg._scene(tris, [0, 0, 1, 1, 2, 2], mats, np.asarray(lights, dtype=np.float32))


def test_planar_grating_matches_oracle(gr, oracle):
    """Grating orders leave at other angles than they arrive: the footprint
    and its wavevector spread become anisotropic (the grating's anamorphic
    factor), which changes the measured distant lobe."""
    scene = sg.grating_scene()
    v = sg.grating_view(width=32, height=32, spp=32)
    img = gr.render_image(scene, v, seed=1, flags=gr.FLAG_ANISO)
    ref = oracle.Scene(scene).render(v, 1, oracle.FLAG_ANISO)
    r = rel_l2(img, ref)
    print("aniso grating rel-L2 =", r)
    assert r <= TOL
    assert elem_err(img, ref) <= ELEM_TOL
    assert rel_l2(gr.render_image(scene, v, seed=1), ref) > 1e-2  # the scalar model differs


@pytest.mark.parametrize("ns", [1, 4])
@pytest.mark.parametrize("nee", [False, True])
def test_emitter_scene_matches_oracle(gr, oracle, ns, nee):
    scene = _emitter_scene()
    v = _view(n_stokes=ns)
    g = gr.FLAG_ANISO | (gr.FLAG_NEE if nee else 0)
    o = oracle.FLAG_ANISO | (oracle.FLAG_NEE if nee else 0)
    img = gr.render_image(scene, v, seed=11, flags=g)
    ref = oracle.Scene(scene).render(v, 11, o)
    r = rel_l2(img, ref)
    print("aniso emitter scene ns=%d nee=%d rel-L2 = %.3g" % (ns, nee, r))
    assert np.linalg.norm(ref) > 1e-3
    assert r <= TOL
    assert elem_err(img, ref) <= ELEM_TOL


def test_procedural_stokes_nee_rr_matches_oracle(gr, oracle):
    scene = sg.procedural_scene(seed=7, n_objects=8, target_tris=4000, n_emitters=2)
    v = sg.procedural_view(width=48, height=40, spp=32, n_bins=8, n_stokes=4, max_depth=4)
    flags = (gr.FLAG_ANISO, oracle.FLAG_ANISO)
    img = gr.render_image(scene, v, seed=4, flags=flags[0] | gr.FLAG_NEE | gr.FLAG_RR)
    ref = oracle.Scene(scene).render(v, 4, flags[1] | oracle.FLAG_NEE | oracle.FLAG_RR)
    r = rel_l2(img, ref)
    print("aniso procedural rel-L2 =", r)
    assert r <= TOL
    assert elem_err(img, ref) <= ELEM_TOL


@pytest.mark.parametrize("cauchy_b", [0.0, 0.0042])
def test_glass_slab_matches_oracle(gr, oracle, cauchy_b):
    """Refraction changes the beam's angle to the interface: Snell's
    anamorphic factor on the footprint, through the slab and back."""
    scene = sg.dielectric_scene(cauchy_b_um2=cauchy_b)
    v = sg.dielectric_view(width=32, height=24, spp=32, n_bins=8, n_stokes=4, max_depth=8)
    img = gr.render_image(scene, v, seed=5, flags=gr.FLAG_ANISO | gr.FLAG_NEE)
    ref = oracle.Scene(scene).render(v, 5, oracle.FLAG_ANISO | oracle.FLAG_NEE)
    r = rel_l2(img, ref)
    print("aniso glass b=%g rel-L2 = %.3g" % (cauchy_b, r))
    assert r <= TOL
    assert elem_err(img, ref) <= ELEM_TOL


def test_mirror_scene_equals_scalar_model(gr):
    """Mirror reflections keep an isotropic footprint isotropic, so the
    anisotropic render equals the scalar one to FP32 rounding."""
    mats = [sg.material(sg.MAT_MIRROR, fresnel=1, n_re=0.3, n_im=3.5),
            sg.material(sg.MAT_EMITTER, Le=1.0, coh_len_um=3.0)]
    tris = np.concatenate([sg._quad((0, 0, 0), (0, 0, 0.5), (0.5, 0, 0)),
                           sg._quad((0.0, 0.29, -0.52), (0.15, 0, 0), (0, 0.131, 0.0729))])
    lights = [sg.light(sg.LIGHT_DISTANT, (0.05, 0.5, -0.86), 1.0, 20.0), sg.light(sg.LIGHT_ENV, (0, 0, 1), 0.1, 0.0)]
    scene = sg._scene(tris, [0, 0, 1, 1], mats, np.asarray(lights, dtype=np.float32))
    for ns in (1, 4):
        v = _view(n_stokes=ns, spp=16)
        a = gr.render_image(scene, v, seed=3, flags=gr.FLAG_ANISO | gr.FLAG_NEE)
        b = gr.render_image(scene, v, seed=3, flags=gr.FLAG_NEE).astype(np.float64)
        assert np.linalg.norm(b) > 0
        assert rel_l2(a, b) <= 1e-5, ns


def test_deterministic_and_graph(gr):
    scene = _emitter_scene()
    v = _view(spp=16, n_stokes=4)
    f = gr.FLAG_ANISO | gr.FLAG_NEE
    a = gr.render_image(scene, v, seed=8, flags=f)
    assert np.array_equal(a, gr.render_image(scene, v, seed=8, flags=f))
    assert np.array_equal(a, gr.render_image(scene, v, seed=8, flags=f, use_graph=True))


def test_hero_and_aniso_rejected(gr):
    scene = _emitter_scene()
    v = _view(spp=8)
    s = gr.Scene(scene)
    f = gr.Frame([v])
    with pytest.raises(gr.GrError) as e:
        gr.render([s], [v], f, flags=gr.FLAG_HERO | gr.FLAG_ANISO)
    assert e.value.status == 1
