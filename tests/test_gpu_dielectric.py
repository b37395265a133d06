"""Dielectric refraction on the CUDA path (Eq. K_reflection_refraction with
refraction) against the FP64 oracle on the same seeded inputs: a dispersive
glass slab over a rough conductor ground under a distant source and an
emitter (Stokes and scalar), the slab white furnace, and the eta^2 radiance
seen from inside glass."""
import numpy as np
import pytest

from paper_2303_15762_gb300 import scenegen as sg

from _parity import ELEM_TOL, assert_parity, elem_err

pytestmark = pytest.mark.gpu
TOL = 1e-3


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-300))


@pytest.mark.parametrize("n_stokes", [4, 1])
def test_slab_scene_matches_oracle(gr, oracle, n_stokes):
    scene = sg.dielectric_scene()
    view = sg.dielectric_view(width=48, height=40, spp=32, n_bins=8, n_stokes=n_stokes, max_depth=8)
    flags = gr.FLAG_NEE | gr.FLAG_RR
    img = gr.render_image(scene, view, seed=9, flags=flags)
    ref = oracle.Scene(scene).render(view, 9, oracle.FLAG_NEE | oracle.FLAG_RR)
    r = rel_l2(img, ref)
    print("dielectric slab, n_stokes", n_stokes, "rel-L2 =", r)
    assert np.linalg.norm(ref) > 0
    assert r <= TOL
    assert elem_err(img, ref) <= ELEM_TOL


def test_slab_white_furnace(gr):
    scene = sg.dielectric_scene(with_ground=False, emitter=False, distant=False, env=1.0)
    view = sg.dielectric_view(width=24, height=20, spp=16, n_bins=4, n_stokes=1, max_depth=64)
    img = gr.render_image(scene, view, seed=3)
    assert np.max(np.abs(img - 1.0)) < 2e-5


def test_camera_inside_glass_sees_eta_squared(gr):
    box = sg._box((0.0, 0.0, 0.0), (0.2, 0.2, 0.2))
    scene = sg._scene(box, [0] * len(box), [sg.material(sg.MAT_DIELECTRIC, n_re=1.5, cauchy_b_um2=0.0042)],
                      [sg.light(sg.LIGHT_ENV, (0, 0, 1), 1.0, 0.0)])
    view = sg.view(eye=(0.0, 0.0, 0.0), look_at=(0.0, 0.0, -1.0), up=(0, 1, 0), vfov_deg=30.0, width=12, height=12,
                   n_bins=4, n_stokes=1, max_depth=64, spp=16)
    img = gr.render_image(scene, view, seed=2)
    lmin, lmax = view["lambda_min_um"], view["lambda_max_um"]
    for b in range(4):
        lam = lmin + b * (lmax - lmin) / 3
        eta = float(np.float32(1.5)) + float(np.float32(0.0042)) / lam ** 2
        assert np.max(np.abs(img[:, :, b, 0] / (eta * eta) - 1.0)) < 2e-5, b


def test_dielectric_with_fp16_tables_and_graph(gr, oracle):
    """The grating-free dielectric scene is unaffected by the table type, and
    the graph launch gives the host loop's image."""
    scene = sg.dielectric_scene()
    view = sg.dielectric_view(width=32, height=24, spp=16, n_bins=4, n_stokes=4, max_depth=6)
    a = gr.render_image(scene, view, seed=4, flags=gr.FLAG_NEE)
    b = gr.render_image(scene, view, seed=4, flags=gr.FLAG_NEE, table_dtype="f16", use_graph=True)
    assert np.array_equal(a, b)
