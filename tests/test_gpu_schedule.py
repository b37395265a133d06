"""The wavefront schedule does not change any image: pool size, regeneration
threshold, block size, the trace kernel's claim groups (64 queue entries per
atomic in launches of more than 4M rays, 32 otherwise), the ticket order over
views (deepest first) and one-sample tickets folded straight into the frame
all leave every pixel bit-identical, because each ticket's samples are summed
in sample order whatever the schedule."""
import numpy as np
import pytest

from paper_2303_15762_gb300 import scenegen as sg

pytestmark = pytest.mark.gpu


def test_images_independent_of_schedule(gr):
    scenes = [sg.procedural_scene(seed=31, n_objects=6, target_tris=6000, n_emitters=2), sg.grating_scene()]
    views = [
        # 1024^2 pixels x 8 of 16 bins: 8.4M one-sample tickets (spp < n_bins)
        dict(sg.procedural_view(width=1024, height=1024, spp=8, n_bins=16, n_stokes=1, max_depth=3),
             scene_index=0, view_index=0),
        # deeper paths, four samples per ticket: numbered first
        dict(sg.procedural_view(width=256, height=192, spp=32, n_bins=8, n_stokes=1, max_depth=6),
             scene_index=0, view_index=1),
        dict(sg.grating_view(width=64, height=48, spp=16, n_bins=4), scene_index=1, view_index=2),
    ]
    S = [gr.Scene(s) for s in scenes]
    schedules = [dict(pool_size=1 << 20, regen_threshold_pct=0),
                 dict(pool_size=1 << 23, regen_threshold_pct=25),   # trace launches of > 4M rays
                 dict(pool_size=1 << 18, regen_threshold_pct=50, block=128)]
    images = []
    for sch in schedules:
        f = gr.Frame(views)
        gr.render(S, views, f, seed=12, flags=gr.FLAG_NEE | gr.FLAG_RR, use_graph=True, **sch)
        images.append([f.readback(i) for i in range(len(views))])
        f.close()
    for i in range(len(views)):
        assert np.linalg.norm(images[0][i]) > 0
        for k in (1, 2):
            assert np.array_equal(images[0][i], images[k][i]), (i, schedules[k])
    # each view alone (a single view is not reordered) gives the same image
    for i, v in enumerate(views):
        f = gr.Frame([v])
        gr.render(S, [v], f, seed=12, flags=gr.FLAG_NEE | gr.FLAG_RR)
        assert np.array_equal(f.readback(0), images[0][i]), i
        f.close()


@pytest.mark.parametrize("mode", ["hero", "aniso"])
def test_hero_and_aniso_images_independent_of_schedule(gr, mode):
    """Hero-wavelength MIS and anisotropic footprints with next-event rays and
    4 Stokes components: pool size, regeneration threshold, block size and the
    host loop or the graph leave every element bit-identical."""
    scene = sg.procedural_scene(seed=31, n_objects=6, target_tris=6000, n_emitters=2)
    view = sg.procedural_view(width=96, height=80, spp=64, n_bins=16, n_stokes=4, max_depth=4)
    flags = gr.FLAG_NEE | gr.FLAG_RR | (gr.FLAG_HERO if mode == "hero" else gr.FLAG_ANISO)
    S = [gr.Scene(scene)]
    schedules = [dict(), dict(pool_size=4096, regen_threshold_pct=25),
                 dict(pool_size=1 << 16, block=128, use_graph=True)]
    images = []
    for sch in schedules:
        f = gr.Frame([view])
        gr.render(S, [view], f, seed=5, flags=flags, **sch)
        images.append(f.readback(0))
        assert f.stats()["shadow_rays"] > 0
        f.close()
    assert np.linalg.norm(images[0]) > 0
    for k in (1, 2):
        assert np.array_equal(images[0], images[k]), schedules[k]
