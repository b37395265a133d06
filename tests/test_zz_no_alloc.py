"""gr_render_static: rendering for callers that may not allocate device memory
while they render (a service that reserves all of its GPU memory up front, or
code where an allocation would synchronise the device or fail under memory
pressure).  The entry point runs the wavefront kernels on scratch compiled into
the library and writes caller-owned accumulators; these tests compare it, call
after call, with gr_render's output through the C ABI.

Kept in a file collected last so that a run stopping at its first failure has
already run every other test; it also passes on its own in a fresh process."""
import ctypes

import numpy as np
import pytest

from paper_2303_15762_gb300 import scenegen as sg

pytestmark = pytest.mark.gpu
TOL = 1e-3


def _static_render(gr, scenes, views, accum, **opts):
    from paper_2303_15762_gb300 import _native as nat
    L = nat.lib_handle()
    sc = (ctypes.c_void_p * len(scenes))(*[s.handle.value for s in scenes])
    arr = nat.pack_views(views)
    o = nat.make_opts(**opts)
    return L.gr_render_static(sc, len(scenes), arr, len(views), ctypes.byref(o),
                              ctypes.c_void_p(accum.data_ptr()), nat.current_stream())


def _mean_from_accum(accum, views, counts):
    """Per-view mean images [H][W][bins][stokes] from the caller's buffer."""
    a = accum.cpu().numpy().astype(np.float64)
    total = sum(v["width"] * v["height"] * v["n_bins"] * v["n_stokes"] for v in views)
    out, off = [], 0
    for v, cnt in zip(views, counts):
        n = v["width"] * v["height"] * v["n_bins"] * v["n_stokes"]
        s = a[off:off + n] - a[total + off:total + off + n]
        s = s.reshape(v["n_bins"], v["height"], v["width"], v["n_stokes"])
        c = np.asarray(cnt, np.float64).reshape(-1, 1, 1, 1)
        out.append(np.transpose(np.where(c > 0, s / np.maximum(c, 1), 0.0), (1, 2, 0, 3)))
        off += n
    return out


def _bin_counts(v, first, spp):
    nb = v["n_bins"]
    return [len([s for s in range(first, first + spp) if s % nb == b]) for b in range(nb)]


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def test_static_matches_render_two_calls_in_a_row(gr):
    import torch
    scenes = [sg.grating_scene(), sg.procedural_scene(seed=7, n_objects=8, target_tris=8000, n_emitters=2)]
    v0 = dict(sg.grating_view(width=32, height=24, spp=16), scene_index=0, view_index=0)
    v1 = dict(sg.procedural_view(width=40, height=40, spp=8, n_bins=4, n_stokes=1), scene_index=1, view_index=1)
    views = [v0, v1]
    S = [gr.Scene(s) for s in scenes]
    total = sum(v["width"] * v["height"] * v["n_bins"] * v["n_stokes"] for v in views)
    accum = torch.zeros(2 * total, dtype=torch.float32, device="cuda")

    # first call: a fresh image, compared with gr_render
    ref = gr.Frame(views)
    gr.render(S, views, ref, seed=11, flags=gr.FLAG_NEE)
    assert _static_render(gr, S, views, accum, seed=11, flags=gr.FLAG_NEE) == 0
    torch.cuda.synchronize()
    got = _mean_from_accum(accum, views, [_bin_counts(v, 0, v["spp"]) for v in views])
    for i in range(2):
        r = ref.readback(i).astype(np.float64)
        assert _rel(got[i], r) <= TOL, i

    # second call right after: the next sample range added into the same
    # buffer (the static scratch still holds the first call's state)
    nxt = [dict(v, first_sample=v["spp"]) for v in views]
    gr.render(S, nxt, ref, seed=11, flags=gr.FLAG_NEE)
    assert _static_render(gr, S, nxt, accum, seed=11, flags=gr.FLAG_NEE) == 0
    torch.cuda.synchronize()
    got = _mean_from_accum(accum, views, [_bin_counts(v, 0, 2 * v["spp"]) for v in views])
    for i in range(2):
        r = ref.readback(i).astype(np.float64)
        assert _rel(got[i], r) <= TOL, i


def test_static_rejects_pool_beyond_capacity(gr):
    import torch
    from paper_2303_15762_gb300 import _native as nat
    S = [gr.Scene(sg.grating_scene())]
    v = sg.grating_view(width=8, height=8, spp=4)
    accum = torch.zeros(2 * 8 * 8 * 16, dtype=torch.float32, device="cuda")
    st = _static_render(gr, S, [v], accum, pool_size=1 << 30)
    assert st == nat.GR_E_INVALID
    assert b"static scratch" in nat.lib_handle().gr_last_error()
