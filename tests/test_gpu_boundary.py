"""The C-ABI boundary: caller-owned accumulators (gr_frame_wrap), rejection
of memory that belongs to no device or another one, and the iteration bound
(GR_E_TIMEOUT), all through the C ABI."""
import ctypes

import numpy as np
import pytest

from paper_2303_15762_gb300 import scenegen as sg

pytestmark = pytest.mark.gpu


def _views():
    scenes = [sg.grating_scene(), sg.procedural_scene(seed=9, n_objects=6, target_tris=5000, n_emitters=2)]
    views = [dict(sg.grating_view(width=24, height=20, spp=32), scene_index=0, view_index=0),
             dict(sg.procedural_view(width=33, height=17, spp=8, n_bins=4, n_stokes=4, max_depth=4),
                  scene_index=1, view_index=1)]
    views[0]["n_stokes"] = 4
    return scenes, views


def test_render_into_caller_tensor_equals_library_frame(gr):
    """gr_render writing into a torch tensor (gr_frame_wrap) gives the
    library-owned frame's image bit for bit, and the tensor holds the sums
    and compensations in the documented layout."""
    import torch
    scenes, views = _views()
    S = [gr.Scene(s) for s in scenes]
    own = gr.Frame(views)
    buf = torch.zeros(gr.accum_floats(views), dtype=torch.float32, device="cuda")
    wrapped = gr.Frame(views, accum=buf)
    for first in (0, 1):
        vv = [dict(v, first_sample=first * v["spp"]) for v in views]
        for f in (own, wrapped):
            gr.render(S, vv, f, seed=4, flags=gr.FLAG_NEE | gr.FLAG_RR)
        for i in range(len(views)):
            assert np.array_equal(wrapped.readback(i), own.readback(i)), (first, i)
    # the documented layout: view 0's sums as [bin][y][x][stokes] from offset 0
    v = views[0]
    T = gr.accum_floats(views) // 2
    n0 = v["width"] * v["height"] * v["n_bins"] * v["n_stokes"]
    a = buf.cpu().numpy()
    s = (a[:n0] - a[T:T + n0]).reshape(v["n_bins"], v["height"], v["width"], v["n_stokes"])
    mean = np.transpose(s, (1, 2, 0, 3)) / np.float32(2 * v["spp"] // v["n_bins"])
    np.testing.assert_allclose(mean, own.readback(0), rtol=1e-6, atol=1e-30)
    # reset zeroes the caller's buffer
    wrapped.reset()
    torch.cuda.synchronize()
    assert torch.count_nonzero(buf) == 0
    wrapped.close()
    assert buf.is_cuda and buf.numel() == gr.accum_floats(views)  # still the caller's


def test_wrap_rejects_host_memory(gr):
    from paper_2303_15762_gb300 import _native as nat
    L = nat.lib_handle()
    _, views = _views()
    host = np.zeros(gr.accum_floats(views), dtype=np.float32)
    out = ctypes.c_void_p()
    st = L.gr_frame_wrap(nat.pack_views(views), len(views), ctypes.c_void_p(host.ctypes.data), nat.current_stream(),
                         ctypes.byref(out))
    assert st == nat.GR_E_INVALID and not out.value
    assert b"device memory" in L.gr_last_error()


@pytest.mark.parametrize("use_graph", [False, True])
def test_iteration_bound_returns_timeout_and_frame_recovers(gr, use_graph):
    """A render cut off by its iteration bound returns GR_E_TIMEOUT with a
    message (the device loop or the host loop stops; nothing faults); after
    gr_frame_reset the same frame renders the image a fresh frame gives."""
    from paper_2303_15762_gb300 import _native as nat
    scenes, views = _views()
    S = [gr.Scene(s) for s in scenes]
    f = gr.Frame(views)
    with pytest.raises(nat.GrError) as exc:
        gr.render(S, views, f, seed=2, flags=gr.FLAG_NEE, use_graph=use_graph, max_iterations=2)
    assert exc.value.status == nat.GR_E_TIMEOUT
    assert "iteration bound" in str(exc.value)
    f.reset()
    gr.render(S, views, f, seed=2, flags=gr.FLAG_NEE, use_graph=use_graph)
    fresh = gr.Frame(views)
    gr.render(S, views, fresh, seed=2, flags=gr.FLAG_NEE, use_graph=use_graph)
    for i in range(len(views)):
        assert np.array_equal(f.readback(i), fresh.readback(i)), i


def test_size_queries_match_what_a_render_holds(gr):
    """gr_render_scratch_bytes predicts the scratch a render keeps in its
    frame, and gr_frame_bytes / gr_scene_bytes report the allocations: the
    accumulators (library-owned only), the counters and that scratch."""
    scenes, views = _views()
    S = [gr.Scene(s) for s in scenes]
    opts = dict(seed=1, flags=gr.FLAG_NEE, pool_size=4096)
    predicted = gr.render_scratch_bytes(S, views, **opts)
    own = gr.Frame(views)
    before = own.device_bytes()
    assert before >= 4 * gr.accum_floats(views)
    gr.render(S, views, own, **opts)
    assert own.device_bytes() - before == predicted
    import torch
    buf = torch.zeros(gr.accum_floats(views), dtype=torch.float32, device="cuda")
    wrapped = gr.Frame(views, accum=buf)
    assert wrapped.device_bytes() == before - 4 * gr.accum_floats(views)  # counters only
    for sc, s in zip(scenes, S):
        n = len(sc["tri_mat"])
        assert 0 < s.device_bytes() < 400 * n + (1 << 16)


def test_pool_beyond_the_largest_is_rejected(gr):
    """Pools above 2^30 - 256 slots are refused before any launch (the trace
    launch tags next-event entries with bit 30 of the slot index)."""
    from paper_2303_15762_gb300 import _native as nat
    scenes, views = _views()
    S = [gr.Scene(s) for s in scenes]
    f = gr.Frame(views)
    with pytest.raises(nat.GrError) as exc:
        gr.render(S, views, f, seed=2, flags=gr.FLAG_NEE, pool_size=(1 << 30) - 255)
    assert exc.value.status == nat.GR_E_INVALID
    assert "bad pool size" in str(exc.value)
