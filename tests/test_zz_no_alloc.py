"""gr_render_static: rendering for callers that may not allocate device memory
while they render (a service that reserves all of its GPU memory up front, or
code where an allocation would synchronise the device or fail under memory
pressure).  The entry point runs the wavefront kernels on scratch compiled into
the library and writes caller-owned accumulators.

Both entry points run the same kernels and a frame element's samples are
summed by one slot in sample order, so the caller's sum and compensation
planes must equal, bit for bit, those of gr_render writing into a wrapped
caller buffer (gr_frame_wrap) -- for two calls in a row, with 4 Stokes
components, and with a pool so small that every view straddles many slot
refills.

Kept in a file collected last so that a run stopping at its first failure has
already run every other test; it also passes on its own in a fresh process."""
import ctypes

import numpy as np
import pytest

from paper_2303_15762_gb300 import scenegen as sg

pytestmark = pytest.mark.gpu


def _static_render(scenes, views, accum_ptr, **opts):
    from paper_2303_15762_gb300 import _native as nat
    L = nat.lib_handle()
    sc = (ctypes.c_void_p * len(scenes))(*[s.handle.value for s in scenes])
    arr = nat.pack_views(views)
    o = nat.make_opts(**opts)
    return L.gr_render_static(sc, len(scenes), arr, len(views), ctypes.byref(o), ctypes.c_void_p(accum_ptr),
                              nat.current_stream())


def _last_error():
    from paper_2303_15762_gb300 import _native as nat
    return nat.lib_handle().gr_last_error()


def _scenes_views(n_stokes):
    scenes = [sg.grating_scene(), sg.procedural_scene(seed=7, n_objects=8, target_tris=8000, n_emitters=2)]
    v0 = dict(sg.grating_view(width=32, height=24, spp=16), scene_index=0, view_index=0)
    v1 = dict(sg.procedural_view(width=40, height=40, spp=8, n_bins=4, n_stokes=n_stokes), scene_index=1,
              view_index=1)
    if n_stokes == 4:
        v0 = dict(v0, n_stokes=4)
    return scenes, [v0, v1]


@pytest.mark.parametrize("n_stokes,pool", [(1, 0), (4, 0), (1, 512)])
def test_static_equals_render_bit_for_bit_two_calls_in_a_row(gr, n_stokes, pool):
    import torch
    scenes, views = _scenes_views(n_stokes)
    S = [gr.Scene(s) for s in scenes]
    n = gr.accum_floats(views)
    mine = torch.zeros(n, dtype=torch.float32, device="cuda")
    ref_buf = torch.zeros(n, dtype=torch.float32, device="cuda")
    ref = gr.Frame(views, accum=ref_buf)
    flags = gr.FLAG_NEE | gr.FLAG_RR
    # first call: a fresh image; second call: the next sample range added into
    # the same buffers (the static scratch still holds the first call's state)
    for first in (0, 1):
        vv = [dict(v, first_sample=first * v["spp"]) for v in views]
        gr.render(S, vv, ref, seed=11, flags=flags, pool_size=pool)
        assert _static_render(S, vv, mine.data_ptr(), seed=11, flags=flags, pool_size=pool) == 0, _last_error()
        torch.cuda.synchronize()
        assert torch.count_nonzero(mine[: n // 2]) > 0
        assert torch.equal(mine, ref_buf), "call %d: sums or compensations differ" % first


def test_static_rejects_pool_beyond_capacity(gr):
    import torch
    from paper_2303_15762_gb300 import _native as nat
    S = [gr.Scene(sg.grating_scene())]
    v = sg.grating_view(width=8, height=8, spp=4)
    accum = torch.zeros(2 * 8 * 8 * 16, dtype=torch.float32, device="cuda")
    assert _static_render(S, [v], accum.data_ptr(), pool_size=1 << 24) == nat.GR_E_INVALID
    assert b"static scratch" in _last_error()
    # beyond the largest pool of any render
    assert _static_render(S, [v], accum.data_ptr(), pool_size=1 << 30) == nat.GR_E_INVALID
    assert b"bad pool size" in _last_error()
    assert _static_render(S, [v], accum.data_ptr(), regen_threshold_pct=101) == nat.GR_E_INVALID
    assert b"regen_threshold_pct" in _last_error()


def test_static_rejects_host_accumulators(gr):
    """A host pointer would be dereferenced by the kernels: rejected before
    any launch."""
    from paper_2303_15762_gb300 import _native as nat
    S = [gr.Scene(sg.grating_scene())]
    v = sg.grating_view(width=8, height=8, spp=4)
    host = np.zeros(2 * 8 * 8 * 16, dtype=np.float32)
    assert _static_render(S, [v], host.ctypes.data) == nat.GR_E_INVALID
    assert b"device memory" in _last_error()
    assert not host.any()


def test_static_descriptor_limit_is_a_clean_rejection(gr):
    """Descriptors (views and grating order tables) that leave fewer than 256
    path slots are rejected with GR_E_INVALID naming the static scratch, also
    in the window where they fit but the slot arrays' alignment padding does
    not.  Table rows grow the descriptors in steps of about 25 KB, tiny extra
    views in steps below 1 KB, so walking up to the limit crosses it in steps
    smaller than that window."""
    import torch
    from paper_2303_15762_gb300 import _native as nat
    gmat = [sg.material(sg.MAT_GRATING, period_um=100.0, height_um=0.2, gdir=(1.0, 0.0, 0.0))] * 128
    big = sg.grating_scene()
    big = dict(big, mats=np.asarray(gmat, np.float32).reshape(-1, 16), tri_mat=np.zeros_like(big["tri_mat"]))
    small = sg.grating_scene()
    small = dict(small, mats=np.asarray([sg.material(sg.MAT_MIRROR)], np.float32).reshape(-1, 16),
                 tri_mat=np.zeros_like(small["tri_mat"]))
    S = [gr.Scene(big), gr.Scene(small)]
    tiny = dict(sg.grating_view(width=1, height=1, spp=0, n_bins=1), scene_index=1)
    accum = torch.zeros(1 << 16, dtype=torch.float32, device="cuda")

    def call(nb, k):
        views = [dict(sg.grating_view(width=1, height=1, spp=0, n_bins=nb), scene_index=0)] + [tiny] * k
        st = _static_render(S, views, accum.data_ptr())
        assert st in (nat.GR_OK, nat.GR_E_INVALID), (nb, k, st, _last_error())
        if st == nat.GR_E_INVALID:
            assert b"static scratch" in _last_error(), _last_error()
        return st == nat.GR_OK

    # largest bin count that fits without extra views (bisection)
    lo, hi = 1, 4096
    assert call(lo, 0) and not call(hi, 0)
    while hi - lo > 1:
        mid = (lo + hi) // 2
        if call(mid, 0):
            lo = mid
        else:
            hi = mid
    # then tiny views, one at a time, until the limit is crossed
    k = 0
    while call(lo, k + 1):
        k += 1
        assert k < 200
    torch.cuda.synchronize()
