"""Integer outputs of the CUDA path are bit-exact with independent CPU
implementations: the Philox4x32-10 stream and the BVH (Morton keys, PLOC
topology and the exact float min/max child boxes)."""
import numpy as np
import pytest

from paper_2303_15762_gb300 import scenegen as sg

pytestmark = pytest.mark.gpu


def test_rng_stream_bit_exact(gr, oracle):
    for seed, view, pixel, sample, seg, call in [(1, 0, 0, 0, 0, 0), (7, 3, 4095, 100, 2, 3),
                                                 (0xDEADBEEF, 63, 2 ** 20, 2 ** 30, 7, 5)]:
        dev = gr.debug_rng(seed, view, pixel, sample, seg, call, 257)
        for i in range(0, 257, 16):
            ref = oracle.philox4x32_10((pixel, sample + i, (seg << 4) | call, 0), (seed, view))
            assert list(dev[i]) == list(ref), (seed, view, pixel, sample + i)


@pytest.mark.parametrize("case", ["one", "two", "three", "grating", "small", "medium", "large"])
def test_bvh_bit_exact(gr, oracle, case):
    if case in ("one", "two", "three"):
        n = {"one": 1, "two": 2, "three": 3}[case]
        rng = np.random.default_rng(n)
        verts = rng.uniform(-1, 1, (n, 3, 3)).astype(np.float32)
        scene = sg._scene(verts, [0] * n, [sg.material(sg.MAT_MIRROR)], np.zeros((0, 8)))
    elif case == "grating":
        scene = sg.grating_scene()
    elif case == "small":
        scene = sg.procedural_scene(seed=5, n_objects=4, target_tris=2100)
    elif case == "medium":
        scene = sg.procedural_scene(seed=6, n_objects=16, target_tris=20000)
    else:
        scene = sg.procedural_scene(seed=2)
    s = gr.Scene(scene)
    k_gpu, c_gpu, b_gpu = s.bvh()
    k_cpu, c_cpu, b_cpu = oracle.lbvh_build(scene["verts"])
    assert np.array_equal(k_gpu, k_cpu)
    assert np.array_equal(c_gpu, c_cpu)
    assert np.array_equal(b_gpu.view(np.uint32), b_cpu.view(np.uint32))
