"""Per-quantity precision of the CUDA path against the FP64 oracle: the
grating order weights as stored in FP32 / FP16 / BF16 tables (Eq. K_grating)
and the FP32 footprint update (Eq. K_free_space_propagation), through the
library's inspection calls, which run the same device code as the render."""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

# round-to-nearest bounds of each table type: relative in the normal range,
# absolute below it (FP16 subnormal spacing 2^-24)
ROUND = {"f32": (2.0 ** -24, 1e-45), "f16": (2.0 ** -11, 2.0 ** -25), "bf16": (2.0 ** -8, 1e-38)}


@pytest.mark.parametrize("dtype", ["f32", "f16", "bf16"])
def test_order_weights_within_type_rounding_of_fp64(gr, oracle, dtype):
    rel, ab = ROUND[dtype]
    # the planar-grating workload's 16 bins (h = 0.2 um, 400-700 nm, period
    # 1.6 um), a deep grating near a zero of J0, and a long-period one
    cases = [(0.2, 0.4 + 0.02 * b, int(2 * 1.6 / (0.4 + 0.02 * b)) + 2) for b in range(16)]
    cases += [(0.306, 0.4, 12), (0.5, 0.45, 40), (0.0, 0.55, 5)]
    worst = 0.0
    for h, lam, jmax in cases:
        got = gr.debug_order_table(h, lam, jmax, dtype).astype(np.float64)
        x = math.pi * float(np.float32(h)) / lam
        ref = np.array([oracle.bessel_j(j, x) ** 2 for j in range(jmax + 1)])
        err = np.abs(got - ref)
        bound = rel * (1 + 1e-6) * ref + ab + 1e-15 * ref
        assert np.all(err <= bound), (h, lam, np.max(err - bound))
        worst = max(worst, float(np.max(err / np.maximum(ref, 1e-30))))
    print(dtype, "max relative order-weight error vs FP64:", worst)


def _kw(lam):
    return np.float32(2 * math.pi / lam)


def test_footprint_update_vs_fp64(gr, oracle):
    """One segment from a range of states the paths visit: camera footprints
    (beta0 = 1 um, rho = 0) and the diverged states after metres of travel;
    all terms are positive for rho >= 0, so the FP32 update is accurate to a
    few ulps."""
    rng = np.random.default_rng(3)
    n = 4000
    beta2 = np.exp(rng.uniform(np.log(0.25), np.log(1e12), n)).astype(np.float32)
    rho = np.where(rng.uniform(size=n) < 0.2, 0.0, np.exp(rng.uniform(np.log(1e-3), np.log(1e6), n))).astype(np.float32)
    t = rng.uniform(1e-5, 10.0, n).astype(np.float32)
    lam = rng.uniform(0.4, 0.7, n)
    kw = np.array([_kw(l) for l in lam], dtype=np.float32)
    out = gr.debug_footprint(np.stack([beta2, rho, t, kw], axis=1))
    worst = 0.0
    for i in range(n):
        zbar = float(t[i]) * 1e6 / float(kw[i])
        b2, r = oracle.propagate(float(beta2[i]), float(rho[i]), zbar)
        eb = abs(out[i, 0] - b2) / b2
        er = abs(out[i, 1] - r) / max(abs(r), 1e-30)
        worst = max(worst, eb, er)
        assert eb <= 2e-6 and er <= 2e-6, (i, beta2[i], rho[i], t[i], kw[i], out[i], b2, r)
    print("max relative footprint error vs FP64 (one segment):", worst)


def test_footprint_chain_vs_fp64(gr, oracle):
    """Three segments chained in FP32 as along a path (depth <= 3), against
    the same chain in FP64."""
    rng = np.random.default_rng(4)
    n = 1000
    seg = rng.uniform(0.05, 5.0, (n, 3)).astype(np.float32)
    lam = rng.uniform(0.4, 0.7, n)
    kw = np.array([_kw(l) for l in lam], dtype=np.float32)
    state = np.stack([np.ones(n, np.float32), np.zeros(n, np.float32)], axis=1)
    ref = [(1.0, 0.0)] * n
    for s in range(3):
        state = gr.debug_footprint(np.stack([state[:, 0], state[:, 1], seg[:, s], kw], axis=1))
        ref = [oracle.propagate(b, r, float(seg[i, s]) * 1e6 / float(kw[i])) for i, (b, r) in enumerate(ref)]
    ref = np.array(ref)
    eb = np.abs(state[:, 0] - ref[:, 0]) / ref[:, 0]
    er = np.abs(state[:, 1] - ref[:, 1]) / np.abs(ref[:, 1])
    print("max relative footprint error vs FP64 (three segments):", eb.max(), er.max())
    assert eb.max() <= 5e-6 and er.max() <= 5e-6
