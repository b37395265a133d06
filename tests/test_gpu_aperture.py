"""Footprint-resolved generalized rays through an aperture on the GPU (the
double-slit validation of Sec. 5.1-5.2 with the accurate propagation of
Sec. 6) against the oracle's FP64 computation of the same sums, and against
exact 2D Rayleigh-Sommerfeld diffraction."""
import numpy as np
import pytest

from paper_2303_15762_gb300 import scenegen as sg

pytestmark = pytest.mark.gpu


def _run(gr, s, rho_cut=None):
    out, ms = gr.aperture_backward_2d(s["x0"], s["x_ap"], s["w_ap"], s["beta"], s["z"], s["k"], s["reach"],
                                      s["dtheta"], s["rho_cut"] if rho_cut is None else rho_cut)
    return out


@pytest.mark.parametrize("d", [100.0, 400.0])
@pytest.mark.parametrize("rho_cut", [2.5, 1e9])
def test_matches_oracle_sums(gr, d, rho_cut):
    from oracle import doubleslit as ds
    s = sg.double_slit_setup(d=d)
    got = _run(gr, s, rho_cut)
    ref = ds.backward_generalized_rays(s["x0"], d, s["beta"], rho_cut=rho_cut)
    err = np.max(np.abs(got - ref)) / np.max(ref)
    print("d", d, "rho_cut", rho_cut, "max error / peak", err)
    assert err < 2e-5


@pytest.mark.parametrize("d", [100.0, 400.0])
def test_truncated_rays_reproduce_exact_diffraction(gr, d):
    from oracle import doubleslit as ds
    s = sg.double_slit_setup(d=d)
    got = _run(gr, s)
    exact = ds.forward_exact(s["x0"], d, s["beta"])
    assert np.max(np.abs(got - exact)) / np.max(exact) < 1e-2


def test_deterministic_and_symmetric(gr):
    s = sg.double_slit_setup(d=200.0, x0=np.linspace(-800, 800, 33))
    a = _run(gr, s)
    b = _run(gr, s)
    assert np.array_equal(a, b)
    # the slits are symmetric about 0: so is the pattern (to FP32 sums)
    assert np.max(np.abs(a - a[::-1])) / np.max(a) < 1e-5
