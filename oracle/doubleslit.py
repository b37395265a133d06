"""Double-slit validation of generalized rays (Sec. 5.1-5.2), in a 2D world.

TEST INFRASTRUCTURE ONLY (used by tests/test_doubleslit.py).

Setup of the paper's experiment: wavelength 1, a plate with two slits of
width b = 40 whose centres are d apart, a screen at z = 10^4; the spatial
standard deviation of a generalized ray at the slits is about 100 (FWHM
about 235).  A coherent plane wave falls normally on the plate.

* Forward, exact: the field on the screen is the Rayleigh-Sommerfeld
  diffraction integral of the first kind with the 2D Green's function,
      U(x) = int_slits (i k z / (2 r)) H1^(1)(k r) dx',  r = sqrt((x - x')^2 + z^2),
  and a detector element at x0 (a distribution of coherent states of width
  beta over all directions, Eq. wdf_coherent_states) measures
      I(x0) = int |U(x)|^2 (pi beta^2)^(-1/2) exp(-(x - x0)^2 / beta^2) dx.
* Backward, generalized rays: each detection state (x0, kappa) is propagated
  back to the plate in closed form (Eq. K_free_space_propagation: beta'^2 =
  beta^2 + zbar^2 / beta^2, rho' = zbar / beta^2, zbar = path length / k;
  the state keeps its tilt kappa and, being propagated against the direction
  of travel, has the wavefront curvature of a beam converging onto the
  screen), truncated at |x' - x_c| > 2.5 beta' (Sec. 6), and overlapped with
  the aperture field; I(x0) = int dkappa/(2 pi) |<U_ap, psi_kappa>|^2.
* The screen-side beta is the root of beta^2 + zbar^2/beta^2 = 2 sigma_slit^2
  with the pixel-scale value (11.29 for sigma_slit = 100).
* Fringe visibility at the screen centre from the exact fields: the
  detection states smooth cos(k d x / z) by exp(-(k d / z)^2 beta^2 / 4),
  which is exp(-d^2 / (8 sigma_slit^2)) in the far field.
"""
import math

import numpy as np
from scipy import special

LAMBDA = 1.0
K = 2 * math.pi / LAMBDA
Z = 1e4
B = 40.0


def screen_beta(sigma_slit=100.0, z=Z, k=K):
    """Smaller root of beta^2 + zbar^2 / beta^2 = 2 sigma^2 (zbar = z / k)."""
    zb = z / k
    s = 2 * sigma_slit ** 2
    disc = s * s - 4 * zb * zb
    return math.sqrt((s - math.sqrt(disc)) / 2)


def _slit_nodes(d, b=B, n=400):
    x, w = np.polynomial.legendre.leggauss(n)
    nodes, weights = [], []
    for c in (-d / 2, d / 2):
        nodes.append(c + 0.5 * b * x)
        weights.append(0.5 * b * w)
    return np.concatenate(nodes), np.concatenate(weights)


def rs_field(xs, d, which=(0, 1), b=B, z=Z, k=K, n=400):
    """Exact 2D Rayleigh-Sommerfeld field on the screen from the chosen slits."""
    xa, wa = _slit_nodes(d, b, n)
    sel = np.zeros(len(xa), bool)
    for s in which:
        sel[s * n:(s + 1) * n] = True
    xa, wa = xa[sel], wa[sel]
    U = np.zeros(len(xs), complex)
    for i0 in range(0, len(xs), 512):
        x = xs[i0:i0 + 512, None]
        r = np.sqrt((x - xa[None, :]) ** 2 + z * z)
        U[i0:i0 + 512] = (1j * k * z / (2 * r) * special.hankel1(1, k * r)) @ wa
    return U


def detect(x0s, xs, intensity, beta):
    """Detector elements: |U|^2 smoothed by the coherent-state density."""
    dx = xs[1] - xs[0]
    out = []
    for x0 in x0s:
        g = np.exp(-((xs - x0) ** 2) / beta ** 2) / math.sqrt(math.pi * beta ** 2)
        out.append(np.sum(intensity * g) * dx)
    return np.array(out)


def forward_exact(x0s, d, beta, step=0.5, margin=8.0):
    xs = np.arange(x0s.min() - margin * beta, x0s.max() + margin * beta + step, step)
    U = rs_field(xs, d)
    return detect(x0s, xs, np.abs(U) ** 2, beta)


def backward_generalized_rays(x0s, d, beta, rho_cut=2.5, b=B, z=Z, k=K, n=400, dkappa=2e-4):
    """Sum over detection states (x0, kappa) propagated back to the plate in
    closed form and truncated at 2.5 beta'."""
    xa, wa = _slit_nodes(d, b, n)
    out = []
    for x0 in x0s:
        # directions whose generalized ray lands within reach of the slits
        reach = d / 2 + b + 8 * 150.0
        t_lo, t_hi = (x0 - reach) / z, (x0 + reach) / z
        th = np.arange(math.atan(t_lo), math.atan(t_hi), dkappa / k)
        kap = k * np.sin(th)
        cos = np.cos(th)
        L = z / cos
        zb = L / k
        b2 = beta ** 2 + zb ** 2 / beta ** 2
        rho = zb / beta ** 2
        xc = x0 - z * np.tan(th)
        u = (xa[None, :] - xc[:, None]) * cos[:, None]
        psi = ((math.pi * b2[:, None]) ** -0.25 * np.sqrt(cos[:, None])
               * np.exp(1j * kap[:, None] * (xa[None, :] - xc[:, None]))
               * np.exp(-(1 + 1j * rho[:, None]) * u ** 2 / (2 * b2[:, None])))
        psi = np.where(np.abs(u) <= rho_cut * np.sqrt(b2)[:, None], psi, 0)
        A = psi @ wa
        dk = k * np.cos(th) * np.gradient(th)
        out.append(np.sum(np.abs(A) ** 2 * dk) / (2 * math.pi))
    return np.array(out)


def visibility_exact(d, beta, step=0.25):
    """Fringe visibility at the screen centre from the exact slit fields."""
    xs = np.arange(-8 * beta, 8 * beta + step, step)
    U1 = rs_field(xs, d, which=(0,))
    U2 = rs_field(xs, d, which=(1,))
    g = np.exp(-xs ** 2 / beta ** 2)
    i1 = np.sum(np.abs(U1) ** 2 * g)
    i2 = np.sum(np.abs(U2) ** 2 * g)
    cross = np.sum(2 * np.real(U1 * np.conj(U2)) * g)
    return cross / (2 * math.sqrt(i1 * i2))


def visibility_predicted(d, beta, z=Z, k=K):
    return math.exp(-((k * d / z) ** 2) * beta ** 2 / 4)
