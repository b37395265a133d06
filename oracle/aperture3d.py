"""Generalized rays through a plane aperture in a 3D world, and the exact
scalar-wave reference -- the double-slit validation of Sec. 5.1-5.2, taken
from a 1D aperture in a 2D world to a 2D aperture (rectangle or disk) and a 2D
screen of detector elements.

TEST INFRASTRUCTURE ONLY (used by tests/ and bench.py): plain numpy FP64.
Inputs (aperture quadrature nodes and weights, detector centres, the
experiment's parameters) come from the seeded input generator
(scenegen.aperture_nodes, scenegen.aperture3d_setup).

Units: lengths in wavelengths (lambda = 1 unless given), k = 2 pi / lambda.
The aperture lies in the plane z = 0 and is lit by a unit plane wave at normal
incidence; the screen is the plane at distance z.

* Exact forward field (Rayleigh-Sommerfeld diffraction integral of the first
  kind):  U(x) = (1 / 2 pi) int_ap U_ap(x') (z / r^2) (1 / r - i k) e^{i k r} d^2x',
  r = |x - x'| with x on the screen.
* A detector element at x0 is a distribution of coherent states of width beta
  over all directions (Eq. wdf_coherent_states); it measures
  I(x0) = int |U(x)|^2 (pi beta^2)^-1 exp(-|x - x0|^2 / beta^2) d^2x.
* Backward generalized rays: the state of direction s (tangent-plane
  coordinates t = (s_x, s_y) / s_z, s_z = (1 + |t|^2)^-1/2) is propagated back
  over the oblique length z / s_z in closed form (Eq. K_free_space_propagation
  from rho = 0: beta'^2 = beta^2 + zbar^2 / beta^2, rho' = zbar / beta^2, zbar
  = length / k).  It meets the aperture plane at x_c = x0 - z t with transverse
  wavevector kappa = k s_z t.  Its field on the plane at offset d = x' - x_c is
  (pi beta'^2)^-1/2 s_z^1/2 exp(i kappa . d) exp(-(1 + i rho') |P d|^2 / (2 beta'^2)),
  where |P d|^2 = |d|^2 - s_z^2 (t . d)^2 is the squared distance from the ray
  measured across it (the oblique projection), and it is truncated at
  |P d| <= rho_cut beta' (Sec. 6).  I(x0) = int d^2kappa / (2 pi)^2 |A|^2 with
  A = <U_ap, psi>, and d^2kappa = k^2 s_z^4 d^2t on the tangent-plane grid.
"""
import math

import numpy as np
from scipy import special


def rs_field(xs, z, k, nodes, weights, chunk=2048):
    """Exact Rayleigh-Sommerfeld (first kind) field at screen points xs [M][2]."""
    xs = np.asarray(xs, np.float64).reshape(-1, 2)
    U = np.zeros(len(xs), complex)
    for i0 in range(0, len(xs), chunk):
        x = xs[i0:i0 + chunk]
        dx = x[:, None, 0] - nodes[None, :, 0]
        dy = x[:, None, 1] - nodes[None, :, 1]
        r = np.sqrt(dx * dx + dy * dy + z * z)
        kern = (z / (r * r)) * (1.0 / r - 1j * k) * np.exp(1j * k * r) / (2 * math.pi)
        U[i0:i0 + chunk] = kern @ weights
    return U


def on_axis_disk(z, k, radius):
    """Closed form of the first-kind Rayleigh-Sommerfeld integral on the axis
    of a uniformly lit disk: e^{ikz} - (z / R) e^{ikR}, R = sqrt(z^2 + a^2)
    (the integrand is the r-derivative of -z e^{ikr} / r)."""
    R = math.sqrt(z * z + radius * radius)
    return np.exp(1j * k * z) - (z / R) * np.exp(1j * k * R)


def fraunhofer_rect(xs, z, k, a, b):
    """Far-field intensity of an a x b rectangle: (k z / (2 pi r^2))^2 (a b)^2
    sinc^2(k a x / 2r) sinc^2(k b y / 2r), sinc(u) = sin(u) / u."""
    xs = np.asarray(xs, np.float64).reshape(-1, 2)
    r = np.sqrt(xs[:, 0] ** 2 + xs[:, 1] ** 2 + z * z)
    sx = np.sinc(k * a * xs[:, 0] / (2 * r) / math.pi)
    sy = np.sinc(k * b * xs[:, 1] / (2 * r) / math.pi)
    return (k * z / (2 * math.pi * r * r)) ** 2 * (a * b * sx * sy) ** 2


def fraunhofer_disk(xs, z, k, radius):
    """Far-field intensity of a disk (Airy pattern):
    (k z / (2 pi r^2))^2 (pi a^2)^2 [2 J1(v) / v]^2, v = k a rho / r."""
    xs = np.asarray(xs, np.float64).reshape(-1, 2)
    r = np.sqrt(xs[:, 0] ** 2 + xs[:, 1] ** 2 + z * z)
    v = k * radius * np.hypot(xs[:, 0], xs[:, 1]) / r
    airy = np.where(v > 1e-12, 2 * special.j1(np.maximum(v, 1e-12)) / np.maximum(v, 1e-12), 1.0)
    return (k * z / (2 * math.pi * r * r)) ** 2 * (math.pi * radius * radius * airy) ** 2


def screen_beta(sigma_ap, z, k):
    """The smaller root of beta^2 + zbar^2 / beta^2 = 2 sigma^2 (zbar = z / k):
    the screen-side width whose state spreads to std sigma at the aperture."""
    zb = z / k
    s = 2 * sigma_ap ** 2
    return math.sqrt((s - math.sqrt(s * s - 4 * zb * zb)) / 2)


def forward_exact(x0s, z, k, nodes, weights, beta, step=0.5, margin=4.5):
    """Detector elements by the exact field: |U|^2 weighted by the coherent
    state density over a screen grid of +-margin beta around each element."""
    out = []
    g = np.arange(-margin * beta, margin * beta + 0.5 * step, step)
    GX, GY = np.meshgrid(g, g, indexing="ij")
    dens = np.exp(-(GX ** 2 + GY ** 2) / beta ** 2) / (math.pi * beta ** 2)
    for x0 in np.asarray(x0s, np.float64).reshape(-1, 2):
        pts = np.stack([(x0[0] + GX).ravel(), (x0[1] + GY).ravel()], axis=1)
        U = rs_field(pts, z, k, nodes, weights)
        out.append(float(np.sum(np.abs(U) ** 2 * dens.ravel()) * step * step))
    return np.array(out)


def direction_grid(x0, z, reach, dt):
    """Tangent-plane directions t whose rays land within +-reach of the
    aperture centre along each axis: t = (x0 - x_c) / z on a grid of step dt
    (n = ceil(2 reach / (z dt)) per axis, first landing point x0 + reach)."""
    n = int(math.ceil(2 * reach / (z * dt)))
    i = np.arange(n)
    tx = (x0[0] - reach) / z + i * dt
    ty = (x0[1] - reach) / z + i * dt
    return tx, ty


def backward_generalized_rays(x0s, z, k, nodes, weights, beta, reach, dt, rho_cut=2.5, chunk=4096):
    """Detector elements by backward generalized rays (module docstring):
    sum over the tangent-plane direction grid of |A|^2 (pi beta'^2)^-1 s_z
    k^2 s_z^4 dt^2 / (2 pi)^2, the overlap A truncated at rho_cut beta'."""
    out = []
    for x0 in np.asarray(x0s, np.float64).reshape(-1, 2):
        tx, ty = direction_grid(x0, z, reach, dt)
        TX, TY = np.meshgrid(tx, ty, indexing="ij")
        TX, TY = TX.ravel(), TY.ravel()
        acc = 0.0
        for i0 in range(0, len(TX), chunk):
            t1, t2 = TX[i0:i0 + chunk, None], TY[i0:i0 + chunk, None]
            sz = 1.0 / np.sqrt(1.0 + t1 * t1 + t2 * t2)
            zb = (z / sz) / k
            b2 = beta * beta + zb * zb / (beta * beta)
            rho = zb / (beta * beta)
            cx, cy = x0[0] - z * t1, x0[1] - z * t2
            dx, dy = nodes[None, :, 0] - cx, nodes[None, :, 1] - cy
            td = t1 * dx + t2 * dy
            p2 = dx * dx + dy * dy - sz * sz * td * td
            kx, ky = k * sz * t1, k * sz * t2
            psi = np.exp(1j * (kx * dx + ky * dy)) * np.exp(-(1 + 1j * rho) * p2 / (2 * b2))
            psi = np.where(p2 <= (rho_cut * rho_cut) * b2, psi, 0.0)
            A = psi @ weights
            amp2 = sz[:, 0] / (math.pi * b2[:, 0])
            acc += float(np.sum(np.abs(A) ** 2 * amp2 * (k * k * sz[:, 0] ** 4 * dt * dt)))
        out.append(acc / (2 * math.pi) ** 2)
    return np.array(out)
