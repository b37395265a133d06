"""Seeded synthetic scenes and views.

This module only writes input data (triangles, material and light parameters,
camera descriptions); it holds none of the rendering method's arithmetic.  Its
outputs are consumed unchanged by both the CUDA library (through the package
binding) and the FP64 oracle (through ``oracle/oracle.py``).

Stand-ins: the paper's own scenes (snake enclosure, bike, CD) are not available,
so every workload here is synthetic, with the shapes and parameter ranges of the
workloads this project measures:

* ``grating_scene``: one planar sinusoidal grating quad (2 triangles, period
  1.6 um, amplitude 0.1 um -> peak-to-peak height 0.2 um), lit by a spatially
  coherent distant source, seen by a 64x64 pinhole camera, 16 wavelengths
  400-700 nm, 1 interaction, 64 spp.
* ``procedural_scene``: ground plane plus ~64 objects (subdivided icospheres and
  displaced height tiles, ~1.3-1.6k triangles each, ~100k total) with rough
  Gaussian-statistics surfaces (sigma_h 0.05-0.5 um, correlation length
  1-10 um) or gratings (period 0.8-3 um), conductor Fresnel indices, and 1-4
  partially coherent emissive quads (coherence length 5-50 um).
* ``batch_views``: 64 views, each its own procedural scene of 5k-200k
  triangles (log-uniform), side 128-1024 (log-uniform), depth 1-8, 16-64 bins.
* ``serving_request``: grating-style scenes with a random source direction and
  grating period, resolutions from {256^2, 512^2, 1280x720, 1920x1080}.

Layouts: material row float32[16] = (type, fresnel, n_re, n_im, period_um,
height_um, gdir xyz, sigma_h_um, corr_len_um, Le, coh_len_um, 0, 0, 0) with
type 0 absorber, 1 grating, 2 rough, 3 mirror, 4 emitter and fresnel 0 unit /
1 conductor; light row float32[8] = (type, direction toward the source xyz, E,
coh_len_um, 0, 0) with type 0 distant, 1 constant environment.
"""
import math

import numpy as np

MAT_ABSORBER, MAT_GRATING, MAT_ROUGH, MAT_MIRROR, MAT_EMITTER, MAT_DIELECTRIC = 0, 1, 2, 3, 4, 5
LIGHT_DISTANT, LIGHT_ENV = 0, 1


def material(type_, fresnel=0, n_re=1.0, n_im=0.0, period_um=0.0, height_um=0.0,
             gdir=(1.0, 0.0, 0.0), sigma_h_um=0.0, corr_len_um=1.0, Le=0.0, coh_len_um=0.0, cauchy_b_um2=0.0):
    row = np.zeros(16, dtype=np.float32)
    row[0] = type_
    row[1] = fresnel
    row[2] = n_re
    row[3] = n_im
    row[4] = period_um
    row[5] = height_um
    row[6:9] = gdir
    row[9] = sigma_h_um
    row[10] = corr_len_um
    row[11] = Le
    row[12] = coh_len_um
    row[13] = cauchy_b_um2
    return row


def light(type_, direction=(0.0, 0.0, 1.0), E=1.0, coh_len_um=0.0):
    row = np.zeros(8, dtype=np.float32)
    row[0] = type_
    d = np.asarray(direction, dtype=np.float64)
    if type_ == LIGHT_DISTANT:
        d = d / np.linalg.norm(d)
    row[1:4] = d
    row[4] = E
    row[5] = coh_len_um
    return row


def view(eye, look_at, up=(0.0, 1.0, 0.0), vfov_deg=28.0, width=64, height=64, p_pix_um=2.0,
         f_beta=0.5, lambda_min_um=0.4, lambda_max_um=0.7, n_bins=16, n_stokes=1, max_depth=1,
         spp=64, first_sample=0, view_index=0, scene_index=0, ortho=0, ortho_half_m=0.0):
    # float fields are rounded to float32 here: the C ABI carries float32, and
    # both implementations must see identical input values
    f = lambda x: float(np.float32(x))  # noqa: E731
    return dict(eye=tuple(f(x) for x in eye), look_at=tuple(f(x) for x in look_at),
                up=tuple(f(x) for x in up), vfov_deg=f(vfov_deg), width=int(width),
                height=int(height), p_pix_um=f(p_pix_um), f_beta=f(f_beta),
                lambda_min_um=f(lambda_min_um), lambda_max_um=f(lambda_max_um),
                n_bins=int(n_bins), n_stokes=int(n_stokes), max_depth=int(max_depth), spp=int(spp),
                first_sample=int(first_sample), view_index=int(view_index),
                scene_index=int(scene_index), ortho=int(ortho), ortho_half_m=f(ortho_half_m))


def _quad(c, a, b):
    """Two triangles of the parallelogram c +- a +- b (normal along a x b)."""
    c, a, b = (np.asarray(x, dtype=np.float64) for x in (c, a, b))
    p00, p10, p11, p01 = c - a - b, c + a - b, c + a + b, c - a + b
    return np.array([[p00, p10, p11], [p00, p11, p01]], dtype=np.float64)


def _scene(tris, tri_mat, mats, lights):
    return dict(verts=np.ascontiguousarray(np.asarray(tris, dtype=np.float32).reshape(-1, 3, 3)),
                tri_mat=np.ascontiguousarray(np.asarray(tri_mat, dtype=np.int32)),
                mats=np.ascontiguousarray(np.asarray(mats, dtype=np.float32).reshape(-1, 16)),
                lights=np.ascontiguousarray(np.asarray(lights, dtype=np.float32).reshape(-1, 8)))


def _box(center, half, rot_y_deg=0.0):
    """12 triangles of a box, wound counter-clockwise seen from outside (outward
    normals), rotated about the vertical axis through its centre."""
    c = np.asarray(center, dtype=np.float64)
    hx, hy, hz = half
    X, Y, Z = np.array([hx, 0, 0]), np.array([0, hy, 0]), np.array([0, 0, hz])
    faces = [_quad(+Z, X, Y), _quad(-Z, Y, X), _quad(+X, Y, Z), _quad(-X, Z, Y), _quad(+Y, Z, X), _quad(-Y, X, Z)]
    t = math.radians(rot_y_deg)
    R = np.array([[math.cos(t), 0, math.sin(t)], [0, 1, 0], [-math.sin(t), 0, math.cos(t)]])
    return np.concatenate(faces, axis=0) @ R.T + c


# ---------------------------------------------------------------- grating workload
def grating_scene(period_um=1.6, amplitude_um=0.1, source_deg=20.0, source_azimuth_deg=0.0,
                  half_size_m=0.05, coh_len_um=0.0, fresnel=0):
    """Planar sinusoidal grating quad in z=0 (normal +z, grooves along y,
    grating vector +x) under one distant source tilted by source_deg."""
    tris = _quad((0, 0, 0), (half_size_m, 0, 0), (0, half_size_m, 0))
    th, az = math.radians(source_deg), math.radians(source_azimuth_deg)
    mats = [material(MAT_GRATING, fresnel=fresnel, n_re=0.2, n_im=3.0, period_um=period_um,
                     height_um=2.0 * amplitude_um, gdir=(1, 0, 0))]
    lights = [light(LIGHT_DISTANT, (math.sin(th) * math.cos(az), math.sin(th) * math.sin(az),
                                    math.cos(th)), 1.0, coh_len_um)]
    return _scene(tris, [0, 0], mats, lights)


def grating_view(width=64, height=64, spp=64, n_bins=16, first_sample=0, view_index=0, n_stokes=1):
    return view(eye=(0, 0, 0.2), look_at=(0, 0, 0), up=(0, 1, 0), vfov_deg=28.0, width=width,
                height=height, n_bins=n_bins, n_stokes=n_stokes, max_depth=1, spp=spp,
                first_sample=first_sample, view_index=view_index)


# ---------------------------------------------------------------- procedural workload
_ICO_CACHE = {}


def _icosphere(subdiv):
    if subdiv in _ICO_CACHE:
        return _ICO_CACHE[subdiv]
    t = (1.0 + 5 ** 0.5) / 2.0
    v = [(-1, t, 0), (1, t, 0), (-1, -t, 0), (1, -t, 0), (0, -1, t), (0, 1, t), (0, -1, -t),
         (0, 1, -t), (t, 0, -1), (t, 0, 1), (-t, 0, -1), (-t, 0, 1)]
    f = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11), (1, 5, 9), (5, 11, 4),
         (11, 10, 2), (10, 7, 6), (7, 1, 8), (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8), (3, 8, 9),
         (4, 9, 5), (2, 4, 11), (6, 2, 10), (8, 6, 7), (9, 8, 1)]
    verts = [np.array(p, dtype=np.float64) / np.linalg.norm(p) for p in v]
    faces = list(f)
    for _ in range(subdiv):
        mid = {}

        def midpoint(a, b):
            key = (min(a, b), max(a, b))
            if key not in mid:
                m = verts[a] + verts[b]
                verts.append(m / np.linalg.norm(m))
                mid[key] = len(verts) - 1
            return mid[key]

        nf = []
        for a, b, c in faces:
            ab, bc, ca = midpoint(a, b), midpoint(b, c), midpoint(c, a)
            nf += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        faces = nf
    V = np.array(verts)
    F = np.array(faces)
    _ICO_CACHE[subdiv] = (V, F)
    return V, F


def _icosphere_tris(center, radius, subdiv, rng):
    V, F = _icosphere(subdiv)
    bump = 1.0 + 0.04 * rng.standard_normal(len(V))
    P = center + radius * V * bump[:, None]
    return P[F]


def _tile_tris(center, size, n, amp, rng, yaw):
    """Displaced height tile: n x n quads over a square of side `size`."""
    xs = np.linspace(-0.5, 0.5, n + 1) * size
    X, Z = np.meshgrid(xs, xs, indexing="xy")
    ph = rng.uniform(0, 2 * np.pi, 3)
    fr = rng.uniform(2, 6, 3) * (2 * np.pi / size)
    Y = amp * (np.sin(fr[0] * X + ph[0]) * np.cos(fr[1] * Z + ph[1])
               + 0.5 * np.sin(fr[2] * (X + Z) + ph[2])) + amp * 1.6
    c, s = math.cos(yaw), math.sin(yaw)
    P = np.stack([c * X - s * Z, Y, s * X + c * Z], axis=-1) + center
    i = np.arange(n)
    a = P[:-1, :-1][..., None, :]
    b = P[:-1, 1:][..., None, :]
    cc = P[1:, 1:][..., None, :]
    d = P[1:, :-1][..., None, :]
    # winding gives normals along +y for a flat tile
    t1 = np.concatenate([a, cc, b], axis=-2)
    t2 = np.concatenate([a, d, cc], axis=-2)
    del i
    return np.concatenate([t1.reshape(-1, 3, 3), t2.reshape(-1, 3, 3)], axis=0)


def procedural_scene(seed=2, n_objects=64, target_tris=100_000, n_emitters=None, extent_m=2.0):
    """Ground plane + objects (rough or grating conductors) + emissive quads."""
    rng = np.random.default_rng(seed)
    tris, tri_mat, mats = [], [], []

    def new_material(kind):
        n_re, n_im = rng.uniform(0.2, 2.0), rng.uniform(2.0, 5.0)
        if kind == MAT_ROUGH:
            mats.append(material(MAT_ROUGH, fresnel=1, n_re=n_re, n_im=n_im,
                                 sigma_h_um=rng.uniform(0.05, 0.5), corr_len_um=rng.uniform(1.0, 10.0)))
        else:
            g = rng.standard_normal(3)
            g /= np.linalg.norm(g)
            mats.append(material(MAT_GRATING, fresnel=1, n_re=n_re, n_im=n_im,
                                 period_um=rng.uniform(0.8, 3.0), height_um=0.2, gdir=g))
        return len(mats) - 1

    # ground: rough conductor, subdivided so it is not one giant primitive
    gm = new_material(MAT_ROUGH)
    ng = 8
    cell = 2 * extent_m / ng
    for iz in range(ng):
        for ix in range(ng):
            c = (-extent_m + (ix + 0.5) * cell, 0.0, -extent_m + (iz + 0.5) * cell)
            q = _quad(c, (0, 0, cell / 2), (cell / 2, 0, 0))  # normal +y
            tris.append(q)
            tri_mat += [gm, gm]
    per_obj = max(200, (target_tris - 2 * ng * ng) // max(1, n_objects))
    side = int(math.ceil(math.sqrt(n_objects)))
    spacing = 2 * extent_m * 0.8 / side
    for o in range(n_objects):
        gx, gz = o % side, o // side
        center = np.array([-extent_m * 0.8 + (gx + 0.5) * spacing + rng.uniform(-0.1, 0.1) * spacing,
                           0.0,
                           -extent_m * 0.8 + (gz + 0.5) * spacing + rng.uniform(-0.1, 0.1) * spacing])
        kind = MAT_ROUGH if rng.uniform() < 0.5 else MAT_GRATING
        mi = new_material(kind)
        r = spacing * rng.uniform(0.25, 0.4)
        if rng.uniform() < 0.5:
            # icosphere: 20 * 4^s triangles, pick s from the per-object budget
            s = max(1, min(5, int(round(math.log(max(per_obj, 20) / 20.0, 4)))))
            t = _icosphere_tris(center + np.array([0, r * 1.05, 0]), r, s, rng)
        else:
            n = max(2, int(round(math.sqrt(per_obj / 2.0))))
            t = _tile_tris(center, 2 * r, n, 0.15 * r, rng, rng.uniform(0, np.pi))
        tris.append(t)
        tri_mat += [mi] * len(t)
    # emitters: downward-facing quads above the scene
    ne = int(rng.integers(1, 5)) if n_emitters is None else int(n_emitters)
    for e in range(ne):
        mats.append(material(MAT_EMITTER, Le=1.0, coh_len_um=rng.uniform(5.0, 50.0)))
        em = len(mats) - 1
        c = (rng.uniform(-0.6, 0.6) * extent_m, rng.uniform(1.2, 1.8), rng.uniform(-0.6, 0.6) * extent_m)
        hs = rng.uniform(0.15, 0.3)
        q = _quad(c, (hs, 0, 0), (0, 0, hs))  # normal (x cross z) = -y: faces down
        tris.append(q)
        tri_mat += [em, em]
    T = np.concatenate([np.asarray(t).reshape(-1, 3, 3) for t in tris], axis=0)
    return _scene(T, tri_mat, mats, np.zeros((0, 8), dtype=np.float32))


def dielectric_scene(n_re=1.5, cauchy_b_um2=0.0042, slab_half=(0.15, 0.1, 0.01), tilt_deg=25.0, with_ground=True,
                     env=0.0, distant=True, emitter=True):
    """A glass slab (index n_re + cauchy_b_um2 / lambda^2, closed box with
    outward faces) tilted about the vertical axis, above a rough conductor
    ground, lit by a distant source, an emissive quad and optionally a
    constant environment."""
    tris, tri_mat, mats, lights = [], [], [], []
    mats.append(material(MAT_DIELECTRIC, n_re=n_re, cauchy_b_um2=cauchy_b_um2))
    box = _box((0.0, 0.12, 0.0), slab_half, tilt_deg)
    tris.append(box)
    tri_mat += [0] * len(box)
    if with_ground:
        mats.append(material(MAT_ROUGH, fresnel=1, n_re=0.3, n_im=3.5, sigma_h_um=0.15, corr_len_um=4.0))
        g = _quad((0, 0, 0), (0, 0, 0.5), (0.5, 0, 0))  # normal +y
        tris.append(g)
        tri_mat += [len(mats) - 1] * 2
    if emitter:
        mats.append(material(MAT_EMITTER, Le=1.0, coh_len_um=20.0))
        q = _quad((0.05, 0.45, 0.1), (0.08, 0, 0), (0, 0, 0.08))  # normal -y: faces down
        tris.append(q)
        tri_mat += [len(mats) - 1] * 2
    if distant:
        lights.append(light(LIGHT_DISTANT, (0.35, 0.9, 0.25), 1.0, 0.0))
    if env > 0.0:
        lights.append(light(LIGHT_ENV, (0, 0, 1), env, 0.0))
    return _scene(np.concatenate([np.asarray(t).reshape(-1, 3, 3) for t in tris]), tri_mat, mats,
                  np.asarray(lights, dtype=np.float32).reshape(-1, 8))


def add_glass(scene, n_glass=8, seed=12, n_re=1.5, cauchy_b_um2=0.0042, extent_m=2.0, env_radiance=0.0):
    """The scene with n_glass closed glass slabs (dielectric, outward faces,
    random size, height and rotation about the vertical) added among its
    objects; the original triangles, materials and lights are unchanged, and
    with env_radiance > 0 a constant environment of that radiance is added to
    the lights (so that paths refracted through the glass reach a light)."""
    rng = np.random.default_rng(seed)
    mats = np.concatenate([scene["mats"], material(MAT_DIELECTRIC, n_re=n_re, cauchy_b_um2=cauchy_b_um2)[None]])
    gm = len(mats) - 1
    boxes = []
    for _ in range(n_glass):
        half = (rng.uniform(0.08, 0.25), rng.uniform(0.1, 0.3), rng.uniform(0.01, 0.05))
        c = (rng.uniform(-0.7, 0.7) * extent_m, half[1] + rng.uniform(0.0, 0.2), rng.uniform(-0.7, 0.7) * extent_m)
        boxes.append(_box(c, half, rng.uniform(0, 180)))
    verts = np.concatenate([scene["verts"], np.concatenate(boxes).astype(np.float32)])
    tri_mat = np.concatenate([scene["tri_mat"], np.full(12 * n_glass, gm, dtype=np.int32)])
    lights = np.asarray(scene["lights"], np.float32).reshape(-1, 8)
    if env_radiance > 0.0:
        lights = np.concatenate([lights, light(LIGHT_ENV, (0, 0, 1), env_radiance, 0.0)[None]])
    return _scene(verts, tri_mat, mats, lights)


def env_only(scene, env_radiance):
    """The scene's geometry and materials with a constant environment of the
    given radiance added to its lights (the glass workload's reference without
    glass)."""
    lights = np.asarray(scene["lights"], np.float32).reshape(-1, 8)
    lights = np.concatenate([lights, light(LIGHT_ENV, (0, 0, 1), env_radiance, 0.0)[None]])
    return _scene(scene["verts"], scene["tri_mat"], scene["mats"], lights)


def dielectric_view(width=48, height=40, spp=32, n_bins=8, n_stokes=4, max_depth=8, first_sample=0):
    """Camera looking through the tilted slab at the ground."""
    return view(eye=(0.0, 0.22, 0.6), look_at=(0.0, 0.08, 0.0), up=(0, 1, 0), vfov_deg=40.0, width=width,
                height=height, n_bins=n_bins, n_stokes=n_stokes, max_depth=max_depth, spp=spp,
                first_sample=first_sample)


def procedural_view(width=512, height=512, spp=256, n_bins=32, n_stokes=4, max_depth=3,
                    first_sample=0, view_index=0, scene_index=0):
    return view(eye=(0.0, 1.3, 3.2), look_at=(0.0, 0.1, 0.0), up=(0, 1, 0), vfov_deg=45.0,
                width=width, height=height, n_bins=n_bins, n_stokes=n_stokes, max_depth=max_depth,
                spp=spp, first_sample=first_sample, view_index=view_index, scene_index=scene_index)


# ---------------------------------------------------------------- double slit (2D world)
def double_slit_setup(d=400.0, b=40.0, z=1e4, wavelength=1.0, sigma_at_slits=100.0, n_per_slit=400,
                      x0=None, rho_cut=2.5, dkappa=2e-4):
    """Inputs of the double-slit experiment of Sec. 5.1-5.2 in units of the
    wavelength: two slits of width b at +-d/2, screen at z, detector states of
    the pixel-scale width beta whose footprint at the slits has std
    sigma_at_slits (the smaller root of beta^2 + zbar^2/beta^2 = 2 sigma^2),
    Gauss-Legendre samples of the unit aperture field, detector centres, and
    the direction grid (reach around the slits, step dkappa / k)."""
    k = 2 * math.pi / wavelength
    zb = z / k
    s2 = 2 * sigma_at_slits ** 2
    beta = math.sqrt((s2 - math.sqrt(s2 * s2 - 4 * zb * zb)) / 2)
    g, w = np.polynomial.legendre.leggauss(n_per_slit)
    xa = np.concatenate([c + 0.5 * b * g for c in (-d / 2, d / 2)])
    wa = np.concatenate([0.5 * b * w, 0.5 * b * w])
    if x0 is None:
        x0 = np.arange(-600, 601, 100.0)
    return dict(x0=np.asarray(x0, dtype=np.float64), x_ap=xa, w_ap=wa, beta=beta, z=z, k=k,
                reach=d / 2 + b + 8 * 150.0, dtheta=dkappa / k, rho_cut=rho_cut, d=d, b=b)


def aperture_nodes(shape, size, n):
    """Quadrature of a unit field over a plane aperture: nodes [N][2] and
    weights [N].  shape 'rect': size = (a, b) full side lengths, n x n
    Gauss-Legendre nodes; 'disk': size = radius, n Gauss-Legendre radii x 2n
    equally spaced angles."""
    x, w = np.polynomial.legendre.leggauss(n)
    if shape == "rect":
        a, b = size
        X, Y = np.meshgrid(0.5 * a * x, 0.5 * b * x, indexing="ij")
        W = np.outer(0.5 * a * w, 0.5 * b * w)
        return np.stack([X.ravel(), Y.ravel()], axis=1), W.ravel()
    if shape == "disk":
        R = float(size)
        r, wr = 0.5 * R * (x + 1), 0.5 * R * w
        m = 2 * n
        ph = 2 * math.pi * (np.arange(m) + 0.5) / m
        rr, pp = np.meshgrid(r, ph, indexing="ij")
        W = np.outer(wr * r, np.full(m, 2 * math.pi / m))
        return np.stack([(rr * np.cos(pp)).ravel(), (rr * np.sin(pp)).ravel()], axis=1), W.ravel()
    raise ValueError(shape)


def aperture3d_setup(shape="disk", size=12.0, z=2000.0, sigma_ap=30.0, n_nodes=24, rho_cut=2.5, dt=5e-4,
                     x0=None, wavelength=1.0):
    """Inputs of the aperture experiment in a 3D world (the double slit of
    Sec. 5.1-5.2 taken to a plane aperture and a 2D screen), in units of the
    wavelength: a disk of radius `size` (or a square of side `size`) lit at
    normal incidence, the screen at z, detector states of the width beta whose
    footprint at the aperture has spatial std sigma_ap (the smaller root of
    beta^2 + zbar^2 / beta^2 = 2 sigma^2; the footprint width there is then
    beta' = sqrt(2) sigma_ap), the aperture quadrature, the detector centres
    (default: a 48 x 48 screen over +-240) and the direction grid (rays
    landing within +-reach of the aperture centre, reach = the aperture's
    half-diagonal + 1.05 rho_cut beta', one landing step = z dt)."""
    k = 2 * math.pi / wavelength
    zb = z / k
    s2 = 2 * sigma_ap ** 2
    beta = math.sqrt((s2 - math.sqrt(s2 * s2 - 4 * zb * zb)) / 2)
    nodes, w = aperture_nodes(shape, size if shape == "disk" else (size, size), n_nodes)
    half = float(np.max(np.hypot(nodes[:, 0], nodes[:, 1])))
    if x0 is None:
        g = np.linspace(-240.0, 240.0, 48)
        X, Y = np.meshgrid(g, g, indexing="ij")
        x0 = np.stack([X.ravel(), Y.ravel()], axis=1)
    return dict(shape=shape, size=size, x0=np.asarray(x0, np.float64).reshape(-1, 2), x_ap=nodes, w_ap=w,
                beta=beta, beta_ap=math.sqrt(2.0) * sigma_ap, z=z, k=k,
                reach=half + 1.05 * rho_cut * math.sqrt(2.0) * sigma_ap, dt=dt, rho_cut=rho_cut)


# ---------------------------------------------------------------- batched workload
def batch_views(seed=4, n_views=64, spp=16, tris_range=(5_000, 200_000), side_range=(128, 1024)):
    """64 views, each with its own seeded procedural scene; returns (scenes, views)."""
    rng = np.random.default_rng(seed)
    scenes, views = [], []
    for i in range(n_views):
        nt = int(round(math.exp(rng.uniform(math.log(tris_range[0]), math.log(tris_range[1])))))
        side = int(round(math.exp(rng.uniform(math.log(side_range[0]), math.log(side_range[1])))))
        n_obj = int(max(4, min(64, nt // 1500)))
        sc = procedural_scene(seed=1000 + i, n_objects=n_obj, target_tris=nt)
        scenes.append(sc)
        views.append(procedural_view(width=side, height=side, spp=spp,
                                     n_bins=int(rng.choice([16, 32, 48, 64])), n_stokes=1,
                                     max_depth=int(rng.integers(1, 9)), view_index=i, scene_index=i))
    return scenes, views


# ---------------------------------------------------------------- serving workload
SERVING_RESOLUTIONS = ((256, 256), (512, 512), (1280, 720), (1920, 1080))


def serving_request(rng, request_index):
    W, H = SERVING_RESOLUTIONS[int(rng.integers(0, len(SERVING_RESOLUTIONS)))]
    scene = grating_scene(period_um=float(rng.uniform(0.8, 3.0)),
                          source_deg=float(rng.uniform(5.0, 35.0)),
                          source_azimuth_deg=float(rng.uniform(0, 360)))
    v = view(eye=(0, 0, 0.2), look_at=(0, 0, 0), up=(0, 1, 0), vfov_deg=28.0, width=W, height=H,
             n_bins=16, n_stokes=1, max_depth=1, spp=1, first_sample=0, view_index=request_index)
    return scene, v


def env_light(L=1.0):
    """Constant environment of radiance L (white-furnace tests)."""
    return light(LIGHT_ENV, (0, 0, 1), L, 0.0)
