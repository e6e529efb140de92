"""Pins of the oracle's projector P (Eq. 1) and its transpose.

Each test compares the FP64 oracle with something other than itself: exact
values of the trilinear line integral, chord lengths of analytic solids, the
paper's projection coordinates (Eq. A6) and Jacobian (Eq. A7), the paper's
closed-form gradient (Eq. 6) in the continuum limit, SciPy's interpolation,
and the explicit transpose of the dense matrix on a tiny problem.
"""
import math

import numpy as np
import pytest

from paper_1001_0599_gb300 import synthetic


def geom(orc, n=(5, 5, 5), h=(2.0, 1.0, 1.0), det=(15, 11), dd=(1.0, 1.0), angles=(0.0,),
         sad=1000.0, sdd=1500.0, step=0.5):
    return orc.Geometry(n[0], n[1], n[2], h[0], h[1], h[2], det[0], det[1], dd[0], dd[1], sad, sdd,
                        np.array(angles, dtype=np.float64), step)


def test_central_ray_single_voxel_is_voxel_width(orc):
    # Central ray (u = v = 0) through the centre voxel of an odd grid: the
    # samples form a uniform grid of spacing dx/4 along the tent of width dx,
    # so the sum is exactly dx (partition of unity), and dy at 90 degrees.
    g = geom(orc, angles=(0.0, math.pi / 2, math.pi))
    vol = np.zeros(g.vol_shape)
    vol[2, 2, 2] = 1.0
    p = orc.forward_project(g, vol)
    assert p[0, 5, 7] == pytest.approx(2.0, abs=1e-12)
    assert p[1, 5, 7] == pytest.approx(1.0, abs=1e-12)
    assert p[2, 5, 7] == pytest.approx(2.0, abs=1e-12)


def test_central_ray_transverse_tent_weights(orc):
    # even ny: the central ray passes half-way between voxel centres in y,
    # each neighbour takes weight 1/2; a voxel one pitch away takes 0.
    g = geom(orc, n=(5, 4, 5))
    for b, w in ((1, 0.5), (2, 0.5), (0, 0.0), (3, 0.0)):
        vol = np.zeros(g.vol_shape)
        vol[2, b, 2] = 1.0
        assert orc.forward_project(g, vol)[0, 5, 7] == pytest.approx(2.0 * w, abs=1e-12)


def test_constant_volume_central_ray_is_grid_length(orc):
    g = geom(orc, n=(7, 5, 5))
    p = orc.forward_project(g, np.ones(g.vol_shape))
    assert p[0, 5, 7] == pytest.approx(7 * 2.0, abs=1e-12)


def test_tilted_ray_chord_pins_sample_weight(orc):
    # u = 0, v != 0: the ray stays in the x-z plane; through a constant slab
    # its integral is the slab thickness nx*dx stretched by L/L_xy.
    g = geom(orc, n=(9, 5, 41), h=(2.0, 1.0, 1.0), det=(15, 41))
    p = orc.forward_project(g, np.ones(g.vol_shape))
    for iv in (20, 24, 27, 30):
        v = (iv - 20) * 1.0
        expect = 9 * 2.0 * math.sqrt(1.0 + (v / 1500.0) ** 2)
        assert p[0, iv, 7] == pytest.approx(expect, rel=1e-12)


def _ball_problem(h, r=20.0, centre=(3.0, -5.0, 2.0), mu=0.02):
    n = int(round(64 / h))
    wl = synthetic.Workload("ball", n, n, n, h, h, h, 96, 64, 0.9, 0.9, 4, photons=1e5)
    ball = [synthetic.Ellipsoid(np.array(centre), np.array([r, r, r]), 0.0, mu)]
    vol = synthetic.voxelise(ball, n, n, n, h, h, h, ss=6)
    return wl, ball, vol


def test_ball_chords_converge(orc):
    # P of a voxelised ball approaches the exact chord lengths 2 sqrt(r^2 - d^2) mu
    # (computed independently by the input generator), with O(h) error.
    errs = []
    for h in (2.0, 1.0):
        wl, ball, vol = _ball_problem(h)
        g = orc.Geometry.from_workload(wl)
        p = orc.forward_project(g, vol)
        exact = synthetic.exact_sinogram(ball, wl)
        errs.append(np.linalg.norm(p - exact) / np.linalg.norm(exact))
    assert errs[0] < 0.05
    assert errs[1] < 0.6 * errs[0]


def test_ellipsoid_phantom_matches_exact_sinogram(orc):
    wl = synthetic.workload("small")
    ells = synthetic.make_phantom(wl)
    vol = synthetic.voxelise(ells, wl.nx, wl.ny, wl.nz, wl.dx, wl.dy, wl.dz)
    g = orc.Geometry.from_workload(wl)
    sub = orc.Geometry(g.nx, g.ny, g.nz, g.dx, g.dy, g.dz, g.nu, g.nv, g.du, g.dv, g.sad, g.sdd,
                       g.angles[::10].copy(), g.step_ratio)
    p = orc.forward_project(sub, vol)
    wl4 = synthetic.Workload("small4", wl.nx, wl.ny, wl.nz, wl.dx, wl.dy, wl.dz, wl.nu, wl.nv,
                             wl.du, wl.dv, 4)
    exact = synthetic.exact_sinogram(ells, wl4)
    assert np.linalg.norm(p - exact) / np.linalg.norm(exact) < 0.05


@pytest.mark.parametrize("theta", [0.0, math.pi / 2, 2.4])
def test_single_voxel_projects_to_eq_a6_with_eq_a7_mass(orc, theta):
    # A small voxel at V projects around (u*, v*) of Eq. A6; its projection
    # integrated over the detector equals voxel volume x L^3/(L0 l^2) (Eq. A7).
    h = 0.5
    n = 101
    sad, sdd = 1000.0, 1500.0
    g = orc.Geometry(n, n, 41, h, h, h, 300, 120, 0.25, 0.25, sad, sdd, np.array([theta]), 0.25)
    a, b, c = 90, 40, 26
    vol = np.zeros(g.vol_shape)
    vol[a, b, c] = 1.0
    x, y, z = (a - 0.5 * (n - 1)) * h, (b - 0.5 * (n - 1)) * h, (c - 0.5 * (41 - 1)) * h
    # rotate into the frame where the projection runs along +x (Appendix)
    xr = x * math.cos(theta) + y * math.sin(theta)
    yr = -x * math.sin(theta) + y * math.cos(theta)
    xs = -sad
    us = -yr * sdd / (xr - xs)
    vs = z * sdd / (xr - xs)
    l2 = (xr - xs) ** 2 + yr ** 2 + z ** 2
    Ls = math.sqrt(sdd ** 2 + us ** 2 + vs ** 2)
    p = orc.forward_project(g, vol)[0]
    uu = (np.arange(g.nu) - 0.5 * (g.nu - 1)) * g.du
    vv = (np.arange(g.nv) - 0.5 * (g.nv - 1)) * g.dv
    m = p.sum()
    assert m > 0
    uc = float((p.sum(axis=0) * uu).sum() / m)
    vc = float((p.sum(axis=1) * vv).sum() / m)
    assert abs(uc - us) < 0.02
    assert abs(vc - vs) < 0.02
    mass = m * g.du * g.dv
    expect = h ** 3 * Ls ** 3 / (sdd * l2)
    assert mass == pytest.approx(expect, rel=2e-3)


def test_interpolation_matches_scipy_map_coordinates(orc):
    # The value of f at every sample is SciPy's order-1 interpolation with
    # zero padding; summing those samples with the ray weight reproduces P.
    scipy_nd = pytest.importorskip("scipy.ndimage")
    rng = np.random.default_rng(5)
    g = geom(orc, n=(9, 8, 7), h=(1.5, 1.25, 1.0), det=(12, 9), dd=(1.1, 1.3),
             angles=(0.3, 1.9), sad=300.0, sdd=450.0, step=0.5)
    vol = rng.random(g.vol_shape)
    p = orc.forward_project(g, vol)
    drho = 0.5 * 1.25
    for view in range(2):
        th = g.angles[view]
        c, s = math.cos(th), math.sin(th)
        S = np.array([-g.sad * c, -g.sad * s, 0.0])
        for iv, iu in ((0, 0), (4, 6), (8, 11), (3, 2)):
            u = (iu - 0.5 * (g.nu - 1)) * g.du
            v = (iv - 0.5 * (g.nv - 1)) * g.dv
            P = np.array([(g.sdd - g.sad) * c + u * s, (g.sdd - g.sad) * s - u * c, v])
            n = P - S
            lxy = math.hypot(n[0], n[1])
            rho = np.arange(int(g.sad / drho) - 40, int(g.sad / drho) + 40) * drho
            pts = S[None, :] + rho[:, None] * (n / lxy)[None, :]
            idx = np.stack([pts[:, 0] / g.dx + 0.5 * (g.nx - 1),
                            pts[:, 1] / g.dy + 0.5 * (g.ny - 1),
                            pts[:, 2] / g.dz + 0.5 * (g.nz - 1)])
            vals = scipy_nd.map_coordinates(vol, idx, order=1, mode="grid-constant", cval=0.0)
            ds = drho * np.linalg.norm(n) / lxy
            assert p[view, iv, iu] == pytest.approx(ds * vals.sum(), rel=1e-12, abs=1e-12)


def _dense(orc, g):
    nvox = g.nx * g.ny * g.nz
    nray = g.n_views * g.nv * g.nu
    A = np.zeros((nray, nvox))
    for j in range(nvox):
        e = np.zeros(nvox)
        e[j] = 1.0
        A[:, j] = orc.forward_project(g, e.reshape(g.vol_shape)).ravel()
    return A


def test_back_projection_is_dense_transpose(orc):
    g = geom(orc, n=(4, 3, 4), h=(2.0, 2.5, 1.5), det=(7, 6), dd=(2.0, 1.7),
             angles=(0.2, 2.0, 4.1), sad=200.0, sdd=320.0)
    A = _dense(orc, g)
    nray = A.shape[0]
    for i in range(nray):
        e = np.zeros(nray)
        e[i] = 1.0
        row = orc.back_project(g, e.reshape(g.sino_shape)).ravel()
        np.testing.assert_allclose(row, A[i], rtol=1e-13, atol=1e-14)
    assert orc.count_terms(g) >= np.count_nonzero(A)


def test_adjoint_identity(orc):
    rng = np.random.default_rng(11)
    g = geom(orc, n=(12, 10, 9), h=(1.5, 1.5, 2.0), det=(24, 16), dd=(1.2, 1.4),
             angles=tuple(np.linspace(0, 2 * np.pi, 9, endpoint=False)), sad=500.0, sdd=800.0)
    f = rng.standard_normal(g.vol_shape)
    s = rng.standard_normal(g.sino_shape)
    a = float(np.sum(orc.forward_project(g, f) * s))
    b = float(np.sum(f * orc.back_project(g, s)))
    assert abs(a - b) <= 1e-12 * max(abs(a), abs(b))


def test_back_projection_continuum_limit_is_eq6(orc):
    # For a smooth detector function T, the matched transpose tends to
    # (voxel volume / pixel area) * L^3/(L0 l^2) * T(u*, v*) per view, i.e.
    # Eq. 6 without its factor 2 (pins A6 signs and the A7 Jacobian).
    n = 24
    h = 1.0
    g = orc.Geometry(n, n, 16, h, h, h, 120, 90, 0.5, 0.5, 600.0, 900.0,
                     np.array([0.0, 1.1, 3.7]), 0.5)
    uu = (np.arange(g.nu) - 0.5 * (g.nu - 1)) * g.du
    vv = (np.arange(g.nv) - 0.5 * (g.nv - 1)) * g.dv
    T = np.empty(g.sino_shape)
    for k in range(g.n_views):
        T[k] = (1.0 + 0.3 * np.cos(uu[None, :] / 9.0 + k) * np.exp(-(vv[:, None] / 30.0) ** 2)
                + 0.01 * uu[None, :] * (k + 1))
    bp = orc.back_project(g, T)
    e6 = orc.eq6_backproject(g, T)
    scale = h ** 3 / (g.du * g.dv) / 2.0
    inner = (slice(4, n - 4), slice(4, n - 4), slice(3, 13))
    rel = np.abs(bp[inner] - scale * e6[inner]) / np.abs(scale * e6[inner])
    assert rel.max() < 0.02
    assert np.median(rel) < 0.005


def test_count_terms_single_voxel_closed_forms(orc):
    # one 2 mm voxel at the isocentre, one pixel at the detector centre, in-plane
    # sample spacing 1 mm on a lattice that hits the isocentre (SAD = 100 mm):
    # along x (0 degrees) the samples at -1, 0, +1 mm lie inside the voxel's
    # open trilinear support (|x| < 2 mm), each with one non-zero corner (the
    # other corners are outside the one-voxel grid or carry weight 0): 3 terms.
    # Along the diagonal (45 degrees) the samples at in-plane offsets -2..+2 mm
    # reach |x|, |y| = 1.41 mm < 2 mm: 5 terms.
    for theta, expect in ((0.0, 3), (np.pi / 4, 5)):
        g = orc.Geometry(1, 1, 1, 2.0, 2.0, 2.0, 1, 1, 1.0, 1.0, 100.0, 150.0, np.array([theta]), 0.5)
        assert orc.count_terms(g) == expect


def test_forward_rays_equal_full_projection(orc):
    g = orc.Geometry(7, 6, 5, 2.0, 2.0, 2.0, 11, 9, 1.7, 1.9, 200.0, 320.0,
                     np.linspace(0, 2 * np.pi, 4, endpoint=False), 0.5)
    rng = np.random.default_rng(31)
    f = rng.random(g.vol_shape)
    full = orc.forward_project(g, f)
    view, iv, iu = np.meshgrid(np.arange(g.n_views), np.arange(g.nv), np.arange(g.nu), indexing="ij")
    rays = orc.forward_rays(g, f, view.ravel(), iv.ravel(), iu.ravel())
    np.testing.assert_array_equal(rays, full.ravel())
