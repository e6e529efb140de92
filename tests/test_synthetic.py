"""Checks of the seeded input generator (exact chords, noise model, seeds)."""
import math

import numpy as np

from paper_1001_0599_gb300 import synthetic


def test_ball_chord_closed_form():
    wl = synthetic.Workload("b", 8, 8, 8, 1.0, 1.0, 1.0, 9, 7, 2.0, 2.0, 3)
    r = 30.0
    ball = [synthetic.Ellipsoid(np.zeros(3), np.array([r, r, r]), 0.0, 1.0)]
    p = synthetic.exact_sinogram(ball, wl)
    src, det = synthetic.ray_endpoints(wl)
    for k in range(3):
        for iv in range(7):
            for iu in range(9):
                S, P = src[k], det[k, iv, iu]
                n = (P - S) / np.linalg.norm(P - S)
                d = np.linalg.norm(np.cross(S, n))       # distance of the line from the centre
                expect = 2 * math.sqrt(max(r * r - d * d, 0.0))
                assert abs(p[k, iv, iu] - expect) < 1e-9


def test_rotated_ellipsoid_volume():
    e = synthetic.Ellipsoid(np.array([1.0, -2.0, 0.5]), np.array([9.0, 5.0, 4.0]), 0.7, 1.0)
    vol = synthetic.voxelise([e], 32, 32, 24, 1.0, 1.0, 1.0, ss=4)
    assert abs(vol.sum() - 4 / 3 * math.pi * 9 * 5 * 4) / (4 / 3 * math.pi * 180) < 0.01


def test_poisson_log_noise_unbiased_and_seeded():
    p = np.full((200, 200), 1.5)
    y1 = synthetic.poisson_log_sinogram(p, 1e5, 3)
    y2 = synthetic.poisson_log_sinogram(p, 1e5, 3)
    np.testing.assert_array_equal(y1, y2)
    sigma = 1.0 / math.sqrt(1e5 * math.exp(-1.5))
    assert abs(y1.mean() - 1.5) < 5 * sigma / 200
    assert abs(y1.std() / sigma - 1.0) < 0.05


def test_workloads_and_phantoms_deterministic():
    for name in ("small", "paper"):
        wl = synthetic.workload(name)
        a = synthetic.make_phantom(wl)
        b = synthetic.make_phantom(wl)
        assert len(a) == len(b) == 11
        for ea, eb in zip(a, b):
            np.testing.assert_array_equal(ea.centre, eb.centre)
    wl = synthetic.workload("paper")
    assert (wl.nx, wl.ny, wl.nz, wl.nu, wl.nv, wl.n_views) == (256, 256, 128, 512, 384, 40)
    assert tuple(wl.iters) == (40, 30, 30)
