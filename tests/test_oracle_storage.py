"""Pins of the oracle's reduced-precision storage model: the rounding matches
PyTorch's own bfloat16 / float16 conversions (a library routine) and the
known tie and range cases; the per-ray sample spacing equals the 3-D distance
between consecutive samples computed from the rotated source and pixel
positions; the storage-mode FBS iteration at FP32 storage agrees with the
plain FP64 iteration to FP32 rounding."""
import numpy as np
import pytest


def test_round_storage_matches_torch_conversions(orc):
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(1)
    x = np.concatenate([rng.standard_normal(20000) * 10.0 ** rng.integers(-6, 4, 20000),
                        rng.random(5000) * 0.04, -rng.random(5000)])
    x32 = x.astype(np.float32)
    t = torch.from_numpy(x32)
    np.testing.assert_array_equal(orc.round_storage(x32, "bf16"), t.to(torch.bfloat16).double().numpy())
    np.testing.assert_array_equal(orc.round_storage(x32, "fp16"), t.to(torch.float16).double().numpy())
    np.testing.assert_array_equal(orc.round_storage(x32, "f32"), x32.astype(np.float64))


def test_round_storage_ties_and_range(orc):
    # bfloat16 keeps 8 significant bits: 1 + 2^-8 is a tie and goes to the even 1
    assert orc.round_storage([1 + 2.0 ** -8], "bf16")[0] == 1.0
    assert orc.round_storage([1 + 3 * 2.0 ** -8], "bf16")[0] == 1 + 2.0 ** -6
    assert orc.round_storage([1 + 2.0 ** -8 + 2.0 ** -20], "bf16")[0] == 1 + 2.0 ** -7
    # binary16 keeps 11: 1 + 2^-11 is a tie, 1 + 3 2^-11 rounds up to 1 + 2^-9
    assert orc.round_storage([1 + 2.0 ** -11], "fp16")[0] == 1.0
    assert orc.round_storage([1 + 3 * 2.0 ** -11], "fp16")[0] == 1 + 2.0 ** -9
    assert orc.round_storage([65504.0], "fp16")[0] == 65504.0
    assert np.isinf(orc.round_storage([70000.0], "fp16")[0])
    assert orc.round_storage([3.0e38], "bf16")[0] == pytest.approx(3.0e38, rel=2.0 ** -8)


def test_ray_spacing_is_distance_between_samples(orc):
    g = orc.Geometry(8, 8, 6, 1.5, 1.5, 2.0, 11, 7, 1.2, 1.7, 300.0, 470.0,
                     np.array([0.3, 2.1]), 0.5)
    ds = orc.ray_ds(g)
    drho = orc.drho(g)
    assert drho == pytest.approx(0.5 * 1.5)
    for th in g.angles:
        c, s = np.cos(th), np.sin(th)
        R = np.array([[c, -s, 0], [s, c, 0], [0, 0, 1.0]])
        src = R @ np.array([-g.sad, 0, 0])
        for iv in range(g.nv):
            for iu in range(g.nu):
                u = (iu - 0.5 * (g.nu - 1)) * g.du
                v = (iv - 0.5 * (g.nv - 1)) * g.dv
                pix = R @ np.array([g.sdd - g.sad, -u, v])
                n = pix - src
                step = n / np.hypot(n[0], n[1]) * drho   # consecutive samples, in-plane step drho
                assert ds[iv, iu] == pytest.approx(np.linalg.norm(step), rel=1e-13)


def test_storage_iteration_at_fp32_matches_fp64_iteration(orc):
    rng = np.random.default_rng(2)
    g = orc.Geometry(6, 5, 4, 2.0, 2.0, 2.0, 10, 8, 2.0, 2.0, 300.0, 450.0,
                     np.linspace(0, 2 * np.pi, 5, endpoint=False), 0.5)
    y = rng.random(g.sino_shape) * 5
    f0 = rng.random(g.vol_shape) * 0.1
    tau = 1.0 / orc.power_lipschitz(g, 30)
    p = orc.TVParams(eps_tv=0.01)
    a, b = f0.copy(), f0.copy()
    e_a, st_a, log_a = orc.fbs_iteration(g, y, a, 0.3, tau, p, clamp=True)
    e_b, st_b, log_b = orc.fbs_iteration_storage(g, orc.round_storage(y, "f32"), b, 0.3, tau, p, "f32",
                                                 clamp=True, replay=list(log_a))
    assert e_b == pytest.approx(e_a, rel=1e-6)
    np.testing.assert_allclose(b, a, rtol=0, atol=1e-6 * np.abs(a).max())
    # bfloat16 storage moves the result by about its rounding, not more
    c = f0.copy()
    orc.fbs_iteration_storage(g, orc.round_storage(y, "bf16"), c, 0.3, tau, p, "bf16", clamp=True,
                              replay=list(log_a))
    err = np.linalg.norm(c - a) / np.linalg.norm(a)
    assert 1e-5 < err < 2.0 ** -6
