"""GPU parity of the ROF pieces (Sec. II.B, Eq. 5) and of the multigrid /
step-size helpers, against the FP64 oracle, through the C ABI."""
import numpy as np
import pytest

from gpu_util import CASES, TOL_CALL, dev, f32, geometries, host, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import torch
    from paper_1001_0599_gb300 import build, cbct
    build.build()
    cbct.load()
    assert torch.cuda.is_available()
    return cbct


def _pair(og, seed, scale=0.02):
    rng = np.random.default_rng(seed)
    g = f32(scale * rng.random(og.vol_shape))
    f = f32(g + 0.1 * scale * rng.standard_normal(og.vol_shape))
    return f, g


@pytest.mark.parametrize("case", ["small", "odd", "one_slice", "tall", "ragged_tma"])
def test_energy_and_gradient(lib, orc, case):
    import torch
    wl, geom, og = geometries(case)
    f, g = _pair(og, 11)
    lam, tau, eps = 0.05, 3e-3, 1e-3
    d = torch.full(og.vol_shape, float("nan"), device="cuda")
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    ws = lib.workspace(lib.cbct_workspace_size(geom))
    lib.cbct_tv_energy_grad(geom, dev(f), dev(g), lam, tau, eps, d, out, ws)
    dref = orc.rof_gradient(og, f, g, lam, tau, eps)
    assert rel_l2(host(d), dref) < TOL_CALL
    e, d2 = out.cpu().numpy()
    assert e == pytest.approx(orc.rof_energy(og, f, g, lam, tau, eps), rel=1e-6)
    assert d2 == pytest.approx(float(np.mean(dref * dref)), rel=1e-5)


@pytest.mark.parametrize("case", ["small", "odd", "ragged_tma"])
def test_trial_energy(lib, orc, case):
    import torch
    wl, geom, og = geometries(case)
    f, g = _pair(og, 12)
    lam, tau, eps = 0.05, 3e-3, 1e-3
    d = f32(orc.rof_gradient(og, f, g, lam, tau, eps))
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    ws = lib.workspace(lib.cbct_workspace_size(geom))
    s = 0.4 * tau
    lib.cbct_tv_trial(geom, dev(f), dev(d), dev(g), s, lam, tau, eps, out, ws)
    ftrial = f32(f - s * d)
    assert float(out.item()) == pytest.approx(orc.rof_energy(og, ftrial, g, lam, tau, eps), rel=1e-6)


@pytest.mark.parametrize("case", ["small", "odd", "ragged_tma"])
def test_rof_solve_matches_oracle(lib, orc, case):
    import torch
    wl, geom, og = geometries(case)
    rng = np.random.default_rng(13)
    clean = np.zeros(og.vol_shape)
    clean[og.nx // 4: 3 * og.nx // 4, og.ny // 4: 3 * og.ny // 4, :] = 0.02
    g = f32(clean + 0.004 * rng.standard_normal(og.vol_shape))
    lam, tau = 0.2, 0.5
    p = orc.TVParams(eps_tv=1e-3, max_inner=30)
    ref = orc.rof_solve(og, g, lam, tau, p)
    f = dev(g)
    ws = lib.workspace(lib.cbct_workspace_size(geom))
    st = lib.stats_buffer(lib.TvStats)
    tv = lib.TvParams(p.eps_tv, p.c, p.alpha, p.rel_tol, p.max_inner, p.max_backtracks, p.s0)
    lib.cbct_tv_denoise(geom, dev(g), f, lam, tau, tv, ws, st)
    stats = lib.read_stats(st, lib.TvStats)
    assert stats.status == 0
    assert stats.n_inner == ref.n_inner and stats.flags == ref.flags
    assert rel_l2(host(f), ref.f) < TOL_CALL
    assert stats.e_last == pytest.approx(ref.e_last, rel=1e-6)


def test_rof_energy_decreases_and_flags(lib, orc):
    import torch
    wl, geom, og = geometries("small")
    rng = np.random.default_rng(14)
    g = f32(0.02 * rng.random(og.vol_shape))
    ws = lib.workspace(lib.cbct_workspace_size(geom))
    st = lib.stats_buffer(lib.TvStats)
    f = dev(g)
    lib.cbct_tv_denoise(geom, dev(g), f, 0.5, 0.05, lib.TvParams(1e-3, 0.01, 0.6, 0.0, 3, 40, 0.0), ws, st)
    s = lib.read_stats(st, lib.TvStats)
    assert s.n_inner == 3 and s.flags & 2 and s.e_last < s.e_first


def test_prolongation_matches_oracle(lib, orc):
    import torch
    rng = np.random.default_rng(15)
    for shape in ((4, 5, 3), (32, 32, 16), (1, 7, 2)):
        c = f32(rng.random(shape))
        out = torch.empty(tuple(2 * n for n in shape), device="cuda")
        lib.cbct_prolongate(dev(c), out)
        assert rel_l2(host(out), orc.prolong(c)) < 1e-6


@pytest.mark.parametrize("level", [0, 1])
def test_power_iteration_matches_oracle(lib, orc, level):
    import torch
    wl, geom, og = geometries("small")
    ws = lib.workspace(lib.cbct_workspace_size(geom))
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    lib.cbct_power_lipschitz(geom, level, 20, out, ws)
    ref = orc.power_lipschitz(og.coarse(2 ** level) if level else og, 20)
    assert float(out.item()) == pytest.approx(ref, rel=1e-5)


def test_barrier_timeout_is_reported_and_context_survives(lib, orc):
    # failure detection on the GPU without a fault: the ROF kernel's grid
    # barrier is never completed, every block's bounded wait (2 s) expires, the
    # kernel returns and the statistics report CBCT_ERR_TIMEOUT; afterwards the
    # same workspace serves a normal solve that matches the oracle
    import time

    import torch
    wl, geom, og = geometries("small")
    ws = lib.workspace(lib.cbct_workspace_size(geom))
    st = lib.stats_buffer(lib.TvStats)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    lib.cbct_check_barrier_timeout(geom, ws, st)
    torch.cuda.synchronize()
    waited = time.perf_counter() - t0
    assert lib.read_stats(st, lib.TvStats).status == 7   # CBCT_ERR_TIMEOUT
    assert 1.5 < waited < 60.0
    rng = np.random.default_rng(23)
    g = f32(0.02 * rng.random(og.vol_shape))
    p = orc.TVParams(eps_tv=1e-3, max_inner=10)
    ref = orc.rof_solve(og, g, 0.2, 0.5, p)
    f = dev(g)
    st2 = lib.stats_buffer(lib.TvStats)
    tv = lib.TvParams(p.eps_tv, p.c, p.alpha, p.rel_tol, p.max_inner, p.max_backtracks, p.s0)
    lib.cbct_tv_denoise(geom, dev(g), f, 0.2, 0.5, tv, ws, st2)
    s = lib.read_stats(st2, lib.TvStats)
    assert s.status == 0 and s.n_inner == ref.n_inner
    assert rel_l2(host(f), ref.f) < TOL_CALL
