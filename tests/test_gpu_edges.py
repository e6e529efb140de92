"""Degenerate cases of Algorithm A1 on the GPU: lambda = 0 without the clamp
is Landweber's iteration (the ROF step returns g), a zero sinogram keeps the
zero start exactly, and multigrid on a grid that does not halve is refused."""
import numpy as np
import pytest

from gpu_util import CASES, TOL_RECON, dev, f32, geometries, host, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import torch
    from paper_1001_0599_gb300 import build, cbct
    build.build()
    cbct.load()
    assert torch.cuda.is_available()
    return cbct


def _recon(lib, g, y, params, init=None):
    import torch
    ws = lib.workspace(lib.cbct_workspace_size(g, params))
    st = lib.stats_buffer()
    vol = torch.zeros(g.vol_shape, device="cuda") if init is None else dev(init)
    lib.cbct_reconstruct(g, dev(y), vol, params, ws, st)
    return host(vol), lib.read_stats(st)


def test_lambda_zero_without_clamp_is_landweber(lib, orc):
    wl, g, og = geometries("odd")
    rng = np.random.default_rng(21)
    y = f32(orc.forward_project(og, rng.random(og.vol_shape) * 0.05) + 0.01 * rng.standard_normal(og.sino_shape))
    tau = 1.0 / orc.power_lipschitz(og, 30)
    params = lib.make_recon_params(0.0, (6,), lib.TvParams.paper(), taus=[tau], clamp=False)
    got, st = _recon(lib, g, y, params)
    assert st.status == 0
    f = np.zeros(og.vol_shape)
    for _ in range(6):
        f = f - tau * orc.kappa(og) * orc.back_project(og, orc.forward_project(og, f) - y)
    assert rel_l2(got, f) < TOL_RECON
    assert np.abs(got).max() > 0.0


def test_zero_sinogram_keeps_zero(lib):
    for case in ("small", "odd"):
        wl, g, og = geometries(case)
        params = lib.make_recon_params(0.05, (3,), lib.TvParams.paper(), power_iters=10)
        got, st = _recon(lib, g, np.zeros(og.sino_shape), params)
        assert st.status == 0
        assert np.all(got == 0.0)


def test_multigrid_on_grid_that_does_not_halve_is_refused(lib):
    wl, g, og = geometries("odd")   # 13 x 11 x 9
    params = lib.make_recon_params(0.05, (2, 2), lib.TvParams.paper())
    with pytest.raises(lib.CbctError) as e:
        _recon(lib, g, np.zeros(og.sino_shape), params)
    assert e.value.status == 6   # CBCT_ERR_UNSUPPORTED
