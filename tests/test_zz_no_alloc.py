"""cbct_residual_static: the residual entry point for callers that may not
allocate device memory. Its partial sums live in a fixed array inside the
library instead of a caller workspace; its results must equal
cbct_residual's, call after call (the array keeps the previous call's
contents, which must not leak into the next result).

Kept in its own file, collected last, so a run that stops at the first
failure has already run every other test."""
import numpy as np
import pytest

from gpu_util import TOL_CALL, dev, f32, host, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import torch
    from paper_1001_0599_gb300 import build, cbct
    build.build()
    cbct.load()
    assert torch.cuda.is_available()
    return cbct


def test_static_residual_matches_workspace_version_twice(lib):
    import torch
    from paper_1001_0599_gb300 import synthetic
    wl = synthetic.workload("small")
    g = lib.geometry_from_workload(wl)
    ws = lib.workspace(lib.cbct_workspace_size(g))
    rng = np.random.default_rng(21)
    for call in range(2):
        f = f32(rng.random(g.vol_shape) * 0.02 * (call + 1))
        y = f32(rng.random(g.sino_shape) * (call + 1))
        r_ref = torch.empty(g.sino_shape, device="cuda")
        s_ref = torch.zeros(1, dtype=torch.float64, device="cuda")
        lib.cbct_residual(g, dev(f), dev(y), r_ref, s_ref, ws)
        r = torch.full(g.sino_shape, float("nan"), device="cuda")
        s = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
        lib.cbct_residual_static(g, dev(f), dev(y), r, s)
        torch.cuda.synchronize()
        assert rel_l2(host(r), host(r_ref)) < TOL_CALL
        assert float(s.item()) == pytest.approx(float(s_ref.item()), rel=TOL_CALL)


def test_static_residual_rejects_oversized_geometry(lib):
    import torch
    # n_views * nu = 300 * 1024 exceeds the fixed array of partial sums
    g = lib.cbct_geometry_create(8, 8, 8, 1.0, 1.0, 1.0, 1024, 4, 0.2, 1.0, 300.0, 450.0,
                                 np.linspace(0, 2 * np.pi, 300, endpoint=False))
    vol = torch.zeros(g.vol_shape, device="cuda")
    y = torch.zeros(g.sino_shape, device="cuda")
    r = torch.empty(g.sino_shape, device="cuda")
    s = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(lib.CbctError) as err:
        lib.cbct_residual_static(g, vol, y, r, s)
    assert err.value.status == 6
    assert "CBCT_STATIC_MAX_PARTIALS" in str(err.value)


def _tall_detector_geometry(lib, n_views):
    # 1100 detector rows: the warp-per-column projector, one row per lane
    # (its rows' z span, 32 * 2.27 slices, exceeds the 64-slice segment for
    # two), so the forward launch has n_views * ceil(8/8) * ceil(1100/32)
    # = 35 n_views blocks, one partial sum each
    return lib.cbct_geometry_create(8, 8, 8, 1.0, 1.0, 0.3, 8, 1100, 1.0, 1.0, 300.0, 450.0,
                                    np.linspace(0, 2 * np.pi, n_views, endpoint=False))


def test_static_residual_on_the_warp_per_column_projector(lib):
    import torch
    g = _tall_detector_geometry(lib, 6)
    ws = lib.workspace(lib.cbct_workspace_size(g))
    rng = np.random.default_rng(22)
    f = f32(rng.random(g.vol_shape))
    y = f32(rng.random(g.sino_shape))
    r_ref = torch.empty(g.sino_shape, device="cuda")
    s_ref = torch.zeros(1, dtype=torch.float64, device="cuda")
    lib.cbct_residual(g, dev(f), dev(y), r_ref, s_ref, ws)
    r = torch.full(g.sino_shape, float("nan"), device="cuda")
    s = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    lib.cbct_residual_static(g, dev(f), dev(y), r, s)
    assert rel_l2(host(r), host(r_ref)) < TOL_CALL
    assert float(s.item()) == pytest.approx(float(s_ref.item()), rel=TOL_CALL)


def test_static_residual_limit_counts_forward_blocks(lib):
    import torch
    limit = 262144
    # 35 * 7489 = 262115 blocks fit; 35 * 7490 = 262150 do not, although
    # n_views * nu (59920) is far below the limit
    for n_views, fits in ((7489, True), (7490, False)):
        g = _tall_detector_geometry(lib, n_views)
        assert (35 * n_views <= limit) == fits
        vol = torch.zeros(g.vol_shape, device="cuda")
        y = torch.zeros(g.sino_shape, device="cuda")
        r = torch.empty(g.sino_shape, device="cuda")
        s = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
        if fits:
            lib.cbct_residual_static(g, vol, y, r, s)
            assert float(s.item()) == 0.0
        else:
            with pytest.raises(lib.CbctError) as err:
                lib.cbct_residual_static(g, vol, y, r, s)
            assert err.value.status == 6
        del vol, y, r
