"""GPU parity of the projector P (Eq. 1), its transpose and the fused residual /
gradient-step epilogues, against the FP64 oracle, through the C ABI."""
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


@pytest.mark.parametrize("case", sorted(CASES))
def test_forward_matches_oracle(lib, orc, case):
    import torch
    wl, g, og = geometries(case)
    f = f32(np.random.default_rng(1).random(og.vol_shape))
    out = torch.full(og.sino_shape, float("nan"), device="cuda")
    lib.cbct_forward_project(g, dev(f), out)
    ref = orc.forward_project(og, f)
    assert rel_l2(host(out), ref) < TOL_CALL


@pytest.mark.parametrize("case", sorted(CASES))
def test_back_projection_matches_oracle(lib, orc, case):
    import torch
    wl, g, og = geometries(case)
    s = f32(np.random.default_rng(2).random(og.sino_shape))
    out = torch.full(og.vol_shape, float("nan"), device="cuda")
    lib.cbct_back_project(g, dev(s), out)
    ref = orc.back_project(og, s)
    got = host(out)
    assert np.all(np.isfinite(got))
    assert rel_l2(got, ref) < TOL_CALL


def test_phantom_projection_matches_oracle(lib, orc):
    import torch
    from paper_1001_0599_gb300 import synthetic
    wl, g, og = geometries("small")
    truth = f32(synthetic.voxelise(synthetic.make_phantom(wl), wl.nx, wl.ny, wl.nz, wl.dx, wl.dy, wl.dz))
    out = torch.empty(og.sino_shape, device="cuda")
    lib.cbct_forward_project(g, dev(truth), out)
    assert rel_l2(host(out), orc.forward_project(og, truth)) < TOL_CALL


@pytest.mark.parametrize("case", ["small", "odd"])
def test_adjoint_identity_on_gpu(lib, case):
    import torch
    wl, g, og = geometries(case)
    rng = np.random.default_rng(3)
    f = f32(rng.standard_normal(og.vol_shape))
    s = f32(rng.standard_normal(og.sino_shape))
    pf = torch.empty(og.sino_shape, device="cuda")
    pts = torch.empty(og.vol_shape, device="cuda")
    lib.cbct_forward_project(g, dev(f), pf)
    lib.cbct_back_project(g, dev(s), pts)
    a = float(np.sum(host(pf) * s))
    b = float(np.sum(f * host(pts)))
    assert abs(a - b) / max(abs(a), abs(b)) < 1e-5


def test_zero_volume_projects_to_zero_and_linearity(lib):
    import torch
    wl, g, og = geometries("odd")
    out = torch.full(og.sino_shape, 7.0, device="cuda")
    lib.cbct_forward_project(g, torch.zeros(og.vol_shape, device="cuda"), out)
    assert float(out.abs().max()) == 0.0
    rng = np.random.default_rng(4)
    a, b = f32(rng.random(og.vol_shape)), f32(rng.random(og.vol_shape))
    pa, pb, pab = (torch.empty(og.sino_shape, device="cuda") for _ in range(3))
    lib.cbct_forward_project(g, dev(a), pa)
    lib.cbct_forward_project(g, dev(b), pb)
    lib.cbct_forward_project(g, dev(f32(a + 2.0 * b)), pab)
    assert rel_l2(host(pab), host(pa) + 2.0 * host(pb)) < 1e-6


def test_residual_and_sum_of_squares(lib, orc):
    import torch
    wl, g, og = geometries("small")
    rng = np.random.default_rng(5)
    f = f32(rng.random(og.vol_shape) * 0.02)
    y = f32(rng.random(og.sino_shape))
    r = torch.empty(og.sino_shape, device="cuda")
    ss = torch.zeros(1, dtype=torch.float64, device="cuda")
    ws = lib.workspace(lib.cbct_workspace_size(g))
    lib.cbct_residual(g, dev(f), dev(y), r, ss, ws)
    ref = orc.forward_project(og, f) - y
    got = host(r)
    assert rel_l2(got, ref) < TOL_CALL
    assert float(ss.item()) == pytest.approx(float(np.sum(ref * ref)), rel=1e-5)
    # the FP64 sum of the FP32 residual itself is exact to reduction order
    assert float(ss.item()) == pytest.approx(float(np.sum(got * got)), rel=1e-9)


def test_gradient_step(lib, orc):
    import torch
    wl, g, og = geometries("odd")
    rng = np.random.default_rng(6)
    r = f32(rng.standard_normal(og.sino_shape))
    f = f32(rng.random(og.vol_shape))
    scale = 0.0123
    out = torch.empty(og.vol_shape, device="cuda")
    lib.cbct_gradient_step(g, dev(r), dev(f), out, scale)
    ref = f - scale * orc.back_project(og, r)
    assert rel_l2(host(out), ref) < TOL_CALL


def _columns_of_p(orc, og, j, views):
    """Non-zero entries of column j of P: rays near the voxel's projection."""
    a, b, c = np.unravel_index(j, og.vol_shape)
    x = (a - 0.5 * (og.nx - 1)) * og.dx
    y = (b - 0.5 * (og.ny - 1)) * og.dy
    z = (c - 0.5 * (og.nz - 1)) * og.dz
    vv, ii, uu = [], [], []
    for k in views:
        th = og.angles[k]
        xr = x * np.cos(th) + y * np.sin(th)
        yr = -x * np.sin(th) + y * np.cos(th)
        us = -yr * og.sdd / (xr + og.sad)
        vs = z * og.sdd / (xr + og.sad)
        iu0 = int(round(us / og.du + 0.5 * (og.nu - 1)))
        iv0 = int(round(vs / og.dv + 0.5 * (og.nv - 1)))
        wu = int(np.ceil(3.0 * og.dx * og.sdd / (og.sad - 200.0) / og.du)) + 2
        wv = int(np.ceil(2.0 * og.dz * og.sdd / (og.sad - 200.0) / og.dv)) + 2
        for iv in range(max(iv0 - wv, 0), min(iv0 + wv, og.nv - 1) + 1):
            for iu in range(max(iu0 - wu, 0), min(iu0 + wu, og.nu - 1) + 1):
                vv.append(k)
                ii.append(iv)
                uu.append(iu)
    vv, ii, uu = (np.array(x, dtype=np.int64) for x in (vv, ii, uu))
    if vv.size == 0:   # the voxel projects outside the detector in every view
        return vv, ii, uu, np.zeros(0)
    e = np.zeros(og.vol_shape)
    e[a, b, c] = 1.0
    w = orc.forward_rays(og, e, vv, ii, uu)
    return vv, ii, uu, w


@pytest.mark.slow
@pytest.mark.parametrize("name", ["paper", "lowdose"])
def test_paper_scale_sampled_parity(lib, orc, name):
    """Full-size workloads (256x256x128, 40 views, 512x384; 256^3, 360 views)
    in the launch configuration of the benchmark: P on 400 sampled rays, P^T on
    sampled voxels through their oracle columns."""
    import torch
    from paper_1001_0599_gb300 import synthetic
    wl = synthetic.workload(name)
    g = lib.geometry_from_workload(wl)
    og = orc.Geometry.from_workload(wl)
    truth = f32(synthetic.voxelise(synthetic.make_phantom(wl), wl.nx, wl.ny, wl.nz, wl.dx, wl.dy, wl.dz))
    p = torch.empty(og.sino_shape, device="cuda")
    lib.cbct_forward_project(g, dev(truth), p)
    ph = host(p)
    rng = np.random.default_rng(7)
    n = 400
    view = rng.integers(0, og.n_views, n)
    iv = rng.integers(0, og.nv, n)
    iu = rng.integers(0, og.nu, n)
    ref = orc.forward_rays(og, truth, view, iv, iu)
    got = ph[view, iv, iu]
    assert rel_l2(got, ref) < TOL_CALL
    # transpose on sampled voxels: (P^T s)_j = <column j of P, s>
    s = f32(rng.random(og.sino_shape))
    bt = torch.empty(og.vol_shape, device="cuda")
    lib.cbct_back_project(g, dev(s), bt)
    bth = host(bt)
    views = list(range(og.n_views))
    got, ref = [], []
    for j in rng.integers(0, og.nx * og.ny * og.nz, 12):
        vv, ii, uu, w = _columns_of_p(orc, og, int(j), views)
        ref.append(float(np.dot(w, s[vv, ii, uu])))
        got.append(bth.ravel()[j])
    assert rel_l2(got, ref) < TOL_CALL


@pytest.mark.parametrize("case", sorted(CASES))
def test_eq6_gradient_matches_oracle(lib, orc, case):
    import torch
    wl, g, og = geometries(case)
    T = f32(np.random.default_rng(8).standard_normal(og.sino_shape))
    out = torch.full(og.vol_shape, float("nan"), device="cuda")
    lib.cbct_eq6_gradient(g, dev(T), out)
    ref = orc.eq6_backproject(og, T)
    got = host(out)
    assert np.all(np.isfinite(got))
    # the kernel carries the detector coordinate in double-float and splits off
    # the integer pixel before rounding the fraction, so the per-call bound is
    # the projector's
    assert rel_l2(got, ref) < TOL_CALL


def test_eq6_tends_to_matched_transpose(lib):
    # on a smooth detector function Eq. 6 approaches the matched transpose
    # scaled by voxel volume / (2 du dv) (the continuum limit of P^T)
    import torch
    from paper_1001_0599_gb300 import synthetic
    wl = synthetic.Workload("fine", 48, 48, 32, 0.5, 0.5, 0.5, 160, 120, 0.4, 0.4, 6, sad=600.0, sdd=900.0)
    g = lib.geometry_from_workload(wl)
    uu = (np.arange(wl.nu) - 0.5 * (wl.nu - 1)) * wl.du
    vv = (np.arange(wl.nv) - 0.5 * (wl.nv - 1)) * wl.dv
    T = np.broadcast_to(1.0 + 0.3 * np.cos(uu[None, None, :] / 9.0) * np.exp(-(vv[None, :, None] / 30.0) ** 2),
                        (wl.n_views, wl.nv, wl.nu))
    a = torch.empty(g.vol_shape, device="cuda")
    b = torch.empty(g.vol_shape, device="cuda")
    lib.cbct_back_project(g, dev(T), a)
    lib.cbct_eq6_gradient(g, dev(T), b)
    scale = wl.dx * wl.dy * wl.dz / (2 * wl.du * wl.dv)
    inner = (slice(6, -6), slice(6, -6), slice(4, -4))
    assert rel_l2(scale * host(b)[inner], host(a)[inner]) < 0.02
