"""Reduced-precision storage (bfloat16 / binary16 volumes and sinograms, FP32
arithmetic): the projector and its transpose against the FP64 oracle applied
to the same rounded inputs, the storage error itself against the plain FP32
path, and Algorithm A1 with stored sinograms against the oracle's storage
model in replay mode."""
import numpy as np
import pytest

from gpu_util import CASES, TOL_CALL, TOL_RECON, dev, f32, geometries, host, rel_l2

pytestmark = pytest.mark.gpu

# significand bits (with the implicit one) and smallest subnormal
BITS = {"bf16": (8, 2.0 ** -133), "fp16": (11, 2.0 ** -24)}


@pytest.fixture(scope="module")
def lib():
    import torch
    from paper_1001_0599_gb300 import build, cbct
    build.build()
    cbct.load()
    assert torch.cuda.is_available()
    return cbct


def _tdtype(storage):
    import torch
    return {"bf16": torch.bfloat16, "fp16": torch.float16}[storage]


def _ulp(x, storage):
    p, tiny = BITS[storage]
    ax = np.maximum(np.abs(x), 1e-300)
    return np.maximum(2.0 ** (np.floor(np.log2(ax)) - (p - 1)), tiny)


def test_convert_matches_torch_rounding(lib):
    import torch
    x = torch.randn(100003, device="cuda") * 3
    for st in ("bf16", "fp16"):
        h = torch.empty(x.shape, dtype=_tdtype(st), device="cuda")
        lib.cbct_convert(x, h)
        assert torch.equal(h, x.to(_tdtype(st)))
        back = torch.empty_like(x)
        lib.cbct_convert(h, back)
        assert torch.equal(back, h.float())


@pytest.mark.parametrize("storage", ["bf16", "fp16"])
@pytest.mark.parametrize("case", sorted(c for c in CASES if c != "very_tall"))
def test_forward_with_storage(lib, orc, case, storage):
    import torch
    wl, g, og = geometries(case)
    f = np.random.default_rng(1).random(og.vol_shape) * 0.05
    fq = orc.round_storage(f, storage)
    vol = torch.from_numpy(f.astype(np.float32)).cuda().to(_tdtype(storage))
    assert np.array_equal(host(vol.float()), fq)
    out = torch.empty(og.sino_shape, dtype=_tdtype(storage), device="cuda")
    lib.cbct_forward_project_ex(g, vol, out)
    got = host(out.float())
    ref = orc.forward_project(og, fq)
    # FP32 accumulation, then one rounding to the storage type: within half an
    # ulp of the stored type plus the FP32 call tolerance
    bound = 0.5 * _ulp(ref, storage) + TOL_CALL * np.abs(ref).max()
    assert np.all(np.abs(got - ref) <= bound)
    # the storage error of the whole call against plain FP32 storage
    full = orc.forward_project(og, f)
    p = BITS[storage][0]
    assert rel_l2(got, full) < 2.0 ** -(p - 1)


def test_forward_storage_unsupported_beyond_1024_rows(lib):
    import torch
    wl, g, og = geometries("very_tall")
    vol = torch.zeros(og.vol_shape, dtype=torch.bfloat16, device="cuda")
    out = torch.empty(og.sino_shape, dtype=torch.bfloat16, device="cuda")
    with pytest.raises(lib.CbctError):
        lib.cbct_forward_project_ex(g, vol, out)


@pytest.mark.parametrize("storage", ["bf16", "fp16"])
@pytest.mark.parametrize("case", sorted(CASES))
def test_transpose_with_storage(lib, orc, case, storage):
    import torch
    wl, g, og = geometries(case)
    # non-negative values as in the FP32 transpose test (no cancellation)
    s = np.random.default_rng(2).random(og.sino_shape)
    sq = orc.round_storage(s, storage)
    sino = torch.from_numpy(s.astype(np.float32)).cuda().to(_tdtype(storage))
    out = torch.full(og.vol_shape, float("nan"), device="cuda")
    lib.cbct_back_project_ex(g, sino, out)
    got = host(out)
    # the stored input is exact in FP64: the transpose itself is FP32-accurate
    assert rel_l2(got, orc.back_project(og, sq)) < TOL_CALL


@pytest.mark.parametrize("storage", ["bf16", "fp16"])
def test_recon_with_storage_replay_parity(lib, orc, storage, record_property):
    import torch
    from paper_1001_0599_gb300 import synthetic
    wl = synthetic.workload("small")
    truth, y = synthetic.make_problem(wl)
    og = orc.Geometry.from_workload(wl)
    y = f32(y)
    p = orc.TVParams(eps_tv=1e-5)
    tau = 1.0 / orc.power_lipschitz(og, 20)
    ref = orc.reconstruct(og, y, wl.lam, (4,), p, taus=[tau], storage=storage)
    plain = orc.reconstruct(og, y, wl.lam, (4,), p, taus=[tau], replay=ref.schedule())
    g = lib.geometry_from_workload(wl)
    tv = lib.TvParams(p.eps_tv, p.c, p.alpha, p.rel_tol, p.max_inner, p.max_backtracks, p.s0)
    params = lib.make_recon_params(wl.lam, (4,), tv, taus=[tau], replay=ref.schedule(), storage=storage)
    ws = lib.workspace(lib.cbct_workspace_size(g, params))
    st = lib.stats_buffer()
    vol = torch.zeros(g.vol_shape, device="cuda")
    lib.cbct_reconstruct(g, dev(y), vol, params, ws, st)
    got = host(vol)
    s = lib.read_stats(st)
    assert s.status == 0
    for k, it in enumerate(ref.iters):
        assert s.iters[k].e2 == pytest.approx(it.e2, rel=1e-5)
    # parity with the oracle's storage model; a stored value may land one ulp
    # apart where FP32 and FP64 arithmetic straddle a rounding boundary
    model_err = rel_l2(got, ref.f)
    assert model_err < 10 * TOL_RECON
    # the storage error of the reconstruction against FP64 arithmetic throughout
    err = rel_l2(got, plain.f)
    assert err < 2.0 ** -(BITS[storage][0] - 1)
    # stated for the record: the GPU result against the FP64 oracle's storage
    # model, and against the FP64 oracle with no reduced storage
    record_property("rel_err_vs_fp64_storage_model", model_err)
    record_property("rel_err_vs_fp64_plain", err)
    print(f"{storage}: GPU vs FP64 oracle storage model {model_err:.3e}, vs FP64 plain {err:.3e}")


def test_multigrid_recon_with_storage_runs_all_levels(lib, orc):
    import torch
    from paper_1001_0599_gb300 import synthetic
    wl = synthetic.Workload("mgs", 32, 32, 16, 4.0, 4.0, 4.0, 64, 48, 1.6, 1.6, 12, photons=5e4,
                            phantom="head_neck", phantom_seed=3, noise_seed=4, lam=0.05, iters=(3, 2, 2))
    truth, y = synthetic.make_problem(wl)
    og = orc.Geometry.from_workload(wl)
    y = f32(y)
    p = orc.TVParams(eps_tv=1e-5)
    ref = orc.reconstruct(og, y, wl.lam, wl.iters, p, storage="fp16")
    g = lib.geometry_from_workload(wl)
    tv = lib.TvParams(p.eps_tv, p.c, p.alpha, p.rel_tol, p.max_inner, p.max_backtracks, p.s0)
    params = lib.make_recon_params(wl.lam, wl.iters, tv, replay=ref.schedule(), storage="fp16")
    ws = lib.workspace(lib.cbct_workspace_size(g, params))
    vol = torch.zeros(g.vol_shape, device="cuda")
    lib.cbct_reconstruct(g, dev(y), vol, params, ws, lib.stats_buffer())
    assert rel_l2(host(vol), ref.f) < 10 * TOL_RECON


@pytest.mark.slow
@pytest.mark.parametrize("storage", ["bf16", "fp16"])
def test_lowdose_sampled_parity_with_storage(lib, orc, storage):
    """Full 360-view 256^3 low-dose workload with stored volume and sinogram:
    P on 300 sampled rays against the oracle's rays through the same rounded
    volume (half an ulp of the stored type plus 1e-5), and the storage error
    against the unrounded volume stated as a bound."""
    import torch
    from paper_1001_0599_gb300 import synthetic
    wl = synthetic.workload("lowdose")
    g = lib.geometry_from_workload(wl)
    og = orc.Geometry.from_workload(wl)
    truth = synthetic.voxelise(synthetic.make_phantom(wl), wl.nx, wl.ny, wl.nz, wl.dx, wl.dy, wl.dz)
    fq = orc.round_storage(truth, storage)
    vol = torch.from_numpy(truth.astype(np.float32)).cuda().to(_tdtype(storage))
    out = torch.empty(og.sino_shape, dtype=_tdtype(storage), device="cuda")
    lib.cbct_forward_project_ex(g, vol, out)
    ph = host(out.float())
    rng = np.random.default_rng(17)
    n = 300
    view, iv, iu = rng.integers(0, og.n_views, n), rng.integers(0, og.nv, n), rng.integers(0, og.nu, n)
    ref = orc.forward_rays(og, fq, view, iv, iu)
    got = ph[view, iv, iu]
    bound = 0.5 * _ulp(ref, storage) + TOL_CALL * np.abs(ref).max()
    assert np.all(np.abs(got - ref) <= bound)
    full = orc.forward_rays(og, truth, view, iv, iu)
    assert rel_l2(got, full) < 2.0 ** -(BITS[storage][0] - 1)
