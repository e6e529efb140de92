"""Autograd over the CUDA projector pair and the TV functional: central finite
differences on seeded voxels at the 128^3 / 60-view / 256x192 workload, the
oracle's transpose as the backward of P (and P as the backward of P^T), the
oracle's TV gradient, and per-iteration checkpointing of unrolled data steps
of Algorithm A1 against the oracle's reverse recursion."""
import numpy as np
import pytest

from gpu_util import TOL_CALL, dev, f32, geometries, host, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ag():
    import torch
    from paper_1001_0599_gb300 import autograd, build, cbct
    build.build()
    cbct.load()
    assert torch.cuda.is_available()
    return autograd


@pytest.fixture(scope="module")
def c4():
    from paper_1001_0599_gb300 import cbct, synthetic
    wl = synthetic.workload("autograd")
    truth, y = synthetic.make_problem(wl)
    return wl, cbct.geometry_from_workload(wl), f32(truth), f32(y)


def test_central_differences_on_64_voxels(ag, c4):
    # L(f) = 1/2 |P f - y|^2 is quadratic, so its central difference equals the
    # directional derivative exactly; only rays through voxel j change between
    # the two evaluations (the projector is deterministic), so the FP32 rounding
    # of the other rays cancels
    import torch
    wl, g, truth, y = c4
    f = dev(0.8 * truth).requires_grad_(True)
    yd = dev(y).double()

    def loss(v):
        return 0.5 * ((ag.forward_project(g, v).double() - yd) ** 2).sum()

    loss(f).backward()
    grad = host(f.grad)
    rng = np.random.default_rng(9)
    idx = rng.integers(0, f.numel(), 64)
    h = 0.25
    num = []
    with torch.no_grad():
        base = f.detach().clone()
        flat = base.view(-1)
        for j in idx:
            old = float(flat[j])
            flat[j] = old + h
            lp = float(loss(base))
            flat[j] = old - h
            lm = float(loss(base))
            flat[j] = old
            num.append((lp - lm) / (2 * h))
    num = np.array(num)
    got = grad.ravel()[idx]
    assert rel_l2(got, num) < 1e-4
    assert np.max(np.abs(got - num)) < 1e-3 * np.max(np.abs(num))


@pytest.mark.parametrize("case", ["small", "odd"])
def test_backward_of_p_is_oracle_transpose(ag, orc, case):
    import torch
    wl, g, og = geometries(case)
    rng = np.random.default_rng(10)
    f = dev(f32(rng.random(og.vol_shape))).requires_grad_(True)
    w = f32(rng.standard_normal(og.sino_shape))
    p = ag.forward_project(g, f)
    assert rel_l2(host(p), orc.forward_project(og, host(f.detach()))) < TOL_CALL
    (p * dev(w)).sum().backward()
    assert rel_l2(host(f.grad), orc.back_project(og, w)) < TOL_CALL


def test_backward_of_transpose_is_oracle_p(ag, orc):
    wl, g, og = geometries("odd")
    rng = np.random.default_rng(11)
    s = dev(f32(rng.standard_normal(og.sino_shape))).requires_grad_(True)
    v = f32(rng.standard_normal(og.vol_shape))
    (ag.back_project(g, s) * dev(v)).sum().backward()
    assert rel_l2(host(s.grad), orc.forward_project(og, v)) < TOL_CALL


def test_batched_leading_dimensions(ag):
    import torch
    wl, g, og = geometries("small")
    rng = np.random.default_rng(12)
    fb = dev(f32(rng.random((2, 3) + og.vol_shape)))
    pb = ag.forward_project(g, fb)
    assert pb.shape == (2, 3) + og.sino_shape
    single = ag.forward_project(g, fb[1, 2].contiguous())
    assert torch.equal(pb[1, 2], single)
    with pytest.raises(ValueError):
        ag.forward_project(g, fb[..., :-1].contiguous())


def test_tv_energy_and_gradient_match_oracle(ag, orc):
    wl, g, og = geometries("odd")
    rng = np.random.default_rng(13)
    fv = f32(rng.random(og.vol_shape))
    f = dev(fv).requires_grad_(True)
    eps = 1e-3
    e1 = ag.tv_energy(g, f, eps)
    assert float(e1.detach()) == pytest.approx(orc.tv_e1(og, fv, eps), rel=1e-5)
    e1.backward()
    ref = orc.rof_gradient(og, fv, fv, 1.0, 1.0, eps) / fv.size
    assert rel_l2(host(f.grad), ref) < TOL_CALL


def test_unrolled_data_steps_checkpointed_match_oracle_recursion(ag, orc):
    # f_K = M^K f0 + sum_k M^k c y with M = I - t kappa P^T P, c = t kappa P^T;
    # d<w, f_K>/dy = sum_{k<K} t kappa P M^k w (M is symmetric)
    import torch
    wl, g, og = geometries("small")
    rng = np.random.default_rng(14)
    y = f32(rng.random(og.sino_shape))
    f0 = f32(rng.random(og.vol_shape) * 0.01)
    w = f32(rng.standard_normal(og.vol_shape))
    K = 4
    tau = 0.5 / orc.power_lipschitz(og, 30)
    kap = orc.kappa(og)
    assert ag.kappa(g) == pytest.approx(kap, rel=1e-15)
    grads = []
    for ckpt in (True, False):
        yt = dev(y).requires_grad_(True)
        ft = dev(f0).requires_grad_(True)
        fK = ag.unrolled_data_steps(g, yt, ft, tau, K, checkpoint=ckpt)
        (fK * dev(w)).sum().backward()
        grads.append((host(fK.detach()), host(yt.grad), host(ft.grad)))
    # recomputation is deterministic: checkpointing changes nothing
    for a, b in zip(grads[0], grads[1]):
        assert np.array_equal(a, b)
    # oracle forward and reverse recursions
    f = f0.copy()
    for _ in range(K):
        f = f - tau * kap * orc.back_project(og, orc.forward_project(og, f) - y)
    gy = np.zeros(og.sino_shape)
    v = w.copy()
    for _ in range(K):
        gy += tau * kap * orc.forward_project(og, v)
        v = v - tau * kap * orc.back_project(og, orc.forward_project(og, v))
    fK, gyt, gft = grads[0]
    assert rel_l2(fK, f) < 1e-4
    assert rel_l2(gyt, gy) < 1e-4
    assert rel_l2(gft, v) < 1e-4


def test_central_differences_with_tv_term(ag, c4):
    # the 128^3 / 60-view workload's loss: data term plus TV, 1/2 |P f - y|^2 +
    # mu N_vox E1(f) with E1 smoothed by eps = 1e-3; the TV part is not
    # quadratic, so the step is small (truncation O(h^2 / |grad f|^2) ~ 1e-3)
    import torch
    wl, g, truth, y = c4
    rng = np.random.default_rng(15)
    f0 = np.asarray(0.8 * truth + 0.002 * rng.standard_normal(truth.shape), dtype=np.float32)
    f = torch.from_numpy(f0).cuda().requires_grad_(True)
    yd = dev(y).double()
    eps, mu = 1e-3, 50.0
    nvox = f.numel()

    def loss(v):
        return 0.5 * ((ag.forward_project(g, v).double() - yd) ** 2).sum() + mu * nvox * ag.tv_energy(g, v, eps)

    loss(f).backward()
    grad = host(f.grad)
    idx = rng.integers(0, nvox, 64)
    h = 1e-4
    num = []
    with torch.no_grad():
        base = f.detach().clone()
        flat = base.view(-1)
        for j in idx:
            old = float(flat[j])
            up = float(np.float32(old + h))
            dn = float(np.float32(old - h))
            flat[j] = up
            lp = float(loss(base))
            flat[j] = dn
            lm = float(loss(base))
            flat[j] = old
            num.append((lp - lm) / (up - dn))
    num = np.array(num)
    got = grad.ravel()[idx]
    assert rel_l2(got, num) < 5e-3


def test_checkpointed_clamped_steps_save_memory(ag, c4):
    # unrolled A1 data steps with the Step-3 clamp at the 128^3 / 60-view
    # workload: each clamp keeps one volume for the backward pass, so 16
    # iterations hold 16 volumes; checkpointed in segments of 4 they hold the 4
    # segment inputs plus one segment recomputed at a time. The gradients are
    # equal bit for bit (the kernels are deterministic) and the peak memory of
    # forward + backward drops by at least 4 volumes.
    import torch
    wl, g, truth, y = c4
    K = 16
    vol_bytes = 4 * wl.nx * wl.ny * wl.nz
    rng = np.random.default_rng(16)
    w = dev(rng.standard_normal(g.vol_shape))
    yd = dev(y)
    # half the step 1/L, L of kappa P^T P from the library's power iteration
    tau = 0.5 / ag_lipschitz(g)
    runs = {}
    for ckpt in (False, True):
        torch.cuda.synchronize()
        torch.cuda.reset_peak_memory_stats()
        base = torch.cuda.memory_allocated()
        ft = dev(0.5 * truth).requires_grad_(True)
        fK = ag.unrolled_data_steps(g, yd, ft, tau, K, checkpoint=ckpt, clamp=True, segment=4)
        (fK * w).sum().backward()
        torch.cuda.synchronize()
        runs[ckpt] = (host(fK.detach()), host(ft.grad), torch.cuda.max_memory_allocated() - base)
        del ft, fK
    assert np.array_equal(runs[True][0], runs[False][0])
    assert np.array_equal(runs[True][1], runs[False][1])
    print(f"peak memory: {runs[False][2] / 1e6:.1f} MB plain, {runs[True][2] / 1e6:.1f} MB checkpointed")
    assert runs[False][2] - runs[True][2] >= 4 * vol_bytes


def ag_lipschitz(g):
    """L of kappa P^T P by the library's power iteration (20 iterations)."""
    import torch
    from paper_1001_0599_gb300 import cbct
    ws = cbct.workspace(cbct.cbct_workspace_size(g))
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    cbct.cbct_power_lipschitz(g, 0, 20, out, ws)
    return float(out.item())


def test_clamped_unrolled_steps_match_oracle(ag, orc):
    # the clamped chain against the oracle's clamped forward recursion
    wl, g, og = geometries("small")
    rng = np.random.default_rng(17)
    y = f32(rng.random(og.sino_shape))
    f0 = f32(rng.random(og.vol_shape) * 0.01)
    K, tau = 4, 0.5 / orc.power_lipschitz(og, 30)
    fK = ag.unrolled_data_steps(g, dev(y), dev(f0).requires_grad_(True), tau, K, checkpoint=True, clamp=True,
                                segment=2)
    f = f0.copy()
    for _ in range(K):
        f = np.maximum(f - tau * orc.kappa(og) * orc.back_project(og, orc.forward_project(og, f) - y), 0.0)
    assert rel_l2(host(fK.detach()), f) < 1e-4
