"""Pins of the oracle's Algorithm A1 pieces: data-term gradient scale, the
Lipschitz step, the FBS iteration, multigrid prolongation (Sec. II.C.3).

Library pins: with lambda = 0 and no clamp, Algorithm A1 is Landweber's
iteration, which from zero converges to NumPy's least-squares solution; the
power-iteration Lipschitz constant equals the largest eigenvalue of the dense
normal matrix (NumPy eigvalsh).
"""
import numpy as np
import pytest


def tiny(orc):
    return orc.Geometry(3, 3, 3, 4.0, 4.0, 4.0, 6, 6, 4.0, 4.0, 200.0, 320.0,
                        np.linspace(0, 2 * np.pi, 6, endpoint=False), 0.5)


def dense(orc, g):
    n = g.nx * g.ny * g.nz
    A = np.zeros((g.n_views * g.nv * g.nu, n))
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        A[:, j] = orc.forward_project(g, e.reshape(g.vol_shape)).ravel()
    return A


def test_data_term_gradient_scale_is_kappa(orc):
    # N_vox * dE2/df_j = kappa (P^T r)_j with kappa = 2 N_vox / (N_theta N_pix)
    rng = np.random.default_rng(1)
    g = tiny(orc)
    f = rng.random(g.vol_shape)
    y = rng.random(g.sino_shape)
    r = orc.forward_project(g, f) - y
    grad = orc.kappa(g) * orc.back_project(g, r)
    n = f.size
    h = 1e-6
    for j in (0, 5, 13, 26):
        e = np.zeros(n)
        e[j] = h
        e = e.reshape(f.shape)
        num = (orc.data_term(g, f + e, y) - orc.data_term(g, f - e, y)) / (2 * h) * n
        assert grad.ravel()[j] == pytest.approx(num, rel=1e-7)


def test_power_iteration_matches_eigvalsh(orc):
    g = tiny(orc)
    A = dense(orc, g)
    lam_max = np.linalg.eigvalsh(orc.kappa(g) * A.T @ A)[-1]
    assert orc.power_lipschitz(g, 300) == pytest.approx(lam_max, rel=1e-12)
    # 20 iterations (the default schedule) already lands within 1 %
    L20 = orc.power_lipschitz(g, 20)
    assert L20 <= lam_max * (1 + 1e-12) and L20 > 0.99 * lam_max


def test_fbs_lambda_zero_is_landweber_to_lstsq(orc):
    g = tiny(orc)
    A = dense(orc, g)
    rng = np.random.default_rng(2)
    y = rng.random(g.sino_shape)
    x_ls = np.linalg.lstsq(A, y.ravel(), rcond=None)[0]
    tau = 1.0 / orc.power_lipschitz(g, 300)
    f = np.zeros(g.vol_shape)
    p = orc.TVParams()
    for _ in range(3500):
        orc.fbs_iteration(g, y, f, 0.0, tau, p, clamp=False)
    np.testing.assert_allclose(f.ravel(), x_ls, rtol=0, atol=1e-9 * np.abs(x_ls).max())


def test_fbs_iteration_steps(orc):
    # One A1 iteration equals: gradient step, ROF from g, clamp.
    rng = np.random.default_rng(3)
    g = orc.Geometry(6, 5, 4, 2.0, 2.0, 2.0, 10, 8, 2.0, 2.0, 300.0, 450.0,
                     np.linspace(0, 2 * np.pi, 5, endpoint=False), 0.5)
    y = rng.random(g.sino_shape) * 5
    f = rng.random(g.vol_shape) * 0.1
    lam, tau = 0.3, 1.0 / orc.power_lipschitz(g, 30)
    p = orc.TVParams(eps_tv=0.01)
    ref = f.copy()
    e2, st, log = orc.fbs_iteration(g, y, f, lam, tau, p, clamp=True)
    r = orc.forward_project(g, ref) - y
    assert e2 == pytest.approx(np.mean(r * r), rel=1e-13)
    gaux = ref - tau * orc.kappa(g) * orc.back_project(g, r)
    rof = orc.rof_solve(g, gaux, lam, tau, p)
    np.testing.assert_allclose(f, np.maximum(rof.f, 0.0), rtol=0, atol=1e-13)
    assert st.n_inner == rof.n_inner and list(log) == list(rof.log)


def test_fbs_decreases_objective(orc):
    # FBS with tau = 1/L is a descent method on E2 + lambda E1 (without clamp).
    rng = np.random.default_rng(4)
    g = orc.Geometry(8, 8, 6, 2.0, 2.0, 2.0, 12, 10, 2.0, 2.0, 300.0, 450.0,
                     np.linspace(0, 2 * np.pi, 8, endpoint=False), 0.5)
    truth = np.zeros(g.vol_shape)
    truth[2:6, 3:6, 1:5] = 0.05
    y = orc.forward_project(g, truth) + 0.002 * rng.standard_normal(g.sino_shape)
    lam = 1e-4
    p = orc.TVParams(eps_tv=1e-3, max_inner=100)
    tau = 1.0 / orc.power_lipschitz(g, 30)
    f = np.zeros(g.vol_shape)
    obj = []
    for _ in range(15):
        orc.fbs_iteration(g, y, f, lam, tau, p, clamp=False)
        obj.append(orc.data_term(g, f, y) + lam * orc.tv_e1(g, f, p.eps_tv))
    assert all(b <= a * (1 + 1e-12) for a, b in zip(obj, obj[1:]))


def test_prolong_linear_fields_exact_inside(orc):
    ncx, ncy, ncz = 4, 5, 3
    I, J, K = np.meshgrid(np.arange(ncx), np.arange(ncy), np.arange(ncz), indexing="ij")
    coarse = 0.3 + 0.5 * I - 0.25 * J + 0.125 * K
    fine = orc.prolong(coarse)
    i, j, k = np.meshgrid(np.arange(2 * ncx), np.arange(2 * ncy), np.arange(2 * ncz), indexing="ij")
    # fine cell centre in coarse index units
    expect = 0.3 + 0.5 * (i / 2 - 0.25) - 0.25 * (j / 2 - 0.25) + 0.125 * (k / 2 - 0.25)
    inner = (slice(1, 2 * ncx - 1), slice(1, 2 * ncy - 1), slice(1, 2 * ncz - 1))
    np.testing.assert_allclose(fine[inner], expect[inner], rtol=0, atol=1e-14)
    const = orc.prolong(np.full((3, 2, 1), 0.7))
    np.testing.assert_allclose(const, 0.7, rtol=0, atol=1e-15)


def test_reconstruct_multigrid_schedule_and_quality_trend(orc):
    # Table 1 trend only (parity with the paper's numbers is unpinned: its
    # phantom is not available): more views, lower relative error.
    from paper_1001_0599_gb300 import synthetic
    rng = np.random.default_rng(5)
    errs = []
    for nviews in (4, 16):
        wl = synthetic.Workload("t", 16, 16, 8, 4.0, 4.0, 4.0, 32, 16, 3.0, 3.0, nviews,
                                sad=500.0, sdd=750.0)
        body = synthetic.Ellipsoid(np.zeros(3), np.array([24.0, 20.0, 12.0]), 0.0, 0.02)
        inner = synthetic.Ellipsoid(np.array([5.0, -4.0, 2.0]), np.array([8.0, 6.0, 6.0]), 0.4, 0.01)
        truth = synthetic.voxelise([body, inner], 16, 16, 8, 4.0, 4.0, 4.0)
        y = synthetic.exact_sinogram([body, inner], wl)
        g = orc.Geometry.from_workload(wl)
        res = orc.reconstruct(g, y, 1e-5, (10, 20), orc.TVParams(eps_tv=1e-4))
        assert res.f.shape == truth.shape and len(res.iters) == 30 and len(res.taus) == 2
        assert res.iters[0].level == 0 and res.iters[-1].level == 1
        errs.append(np.linalg.norm(res.f - truth) / np.linalg.norm(truth))
    assert errs[1] < errs[0]


def test_warm_started_power_iteration_converges_to_eigvalsh(orc):
    # start vector: prolongation of the coarse grid's dominant eigenvector
    g = orc.Geometry(6, 6, 4, 2.0, 2.0, 2.0, 12, 8, 2.0, 2.0, 200.0, 320.0,
                     np.linspace(0, 2 * np.pi, 5, endpoint=False), 0.5)
    gc = g.coarse(2)
    A = dense(orc, g)
    lam_max = np.linalg.eigvalsh(orc.kappa(g) * A.T @ A)[-1]
    _, vc = orc.power_lipschitz_from(gc, np.ones(gc.vol_shape), 50)
    L_warm, v = orc.power_lipschitz_from(g, orc.prolong(vc), 40)
    assert L_warm == pytest.approx(lam_max, rel=1e-10)
    assert np.linalg.norm(v) == pytest.approx(1.0, rel=1e-12)
    # from ones the same start behaves like the plain routine
    L_cold, _ = orc.power_lipschitz_from(g, np.ones(g.vol_shape), 25)
    assert L_cold == pytest.approx(orc.power_lipschitz(g, 25), rel=1e-14)
    assert L_cold <= lam_max * (1 + 1e-12)


def test_eq6_step_tends_to_matched_step(orc):
    # Step 1 through Eq. 6 (with the voxel volume / (2 du dv) factor) approaches
    # the matched gradient step on a smooth residual: with lambda = 0 and no
    # clamp, one iteration of each moves f by nearly the same amount inside the
    # volume (pins the scale factor and its sign)
    n = 24
    g = orc.Geometry(n, n, 16, 1.0, 1.0, 1.0, 120, 90, 0.5, 0.5, 600.0, 900.0,
                     np.array([0.0, 1.1, 3.7]), 0.5)
    rng = np.random.default_rng(41)
    f0 = 0.02 * rng.random(g.vol_shape)
    uu = (np.arange(g.nu) - 0.5 * (g.nu - 1)) * g.du
    vv = (np.arange(g.nv) - 0.5 * (g.nv - 1)) * g.dv
    T = np.broadcast_to(1.0 + 0.3 * np.cos(uu[None, None, :] / 9.0) * np.exp(-(vv[None, :, None] / 30.0) ** 2),
                        g.sino_shape).copy()
    y = orc.forward_project(g, f0) - T      # residual P f0 - y = T, smooth
    tau = 1.0 / orc.power_lipschitz(g, 20)
    p = orc.TVParams()
    fm, f6 = f0.copy(), f0.copy()
    orc.fbs_iteration(g, y, fm, 0.0, tau, p, clamp=False)
    orc.fbs_iteration_eq6(g, y, f6, 0.0, tau, p, clamp=False)
    inner = (slice(4, n - 4), slice(4, n - 4), slice(3, 13))
    dm, d6 = (fm - f0)[inner], (f6 - f0)[inner]
    assert np.all(dm < 0) and np.all(d6 < 0)       # both descend along -P^T T
    assert np.max(np.abs(d6 - dm) / np.abs(dm)) < 0.03
