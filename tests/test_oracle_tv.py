"""Pins of the oracle's TV energy, its gradient and the ROF solver (Sec. II.B).

Closed forms for E1 on constant and ramp volumes fix the discretisation and
the boundary conditions (zero on x and y, reflective on z); central finite
differences fix the gradient against the energy; the lambda = 0 case reduces
the ROF model to a quadratic whose minimiser is g itself; the Armijo rule
(Eq. 5) and the stopping rule are checked on every accepted step.
"""
import json
import math
import os

import numpy as np
import pytest


def g3(orc, n=(5, 4, 6), h=(2.0, 1.5, 1.0)):
    return orc.Geometry(n[0], n[1], n[2], h[0], h[1], h[2], 4, 4, 1.0, 1.0, 1000.0, 1500.0,
                        np.array([0.0]), 0.5)


def test_tv_constant_volume_closed_form(orc):
    # Only the last x face and last y face see a jump (to the zero ghost).
    nx, ny, nz = 5, 4, 6
    dx, dy, dz = 2.0, 1.5, 1.0
    cval, eps = 0.7, 1e-3
    g = g3(orc)
    f = np.full((nx, ny, nz), cval)
    n_inner = (nx - 1) * (ny - 1) * nz
    n_xface = (ny - 1) * nz
    n_yface = (nx - 1) * nz
    n_edge = nz
    expect = (n_inner * eps + n_xface * math.sqrt(eps ** 2 + (cval / dx) ** 2)
              + n_yface * math.sqrt(eps ** 2 + (cval / dy) ** 2)
              + n_edge * math.sqrt(eps ** 2 + (cval / dx) ** 2 + (cval / dy) ** 2)) / (nx * ny * nz)
    assert orc.tv_e1(g, f, eps) == pytest.approx(expect, rel=1e-14)


def test_tv_z_ramp_reflective_top(orc):
    # f = s * c along z, constant in x, y: every slice but the last has
    # |D_z| = s/dz; the last slice has zero z difference (reflective);
    # the x/y boundary faces add their jump to zero.
    nx, ny, nz = 3, 3, 5
    dx, dy, dz = 1.0, 1.0, 2.0
    s, eps = 0.3, 0.0
    g = g3(orc, (nx, ny, nz), (dx, dy, dz))
    f = np.broadcast_to(s * np.arange(nz, dtype=float), (nx, ny, nz)).copy()
    total = 0.0
    for a in range(nx):
        for b in range(ny):
            for c in range(nz):
                Dx = -f[a, b, c] / dx if a == nx - 1 else 0.0
                Dy = -f[a, b, c] / dy if b == ny - 1 else 0.0
                Dz = s / dz if c < nz - 1 else 0.0
                total += math.sqrt(Dx * Dx + Dy * Dy + Dz * Dz)
    assert orc.tv_e1(g, f, eps) == pytest.approx(total / f.size, rel=1e-14)


def test_rof_gradient_matches_central_differences(orc):
    rng = np.random.default_rng(3)
    g = g3(orc)
    f = rng.random(g.vol_shape)
    gg = rng.random(g.vol_shape)
    lam, tau, eps = 0.7, 0.3, 0.05
    d = orc.rof_gradient(g, f, gg, lam, tau, eps)
    n = f.size
    h = 1e-6
    for j in range(0, n, 7):
        e = np.zeros(n)
        e[j] = h
        e = e.reshape(f.shape)
        num = (orc.rof_energy(g, f + e, gg, lam, tau, eps)
               - orc.rof_energy(g, f - e, gg, lam, tau, eps)) / (2 * h) * n
        assert d.ravel()[j] == pytest.approx(num, rel=1e-7, abs=1e-8)


def test_rof_lambda_zero_one_step_to_g(orc):
    # lambda = 0: E_ROF is the quadratic fidelity; the first trial step s0 = tau
    # along d = (f - g)/tau lands exactly on g, and Armijo accepts it.
    rng = np.random.default_rng(4)
    g = g3(orc)
    gg = rng.random(g.vol_shape)
    f0 = rng.random(g.vol_shape)
    r = orc.rof_solve(g, gg, 0.0, 0.25, orc.TVParams(), f0=f0)
    assert r.n_inner == 1
    assert list(r.log) == [0]
    np.testing.assert_allclose(r.f, gg, rtol=0, atol=1e-15)
    # starting at g there is nothing to do
    r2 = orc.rof_solve(g, gg, 0.0, 0.25, orc.TVParams())
    assert r2.n_inner == 0
    np.testing.assert_array_equal(r2.f, gg)


def test_rof_armijo_and_stop_rule(orc):
    rng = np.random.default_rng(5)
    g = g3(orc, (8, 7, 6), (1.0, 1.0, 1.0))
    gg = rng.random(g.vol_shape)
    lam, tau = 0.5, 0.05
    p = orc.TVParams(eps_tv=0.05)
    r = orc.rof_solve(g, gg, lam, tau, p)
    assert r.n_inner >= 2 and r.flags & 1 == 0
    # walk the same path: every accepted step satisfies Eq. 5 and the one
    # before it (if any) did not; the energy decreases monotonically
    f = gg.copy()
    energies = [orc.rof_energy(g, f, gg, lam, tau, p.eps_tv)]
    for i, m in enumerate(r.log):
        d = orc.rof_gradient(g, f, gg, lam, tau, p.eps_tv)
        d2 = float(np.mean(d * d))
        E0 = energies[-1]
        s = tau * p.alpha ** m
        Enew = orc.rof_energy(g, f - s * d, gg, lam, tau, p.eps_tv)
        assert Enew <= E0 - p.c * s * d2
        if m > 0:
            sp = s / p.alpha
            assert orc.rof_energy(g, f - sp * d, gg, lam, tau, p.eps_tv) > E0 - p.c * sp * d2
        f = f - s * d
        energies.append(Enew)
        rel = abs(Enew - E0) / E0
        if i < r.n_inner - 1:
            assert rel >= p.rel_tol
        else:
            assert rel < p.rel_tol or r.flags & 2
    assert all(b < a for a, b in zip(energies, energies[1:]))
    np.testing.assert_allclose(f, r.f, rtol=0, atol=1e-14)
    assert r.e_last == pytest.approx(energies[-1], rel=1e-14)


def test_rof_replay_reproduces_free_run(orc):
    rng = np.random.default_rng(6)
    g = g3(orc, (6, 6, 6), (1.0, 1.0, 1.0))
    gg = rng.random(g.vol_shape)
    p = orc.TVParams(eps_tv=0.05)
    r = orc.rof_solve(g, gg, 0.4, 0.05, p)
    rr = orc.rof_solve(g, gg, 0.4, 0.05, p, replay=list(r.log))
    np.testing.assert_array_equal(r.f, rr.f)


def test_rof_reduces_tv(orc):
    rng = np.random.default_rng(7)
    g = g3(orc, (10, 9, 8), (1.0, 1.0, 1.0))
    clean = np.zeros(g.vol_shape)
    clean[2:7, 2:6, 2:6] = 1.0
    noisy = clean + 0.2 * rng.standard_normal(g.vol_shape)
    r = orc.rof_solve(g, noisy, 0.2, 0.05, orc.TVParams(eps_tv=1e-3, max_inner=200))
    assert r.e_last < r.e_first
    assert orc.tv_e1(g, r.f, 1e-3) < 0.95 * orc.tv_e1(g, noisy, 1e-3)
    assert np.linalg.norm(r.f - clean) < 0.95 * np.linalg.norm(noisy - clean)


def test_paper_constants_golden(orc):
    path = os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")
    with open(path) as fh:
        gold = json.load(fh)
    p = orc.TVParams()
    assert p.c == gold["armijo_c"]["value"]
    assert p.alpha == gold["armijo_alpha"]["value"]
    assert p.rel_tol == gold["rof_rel_tol"]["value"]
