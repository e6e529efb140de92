"""Host-side checks of the autograd wrappers (no GPU needed): argument
validation happens before any library call."""
import types

import pytest


def _fake_geometry(wl):
    desc = types.SimpleNamespace(nx=wl.nx, ny=wl.ny, nz=wl.nz, nu=wl.nu, nv=wl.nv, n_views=wl.n_views)
    return types.SimpleNamespace(desc=desc, vol_shape=(wl.nx, wl.ny, wl.nz), sino_shape=(wl.n_views, wl.nv, wl.nu))


def test_inputs_must_be_cuda_float32_with_geometry_shape():
    torch = pytest.importorskip("torch")
    from paper_1001_0599_gb300 import autograd, synthetic
    wl = synthetic.workload("small")
    g = _fake_geometry(wl)
    with pytest.raises(TypeError):
        autograd.forward_project(g, torch.zeros(g.vol_shape))
    with pytest.raises(TypeError):
        autograd.back_project(g, torch.zeros(g.sino_shape, dtype=torch.float64))
    assert autograd.kappa(g) == pytest.approx(2.0 * wl.nx * wl.ny * wl.nz / (wl.n_views * wl.nv * wl.nu))
