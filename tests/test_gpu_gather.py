"""The gather microbenchmark used as the projector pair's gather roofline:
its trilinear weights form a partition of unity (a constant volume returns
the constant at every sample) and it stays inside the volume on the
smallest grids it accepts."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import torch
    from paper_1001_0599_gb300 import build, cbct
    build.build()
    cbct.load()
    assert torch.cuda.is_available()
    return cbct


@pytest.mark.parametrize("shape", [(2, 2, 2), (17, 9, 33), (64, 64, 32)])
def test_gather_bench_constant_volume(lib, shape):
    import torch
    n_lines, n_samples = 300, 37
    vol = torch.full(shape, 0.25, device="cuda")
    out = torch.full((n_lines * 32,), float("nan"), device="cuda")
    lib.cbct_gather_bench(vol, n_lines, n_samples, out)
    got = out.cpu().numpy()
    assert np.allclose(got, 0.25 * n_samples, rtol=1e-5)


def test_gather_bench_rejects_degenerate(lib):
    import torch
    vol = torch.zeros((1, 4, 4), device="cuda")
    out = torch.empty(32, device="cuda")
    with pytest.raises(lib.CbctError):
        lib.cbct_gather_bench(vol, 1, 1, out)
