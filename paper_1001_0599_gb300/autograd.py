"""PyTorch autograd over the cone-beam operators.

The projector P of Eq. 1 (ray-driven trilinear samples) and its matched
transpose P^T are linear maps, so each is the other's backward: the gradient
of a loss through P is P^T applied to the incoming sinogram gradient, and the
gradient through P^T is P applied to the incoming volume gradient. Both run in
the CUDA library through its C ABI (cbct_forward_project and cbct_back_project);
nothing here computes on the host.

The TV functional E1 of Eq. 2 (mean of phi_j = sqrt(eps^2 + |grad f|_j^2),
forward differences, zero boundary on x and y and reflective on z, Sec. II.C.2)
is exposed as a scalar function with its first derivative from
cbct_tv_energy_grad (the ROF energy of Eq. 4 with g = f, so the fidelity term
and its gradient vanish). Its backward is first order only.

unrolled_data_steps chains the data step of Algorithm A1
(g = f - tau kappa P^T (P f - y), Sec. II.C.1) differentiably and keeps only f
per iteration when checkpointing (each iteration's sinograms are recomputed in
the backward pass).
"""
from __future__ import annotations

from . import cbct


def _check_tensor(t, shape, name):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float32:
        raise TypeError(f"{name} must be a float32 CUDA tensor")
    if tuple(t.shape[-3:]) != tuple(shape):
        raise ValueError(f"{name} has trailing shape {tuple(t.shape[-3:])}, expected {tuple(shape)}")


def _apply_batched(op, geom, x, in_shape, out_shape):
    """Apply a single-item C-ABI operator over any leading batch dimensions."""
    import torch
    _check_tensor(x, in_shape, "input")
    lead = tuple(x.shape[:-3])
    xs = x.contiguous().reshape((-1,) + tuple(in_shape))
    out = torch.empty((xs.shape[0],) + tuple(out_shape), device=x.device, dtype=torch.float32)
    with torch.cuda.device(x.device):
        for b in range(xs.shape[0]):
            op(geom, xs[b], out[b])
    return out.reshape(lead + tuple(out_shape))


def _fp(geom, vol):
    return _apply_batched(cbct.cbct_forward_project, geom, vol, geom.vol_shape, geom.sino_shape)


def _bp(geom, sino):
    return _apply_batched(cbct.cbct_back_project, geom, sino, geom.sino_shape, geom.vol_shape)


def _function_classes():
    import torch

    class ForwardProjectFn(torch.autograd.Function):
        @staticmethod
        def forward(ctx, vol, geom):
            ctx.geom = geom
            return _fp(geom, vol)

        @staticmethod
        def backward(ctx, grad_sino):
            return _bp(ctx.geom, grad_sino.float()), None

    class BackProjectFn(torch.autograd.Function):
        @staticmethod
        def forward(ctx, sino, geom):
            ctx.geom = geom
            return _bp(geom, sino)

        @staticmethod
        def backward(ctx, grad_vol):
            return _fp(ctx.geom, grad_vol.float()), None

    class TvEnergyFn(torch.autograd.Function):
        @staticmethod
        def forward(ctx, vol, geom, eps_tv):
            _check_tensor(vol, geom.vol_shape, "vol")
            if vol.dim() != 3:
                raise ValueError("tv_energy takes one volume")
            v = vol.contiguous()
            d = torch.empty_like(v)
            out = torch.zeros(2, dtype=torch.float64, device=v.device)
            ws = cbct.workspace(cbct.cbct_workspace_size(geom), device=v.device)
            # E_ROF with g = f, lambda = 1, tau = 1: the fidelity term is zero,
            # so out[0] = E1 and d = N_vox dE1/df
            cbct.cbct_tv_energy_grad(geom, v, v, 1.0, 1.0, float(eps_tv), d, out, ws)
            ctx.save_for_backward(d)
            ctx.n_vox = v.numel()
            return out[0].clone()

        @staticmethod
        def backward(ctx, grad_e):
            (d,) = ctx.saved_tensors
            return (grad_e.to(torch.float32) / ctx.n_vox) * d, None, None

    return ForwardProjectFn, BackProjectFn, TvEnergyFn


_FNS = None


def _fns():
    global _FNS
    if _FNS is None:
        cbct.load()
        _FNS = _function_classes()
    return _FNS


def forward_project(geom: "cbct.Geometry", vol):
    """Differentiable P (Eq. 1): (..., nx, ny, nz) -> (..., n_views, nv, nu)."""
    return _fns()[0].apply(vol, geom)


def back_project(geom: "cbct.Geometry", sino):
    """Differentiable P^T (the matched transpose): (..., n_views, nv, nu) -> (..., nx, ny, nz)."""
    return _fns()[1].apply(sino, geom)


def tv_energy(geom: "cbct.Geometry", vol, eps_tv: float = 1e-5):
    """Differentiable E1 (mean smoothed isotropic TV of Eq. 2), a float64 scalar."""
    return _fns()[2].apply(vol, geom, eps_tv)


def kappa(geom: "cbct.Geometry") -> float:
    """Scale of the mean-metric data-term gradient: 2 N_vox / (N_theta N_pix)."""
    nx, ny, nz = geom.vol_shape
    nv, nu = geom.desc.nv, geom.desc.nu
    return 2.0 * nx * ny * nz / (geom.desc.n_views * nv * nu)


def unrolled_data_steps(geom: "cbct.Geometry", y, f0, tau: float, n_iter: int, checkpoint: bool = True,
                        clamp: bool = False, segment: int = 1):
    """n_iter differentiable iterations of the data step of Algorithm A1,
    f <- f - tau kappa P^T (P f - y) (Sec. II.C.1), differentiable in f0 and
    y; with clamp=True each step is followed by the nonnegativity projection
    of Step 3 (f <- max(f, 0)).

    The data step alone is linear, so autograd saves no tensor for it; the
    clamp saves its output, one volume per iteration. With checkpoint=True the
    chain is cut into segments of ``segment`` iterations: only each segment's
    input volume is kept, and the backward pass recomputes the segment's
    projections and clamps, so a chain of n iterations holds about
    n / segment volumes instead of n."""
    import torch
    import torch.utils.checkpoint as ckpt

    k = kappa(geom)

    def step(f, y):
        f = f - (tau * k) * back_project(geom, forward_project(geom, f) - y)
        return torch.clamp(f, min=0.0) if clamp else f

    def run(f, y, n):
        for _ in range(n):
            f = step(f, y)
        return f

    f = f0
    seg = max(int(segment), 1)
    done = 0
    while done < n_iter:
        n = min(seg, n_iter - done)
        if checkpoint and (f.requires_grad or y.requires_grad):
            f = ckpt.checkpoint(run, f, y, n, use_reentrant=False)
        else:
            f = run(f, y, n)
        done += n
    return f
