"""torch.autograd.Function over the C ABI (replaces the paper's PyTorch
autograd of the multislice chain, Sec. 3-4, with the hand-written adjoint).

forward:  vol (complex64 [ns][nz][ny], delta + i beta) -> I (float32 [nw][nz][ny])
backward: dL/dI -> g_Psi = 2 dL/dI Psi (kernel) -> mslice_adjoint -> dL/ddelta + i dL/dbeta

The complex gradient returned for ``vol`` is dL/dRe(vol) + i dL/dIm(vol),
which is torch's convention for a real loss of a complex leaf.  PyTorch only
supplies memory and the stream; all arithmetic runs in libmslice.
"""
from __future__ import annotations

import torch

from . import binding as B


class MultisliceIntensity(torch.autograd.Function):
    @staticmethod
    def forward(ctx, vol, params, probe=None):
        if vol.dtype != torch.complex64 or not vol.is_cuda:
            raise TypeError("vol must be a complex64 CUDA tensor")
        vol = vol.contiguous()
        p = params
        shape = (p.nw, p.nz, p.ny)
        ws = B.workspace(p, B.MSLICE_OP_FORWARD, vol.device)
        inten = torch.empty(shape, dtype=torch.float32, device=vol.device)
        psi = torch.empty(shape, dtype=torch.complex64, device=vol.device)
        B.mslice_forward(p, vol, probe, inten, psi, ws)
        ctx.params = p
        ctx.save_for_backward(vol, psi, probe if probe is not None else torch.empty(0))
        ctx.has_probe = probe is not None
        return inten

    @staticmethod
    def backward(ctx, grad_inten):
        vol, psi, probe = ctx.saved_tensors
        probe = probe if ctx.has_probe else None
        p = ctx.params
        g_psi = torch.empty_like(psi)
        B.mslice_intensity_vjp(psi, grad_inten.contiguous().to(torch.float32), g_psi)
        ws = B.workspace(p, B.MSLICE_OP_ADJOINT, vol.device)
        grad = torch.empty_like(vol)
        B.mslice_adjoint(p, vol, probe, g_psi, grad, ws)
        return grad, None, None


def multislice_intensity(vol, params, probe=None):
    """Detector intensity of the multislice model, differentiable in ``vol``."""
    return MultisliceIntensity.apply(vol, params, probe)
