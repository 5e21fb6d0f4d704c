"""Shared helpers of the GPU tests: run the CUDA path through the C ABI binding."""
import numpy as np
import torch

from paper_2212_01253_gb300 import binding as B


def params(geo, checkpoint_every=32, flags=0, schedule=0):
    if getattr(geo, "exact_transmission", False):
        flags |= B.MSLICE_EXACT_TRANSMISSION
    if getattr(geo, "strang", False):
        flags |= B.MSLICE_STRANG
    if getattr(geo, "angular", False):
        flags |= B.MSLICE_ANGULAR
    return B.make_params(geo.ny, geo.nz, geo.ns, np.rad2deg(geo.alpha_i_rad), geo.wavelength_nm,
                         geo.slice_nm, geo.dy_nm, geo.dz_nm, checkpoint_every, flags, schedule=schedule,
                         psi_rad=getattr(geo, "psi_rad_w", 0.0))


def dev(a, dtype):
    return torch.from_numpy(np.ascontiguousarray(a).astype(dtype)).cuda()


def forward(geo, vol, probe=None, exit_wave=False, return_field=False, schedule=0):
    p = params(geo, flags=B.MSLICE_EXIT_WAVE if exit_wave else 0, schedule=schedule)
    ws = B.workspace(p, B.MSLICE_OP_FORWARD)
    v = dev(vol, np.complex64)
    pr = None if probe is None else dev(probe, np.complex64)
    I = torch.empty((geo.nw, geo.nz, geo.ny), dtype=torch.float32, device="cuda")
    F = torch.empty((geo.nw, geo.nz, geo.ny), dtype=torch.complex64, device="cuda")
    B.mslice_forward(p, v, pr, I, F, ws)
    torch.cuda.synchronize()
    assert B.mslice_status(ws) == 0
    if exit_wave:
        return F.cpu().numpy()
    return (I.cpu().numpy(), F.cpu().numpy()) if return_field else I.cpu().numpy()


def loss_grad(geo, vol, meas, scale, probe=None, checkpoint_every=32, return_intensity=False, schedule=0):
    p = params(geo, checkpoint_every, schedule=schedule)
    ws = B.workspace(p, B.MSLICE_OP_LOSS_GRAD)
    v = dev(vol, np.complex64)
    pr = None if probe is None else dev(probe, np.complex64)
    m = dev(meas, np.float32)
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    g = torch.empty((geo.ns, geo.nz, geo.ny), dtype=torch.complex64, device="cuda")
    I = torch.empty((geo.nw, geo.nz, geo.ny), dtype=torch.float32, device="cuda")
    B.mslice_loss_grad(p, v, pr, m, float(scale), loss, g, I, ws)
    torch.cuda.synchronize()
    assert B.mslice_status(ws) == 0
    out = (float(loss.item()), g.cpu().numpy())
    return out + (I.cpu().numpy(),) if return_intensity else out


def adjoint(geo, vol, gpsi, probe=None, checkpoint_every=32):
    p = params(geo, checkpoint_every)
    ws = B.workspace(p, B.MSLICE_OP_ADJOINT)
    g = torch.empty((geo.ns, geo.nz, geo.ny), dtype=torch.complex64, device="cuda")
    B.mslice_adjoint(p, dev(vol, np.complex64), None if probe is None else dev(probe, np.complex64),
                     dev(gpsi, np.complex64), g, ws)
    torch.cuda.synchronize()
    assert B.mslice_status(ws) == 0
    return g.cpu().numpy()


def rel(a, b):
    a, b = np.ravel(a).astype(np.complex128), np.ravel(b).astype(np.complex128)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))
