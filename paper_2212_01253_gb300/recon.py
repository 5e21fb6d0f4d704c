"""Gradient reconstruction of a coarse delta volume from detector amplitudes
(Sec. 4: coarse reconstruction voxels mapped onto the multislice grid, amplitude
loss of Eq. 4, ADAM).  Every step runs in libmslice kernels:

    E (coarse -> fine) -> mslice_loss_grad -> E^T -> ADAM (clamped to [lo, hi])
    [-> shrink-wrap support every shrinkwrap_every iterations]
    [-> material snapping every snap_every iterations]

The fine volume keeps its fixed part (substrate, vacuum) outside the coarse
block.  The stopping rule is the reduced chi^2 of Poisson amplitudes,
chi2_red = 4 L / N_pix (Var(sqrt(Poisson)) ~ 1/4).
"""
from __future__ import annotations

import time

import torch

from . import binding as B


class Reconstructor:
    def __init__(self, params, coarse, base_vol, meas_amp, scale, theta0=None, lr=2e-6, lo=0.0, hi=4.7e-5,
                 b1=0.9, b2=0.999, eps=1e-20, probe=None, snap_every=0, snap_levels=None, snap_start=0,
                 shrinkwrap_every=0, shrinkwrap_sigma=1.0, shrinkwrap_threshold=0.2):
        dev = base_vol.device
        self.p, self.c = params, coarse
        self.vol = base_vol.clone()
        self.meas = meas_amp.contiguous()
        self.scale = float(scale)
        self.probe = probe
        n = coarse.cx * coarse.cz * coarse.cy
        self.theta = (torch.zeros(n, dtype=torch.float32, device=dev) if theta0 is None
                      else theta0.reshape(-1).to(torch.float32).contiguous().clone())
        self.m = torch.zeros_like(self.theta)
        self.v = torch.zeros_like(self.theta)
        self.g_theta = torch.zeros_like(self.theta)
        self.grad = torch.empty_like(self.vol)
        self.loss = torch.zeros(1, dtype=torch.float64, device=dev)
        self.ws = B.workspace(params, B.MSLICE_OP_LOSS_GRAD, dev)
        self.lr, self.lo, self.hi, self.b1, self.b2, self.eps = lr, lo, hi, b1, b2, eps
        self.t = 0
        self.npix = params.nw * params.ny * params.nz
        # material snapping (Sec. 4.1): every snap_every iterations (from
        # iteration snap_start on) each coarse voxel becomes the nearest of snap_levels
        self.snap_every = int(snap_every)
        self.snap_levels = list(snap_levels) if snap_levels is not None else None
        self.snap_start = int(snap_start)
        # shrink-wrap support (Sec. 4.2): every shrinkwrap_every iterations the
        # coarse voxels outside the thresholded Gaussian blur of theta go to 0
        self.sw_every = int(shrinkwrap_every)
        self.sw_sigma, self.sw_threshold = float(shrinkwrap_sigma), float(shrinkwrap_threshold)
        self.sw_ws = (torch.empty(B._load().mslice_shrinkwrap_workspace(n), dtype=torch.uint8, device=dev)
                      if self.sw_every else None)

    def step(self):
        """One iteration; returns nothing (the loss of the current theta lands in self.loss)."""
        self.t += 1
        B.mslice_coarse_to_fine(self.p, self.c, self.theta, self.vol)
        B.mslice_loss_grad(self.p, self.vol, self.probe, self.meas, self.scale, self.loss, self.grad, None,
                           self.ws)
        B.mslice_fine_to_coarse(self.p, self.c, self.grad, self.g_theta)
        B.mslice_adam_step(self.theta, self.m, self.v, self.g_theta, self.lr, self.b1, self.b2, self.eps,
                           self.t, self.lo, self.hi)
        if self.sw_every and self.t % self.sw_every == 0:
            B.mslice_shrinkwrap(self.theta.view(self.c.cx, self.c.cz, self.c.cy), self.sw_sigma, self.sw_threshold,
                                ws=self.sw_ws)
        if self.snap_every and self.snap_levels and self.t >= self.snap_start and self.t % self.snap_every == 0:
            B.mslice_snap(self.theta, self.snap_levels)

    def save(self, path):
        """Write theta, the ADAM moments and the iteration count to `path`
        (.npz), so that a later Reconstructor resumes exactly where this one
        stopped (the fixed part of the volume, the target and the settings are
        the caller's to rebuild)."""
        import numpy as np
        torch.cuda.synchronize()
        np.savez(path, theta=self.theta.cpu().numpy(), m=self.m.cpu().numpy(), v=self.v.cpu().numpy(),
                 t=np.int64(self.t))

    def load(self, path):
        """Resume from a file written by `save`."""
        import numpy as np
        d = np.load(path)
        for name in ("theta", "m", "v"):
            src = torch.from_numpy(d[name])
            if src.numel() != self.theta.numel():
                raise ValueError("%s in %s has %d values, expected %d" % (name, path, src.numel(),
                                                                          self.theta.numel()))
            getattr(self, name).copy_(src.to(self.theta.device))
        self.t = int(d["t"])

    def chi2(self):
        return 4.0 * float(self.loss.item()) / self.npix

    def run(self, chi2_target, max_iters=1000, check_every=5):
        """Iterate until chi2_red <= chi2_target; returns (iterations, seconds, history)."""
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        hist = []
        for it in range(1, max_iters + 1):
            self.step()
            if it % check_every == 0 or it == max_iters:
                c2 = self.chi2()          # loss of the theta before this iteration's update
                hist.append((it, c2))
                if c2 <= chi2_target:
                    break
        torch.cuda.synchronize()
        if B.mslice_status(self.ws) != 0:
            raise RuntimeError("device-side wait timed out during reconstruction")
        return it, time.perf_counter() - t0, hist
