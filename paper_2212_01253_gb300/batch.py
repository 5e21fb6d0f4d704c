"""Loss and gradient of many independent structures of uneven shape in one
call of the library's batched entry point (mslice_loss_grad_batched).

The library groups the jobs by grid shape, advances each group as one
persistent per-structure run and spreads the groups over concurrent lanes;
this module only marshals the jobs (and, optionally, each shape's tuned
column-group width), and records the call into one CUDA graph.
"""
from __future__ import annotations

import collections

import torch

from . import autotune
from . import binding as B


class BatchedLossGrad:
    def __init__(self, jobs, wavelength_nm=0.155, slice_nm=20.0, dy_nm=2.0, dz_nm=2.0, checkpoint_every=32,
                 tune=True, device="cuda", lanes=1, flags=0):
        """jobs: list of dicts with 'vol' (complex64 [ns][nz][ny], CUDA), 'meas' (float32 [nz][ny], CUDA),
        'scale' (float) and 'alpha_deg' (float).  lanes: concurrent lanes of the batched call (1..16)."""
        self.device = torch.device(device)
        self.lanes = int(lanes)
        counts = collections.Counter(tuple(jb["vol"].shape) for jb in jobs)
        self.jobs = []
        for jb in jobs:
            ns, nz, ny = jb["vol"].shape
            cw = 0
            if tune:
                nw = min(counts[(ns, nz, ny)], B.MSLICE_MAX_ANGLES)
                cw = autotune.tune(ny, nz, nw, self.device)[1]
            self.jobs.append(dict(vol=jb["vol"], meas=jb["meas"], scale=float(jb["scale"]),
                                  alpha_deg=float(jb["alpha_deg"]), col_width=cw,
                                  grad=torch.empty_like(jb["vol"]),
                                  loss=torch.zeros(1, dtype=torch.float64, device=self.device)))
        self.common = B.make_params(64, 64, 1, (0.0,), wavelength_nm, slice_nm, dy_nm, dz_nm, checkpoint_every,
                                    flags=flags)
        self.arr = B.make_jobs(self.jobs)
        self.ws = torch.empty(B.mslice_batched_workspace_size(self.common, self.arr, B.MSLICE_OP_LOSS_GRAD,
                                                              self.lanes), dtype=torch.uint8, device=self.device)
        self.loss_total = torch.zeros(1, dtype=torch.float64, device=self.device)
        self.group_of_job, self.lane_of_group = B.mslice_batched_plan(self.common, self.arr, B.MSLICE_OP_LOSS_GRAD,
                                                                      self.lanes)
        self.units = sum(int(jb["vol"].numel()) for jb in self.jobs)
        self.graph = None

    @property
    def ngroups(self):
        return len(self.lane_of_group)

    def run(self):
        """Enqueue the batched loss and gradient on the current stream."""
        B.mslice_loss_grad_batched(self.common, self.arr, self.lanes, self.loss_total, self.ws)

    def capture(self):
        """Record run() into one CUDA graph (after one eager warm-up run)."""
        self.run()
        torch.cuda.synchronize()
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            self.run()
        return self.graph

    def replay(self):
        if self.graph is None:
            self.capture()
        self.graph.replay()

    def loss(self):
        return float(self.loss_total.item())

    def job_loss(self, job):
        return float(self.jobs[job]["loss"].item())

    def grad(self, job):
        return self.jobs[job]["grad"]

    def check(self):
        if B.mslice_batched_status(self.common, self.arr, B.MSLICE_OP_LOSS_GRAD, self.lanes, self.ws) != 0:
            raise RuntimeError("device-side wait timed out in a batched launch")
