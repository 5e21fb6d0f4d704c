"""Loss and gradient of many independent structures of uneven shape in one
graph launch.

Jobs (volume, incidence angle, detector amplitudes, flux scale) are grouped by
grid shape (ny, nz, ns); each group advances as the wavefields of one
persistent multi-structure launch sequence (mslice_loss_grad_multi: every
wavefield has its own volume and gradient), with the launch shape picked by
the autotuner.  The calls of all groups are captured into one CUDA graph, so a
whole batch evaluation is a single cudaGraphLaunch.
"""
from __future__ import annotations

import collections

import numpy as np
import torch

from . import autotune
from . import binding as B


def assign_lanes(costs, lanes):
    """Greedy longest-first assignment of jobs with the given costs to `lanes`
    queues, each job onto the least loaded queue (ties: the lowest index).
    Returns the job indices of each queue, in the order they were placed."""
    out = [[] for _ in range(max(1, int(lanes)))]
    load = [0.0] * len(out)
    for i in sorted(range(len(costs)), key=lambda i: (-costs[i], i)):
        k = load.index(min(load))
        out[k].append(i)
        load[k] += costs[i]
    return out


def group_cost(p):
    """Modelled time of one group's loss + gradient: its work plus a per-slice
    latency term (grid barriers and launch-bound slice steps)."""
    return p.nw * p.ny * p.nz * p.ns / 4e10 + p.ns * 2.5e-5


class BatchedLossGrad:
    def __init__(self, jobs, wavelength_nm=0.155, slice_nm=20.0, dy_nm=2.0, dz_nm=2.0, checkpoint_every=32,
                 tune=True, device="cuda", lanes=1):
        """jobs: list of dicts with 'vol' (complex64 [ns][nz][ny], CUDA), 'meas' (float32 [nz][ny], CUDA),
        'scale' (float) and 'alpha_deg' (float).

        lanes > 1 runs the groups on that many streams at once, each group's
        persistent kernels on SMs / lanes blocks, so that the grids of the
        concurrent launches fit on the GPU together (one block per SM each) and
        small groups, whose slice loops are latency-bound, overlap."""
        self.device = torch.device(device)
        groups = collections.OrderedDict()
        for i, jb in enumerate(jobs):
            ns, nz, ny = jb["vol"].shape
            groups.setdefault((ny, nz, ns), []).append(i)
        self.groups = []
        self.where = {}
        for (ny, nz, ns), idx in groups.items():
            for c0 in range(0, len(idx), B.MSLICE_MAX_ANGLES):
                chunk = idx[c0:c0 + B.MSLICE_MAX_ANGLES]
                nw = len(chunk)
                p = B.make_params(ny, nz, ns, [jobs[i]["alpha_deg"] for i in chunk], wavelength_nm, slice_nm,
                                  dy_nm, dz_nm, checkpoint_every, flags=B.MSLICE_PER_STRUCTURE)
                if tune:
                    autotune.apply(p, self.device)
                if lanes > 1:
                    sms = torch.cuda.get_device_properties(self.device).multi_processor_count
                    p.grid_blocks = max(1, sms // int(lanes))
                vols = torch.stack([jobs[i]["vol"] for i in chunk]).contiguous()
                meas = torch.stack([jobs[i]["meas"] for i in chunk]).contiguous()
                g = dict(p=p, vols=vols, meas=meas, scales=[float(jobs[i]["scale"]) for i in chunk],
                         grad=torch.empty_like(vols), loss=torch.zeros(1, dtype=torch.float64, device=self.device),
                         ws=B.workspace(p, B.MSLICE_OP_LOSS_GRAD, self.device), jobs=chunk)
                for k, i in enumerate(chunk):
                    self.where[i] = (len(self.groups), k)
                self.groups.append(g)
        self.graph = None
        self.units = sum(g["p"].nw * g["p"].ny * g["p"].nz * g["p"].ns for g in self.groups)
        # groups to lanes, longest first onto the least loaded lane
        self.lanes = assign_lanes([group_cost(g["p"]) for g in self.groups], lanes)
        self.streams = [torch.cuda.Stream(self.device) for _ in self.lanes] if len(self.lanes) > 1 else []

    def _enqueue(self, g, stream=None):
        B.mslice_loss_grad_multi(g["p"], g["vols"], None, g["meas"], g["scales"], g["loss"], g["grad"], None,
                                 g["ws"], stream=stream)

    def run(self):
        """Enqueue every group's loss and gradient: on the current stream, or
        forked onto the lane streams and joined back into the current one."""
        if not self.streams:
            for g in self.groups:
                self._enqueue(g)
            return
        main = torch.cuda.current_stream(self.device)
        for st in self.streams:
            st.wait_stream(main)
        for st, lane in zip(self.streams, self.lanes):
            for gi in lane:
                self._enqueue(self.groups[gi], st)
        for st in self.streams:
            main.wait_stream(st)

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
        return float(sum(g["loss"].item() for g in self.groups))

    def grad(self, job):
        gi, k = self.where[job]
        return self.groups[gi]["grad"][k]

    def check(self):
        for g in self.groups:
            if B.mslice_status(g["ws"]) != 0:
                raise RuntimeError("device-side wait timed out in a batched launch")
