"""Loss + gradient for problems that live in host memory, with the host-device
copies of one problem overlapping the GPU work of its neighbours.

A caller whose volumes and detector images sit in (pinned) host memory, and
who needs each gradient back on the host, would otherwise pay the copies in
series with the slice loop: at 512x512x1024 with 9 angles that is 2.2 GB in and
2.1 GB out per problem.  `HostPipeline` keeps `slots` device slots and three
streams:

    copy-in stream   vol, meas  -> slot b          (waits until slot b's last
                                                    gradient has been copied out)
    compute stream   mslice_loss_grad on slot b    (waits for its copy-in)
    copy-out stream  grad, loss -> host            (waits for its compute)

so problem k+1 is copied in and problem k-1 copied out while problem k runs.
With two slots the copy-in of k+1 reuses k-1's slot and waits for its
copy-out, so the two copies run one after the other; with three they run at
once, on the two copy directions.
Ordering between the streams is by CUDA events only; the host never blocks
unless it asks for a result.  The arithmetic is exactly `mslice_loss_grad`'s.
"""
from __future__ import annotations

import torch

from . import binding as B


class HostPipeline:
    def __init__(self, params, scale, device=None, slots=2):
        self.p = params
        self.scale = float(scale)
        self.dev = torch.device(device or "cuda")
        nvol, nfield = B._sizes(params)
        self.shape_vol = (nvol,)
        self.ws = B.workspace(params, B.MSLICE_OP_LOSS_GRAD, self.dev)
        self.slots = []
        for _ in range(int(slots)):
            self.slots.append(dict(
                vol=torch.empty(nvol, dtype=torch.complex64, device=self.dev),
                meas=torch.empty(nfield, dtype=torch.float32, device=self.dev),
                grad=torch.empty(nvol, dtype=torch.complex64, device=self.dev),
                loss=torch.zeros(1, dtype=torch.float64, device=self.dev),
                copied_in=torch.cuda.Event(), computed=torch.cuda.Event(), copied_out=torch.cuda.Event(),
                used=False))
        self.s_in = torch.cuda.Stream(self.dev)
        self.s_comp = torch.cuda.Stream(self.dev)
        self.s_out = torch.cuda.Stream(self.dev)
        self.k = 0

    def submit(self, vol_host, meas_host, grad_host, loss_host):
        """Enqueue one problem: vol_host (complex64) and meas_host (float32) are
        read, grad_host (complex64) and loss_host (float64[1]) written, all
        pinned host tensors of the problem's sizes.  Returns the event that
        completes when grad_host and loss_host hold the result."""
        sl = self.slots[self.k % len(self.slots)]
        self.k += 1
        if sl["used"]:
            self.s_in.wait_event(sl["copied_out"])      # the slot's previous result is on the host
        with torch.cuda.stream(self.s_in):
            sl["vol"].copy_(vol_host.reshape(-1), non_blocking=True)
            sl["meas"].copy_(meas_host.reshape(-1), non_blocking=True)
            sl["copied_in"].record(self.s_in)
        self.s_comp.wait_event(sl["copied_in"])
        B.mslice_loss_grad(self.p, sl["vol"], None, sl["meas"], self.scale, sl["loss"], sl["grad"], None, self.ws,
                           stream=self.s_comp)
        sl["computed"].record(self.s_comp)
        self.s_out.wait_event(sl["computed"])
        with torch.cuda.stream(self.s_out):
            grad_host.reshape(-1).copy_(sl["grad"], non_blocking=True)
            loss_host.copy_(sl["loss"], non_blocking=True)
            sl["copied_out"].record(self.s_out)
        sl["used"] = True
        return sl["copied_out"]

    def status(self):
        """Bounded-wait status word of the workspace (0 = no device wait timed out)."""
        self.s_comp.synchronize()
        return B.mslice_status(self.ws, stream=self.s_comp)
