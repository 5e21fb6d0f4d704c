"""HostPipeline (copies on their own streams, two or three device slots) gives the same
loss and gradient as mslice_loss_grad on device tensors, bit for bit, for a
sequence of different host-resident problems."""
import numpy as np
import pytest
import torch

import cssi_inputs as ci
import oracle
from tests import _gpu as G

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2212_01253_gb300 import build
    build.build()


@pytest.mark.parametrize("slots", [2, 3])
def test_host_pipeline_matches_device_calls(slots):
    from paper_2212_01253_gb300 import binding as B
    from paper_2212_01253_gb300.pipeline import HostPipeline
    geo = oracle.Geometry(128, 64, 20, alpha_i_deg=(0.2, 0.35))
    p = G.params(geo, checkpoint_every=8)
    vols = [ci.random_volume(40 + k, 128, 64, 20, scale=40) for k in range(5)]
    meas = (np.sqrt(oracle.forward(geo, vols[0])) * 1.1).astype(np.float32)
    pipe = HostPipeline(p, 0.8, slots=slots)
    meas_pin = torch.from_numpy(meas).pin_memory()
    outs = []
    for v in vols:
        g = torch.empty(v.shape, dtype=torch.complex64).pin_memory()
        l = torch.empty(1, dtype=torch.float64).pin_memory()
        pipe.submit(torch.from_numpy(v).pin_memory(), meas_pin, g, l)
        outs.append((g, l))
    torch.cuda.synchronize()
    assert pipe.status() == 0
    ws = B.workspace(p, B.MSLICE_OP_LOSS_GRAD)
    for v, (g, l) in zip(vols, outs):
        grad = torch.empty(v.shape, dtype=torch.complex64, device="cuda")
        loss = torch.zeros(1, dtype=torch.float64, device="cuda")
        B.mslice_loss_grad(p, G.dev(v, np.complex64), None, G.dev(meas, np.float32), 0.8, loss, grad, None, ws)
        torch.cuda.synchronize()
        assert float(l.item()) == float(loss.item())
        assert torch.equal(g, grad.cpu())
