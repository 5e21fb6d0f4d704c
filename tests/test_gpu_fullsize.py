"""Parity at the benchmark's full size and launch configuration: 512x512 grid,
1024 slices of 20 nm, 9 incidence angles 0.10-0.50 deg through one Si + Au
pillar volume, loss and gradient against Poisson targets, with the launch shape
from the autotuner and every a_j kept (one checkpoint segment), exactly as
``bench.py`` times it.  The FP64 oracle computes the same step on the host
cores (about half a minute)."""
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
    oracle.build()


def test_full_size_loss_gradient_in_bench_launch_configuration():
    from paper_2212_01253_gb300 import autotune
    from paper_2212_01253_gb300 import binding as B
    ny = nz = 512
    ns, nw = 1024, 9
    angles = np.linspace(0.1, 0.5, nw)
    geo = oracle.Geometry(ny, nz, ns, alpha_i_deg=angles)
    vol = ci.pillars_large(0, ns=ns)
    truth = ci.pillars_large(1000, ns=ns)
    I_gt = oracle.forward(geo, truth)
    meas = np.empty(I_gt.shape, np.float32)
    scales = []
    for w in range(nw):
        meas[w], s_w = ci.poisson_target(I_gt[w], 1e6, seed=w)
        scales.append(s_w)
    s = float(np.mean(scales))
    L_ref, g_ref, I_ref = oracle.loss_grad(geo, vol, meas, s, return_intensity=True)

    p = G.params(geo, checkpoint_every=ns)
    autotune.apply(p)
    ws = B.workspace(p, B.MSLICE_OP_LOSS_GRAD)
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    grad = torch.empty((ns, nz, ny), dtype=torch.complex64, device="cuda")
    inten = torch.empty((nw, nz, ny), dtype=torch.float32, device="cuda")
    B.mslice_loss_grad(p, G.dev(vol, np.complex64), None, G.dev(meas, np.float32), s, loss, grad, inten, ws)
    torch.cuda.synchronize()
    assert B.mslice_status(ws) == 0
    assert G.rel(inten.cpu().numpy(), I_ref) <= 1e-4
    assert abs(float(loss.item()) - L_ref) <= 1e-4 * abs(L_ref)
    assert G.rel(grad.cpu().numpy(), g_ref) <= 1e-3
