"""Batched multi-structure launches, graph capture and the launch-shape
autotuner: results equal the single-structure calls."""
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


def _jobs(seed):
    rng = np.random.default_rng(seed)
    shapes = [(64, 64, 12), (128, 64, 9), (64, 64, 12), (64, 128, 7), (64, 64, 12)]
    jobs = []
    for k, (ny, nz, ns) in enumerate(shapes):
        vol = ci.random_volume(100 + k, ny, nz, ns, scale=40)
        a = float(rng.uniform(0.1, 0.5))
        geo = oracle.Geometry(ny, nz, ns, alpha_i_deg=(a,))
        I = oracle.forward(geo, vol)
        meas = (np.sqrt(I[0]) * rng.uniform(0.8, 1.2, I[0].shape)).astype(np.float32)
        jobs.append(dict(vol=G.dev(vol, np.complex64), meas=G.dev(meas, np.float32),
                         scale=float(rng.uniform(0.5, 2.0)), alpha_deg=a, geo=geo, vol_h=vol, meas_h=meas))
    return jobs


def test_batched_equals_single_and_oracle():
    from paper_2212_01253_gb300.batch import BatchedLossGrad
    jobs = _jobs(1)
    bat = BatchedLossGrad(jobs, tune=False)
    assert len(bat.groups) == 3          # three structures share 64x64x12
    bat.run()
    torch.cuda.synchronize()
    bat.check()
    total = 0.0
    for i, jb in enumerate(jobs):
        L1, g1 = G.loss_grad(jb["geo"], jb["vol_h"], jb["meas_h"][None], jb["scale"])
        total += L1
        assert np.array_equal(bat.grad(i).cpu().numpy(), g1)     # same arithmetic per element
        Lr, gr = oracle.loss_grad(jb["geo"], jb["vol_h"], jb["meas_h"][None], jb["scale"])
        assert G.rel(g1, gr) <= 1e-3
    assert abs(bat.loss() - total) <= 1e-9 * total


@pytest.mark.parametrize("lanes", [1, 3])
def test_graph_replay_equals_eager(lanes):
    """One CUDA graph of the whole batch, on one stream or forked onto lanes
    (concurrent groups on a split grid), equals the eager single-stream run."""
    from paper_2212_01253_gb300.batch import BatchedLossGrad
    jobs = _jobs(2)
    bat = BatchedLossGrad(jobs, tune=False, lanes=lanes)
    bat.run()
    torch.cuda.synchronize()
    eager = [bat.grad(i).clone() for i in range(len(jobs))]
    L_eager = bat.loss()
    for g in bat.groups:
        g["grad"].zero_()
    bat.capture()
    bat.replay()
    torch.cuda.synchronize()
    bat.check()
    for i in range(len(jobs)):
        assert torch.equal(bat.grad(i), eager[i])
    assert abs(bat.loss() - L_eager) <= 1e-12 * L_eager


def test_launch_shape_does_not_change_results():
    from paper_2212_01253_gb300 import autotune
    from paper_2212_01253_gb300 import binding as B
    geo = oracle.Geometry(256, 512, 6, alpha_i_deg=(0.2, 0.4))
    vol = ci.random_volume(7, 256, 512, 6, scale=40)
    ref = None
    for g, cw in [(0, 0), (16, 4), (152, 8), (38, 16)]:
        p = G.params(geo)
        p.grid_blocks, p.col_width = g, cw
        ws = B.workspace(p, B.MSLICE_OP_FORWARD)
        I = torch.empty((2, 512, 256), dtype=torch.float32, device="cuda")
        B.mslice_forward(p, G.dev(vol, np.complex64), None, I, None, ws)
        out = I.cpu().numpy()
        if ref is None:
            ref = out
            assert G.rel(out, oracle.forward(geo, vol)) <= 1e-4
        else:
            assert np.array_equal(out, ref), (g, cw)
    g, cw, sc = autotune.tune(256, 512, 2, force=True)
    assert cw in autotune.col_widths(512) and sc in (1, 2)
