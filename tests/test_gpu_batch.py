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
    assert bat.ngroups == 3              # three structures share 64x64x12
    bat.run()
    torch.cuda.synchronize()
    bat.check()
    total = 0.0
    for i, jb in enumerate(jobs):
        L1, g1 = G.loss_grad(jb["geo"], jb["vol_h"], jb["meas_h"][None], jb["scale"])
        total += L1
        assert np.array_equal(bat.grad(i).cpu().numpy(), g1)     # same arithmetic per element
        assert bat.job_loss(i) == L1
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
    for jb in bat.jobs:
        jb["grad"].zero_()
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


def _mix(seed, shapes):
    """A mix of uneven structures in the manner of the 64-structure batch: Si
    substrate with Au pillars, grids 128..512, 128..1024 slices, 0.1-0.5 deg."""
    rng = np.random.default_rng(seed)
    jobs = []
    for k, (ny, nz, ns) in enumerate(shapes):
        vol = ci.pillars_large(1000 * seed + k, ny, nz, ns, count=max(4, ny // 16))
        a = float(rng.uniform(0.1, 0.5))
        jobs.append(dict(shape=(ny, nz, ns), alpha_deg=a, vol_h=vol, scale=float(rng.uniform(0.5, 2.0)),
                         geo=oracle.Geometry(ny, nz, ns, alpha_i_deg=(a,))))
    return jobs


MIX = [(512, 512, 1024), (128, 128, 128), (256, 128, 256), (128, 256, 128), (256, 128, 256),
       (128, 128, 512), (256, 256, 128), (128, 128, 128), (512, 128, 128)]


@pytest.fixture(scope="module")
def mix_with_oracle():
    """Each job's target: Poisson counts (1e6 in all) of another pillar layout
    of its shape, as in a reconstruction; its flux scale from the counts."""
    jobs = _mix(4, MIX)
    for k, jb in enumerate(jobs):
        ny, nz, ns = jb["shape"]
        truth = ci.pillars_large(7000 + k, ny, nz, ns, count=max(4, ny // 16))
        I_gt = oracle.forward(jb["geo"], truth)[0]
        jb["meas_h"], jb["scale"] = ci.poisson_target(I_gt, 1e6, seed=k)
        jb["meas_h"] = jb["meas_h"].astype(np.float32)
        jb["I_ref"] = oracle.forward(jb["geo"], jb["vol_h"])[0]
        jb["ref"] = oracle.loss_grad(jb["geo"], jb["vol_h"], jb["meas_h"][None], jb["scale"])
    return jobs


@pytest.mark.parametrize("lanes", [1, 4])
def test_batched_uneven_mix_vs_oracle_and_single_calls(mix_with_oracle, lanes):
    """mslice_loss_grad_batched on nine structures of seven shapes (one
    512x512x1024, one 128x128x128 ...): every job's loss and gradient match
    the FP64 oracle, and equal the single-structure call bit for bit."""
    from paper_2212_01253_gb300.batch import BatchedLossGrad
    jobs = mix_with_oracle
    dj = [dict(vol=G.dev(jb["vol_h"], np.complex64), meas=G.dev(jb["meas_h"], np.float32), scale=jb["scale"],
               alpha_deg=jb["alpha_deg"]) for jb in jobs]
    bat = BatchedLossGrad(dj, tune=False, lanes=lanes)
    assert bat.ngroups == 7
    bat.run()
    torch.cuda.synchronize()
    bat.check()
    total = 0.0
    for i, jb in enumerate(jobs):
        L_ref, g_ref = jb["ref"]
        g = bat.grad(i).cpu().numpy()
        L = bat.job_loss(i)
        total += L
        assert abs(L - L_ref) <= 1e-4 * abs(L_ref), (jb["shape"], L, L_ref)
        assert G.rel(g, g_ref) <= 1e-3, jb["shape"]
        L1, g1 = G.loss_grad(jb["geo"], jb["vol_h"], jb["meas_h"][None], jb["scale"])
        assert L == L1 and np.array_equal(g, g1), jb["shape"]
    assert bat.loss() == pytest.approx(total, rel=1e-12)


def test_forward_batched_vs_oracle_and_single_calls(mix_with_oracle):
    from paper_2212_01253_gb300 import binding as B
    jobs = mix_with_oracle
    dj = [dict(vol=G.dev(jb["vol_h"], np.complex64), alpha_deg=jb["alpha_deg"],
               intensity=torch.full(jb["shape"][1::-1], float("nan"), dtype=torch.float32, device="cuda"))
          for jb in jobs]
    common = B.make_params(64, 64, 1)
    arr = B.make_jobs(dj)
    ws = torch.empty(B.mslice_batched_workspace_size(common, arr, B.MSLICE_OP_FORWARD, 3), dtype=torch.uint8,
                     device="cuda")
    B.mslice_forward_batched(common, arr, 3, ws)
    torch.cuda.synchronize()
    assert B.mslice_batched_status(common, arr, B.MSLICE_OP_FORWARD, 3, ws) == 0
    for jb, d in zip(jobs, dj):
        I = d["intensity"].cpu().numpy()
        assert G.rel(I, jb["I_ref"]) <= 1e-4, jb["shape"]
        assert np.array_equal(I, G.forward(jb["geo"], jb["vol_h"])[0])
