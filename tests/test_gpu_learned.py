"""Learned initialiser kernels on the GPU against the FP64 network oracle, and
what the trained network gains over starting the reconstruction from bare
silicon."""
import numpy as np
import pytest
import torch

from oracle import nn as onn
from tests import _gpu as G

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2212_01253_gb300 import build
    build.build()


def _gemm_ref(A, sam, sak, Bm, sbn, sbk, M, N, K, bias, relu, beta, C0):
    Am = np.lib.stride_tricks.as_strided(A, (M, K), (sam * A.itemsize, sak * A.itemsize))
    Bv = np.lib.stride_tricks.as_strided(Bm, (N, K), (sbn * Bm.itemsize, sbk * Bm.itemsize))
    z = onn.dense(np.array(Am), np.array(Bv))
    if bias is not None:
        z = z + bias
    if relu:
        z = np.maximum(z, 0)
    return z + beta * C0 if beta else z


@pytest.mark.parametrize("M,N,K,trans_a,trans_b,use_bias,relu,beta", [
    (67, 45, 37, False, False, True, True, 0.0),       # ragged tiles in every dimension
    (130, 70, 200, True, True, False, False, 0.5),     # transposed operands, accumulate into C
    (64, 32, 20000, False, True, True, False, 0.0),    # long K: split over CTAs
    (300, 17, 4096, True, False, True, True, 0.0),
])
def test_gemm_vs_oracle(M, N, K, trans_a, trans_b, use_bias, relu, beta):
    from paper_2212_01253_gb300 import binding as B
    rng = np.random.default_rng(M + N + K)
    A = rng.standard_normal(M * K).astype(np.float32)
    Bm = rng.standard_normal(N * K).astype(np.float32)
    sam, sak = (1, M) if trans_a else (K, 1)
    sbn, sbk = (1, N) if trans_b else (K, 1)
    bias = rng.standard_normal(N).astype(np.float32) if use_bias else None
    C0 = rng.standard_normal((M, N)).astype(np.float32)
    C = G.dev(C0, np.float32)
    need = B.mslice_nn_gemm_workspace(M, N, K)
    if K >= 20000:
        assert need > 0, "long K should split"
    ws = torch.empty(max(need, 16), dtype=torch.uint8, device="cuda")
    B.mslice_nn_gemm(M, N, K, G.dev(A, np.float32), sam, sak, G.dev(Bm, np.float32), sbn, sbk, C, N,
                     None if bias is None else G.dev(bias, np.float32), relu, beta, ws)
    ref = _gemm_ref(A, sam, sak, Bm, sbn, sbk, M, N, K, bias, relu, beta, C0)
    assert G.rel(C.cpu().numpy(), ref) <= 1e-5


def test_gemm_padded_rows_ragged_k():
    """Row strides larger than K (padded rows, 16-byte loads along k) with K not
    a multiple of 4: the last group of each row is read element by element."""
    from paper_2212_01253_gb300 import binding as B
    rng = np.random.default_rng(11)
    M, N, K, lda, ldb = 70, 65, 4097, 4100, 4104
    A = rng.standard_normal(M * lda).astype(np.float32)
    Bm = rng.standard_normal(N * ldb).astype(np.float32)
    C = torch.empty((M, N), dtype=torch.float32, device="cuda")
    ws = torch.empty(max(B.mslice_nn_gemm_workspace(M, N, K), 16), dtype=torch.uint8, device="cuda")
    B.mslice_nn_gemm(M, N, K, G.dev(A, np.float32), lda, 1, G.dev(Bm, np.float32), ldb, 1, C, N, ws=ws)
    ref = onn.dense(A.reshape(M, lda)[:, :K], Bm.reshape(N, ldb)[:, :K])
    assert G.rel(C.cpu().numpy(), ref) <= 1e-5


def test_gemm_constant_a_column_sums():
    """sam = sak = 0 reads A as a constant: the bias-gradient form 1^T dZ."""
    from paper_2212_01253_gb300 import binding as B
    rng = np.random.default_rng(9)
    rows, N = 5000, 100
    dZ = rng.standard_normal((rows, N)).astype(np.float32)
    out = torch.empty(N, dtype=torch.float32, device="cuda")
    ws = torch.empty(max(B.mslice_nn_gemm_workspace(1, N, rows), 16), dtype=torch.uint8, device="cuda")
    B.mslice_nn_gemm(1, N, rows, torch.ones(1, device="cuda"), 0, 0, G.dev(dZ, np.float32), 1, N, out, N,
                     ws=ws)
    ref = onn.bf16_round(dZ).sum(axis=0)
    assert G.rel(out.cpu().numpy(), ref) <= 1e-5


def test_space_to_depth_bit_exact():
    from paper_2212_01253_gb300 import binding as B
    rng = np.random.default_rng(1)
    x = rng.standard_normal((3, 16, 16, 5)).astype(np.float32)
    y = torch.empty(x.size, dtype=torch.float32, device="cuda")
    B.mslice_nn_space_to_depth(G.dev(x, np.float32).reshape(-1), y, 3, 16, 16, 5, 4)
    np.testing.assert_array_equal(y.cpu().numpy().reshape(3, 4, 4, 4, 4, 5), onn.space_to_depth(x, 4))
    back = torch.empty_like(y)
    B.mslice_nn_space_to_depth(y, back, 3, 16, 16, 5, 4, inverse=True)
    np.testing.assert_array_equal(back.cpu().numpy().reshape(x.shape), x)


def test_detector_features_vs_oracle():
    from paper_2212_01253_gb300 import binding as B
    rng = np.random.default_rng(2)
    I = (rng.random((3, 32, 64)) ** 4).astype(np.float32)
    noise = rng.standard_normal(I.shape).astype(np.float32)
    x = torch.empty(I.size, dtype=torch.float32, device="cuda")
    for nz_, counts in ((noise, 1e6), (None, 1e5), (None, 0.0), (noise, -1.0)):
        B.mslice_nn_detector_features(G.dev(I, np.float32), None if nz_ is None else G.dev(nz_, np.float32), x,
                                      3, 32, 64, counts, 0.25)
        ref = onn.detector_features(I, nz_, counts, 0.25)
        assert np.abs(x.cpu().numpy().reshape(I.shape) - ref).max() <= 2e-6 * np.abs(ref).max()


def test_rasterize_boxes_bit_exact():
    from paper_2212_01253_gb300 import binding as B
    rng = np.random.default_rng(3)
    lo = rng.integers(0, 6, (4, 5, 3))
    hi = lo + rng.integers(0, 5, (4, 5, 3))
    boxes = np.stack([lo[..., 0], hi[..., 0], lo[..., 1], hi[..., 1], lo[..., 2], hi[..., 2]], -1)
    out = torch.empty(4 * 8 * 7 * 9, dtype=torch.float32, device="cuda")
    B.mslice_nn_rasterize_boxes(torch.from_numpy(boxes.astype(np.int32)).cuda(), out, (8, 7, 9), 0.75)
    np.testing.assert_array_equal(out.cpu().numpy().reshape(4, 8, 7, 9),
                                  onn.rasterize_boxes(boxes, (8, 7, 9), 0.75))


def test_sigmoid_mse_vs_oracle():
    from paper_2212_01253_gb300 import binding as B
    rng = np.random.default_rng(4)
    rows, cols = 5, 3000
    z = (3 * rng.standard_normal((rows, cols))).astype(np.float32)
    t = (rng.random((rows, cols)) < 0.2).astype(np.float32)
    y = torch.empty(rows * cols, device="cuda")
    dz = torch.empty_like(y)
    rl = torch.empty(rows, dtype=torch.float64, device="cuda")
    B.mslice_nn_sigmoid_mse(G.dev(z, np.float32).reshape(-1), G.dev(t, np.float32).reshape(-1), y, dz, rl, rows,
                            cols, 1.0)
    yr, lr_, dzr = onn.sigmoid_mse(z, t, 1.0)
    assert G.rel(y.cpu().numpy(), yr.ravel()) <= 1e-6
    assert G.rel(dz.cpu().numpy(), dzr.ravel()) <= 1e-5
    assert abs(rl.sum().item() - lr_) <= 1e-6 * lr_


SMALL = dict(in_hw=32, enc=[(2, 8), (2, 16)], latent=24, dec_c0=12, dec=[(2, 8), (2, 6)])


@pytest.mark.parametrize("tensor_cores", [False, True])
def test_network_forward_and_gradients_vs_oracle(tensor_cores, monkeypatch):
    """Forward, loss and every parameter gradient against the oracle, with the
    layers' forward and input-gradient GEMMs on mslice_nn_gemm or, with the
    thresholds at 1, all on the tcgen05 path (BF16 weight copies)."""
    from paper_2212_01253_gb300 import learned
    from paper_2212_01253_gb300.learned import EncoderDecoder
    for name in ("TC_MIN_ROWS", "TC_MIN_K", "TC_MIN_N"):
        monkeypatch.setattr(learned, name, 1 if tensor_cores else 1 << 30)
    rng = np.random.default_rng(6)
    net = EncoderDecoder(SMALL, max_batch=4)
    assert net.n_params == onn.n_params(SMALL)
    th = (rng.standard_normal(net.n_params) * 0.2).astype(np.float32)
    net.theta.copy_(torch.from_numpy(th))
    net.refresh_bf16()
    x = rng.standard_normal((3, 32, 32)).astype(np.float32)
    tgt = (rng.random((3, 32, 32, 6)) < 0.3).astype(np.float32)
    rl = net.loss_grad(G.dev(x, np.float32), G.dev(tgt, np.float32), nb=3)
    loss_ref, g_ref, y_ref = onn.loss_and_grad(SMALL, th, x, tgt)
    assert abs(rl.sum().item() - loss_ref) <= 1e-4 * loss_ref
    assert G.rel(net.y[:y_ref.size].cpu().numpy(), y_ref.ravel()) <= 1e-4
    g = net.grad.cpu().numpy()
    o = 0
    for L in onn.layer_table(SMALL):
        n = L["N"] * L["K"] + L["N"]
        assert G.rel(g[o:o + n], g_ref[o:o + n]) <= 1e-3, L
        o += n


def test_trained_network_gains_over_zero_and_constant_starts():
    """64x64 grid, 64 slices, 16x16x8 coarse Au voxels, 1-3 pillars 12-40 nm tall.
    A network trained on 8192 fresh forward-model samples gives starting volumes
    from which ADAM on the CUDA gradient lowers the reduced chi^2 of held-out
    Poisson targets far below what the bare-substrate start (zero) and the
    mean-occupancy start (constant) reach in the same number of iterations;
    those two stall in the same local minimum."""
    import cssi_inputs as ci
    from paper_2212_01253_gb300 import binding as B
    from paper_2212_01253_gb300.learned import AU_DELTA, EncoderDecoder, PillarSampler, train
    from paper_2212_01253_gb300.recon import Reconstructor
    ny = nz = ns = 64
    p = B.make_params(ny, nz, ns, (0.3,))
    c = B.make_coarse((16, 16, 8), (4, 2, 8), (0, 32, 0))
    base = torch.from_numpy(ci.substrate(ny, nz, ns)).cuda()
    sampler = PillarSampler(p, c, base, n_pillars=(1, 3), foot=(1, 5), height=(3, 11))
    net = EncoderDecoder(dict(in_hw=64, enc=[(4, 16), (2, 32)], latent=64, dec_c0=32, dec=[(2, 8)]), 64)
    losses = train(net, sampler, 8192, 64, lr=1e-3, seed=1000)
    k = len(losses) // 10
    assert np.mean(losses[-k:]) < 0.9 * np.mean(losses[:k]), losses
    _, occ, _ = sampler.sample(np.random.default_rng(999), 256, noise=False)
    occ_mean = float(occ.cpu().numpy().mean())
    ws = B.workspace(p, B.MSLICE_OP_FORWARD)
    for seed in (100001, 100002, 100003):
        _, _, theta = sampler.sample(np.random.default_rng(seed), 1, noise=False)
        vol = base.clone()
        B.mslice_coarse_to_fine(p, c, theta.reshape(-1).contiguous(), vol)
        inten = torch.empty(nz * ny, dtype=torch.float32, device="cuda")
        B.mslice_forward(p, vol, None, inten, None, ws)
        I_gt = inten.cpu().numpy().astype(np.float64).reshape(nz, ny)
        meas, s = ci.poisson_target(I_gt, 1e6, seed=seed)
        chi2_gt = 4 * ((np.sqrt(s * I_gt) - meas) ** 2).sum() / meas.size
        measd = torch.from_numpy(meas).cuda()
        starts = {"zero": None,
                  "constant": torch.full((16 * 16 * 8,), occ_mean * AU_DELTA, dtype=torch.float32, device="cuda"),
                  "learned": net.predict(sampler.features_of(measd)).reshape(-1).contiguous()}
        end = {}
        for name, th0 in starts.items():
            R = Reconstructor(p, c, base, measd, s, theta0=th0, lr=5e-6)
            _, _, hist = R.run(chi2_target=0.0, max_iters=100, check_every=100)
            end[name] = hist[-1][1]
        assert end["learned"] < 0.2 * min(end["zero"], end["constant"]), (seed, end, chi2_gt)
        assert end["learned"] < 3.0 * chi2_gt, (seed, end, chi2_gt)
