"""Pins of the learned initialiser's network oracle (CPU, no GPU).

Each test ties ``oracle.nn`` to something other than itself: the definition of
BF16 (and torch's independent conversion), a brute-force convolution, central
finite differences, numpy's fftshift, and explicit loops.
"""
import numpy as np
import pytest
import torch

from oracle import nn


def test_bf16_round_ties_to_even_and_spacing():
    # BF16 spacing at 1 is 2^-7; midpoints go to the even significand
    assert nn.bf16_round(1.0 + 2.0 ** -8) == 1.0
    assert nn.bf16_round(1.0 + 3 * 2.0 ** -8) == 1.0 + 2.0 ** -6
    assert nn.bf16_round(1.0 + 2.0 ** -8 + 2.0 ** -20) == 1.0 + 2.0 ** -7
    assert nn.bf16_round(-3.0) == -3.0 and nn.bf16_round(0.0) == 0.0
    assert nn.bf16_round(255.0) == 255.0 and nn.bf16_round(257.0) == 256.0


def test_bf16_round_matches_torch_conversion():
    rng = np.random.default_rng(0)
    x = (rng.standard_normal(20000) * np.exp(rng.uniform(-20, 20, 20000))).astype(np.float32)
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(nn.bf16_round(x), ref)


def test_space_to_depth_round_trip_and_patch_order():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((2, 8, 12, 3))
    y = nn.space_to_depth(x, 4)
    assert y.shape == (2, 2, 3, 4, 4, 3)
    np.testing.assert_array_equal(nn.depth_to_space(y, 4), x)
    # patch (i, j) element (di, dj, c) is input row 4i+di, column 4j+dj
    for i, j, di, dj, c in [(1, 2, 3, 0, 2), (0, 0, 0, 0, 0), (1, 1, 2, 3, 1)]:
        assert y[1, i, j, di, dj, c] == x[1, 4 * i + di, 4 * j + dj, c]


def test_patch_convolution_equals_brute_force_conv():
    """A stride-p, kernel-p convolution written as loops equals space_to_depth + dense."""
    rng = np.random.default_rng(2)
    B, H, C, p, co = 2, 8, 3, 2, 5
    x = rng.standard_normal((B, H, H, C))
    w4 = rng.standard_normal((co, p, p, C))     # [c_out][di][dj][c_in]
    b = rng.standard_normal(co)
    ref = np.zeros((B, H // p, H // p, co))
    for n in range(B):
        for i in range(H // p):
            for j in range(H // p):
                for o in range(co):
                    s = b[o]
                    for di in range(p):
                        for dj in range(p):
                            for c in range(C):
                                s += w4[o, di, dj, c] * x[n, p * i + di, p * j + dj, c]
                    ref[n, i, j, o] = s
    X = nn.space_to_depth(x, p).reshape(-1, p * p * C)
    got = nn.dense(X, w4.reshape(co, -1), b, rounding=False).reshape(ref.shape)
    np.testing.assert_allclose(got, ref, rtol=1e-13, atol=1e-13)


def test_transposed_patch_convolution_equals_brute_force():
    rng = np.random.default_rng(3)
    B, h, C, p, co = 2, 3, 4, 2, 3
    a = rng.standard_normal((B, h, h, C))
    w = rng.standard_normal((p * p * co, C))
    ref = np.zeros((B, h * p, h * p, co))
    w4 = w.reshape(p, p, co, C)
    for n in range(B):
        for i in range(h):
            for j in range(h):
                for di in range(p):
                    for dj in range(p):
                        for o in range(co):
                            ref[n, p * i + di, p * j + dj, o] = (w4[di, dj, o] * a[n, i, j]).sum()
    Y = nn.dense(a.reshape(-1, C), w, rounding=False)
    got = nn.depth_to_space(Y.reshape(B, h, h, p, p, co), p)
    np.testing.assert_allclose(got, ref, rtol=1e-13, atol=1e-13)


ARCH = dict(in_hw=32, enc=[(2, 4), (2, 6)], latent=5, dec_c0=3, dec=[(2, 4), (2, 3)])


def test_network_gradient_matches_central_differences():
    rng = np.random.default_rng(4)
    th = rng.standard_normal(nn.n_params(ARCH)) * 0.3
    x = rng.standard_normal((2, 32, 32))
    tgt = (rng.random((2, 32, 32, 3)) < 0.3).astype(float)
    loss, g, _ = nn.loss_and_grad(ARCH, th, x, tgt, rounding=False)
    # parameters of every layer, hidden and output
    offs, o = [], 0
    for L in nn.layer_table(ARCH):
        offs.append((o, o + L["N"] * L["K"] + L["N"]))
        o += L["N"] * L["K"] + L["N"]
    idx = [rng.integers(a, b) for a, b in offs for _ in range(3)] + [b - 1 for _, b in offs]
    checked = 0
    for i in idx:
        h = 1e-6
        tp, tm = th.copy(), th.copy()
        tp[i] += h
        tm[i] -= h
        fd = (nn.loss_and_grad(ARCH, tp, x, tgt, rounding=False)[0]
              - nn.loss_and_grad(ARCH, tm, x, tgt, rounding=False)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1e-3, abs(fd)) + 1e-10, (i, fd, g[i])
        checked += g[i] != 0
    assert checked >= len(offs)


def test_sigmoid_mse_derivative():
    rng = np.random.default_rng(5)
    z = rng.standard_normal(50)
    t = rng.random(50)
    _, loss, dz = nn.sigmoid_mse(z, t, 2.5)
    for i in range(0, 50, 7):
        h = 1e-6
        zp, zm = z.copy(), z.copy()
        zp[i] += h
        zm[i] -= h
        fd = (nn.sigmoid_mse(zp, t, 2.5)[1] - nn.sigmoid_mse(zm, t, 2.5)[1]) / (2 * h)
        assert abs(fd - dz[i]) < 1e-9


def test_detector_features_scaling_and_centring():
    rng = np.random.default_rng(6)
    I = rng.random((2, 8, 16))
    x = nn.detector_features(I, counts=1e4, gain=1.0)
    # undo the log and the shift: the amplitudes squared sum to the counts
    a2 = np.expm1(np.fft.ifftshift(x, axes=(1, 2)))
    np.testing.assert_allclose(a2.sum(axis=(1, 2)), [1e4, 1e4], rtol=1e-12)
    # the DC pixel lands at the centre
    assert x[0, 4, 8] == pytest.approx(np.log1p(1e4 * I[0, 0, 0] / I[0].sum()), rel=1e-13)
    # counts == 0: input already in counts; counts < 0: input is the amplitude
    np.testing.assert_allclose(nn.detector_features(I, counts=0, gain=2.0)[1, 4, 8], 2 * np.log1p(I[1, 0, 0]))
    np.testing.assert_allclose(nn.detector_features(I, counts=-1, gain=2.0)[1, 4, 8],
                               2 * np.log1p(I[1, 0, 0] ** 2))


def test_rasterize_boxes_by_loops():
    boxes = np.array([[[0, 2, 1, 3, 0, 1], [3, 4, 0, 1, 2, 4]], [[0, 0, 0, 0, 0, 0], [1, 4, 2, 3, 0, 4]]])
    out = nn.rasterize_boxes(boxes, (4, 3, 4), 0.5)
    for s in range(2):
        for i in range(4):
            for j in range(3):
                for k in range(4):
                    inside = any(b[0] <= i < b[1] and b[2] <= j < b[3] and b[4] <= k < b[5] for b in boxes[s])
                    assert out[s, i, j, k] == (0.5 if inside else 0.0)
