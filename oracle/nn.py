"""FP64 oracle of the learned initialiser's network (numpy).

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``: imported by ``tests/``
and by ``bench.py``'s CPU legs, never by the product package, and sharing no
code with it.

The paper has no network: its reconstructions start from a guessed structure
(Sec. 4.1 starts from bare silicon, Sec. 4.2 from AFM-derived rectangles).  The
learned initialiser proposes that starting volume from the detector image.
What it computes is plain textbook algebra, written out here without any
blocking or fusion:

* a dense layer is z = x W^T + b with the operands x and W rounded to BF16
  (8 significant bits, round to nearest, ties to even) and the products summed
  exactly (FP64 stands in for the FP32 accumulator);
* a convolution whose kernel equals its stride p is that dense layer applied
  to non-overlapping p x p patches (``space_to_depth``), and its transpose is
  the dense layer followed by the inverse patch permutation;
* ReLU on hidden layers, a logistic sigmoid scaled by ``hi`` on the output,
  and the mean squared error against the target volume;
* gradients by the chain rule (no autograd), checked against central
  differences in ``tests/test_oracle_pins.py``.

Layouts follow the C ABI: activations NHWC, weights W[n_out][k_in], and all
parameters in one flat vector, layer by layer, W then b.
"""
from __future__ import annotations

import numpy as np


# --- BF16 rounding -------------------------------------------------------------

def bf16_round(x):
    """Nearest value with an 8-bit significand (BF16), ties to even, of the
    FP32 value of x; zeros stay zeros.  Computed from the definition: split
    x = m 2^e with 0.5 <= |m| < 1, round m 2^8 to an integer (half to even),
    scale back.  BF16 has FP32's exponent range, so no subnormal case arises
    for the magnitudes used here (> 1e-30)."""
    x32 = np.asarray(x, dtype=np.float32).astype(np.float64)
    m, e = np.frexp(x32)
    return np.ldexp(np.round(m * 256.0), e - 8)


def _rnd(x, rounding):
    return bf16_round(x) if rounding else np.asarray(x, np.float64)


def dense(x, w, b=None, rounding=True):
    """z[m][n] = sum_k x[m][k] w[n][k] (+ b[n]) on BF16-rounded x and w."""
    z = _rnd(x, rounding) @ _rnd(w, rounding).T
    return z if b is None else z + np.asarray(b, np.float64)


# --- patch permutation ---------------------------------------------------------

def space_to_depth(x, p):
    """NHWC [B][H][W][C] -> [B][H/p][W/p][p][p][C]: the p x p patch of output
    position (i, j) is rows p i + di, columns p j + dj of the input."""
    B, H, W, C = x.shape
    return x.reshape(B, H // p, p, W // p, p, C).transpose(0, 1, 3, 2, 4, 5).copy()


def depth_to_space(y, p):
    """Inverse of space_to_depth: [B][h][w][p][p][C] -> [B][h p][w p][C]."""
    B, h, w, _, _, C = y.shape
    return y.transpose(0, 1, 3, 2, 4, 5).reshape(B, h * p, w * p, C).copy()


# --- network input and training targets ------------------------------------------

def detector_features(intensity, noise=None, counts=1e6, gain=1.0):
    """x = gain log(1 + a^2) with a = sqrt(s I) (+ 0.5 noise, clamped at 0),
    s = counts / sum(I) per image (s = 1 for counts == 0; for counts < 0 the
    input is the amplitude a itself), centred with fftshift.
    intensity [nimg][nz][ny]."""
    I = np.asarray(intensity, np.float64)
    out = np.empty_like(I)
    for i in range(I.shape[0]):
        if counts < 0:
            a = I[i].copy()
        else:
            s = counts / I[i].sum() if counts > 0 else 1.0
            a = np.sqrt(s * I[i])
        if noise is not None:
            a = np.maximum(a + 0.5 * np.asarray(noise[i], np.float64), 0.0)
        out[i] = gain * np.fft.fftshift(np.log1p(a * a))
    return out


def rasterize_boxes(boxes, shape, value):
    """out[s] = value inside any half-open box (lo0, hi0, lo1, hi1, lo2, hi2) of sample s."""
    boxes = np.asarray(boxes)
    out = np.zeros((boxes.shape[0],) + tuple(shape), np.float64)
    for s in range(boxes.shape[0]):
        for b in boxes[s]:
            out[s, b[0]:b[1], b[2]:b[3], b[4]:b[5]] = value
    return out


def sigmoid_mse(z, target, hi):
    """y = hi sigmoid(z); loss = mean((y - t)^2); dz = dloss/dz."""
    z = np.asarray(z, np.float64)
    s = 1.0 / (1.0 + np.exp(-z))
    y = hi * s
    d = y - np.asarray(target, np.float64)
    loss = np.mean(d * d)
    dz = 2.0 * d / d.size * hi * s * (1.0 - s)
    return y, loss, dz


# --- the encoder-decoder ---------------------------------------------------------

def layer_table(arch):
    """Layers of the network described by ``arch`` (a dict):

    in_hw   detector side (square image, one channel)
    enc     [(p, c_out), ...] patch convolutions down to an 8 x 8 map
    latent  width of the dense bottleneck
    dec_c0  channels of the 8 x 8 map the bottleneck expands to
    dec     [(p, c_out), ...] transposed patch convolutions; the last c_out is
            the output depth, the output map side is 8 * prod(p)

    Returns dicts with kind ('enc', 'dense', 'dec'), K (inputs), N (outputs),
    p, the input map side, channel counts and whether ReLU follows.
    """
    layers = []
    h, c = arch["in_hw"], 1
    for p, co in arch["enc"]:
        layers.append(dict(kind="enc", p=p, hin=h, cin=c, K=p * p * c, N=co, relu=True))
        h, c = h // p, co
    assert h == 8, "encoder must end on an 8 x 8 map"
    layers.append(dict(kind="dense", K=h * h * c, N=arch["latent"], relu=True, to_map=False))
    layers.append(dict(kind="dense", K=arch["latent"], N=64 * arch["dec_c0"], relu=True, to_map=True))
    h, c = 8, arch["dec_c0"]
    for i, (p, co) in enumerate(arch["dec"]):
        last = i == len(arch["dec"]) - 1
        layers.append(dict(kind="dec", p=p, hin=h, cin=c, K=c, N=p * p * co, cout=co, relu=not last))
        h, c = h * p, co
    if not arch["dec"]:
        layers[-1]["relu"] = False
    return layers


def n_params(arch):
    return sum(L["N"] * L["K"] + L["N"] for L in layer_table(arch))


def unpack(arch, theta):
    out, o = [], 0
    for L in layer_table(arch):
        w = np.asarray(theta[o:o + L["N"] * L["K"]], np.float64).reshape(L["N"], L["K"])
        o += L["N"] * L["K"]
        b = np.asarray(theta[o:o + L["N"]], np.float64)
        o += L["N"]
        out.append((w, b))
    return out


def forward(arch, theta, x, rounding=True):
    """x [B][H][W] features -> (pre-sigmoid output [B][side][side][depth], cache)."""
    B = x.shape[0]
    a = np.asarray(x, np.float64).reshape(B, x.shape[1], x.shape[2], 1)
    cache = []
    for L, (w, b) in zip(layer_table(arch), unpack(arch, theta)):
        if L["kind"] == "enc":
            X = space_to_depth(a, L["p"]).reshape(-1, L["K"])
        elif L["kind"] == "dense":
            X = a.reshape(B, -1)
        else:
            X = a.reshape(-1, L["K"])
        Z = dense(X, w, b, rounding)
        Y = np.maximum(Z, 0.0) if L["relu"] else Z
        cache.append((X, Y))
        if L["kind"] == "enc":
            h = L["hin"] // L["p"]
            a = Y.reshape(B, h, h, L["N"])
        elif L["kind"] == "dense":
            a = Y.reshape(B, 8, 8, -1) if L["to_map"] else Y
        else:
            h, p = L["hin"], L["p"]
            a = depth_to_space(Y.reshape(B, h, h, p, p, L["cout"]), p)
    return a, cache


def backward(arch, theta, cache, dout, rounding=True):
    """Gradient of a scalar loss with respect to the flat parameters, given
    dloss/d(pre-sigmoid output) ``dout`` [B][side][side][depth]."""
    layers = layer_table(arch)
    params = unpack(arch, theta)
    B = dout.shape[0]
    grads = [None] * len(layers)
    da = np.asarray(dout, np.float64)
    for li in range(len(layers) - 1, -1, -1):
        L, (w, _), (X, Y) = layers[li], params[li], cache[li]
        if L["kind"] == "dec":
            p, h = L["p"], L["hin"]
            dY = space_to_depth(da.reshape(B, h * p, h * p, L["cout"]), p).reshape(-1, L["N"])
        else:
            dY = da.reshape(Y.shape)
        dZ = dY * (Y > 0) if L["relu"] else dY
        dW = _rnd(dZ, rounding).T @ _rnd(X, rounding)
        db = _rnd(dZ, rounding).sum(axis=0)
        grads[li] = (dW, db)
        dX = _rnd(dZ, rounding) @ _rnd(w, rounding)
        if L["kind"] == "enc":
            hp = L["hin"] // L["p"]
            da = depth_to_space(dX.reshape(B, hp, hp, L["p"], L["p"], L["cin"]), L["p"])
        else:
            da = dX
    return np.concatenate([np.concatenate([g[0].ravel(), g[1]]) for g in grads])


def loss_and_grad(arch, theta, x, target, hi=1.0, rounding=True):
    """MSE of hi sigmoid(net(x)) against target [B][side][side][depth]: (loss, grad, y)."""
    z, cache = forward(arch, theta, x, rounding)
    y, loss, dz = sigmoid_mse(z, np.asarray(target, np.float64).reshape(z.shape), hi)
    return loss, backward(arch, theta, cache, dz, rounding), y
