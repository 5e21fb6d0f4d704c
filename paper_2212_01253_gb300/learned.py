"""Learned initialiser: a patch-convolution encoder-decoder that maps a
detector image to a coarse delta volume, the starting point of the gradient
reconstruction (``recon.Reconstructor``).

The paper starts its reconstructions from a guess (bare silicon in Sec. 4.1,
AFM-derived rectangles in Sec. 4.2) and has no network; this module replaces
the guess by a prediction.  Training pairs (detector image, coarse volume) come
from the forward model itself: random Au pillar layouts are rasterised on the
coarse grid, mapped onto the multislice grid (E), pushed through
``mslice_forward`` in per-structure batches, and turned into network inputs
with Poisson-amplitude noise.  Every step runs in libmslice kernels:

* layers: ``mslice_nn_space_to_depth`` (patch permutation) + a GEMM with BF16
  operands and FP32 accumulation, fused bias and ReLU: the forward and the
  input gradient of dense enough layers (``_use_tc``) run on the tcgen05
  tensor cores (``mslice_nn_gemm_bf16``, activations packed to BF16
  by ``mslice_nn_pack_bf16``, weights from BF16 copies refreshed after every
  ADAM step); the rest, and the weight gradients (long k, split over CTAs),
  run ``mslice_nn_gemm``;
* loss: ``mslice_nn_sigmoid_mse``; backward: the same GEMM with transposed
  strides, ``mslice_nn_relu_backward``; optimiser: ``mslice_adam_step`` over
  the flat FP32 master parameters (FP32 is the master copy; the GEMMs read
  weights rounded to BF16, nearest even, either way).

Architecture (``arch`` dict): ``in_hw`` detector side; ``enc`` list of
(p, c_out) patch convolutions (kernel = stride = p, ReLU) down to an 8 x 8 map;
a dense bottleneck of width ``latent`` and a dense expansion to an 8 x 8 x
``dec_c0`` map (both ReLU); ``dec`` list of (p, c_out) transposed patch
convolutions (ReLU except the last).  The output map (side 8 * prod p, depth
the last c_out) is read as theta[cx][cz][cy]: map rows = coarse x (along the
beam), map columns = coarse z (height), channels = coarse y.  Parameters are
one flat vector, layer by layer, W[n_out][k_in] then b[n_out].
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import binding as B

AU_DELTA = 4.7e-5
AU_BETA = 4.9e-6

# ~4.5M parameters: 256^2 detector -> 64^3 coarse volume
ARCH_256 = dict(in_hw=256, enc=[(4, 32), (2, 64), (2, 128), (2, 256)], latent=128, dec_c0=256,
                dec=[(2, 64), (2, 32), (2, 64)])


# GEMMs with at least this many rows, this long a reduction and this many
# output columns use the tcgen05 path (128 x 256 tiles); thinner ones are
# bound by memory, where packing the activations to BF16 costs more than the
# tensor cores save (ARCH_256 at batch 64: 2.12 ms per step on mslice_nn_gemm,
# 2.34 ms with every layer of >= 1024 rows on the tcgen05 path)
TC_MIN_ROWS = 1024
TC_MIN_K = 256
TC_MIN_N = 128


def _use_tc(rows, n_out, k_red):
    return rows >= TC_MIN_ROWS and k_red >= TC_MIN_K and n_out >= TC_MIN_N


def _ld8(n):
    return (int(n) + 7) // 8 * 8


def layers_of(arch):
    """Per-layer shapes of ``arch`` (kind, p, map side in, channels, K, N, ReLU)."""
    out = []
    side, ch = int(arch["in_hw"]), 1
    for p, co in arch["enc"]:
        out.append(dict(kind="enc", p=p, side=side, cin=ch, K=p * p * ch, N=co, relu=True))
        side, ch = side // p, co
    if side != 8:
        raise ValueError("the encoder must reduce the detector to an 8 x 8 map")
    out.append(dict(kind="dense", side=8, cin=ch, K=64 * ch, N=arch["latent"], relu=True))
    out.append(dict(kind="dense", side=8, cin=arch["latent"], K=arch["latent"], N=64 * arch["dec_c0"],
                    relu=bool(arch["dec"])))
    side, ch = 8, arch["dec_c0"]
    for i, (p, co) in enumerate(arch["dec"]):
        out.append(dict(kind="dec", p=p, side=side, cin=ch, K=ch, N=p * p * co, cout=co,
                        relu=i < len(arch["dec"]) - 1))
        side, ch = side * p, co
    return out, side, ch


class EncoderDecoder:
    """Network state on one device: flat parameters, gradients, ADAM moments and
    the activation buffers of a batch of up to ``max_batch`` images."""

    def __init__(self, arch, max_batch, device=None, seed=0):
        self.arch = arch
        self.dev = torch.device(device or "cuda")
        self.layers, self.side, self.depth = layers_of(arch)
        self.max_batch = int(max_batch)
        self.n_params = sum(L["N"] * L["K"] + L["N"] for L in self.layers)
        f32 = dict(dtype=torch.float32, device=self.dev)
        self.theta = torch.zeros(self.n_params, **f32)
        self.grad = torch.zeros(self.n_params, **f32)
        self.m = torch.zeros(self.n_params, **f32)
        self.v = torch.zeros(self.n_params, **f32)
        self.t = 0
        o = 0
        gen = torch.Generator().manual_seed(seed)
        for L in self.layers:
            nw, nb = L["N"] * L["K"], L["N"]
            L["w"], L["b"] = self.theta[o:o + nw], self.theta[o + nw:o + nw + nb]
            L["gw"], L["gb"] = self.grad[o:o + nw], self.grad[o + nw:o + nw + nb]
            # He initialisation (random numbers drawn by torch, used as inputs)
            L["w"].copy_(torch.randn(nw, generator=gen) * math.sqrt(2.0 / L["K"]))
            o += nw + nb
        last = self.layers[-1]
        last["b"].fill_(-2.0)      # sigmoid(-2) ~ 0.12: a sparse volume before training
        Bm = self.max_batch
        self.ones = torch.ones(1, **f32)
        ws = 0
        for L in self.layers:
            L["M"] = self._rows(L, 1)
            rows = self._rows(L, Bm)
            # X: layer input in GEMM layout (own buffer for patch layers), Y: output
            L["X"] = torch.empty(rows * L["K"], **f32) if L["kind"] == "enc" else None
            L["Y"] = torch.empty(rows * L["N"], **f32)
            L["dY"] = torch.empty(rows * L["N"], **f32)
            L["dZ"] = torch.empty(rows * L["N"], **f32)
            L["dX"] = torch.empty(rows * L["K"], **f32)
            L["A"] = torch.empty(Bm * (L["side"] * L["p"]) ** 2 * L["cout"], **f32) if L["kind"] == "dec" else None
            ws = max(ws, B.mslice_nn_gemm_workspace(rows, L["N"], L["K"]),
                     B.mslice_nn_gemm_workspace(L["N"], L["K"], rows),
                     B.mslice_nn_gemm_workspace(1, L["N"], rows),
                     B.mslice_nn_gemm_workspace(rows, L["K"], L["N"]))
        # BF16 operands of the tcgen05 path: weights W [N][K] and W^T [K][N]
        # (refreshed after every ADAM step), and per-call activation packs
        bf = dict(dtype=torch.bfloat16, device=self.dev)
        pack = 8
        for L in self.layers:
            rows = self._rows(L, Bm)
            L["ldK"], L["ldN"] = _ld8(L["K"]), _ld8(L["N"])
            L["w16"] = torch.empty(L["N"] * L["ldK"], **bf)
            L["w16t"] = torch.empty(L["K"] * L["ldN"], **bf)
            pack = max(pack, rows * max(L["ldK"], L["ldN"]))
        self.pack16 = torch.empty(pack, **bf)
        self.refresh_bf16()
        self.dA0 = torch.empty(Bm * arch["in_hw"] ** 2, **f32)
        self.ws = torch.empty(max(ws, 16) // 4 + 4, **f32)
        self.out_numel = self.side * self.side * self.depth
        self.y = torch.empty(Bm * self.out_numel, **f32)
        self.dz = torch.empty(Bm * self.out_numel, **f32)
        self.row_loss = torch.zeros(Bm, dtype=torch.float64, device=self.dev)

    @staticmethod
    def _rows(L, nb):
        if L["kind"] == "enc":
            return nb * (L["side"] // L["p"]) ** 2
        if L["kind"] == "dense":
            return nb
        return nb * L["side"] ** 2

    def _gemm(self, M, N, K, A, sam, sak, Bt, sbn, sbk, C, ldc, bias=None, relu=False):
        B.mslice_nn_gemm(M, N, K, A, sam, sak, Bt, sbn, sbk, C, ldc, bias, relu, 0.0, self.ws)

    def refresh_bf16(self):
        """BF16 copies of every layer's weights and their transposes (after
        ADAM steps this runs by itself; call it after writing theta directly)."""
        for L in self.layers:
            N, K = L["N"], L["K"]
            B.mslice_nn_pack_bf16(L["w"], K, 1, N, K, L["w16"], L["ldK"])
            B.mslice_nn_pack_bf16(L["w"], 1, K, K, N, L["w16t"], L["ldN"])

    def _gemm_w(self, M, N, K, X, W16, ldw, C, bias=None, relu=False):
        """C[M][N] = X[M][K] W^T (+ bias) (ReLU): X float32 row-major, W16 the
        layer's BF16 copy [N][ldw], on the tcgen05 tensor cores."""
        ldx = _ld8(K)
        X16 = self.pack16[:M * ldx]
        B.mslice_nn_pack_bf16(X, K, 1, M, K, X16, ldx)
        B.mslice_nn_gemm_bf16(M, N, K, X16, ldx, W16, ldw, C, N, bias, relu, 0.0)

    def forward(self, x, nb=None):
        """x: features [nb][in_hw][in_hw] (float32, contiguous) -> pre-sigmoid
        output [nb * side * side * depth] (a view of the last activation)."""
        nb = int(nb or x.shape[0])
        if nb > self.max_batch:
            raise ValueError("batch larger than max_batch")
        self._x, self._nb = x.reshape(-1), nb
        a = self._x
        for L in self.layers:
            rows = self._rows(L, nb)
            if L["kind"] == "enc":
                s = L["side"]
                X = L["X"][:rows * L["K"]]
                B.mslice_nn_space_to_depth(a[:nb * s * s * L["cin"]], X, nb, s, s, L["cin"], L["p"])
            else:
                X = a[:rows * L["K"]]
            L["Xin"] = X
            Y = L["Y"][:rows * L["N"]]
            if _use_tc(rows, L["N"], L["K"]):
                self._gemm_w(rows, L["N"], L["K"], X, L["w16"], L["ldK"], Y, L["b"], L["relu"])
            else:
                self._gemm(rows, L["N"], L["K"], X, L["K"], 1, L["w"], L["K"], 1, Y, L["N"], L["b"], L["relu"])
            if L["kind"] == "dec":
                so = L["side"] * L["p"]
                Aout = L["A"][:nb * so * so * L["cout"]]
                B.mslice_nn_space_to_depth(Y, Aout, nb, so, so, L["cout"], L["p"], inverse=True)
                a = Aout
            else:
                a = Y
        self._out = a
        return a

    def backward(self, dout):
        """Gradient of the loss into ``self.grad`` given dloss/d(pre-sigmoid output)."""
        nb = self._nb
        da = dout
        for li in range(len(self.layers) - 1, -1, -1):
            L = self.layers[li]
            rows = self._rows(L, nb)
            Y = L["Y"][:rows * L["N"]]
            if L["kind"] == "dec":
                so = L["side"] * L["p"]
                dY = L["dY"][:rows * L["N"]]
                B.mslice_nn_space_to_depth(da[:nb * so * so * L["cout"]], dY, nb, so, so, L["cout"], L["p"])
            else:
                dY = da[:rows * L["N"]]
            if L["relu"]:
                dZ = L["dZ"][:rows * L["N"]]
                B.mslice_nn_relu_backward(Y, dY, dZ)
            else:
                dZ = dY
            N, K = L["N"], L["K"]
            # dW[n][k] = sum_m dZ[m][n] X[m][k];  db[n] = sum_m dZ[m][n]
            self._gemm(N, K, rows, dZ, 1, N, L["Xin"], 1, K, L["gw"], K)
            self._gemm(1, N, rows, self.ones, 0, 0, dZ, 1, N, L["gb"], N)
            if li == 0:
                break
            # dX[m][k] = sum_n dZ[m][n] W[n][k]
            dX = L["dX"][:rows * K]
            if _use_tc(rows, K, N):
                self._gemm_w(rows, K, N, dZ, L["w16t"], L["ldN"], dX)
            else:
                self._gemm(rows, K, N, dZ, N, 1, L["w"], 1, K, dX, K)
            if L["kind"] == "enc":
                s, hp = L["side"], L["side"] // L["p"]
                dA = self.layers[li - 1]["dY"] if li > 0 else self.dA0
                dA = dA[:nb * s * s * L["cin"]]
                B.mslice_nn_space_to_depth(dX, dA, nb, s, s, L["cin"], L["p"], inverse=True)
                da = dA
            else:
                da = dX
        return self.grad

    def loss_grad(self, x, target, nb=None):
        """Forward, MSE of sigmoid(output) against the occupancy target
        [nb][cx][cz][cy] and backward; returns the per-sample loss (device FP64)."""
        nb = int(nb or x.shape[0])
        z = self.forward(x, nb)
        n = nb * self.out_numel
        B.mslice_nn_sigmoid_mse(z[:n], target.reshape(-1)[:n], self.y[:n], self.dz[:n], self.row_loss[:nb], nb,
                                self.out_numel, 1.0)
        self.backward(self.dz[:n])
        return self.row_loss[:nb]

    def adam(self, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
        self.t += 1
        B.mslice_adam_step(self.theta, self.m, self.v, self.grad, lr, b1, b2, eps, self.t, -3.0e38, 3.0e38)
        self.refresh_bf16()

    def predict(self, x, nb=None, hi=AU_DELTA):
        """Coarse volume theta = hi * sigmoid(net(x)), [nb][cx][cz][cy]."""
        nb = int(nb or x.shape[0])
        z = self.forward(x, nb)
        n = nb * self.out_numel
        y = torch.empty(n, dtype=torch.float32, device=self.dev)
        B.mslice_nn_sigmoid_mse(z[:n], None, y, None, None, nb, self.out_numel, hi)
        return y.view(nb, self.side, self.side, self.depth)


class PillarSampler:
    """Training pairs from the forward model: random Au pillars on Si.

    Each sample has ``n_pillars`` boxes in coarse units (cx, cz, cy): x
    extent and y extent uniform in ``foot`` (lengths), height uniform in
    ``height`` (coarse rows from the surface, which is coarse row 0 of the
    block).  The fine volume is the substrate ``base`` (Si below the surface)
    with the coarse block mapped on top (delta = Au delta times occupancy,
    beta in the Au ratio).  Intensities go through ``mslice_nn_detector_features``
    with ``counts`` expected photons and Poisson-amplitude noise."""

    def __init__(self, params, coarse, base, n_pillars=(4, 16), foot=(2, 9), height=(1, 9), counts=1e6,
                 chunk=16, gain=0.25, tune=False):
        self.p1 = params
        self.c = coarse
        self.shape = (coarse.cx, coarse.cz, coarse.cy)
        self.npill, self.foot, self.height = n_pillars, foot, height
        self.counts, self.gain = counts, gain
        ny, nz, ns = params.ny, params.nz, params.ns
        self.chunk = int(chunk)
        alphas = [math.degrees(params.alpha_i_rad[0])] * self.chunk
        self.pb = B.make_params(ny, nz, ns, alphas, wavelength_nm=params.wavelength_nm,
                                slice_nm=params.slice_nm, dy_nm=params.dy_nm, dz_nm=params.dz_nm,
                                flags=B.MSLICE_PER_STRUCTURE)
        dev = base.device
        if tune:
            from . import autotune
            autotune.apply(self.pb, dev)
        self.npx = ny * nz
        self.vols = base.reshape(1, ns, nz, ny).repeat(self.chunk, 1, 1, 1).contiguous()
        self.ws = B.workspace(self.pb, B.MSLICE_OP_FORWARD, dev)
        self.inten = torch.empty(self.chunk * self.npx, dtype=torch.float32, device=dev)
        self.dev = dev

    def boxes(self, rng, n):
        """int32 [n][max pillars][6] coarse boxes (unused slots are empty boxes)."""
        cx, cz, cy = self.shape
        nmax = self.npill[1]
        out = np.zeros((n, nmax, 6), np.int32)
        for s in range(n):
            k = rng.integers(self.npill[0], self.npill[1] + 1)
            for b in range(k):
                lx, ly = rng.integers(*self.foot, size=2)
                h = rng.integers(*self.height)
                x0, y0 = rng.integers(0, max(1, cx - lx + 1)), rng.integers(0, max(1, cy - ly + 1))
                out[s, b] = (x0, x0 + lx, 0, min(h, cz), y0, y0 + ly)
        return out

    def sample(self, rng, n, noise=True, gen=None):
        """(features [n][nz][ny], occupancy [n][cx][cz][cy], theta [n][cx][cz][cy]) on the device."""
        boxes = torch.from_numpy(self.boxes(rng, n)).to(self.dev)
        cx, cz, cy = self.shape
        occ = torch.empty(n * cx * cz * cy, dtype=torch.float32, device=self.dev)
        theta = torch.empty_like(occ)
        B.mslice_nn_rasterize_boxes(boxes, occ, self.shape, 1.0)
        B.mslice_nn_rasterize_boxes(boxes, theta, self.shape, AU_DELTA)
        feats = torch.empty(n * self.npx, dtype=torch.float32, device=self.dev)
        ncoarse = cx * cz * cy
        for s0 in range(0, n, self.chunk):
            k = min(self.chunk, n - s0)
            for w in range(k):
                B.mslice_coarse_to_fine(self.p1, self.c, theta[(s0 + w) * ncoarse:(s0 + w + 1) * ncoarse],
                                        self.vols[w])
            B.mslice_forward(self.pb, self.vols, None, self.inten, None, self.ws)
            nz_ = (torch.randn(k * self.npx, generator=gen, device=self.dev) if noise else None)
            B.mslice_nn_detector_features(self.inten[:k * self.npx], nz_, feats[s0 * self.npx:(s0 + k) * self.npx],
                                          k, self.p1.nz, self.p1.ny, self.counts, self.gain)
        return feats.view(n, self.p1.nz, self.p1.ny), occ.view(n, cx, cz, cy), theta.view(n, cx, cz, cy)

    def features_of(self, meas_amp):
        """Network input from a measured amplitude sqrt(counts) [nz][ny]."""
        x = torch.empty(self.npx, dtype=torch.float32, device=self.dev)
        B.mslice_nn_detector_features(meas_amp.reshape(-1).contiguous(), None, x, 1, self.p1.nz, self.p1.ny, -1.0,
                                      self.gain)
        return x.view(1, self.p1.nz, self.p1.ny)


def train(net, sampler, n_samples, batch, lr=1e-3, seed=1000, log_every=0):
    """Train on ``n_samples`` fresh forward-model samples (one pass, batches of
    ``batch``); returns the mean training loss of each batch (host list)."""
    rng = np.random.default_rng(seed)
    gen = torch.Generator(device=sampler.dev).manual_seed(seed)
    losses = []
    for i in range(0, n_samples, batch):
        nb = min(batch, n_samples - i)
        x, occ, _ = sampler.sample(rng, nb, gen=gen)
        rl = net.loss_grad(x, occ, nb)
        net.adam(lr)
        losses.append(rl.clone())
        if log_every and (i // batch) % log_every == 0:
            print("samples %d loss %.5f" % (i + nb, float(losses[-1].cpu().numpy().sum())), flush=True)
    return [float(v.sum()) for v in (t.cpu().numpy() for t in losses)]
