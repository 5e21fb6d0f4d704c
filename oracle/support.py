"""Oracle of the shrink-wrap support update (Sec. 4.2: every twenty epochs a
shrink-wrap support, after Marchesini et al. 2003, which also acts as a
nearest-neighbour filter between material and air).

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle``.

On a coarse parameter grid theta[cx][cz][cy]:
  1. blur theta with a normalised Gaussian of width sigma (in coarse voxels),
     separably along y, then z, then x, with taps t = -r..r,
     r = floor(3 sigma + 0.5), and zero outside the grid;
  2. the support is where the blur is at least threshold * its maximum;
  3. theta outside the support is set to 0 (air, or the host material of a
     buried pattern).

The support is an integer decision taken from floating point, so this oracle
takes it in the same precision as the CUDA kernel: FP32 weights (formed in
double, normalised, rounded once), FP32 products and sums, each rounded on
its own, in tap order.  `blur64` is the same blur in double, for the pin
against a library Gaussian filter.
"""
from __future__ import annotations

import numpy as np


def taps(sigma):
    """Normalised Gaussian weights for t = -r..r (double): libm exp and a sum
    in tap order, so that the FP32 weights come out as the library's do."""
    import math
    r = int(math.floor(3.0 * sigma + 0.5))
    w = [math.exp(-float(t * t) / (2.0 * sigma * sigma)) for t in range(-r, r + 1)]
    total = 0.0
    for x in w:
        total += x
    return np.array([x / total for x in w])


def _shift(a, t, axis):
    """out[i] = a[i + t] along axis, 0 where i + t is outside."""
    out = np.zeros_like(a)
    n = a.shape[axis]
    if abs(t) >= n:
        return out
    src = [slice(None)] * a.ndim
    dst = [slice(None)] * a.ndim
    src[axis] = slice(max(t, 0), n + min(t, 0))
    dst[axis] = slice(max(-t, 0), n - max(t, 0))
    out[tuple(dst)] = a[tuple(src)]
    return out


def _blur(a, w, dtype):
    r = (len(w) - 1) // 2
    wd = w.astype(dtype)
    for axis in (2, 1, 0):
        acc = np.zeros_like(a)
        for k, t in enumerate(range(-r, r + 1)):
            acc = acc + wd[k] * _shift(a, t, axis)
        a = acc
    return a


def blur(theta, sigma):
    """The FP32 blur of step 1, rounded as the kernel rounds it."""
    return _blur(np.asarray(theta, dtype=np.float32), taps(sigma), np.float32)


def blur64(theta, sigma):
    return _blur(np.asarray(theta, dtype=np.float64), taps(sigma), np.float64)


def shrinkwrap(theta, sigma, threshold):
    """(theta with zeros outside the support, support mask)."""
    theta = np.asarray(theta, dtype=np.float32)
    b = blur(theta, sigma)
    thr = np.float32(threshold) * b.max()
    mask = b >= thr
    return np.where(mask, theta, np.float32(0)), mask
