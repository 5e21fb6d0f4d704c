"""FP64 CPU oracle for the reflection-geometry multislice model (arxiv 2212.01253).

TEST INFRASTRUCTURE ONLY.  This package is imported by ``tests/``, by
``__graft_entry__.smoke()`` and by the CPU-baseline / reference leg of
``bench.py``; the product package never imports it and it never imports the
product package.  It shares no code with the CUDA path.

The numerical work lives in ``mslice_oracle.c`` (plain C99 + OpenMP, double
precision, own DFT/FFT); this module compiles it with gcc on first use and
wraps it with ctypes.  Every entry point follows the steps written out in the
C file's header:

* Eq. 1 (Sec. 1): transmission exp(-i k Delta (delta - i beta)) then the
  paraxial Fresnel propagator exp(-i Delta (k_y^2 + k_z^2) / 2k) in Fourier
  space, slice after slice.
* Fig. 1a: the last exit wave is Fourier transformed and squared.
* Eq. 4 (Sec. 4.1): squared error of amplitudes, here summed (no 1/N).
* The gradient is the exact adjoint of those steps (the paper used autograd).

Parity is pinned by ``tests/test_oracle_pins.py`` (closed forms, physics,
brute force, finite differences); no oracle function is "parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mslice_oracle.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "libmslice_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle shared library (gcc, -O2, OpenMP, IEEE math)."""
    os.makedirs(_BUILD_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-std=c11", "-O2", "-fopenmp", "-fPIC", "-shared", "-Wall",
           "-o", tmp, _SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class OrcParams(ctypes.Structure):
    _fields_ = [
        ("wavelength_nm", ctypes.c_double),
        ("slice_nm", ctypes.c_double),
        ("dy_nm", ctypes.c_double),
        ("dz_nm", ctypes.c_double),
        ("ny", ctypes.c_int32),
        ("nz", ctypes.c_int32),
        ("ns", ctypes.c_int32),
        ("nw", ctypes.c_int32),
        ("alpha_i_rad", ctypes.POINTER(ctypes.c_double)),
        ("force_naive_dft", ctypes.c_int32),
        ("exit_wave", ctypes.c_int32),
        ("exact", ctypes.c_int32),
        ("psi_rad", ctypes.POINTER(ctypes.c_double)),
        ("strang", ctypes.c_int32),
        ("angular", ctypes.c_int32),
    ]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            vp, dp = ctypes.c_void_p, ctypes.POINTER(OrcParams)
            lib.orc_forward.argtypes = [dp, vp, vp, vp, vp]
            lib.orc_adjoint.argtypes = [dp, vp, vp, vp, vp]
            lib.orc_loss_grad.argtypes = [dp, vp, vp, vp, ctypes.c_double, vp, vp, vp]
            lib.orc_propagator_1d.argtypes = [dp, vp, vp]
            lib.orc_dft1d.argtypes = [ctypes.c_int, vp, ctypes.c_int, ctypes.c_int]
            lib.orc_dft2d.argtypes = [ctypes.c_int, ctypes.c_int, vp, ctypes.c_int, ctypes.c_int]
            for f in ("orc_forward", "orc_adjoint", "orc_loss_grad", "orc_propagator_1d",
                      "orc_dft1d", "orc_dft2d", "orc_num_threads"):
                getattr(lib, f).restype = ctypes.c_int
            _lib = lib
    return _lib


def num_threads() -> int:
    """OpenMP threads the oracle runs with."""
    return int(_load().orc_num_threads())


class Geometry:
    """Grid and beam: lambda, Delta, dy, dz, (Ny, Nz, Ns) and the incidence angles."""

    def __init__(self, ny, nz, ns, wavelength_nm=0.155, slice_nm=20.0, dy_nm=2.0,
                 dz_nm=2.0, alpha_i_deg=(0.3,), exact_transmission=False, psi_deg=0.0, strang=False,
                 angular=False):
        self.ny, self.nz, self.ns = int(ny), int(nz), int(ns)
        # symmetric splitting: half a step of propagation before the first
        # slice (and after the last, for the exit wave)
        self.strang = bool(strang)
        # angular-spectrum propagator exp(i Delta (sqrt(k^2 - k_perp^2) - k))
        # instead of the paraxial Fresnel one
        self.angular = bool(angular)
        # exact 1 - n^2 in the transmission of Eq. 1 instead of 2 (delta - i beta)
        self.exact_transmission = bool(exact_transmission)
        # in-plane angle of each view's default probe (one value for all views,
        # or one per incidence angle)
        self.psi_rad_w = np.deg2rad(np.broadcast_to(np.asarray(psi_deg, dtype=np.float64),
                                                    np.atleast_1d(np.asarray(alpha_i_deg)).shape)).copy()
        self.wavelength_nm = float(wavelength_nm)
        self.slice_nm = float(slice_nm)
        self.dy_nm, self.dz_nm = float(dy_nm), float(dz_nm)
        self.alpha_i_rad = np.deg2rad(np.atleast_1d(np.asarray(alpha_i_deg, dtype=np.float64)))

    @property
    def nw(self):
        return int(self.alpha_i_rad.size)

    @property
    def psi_rad(self):
        """The in-plane angle when all views share one, else the per-view array."""
        return float(self.psi_rad_w[0]) if np.all(self.psi_rad_w == self.psi_rad_w[0]) else self.psi_rad_w

    def _params(self, naive=False, exit_wave=False):
        self._alpha_keep = np.ascontiguousarray(self.alpha_i_rad, dtype=np.float64)
        self._psi_keep = np.ascontiguousarray(self.psi_rad_w, dtype=np.float64)
        return OrcParams(self.wavelength_nm, self.slice_nm, self.dy_nm, self.dz_nm,
                         self.ny, self.nz, self.ns, self.nw,
                         self._alpha_keep.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                         int(bool(naive)), int(bool(exit_wave)), int(self.exact_transmission),
                         self._psi_keep.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                         int(self.strang), int(self.angular))


def _c128(a, shape):
    a = np.ascontiguousarray(a, dtype=np.complex128)
    if a.shape != tuple(shape):
        raise ValueError("expected shape %s, got %s" % (shape, a.shape))
    return a


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _rc(rc, name):
    if rc != 0:
        raise RuntimeError("%s failed with code %d" % (name, rc))


def forward(geo: Geometry, vol, probe=None, naive=False, exit_wave=False, return_field=False):
    """Detector intensity I [nw][nz][ny] (and Psi, or phi_Ns with exit_wave)."""
    vol = _c128(vol, (geo.ns, geo.nz, geo.ny))
    if probe is not None:
        probe = _c128(probe, (geo.nw, geo.nz, geo.ny))
    shape = (geo.nw, geo.nz, geo.ny)
    inten = np.zeros(shape, np.float64)
    field = np.zeros(shape, np.complex128) if (return_field or exit_wave) else None
    p = geo._params(naive, exit_wave)
    _rc(_load().orc_forward(ctypes.byref(p), _ptr(vol), _ptr(probe), _ptr(inten), _ptr(field)),
        "orc_forward")
    if exit_wave:
        return field
    return (inten, field) if return_field else inten


def adjoint(geo: Geometry, vol, g_psi, probe=None, naive=False):
    """grad = dL/ddelta + i dL/dbeta [ns][nz][ny] for a detector gradient g_psi."""
    vol = _c128(vol, (geo.ns, geo.nz, geo.ny))
    g_psi = _c128(g_psi, (geo.nw, geo.nz, geo.ny))
    if probe is not None:
        probe = _c128(probe, (geo.nw, geo.nz, geo.ny))
    grad = np.zeros((geo.ns, geo.nz, geo.ny), np.complex128)
    p = geo._params(naive)
    _rc(_load().orc_adjoint(ctypes.byref(p), _ptr(vol), _ptr(probe), _ptr(g_psi), _ptr(grad)),
        "orc_adjoint")
    return grad


def loss_grad(geo: Geometry, vol, meas_amp, scale, probe=None, naive=False,
              return_intensity=False):
    """(L, grad) with L = sum (sqrt(scale I) - meas_amp)^2, grad as in adjoint()."""
    vol = _c128(vol, (geo.ns, geo.nz, geo.ny))
    meas_amp = np.ascontiguousarray(meas_amp, dtype=np.float64)
    if meas_amp.shape != (geo.nw, geo.nz, geo.ny):
        raise ValueError("meas_amp shape %s" % (meas_amp.shape,))
    if probe is not None:
        probe = _c128(probe, (geo.nw, geo.nz, geo.ny))
    grad = np.zeros((geo.ns, geo.nz, geo.ny), np.complex128)
    inten = np.zeros((geo.nw, geo.nz, geo.ny), np.float64)
    loss = ctypes.c_double(0.0)
    p = geo._params(naive)
    _rc(_load().orc_loss_grad(ctypes.byref(p), _ptr(vol), _ptr(probe), _ptr(meas_amp),
                              float(scale), ctypes.cast(ctypes.byref(loss), ctypes.c_void_p),
                              _ptr(grad), _ptr(inten)), "orc_loss_grad")
    if return_intensity:
        return loss.value, grad, inten
    return loss.value, grad


def propagator_1d(geo: Geometry):
    """(P_y [ny], P_z [nz]) with P = exp(-i Delta k^2 / 2k)."""
    py = np.zeros(geo.ny, np.complex128)
    pz = np.zeros(geo.nz, np.complex128)
    p = geo._params()
    _rc(_load().orc_propagator_1d(ctypes.byref(p), _ptr(py), _ptr(pz)), "orc_propagator_1d")
    return py, pz


def dft1d(x, sign=-1, naive=False):
    """Unnormalised 1-D DFT with kernel exp(sign * 2 pi i m k / n)."""
    x = np.array(x, dtype=np.complex128, copy=True)
    _rc(_load().orc_dft1d(x.size, _ptr(x), int(sign), int(bool(naive))), "orc_dft1d")
    return x


def dft2d(x, sign=-1, naive=False):
    """Unnormalised 2-D DFT of x[nz][ny]."""
    x = np.array(x, dtype=np.complex128, copy=True)
    nz, ny = x.shape
    _rc(_load().orc_dft2d(ny, nz, _ptr(x), int(sign), int(bool(naive))), "orc_dft2d")
    return x


# ---------------------------------------------------------------------------
# Reconstruction helpers (Sec. 4): coarse reconstruction voxels on the fine
# multislice grid, and the ADAM update the paper optimises them with.
# Plain numpy in double precision; definitions written out.
# ---------------------------------------------------------------------------
def coarse_to_fine(theta, fine_shape, block, offset=(0, 0, 0), beta_ratio=4.9e-6 / 4.7e-5, base=None,
                   block_index=0j):
    """E: theta[cx][cz][cy] -> volume [ns][nz][ny]; every fine voxel of a coarse
    block gets delta = Re(block_index) + theta and beta = Im(block_index) +
    beta_ratio * theta (block_index: the index at theta = 0, e.g. the host
    material of buried inclusions); voxels outside the blocks keep ``base``."""
    theta = np.asarray(theta, dtype=np.float64)
    vol = np.zeros(fine_shape, np.complex128) if base is None else np.array(base, np.complex128)
    cx, cz, cy = theta.shape
    bx, bz, by = block
    x0, z0, y0 = offset
    for a in range(cx):
        for b in range(cz):
            for c in range(cy):
                d = theta[a, b, c]
                vol[x0 + a * bx:x0 + (a + 1) * bx, z0 + b * bz:z0 + (b + 1) * bz,
                    y0 + c * by:y0 + (c + 1) * by] = complex(block_index) + d + 1j * beta_ratio * d
    return vol


def fine_to_coarse(grad, coarse_shape, block, offset=(0, 0, 0), beta_ratio=4.9e-6 / 4.7e-5):
    """E^T: sum of dL/ddelta + beta_ratio dL/dbeta over each coarse block."""
    grad = np.asarray(grad, dtype=np.complex128)
    cx, cz, cy = coarse_shape
    bx, bz, by = block
    x0, z0, y0 = offset
    g = np.zeros(coarse_shape, np.float64)
    for a in range(cx):
        for b in range(cz):
            for c in range(cy):
                blk = grad[x0 + a * bx:x0 + (a + 1) * bx, z0 + b * bz:z0 + (b + 1) * bz,
                           y0 + c * by:y0 + (c + 1) * by]
                g[a, b, c] = (blk.real + beta_ratio * blk.imag).sum()
    return g


def snap(theta, levels):
    """Material snapping (Sec. 4.1): each parameter becomes the nearest level,
    the lower one when two are equally near."""
    theta = np.asarray(theta, dtype=np.float64)
    lv = np.sort(np.asarray(levels, dtype=np.float64))
    d = np.abs(theta[..., None] - lv)            # argmin takes the first (lowest) level on a tie
    return lv[np.argmin(d, axis=-1)]


def adam_step(theta, m, v, grad, lr, b1, b2, eps, t, lo=-np.inf, hi=np.inf):
    """One ADAM step (Kingma & Ba): returns new (theta, m, v)."""
    m = b1 * m + (1 - b1) * grad
    v = b2 * v + (1 - b2) * grad * grad
    mhat = m / (1 - b1 ** t)
    vhat = v / (1 - b2 ** t)
    theta = np.clip(theta - lr * mhat / (np.sqrt(vhat) + eps), lo, hi)
    return theta, m, v
