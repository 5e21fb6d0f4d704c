"""Python binding of libmslice (include/mslice.h): argument marshalling only.

Every function has the name of the C entry point it calls.  Arrays are torch
tensors on the current CUDA device (complex arrays as complex64); the call is
enqueued on torch's current stream.  All arithmetic runs in the library's
CUDA kernels; if the library is missing, loading fails with an error (there
is no CPU fallback).
"""
from __future__ import annotations

import ctypes
import math
import os
import threading

import torch

from . import build as _build

MSLICE_MAX_ANGLES = 64
MSLICE_OP_FORWARD, MSLICE_OP_ADJOINT, MSLICE_OP_LOSS_GRAD = 0, 1, 2
MSLICE_EXIT_WAVE = 1
MSLICE_PER_STRUCTURE = 2
MSLICE_EXACT_TRANSMISSION = 4
MSLICE_STRANG = 8
MSLICE_ANGULAR = 16
ERRORS = {-1: "MSLICE_EINVAL", -2: "MSLICE_EUNSUPPORTED", -3: "MSLICE_ELAUNCH",
          -4: "MSLICE_ETIMEDOUT", -5: "MSLICE_EWORKSPACE"}


class MsliceError(RuntimeError):
    def __init__(self, code, what):
        self.code = code
        msg = "%s failed: %s (%s)" % (what, ERRORS.get(code, code), mslice_strerror(code))
        if code == -3:
            msg += ": " + _load().mslice_last_cuda_error().decode()
        super().__init__(msg)


class mslice_params(ctypes.Structure):
    _fields_ = [
        ("wavelength_nm", ctypes.c_double),
        ("slice_nm", ctypes.c_double),
        ("dy_nm", ctypes.c_double),
        ("dz_nm", ctypes.c_double),
        ("ny", ctypes.c_int32),
        ("nz", ctypes.c_int32),
        ("ns", ctypes.c_int32),
        ("nw", ctypes.c_int32),
        ("alpha_i_rad", ctypes.c_double * MSLICE_MAX_ANGLES),
        ("psi_rad", ctypes.c_double * MSLICE_MAX_ANGLES),
        ("checkpoint_every", ctypes.c_int32),
        ("flags", ctypes.c_uint32),
        ("grid_blocks", ctypes.c_int32),
        ("col_width", ctypes.c_int32),
        ("schedule", ctypes.c_int32),
    ]


def make_params(ny, nz, ns, alpha_i_deg=(0.3,), wavelength_nm=0.155, slice_nm=20.0,
                dy_nm=2.0, dz_nm=2.0, checkpoint_every=32, flags=0, psi_rad=0.0, grid_blocks=0,
                col_width=0, schedule=0):
    """mslice_params from plain numbers (incidence angles in degrees; psi_rad, the
    in-plane angle in radians, one value for all wavefields or one per wavefield)."""
    alphas = [math.radians(float(a)) for a in (alpha_i_deg if hasattr(alpha_i_deg, "__len__")
                                               else [alpha_i_deg])]
    if not 1 <= len(alphas) <= MSLICE_MAX_ANGLES:
        raise ValueError("1..%d incidence angles" % MSLICE_MAX_ANGLES)
    p = mslice_params()
    p.wavelength_nm, p.slice_nm, p.dy_nm, p.dz_nm = wavelength_nm, slice_nm, dy_nm, dz_nm
    p.ny, p.nz, p.ns, p.nw = int(ny), int(nz), int(ns), len(alphas)
    for i, a in enumerate(alphas):
        p.alpha_i_rad[i] = a
    psis = list(psi_rad) if hasattr(psi_rad, "__len__") else [psi_rad] * len(alphas)
    if len(psis) != len(alphas):
        raise ValueError("one in-plane angle, or one per incidence angle")
    for i, v in enumerate(psis):
        p.psi_rad[i] = float(v)
    p.checkpoint_every = int(checkpoint_every)
    p.flags = int(flags)
    p.grid_blocks = int(grid_blocks)
    p.col_width = int(col_width)
    p.schedule = int(schedule)
    return p


class mslice_coarse(ctypes.Structure):
    _fields_ = [("cx", ctypes.c_int32), ("cz", ctypes.c_int32), ("cy", ctypes.c_int32),
                ("bx", ctypes.c_int32), ("bz", ctypes.c_int32), ("by", ctypes.c_int32),
                ("x0", ctypes.c_int32), ("z0", ctypes.c_int32), ("y0", ctypes.c_int32),
                ("beta_ratio", ctypes.c_float), ("base_delta", ctypes.c_float), ("base_beta", ctypes.c_float)]


def make_coarse(shape, block, offset=(0, 0, 0), beta_ratio=4.9e-6 / 4.7e-5, base=0j):
    """mslice_coarse for a coarse grid shape (cx, cz, cy), block (bx, bz, by), fine
    offset, d beta / d theta and the block's index at theta = 0 (``base``, complex)."""
    c = mslice_coarse()
    c.cx, c.cz, c.cy = (int(v) for v in shape)
    c.bx, c.bz, c.by = (int(v) for v in block)
    c.x0, c.z0, c.y0 = (int(v) for v in offset)
    c.beta_ratio = float(beta_ratio)
    c.base_delta, c.base_beta = float(complex(base).real), float(complex(base).imag)
    return c


class mslice_job(ctypes.Structure):
    _fields_ = [("ny", ctypes.c_int32), ("nz", ctypes.c_int32), ("ns", ctypes.c_int32),
                ("col_width", ctypes.c_int32), ("alpha_i_rad", ctypes.c_double), ("psi_rad", ctypes.c_double),
                ("scale", ctypes.c_float),
                ("reserved", ctypes.c_float), ("vol", ctypes.c_void_p), ("meas_amp", ctypes.c_void_p),
                ("grad_vol", ctypes.c_void_p), ("intensity", ctypes.c_void_p), ("loss_out", ctypes.c_void_p)]


def make_jobs(jobs):
    """A ctypes array of mslice_job from dicts with 'vol' (complex64 [ns][nz][ny]),
    'alpha_deg' and optionally 'meas' (float32 [nz][ny]), 'scale', 'grad'
    (complex64 like vol), 'intensity' (float32 [nz][ny]), 'loss' (float64 [1]),
    'col_width' -- CUDA tensors, kept alive by the caller."""
    arr = (mslice_job * len(jobs))()
    for i, jb in enumerate(jobs):
        ns, nz, ny = jb["vol"].shape
        j = arr[i]
        j.ny, j.nz, j.ns = int(ny), int(nz), int(ns)
        j.col_width = int(jb.get("col_width", 0))
        j.alpha_i_rad = math.radians(float(jb["alpha_deg"]))
        j.psi_rad = float(jb.get("psi_rad", 0.0))
        j.scale = float(jb.get("scale", 1.0))
        j.vol = _ptr(jb["vol"], torch.complex64, ns * nz * ny, "vol")
        j.meas_amp = _ptr(jb.get("meas"), torch.float32, nz * ny, "meas")
        j.grad_vol = _ptr(jb.get("grad"), torch.complex64, ns * nz * ny, "grad")
        j.intensity = _ptr(jb.get("intensity"), torch.float32, nz * ny, "intensity")
        j.loss_out = _ptr(jb.get("loss"), torch.float64, 1, "loss")
    return arr


class mslice_kernel_time(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("launches", ctypes.c_int32),
                ("total_ms", ctypes.c_double), ("units", ctypes.c_double)]


_lock = threading.Lock()
_lib = None


def _load():
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(_build.LIB):
                raise RuntimeError("libmslice.so is not built (%s); run "
                                   "paper_2212_01253_gb300.build.build()" % _build.LIB)
            lib = ctypes.CDLL(_build.LIB)
            P, vp, sz = ctypes.POINTER(mslice_params), ctypes.c_void_p, ctypes.c_size_t
            ll = ctypes.c_longlong
            sig = {
                "mslice_workspace_size": ([P, ctypes.c_int], sz),
                "mslice_forward": ([P, vp, vp, vp, vp, vp, sz, vp], ctypes.c_int),
                "mslice_forward_static": ([P, vp, vp, vp, vp, vp], ctypes.c_int),
                "mslice_forward_static_status": ([vp], ctypes.c_int),
                "mslice_adjoint": ([P, vp, vp, vp, vp, vp, sz, vp], ctypes.c_int),
                "mslice_loss_grad": ([P, vp, vp, vp, ctypes.c_float, vp, vp, vp, vp, sz, vp],
                                     ctypes.c_int),
                "mslice_plan_tables": ([P, vp, vp, vp, vp, sz, vp], ctypes.c_int),
                "mslice_loss_grad_multi": ([P, vp, vp, vp, vp, vp, vp, vp, vp, sz, vp], ctypes.c_int),
                "mslice_batched_workspace_size": ([P, vp, ctypes.c_int, ctypes.c_int, ctypes.c_int], sz),
                "mslice_loss_grad_batched": ([P, vp, ctypes.c_int, ctypes.c_int, vp, vp, sz, vp], ctypes.c_int),
                "mslice_forward_batched": ([P, vp, ctypes.c_int, ctypes.c_int, vp, sz, vp], ctypes.c_int),
                "mslice_batched_status": ([P, vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, vp, vp], ctypes.c_int),
                "mslice_batched_plan": ([P, vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, vp, vp, vp, vp],
                                        ctypes.c_int),
                "mslice_transmission": ([P, vp, vp, vp], ctypes.c_int),
                "mslice_status": ([vp, vp], ctypes.c_int),
                "mslice_intensity_vjp": ([vp, vp, vp, sz, vp], ctypes.c_int),
                "mslice_debug_wait": ([ctypes.c_int, ctypes.c_int, ctypes.c_longlong, vp, sz, vp],
                                      ctypes.c_int),
                "mslice_strerror": ([ctypes.c_int], ctypes.c_char_p),
                "mslice_last_cuda_error": ([], ctypes.c_char_p),
                "mslice_profile_enable": ([ctypes.c_int], ctypes.c_int),
                "mslice_coarse_to_fine": ([P, ctypes.POINTER(mslice_coarse), vp, vp, vp], ctypes.c_int),
                "mslice_fine_to_coarse": ([P, ctypes.POINTER(mslice_coarse), vp, vp, vp], ctypes.c_int),
                "mslice_snap": ([vp, sz, ctypes.POINTER(ctypes.c_float), ctypes.c_int, vp], ctypes.c_int),
                "mslice_shrinkwrap_workspace": ([sz], sz),
                "mslice_shrinkwrap": ([vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_float, ctypes.c_float,
                                       vp, vp, sz, vp], ctypes.c_int),
                "mslice_rotate": ([P, ctypes.c_double, ctypes.c_double, ctypes.POINTER(ctypes.c_double), vp, vp,
                                   vp], ctypes.c_int),
                "mslice_rotate_adjoint": ([P, ctypes.c_double, ctypes.c_double, ctypes.POINTER(ctypes.c_double),
                                           vp, vp, vp], ctypes.c_int),
                "mslice_adam_step": ([vp, vp, vp, vp, sz, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                                      ctypes.c_float, ctypes.c_int, ctypes.c_float, ctypes.c_float, vp],
                                     ctypes.c_int),
                "mslice_profile_read": ([ctypes.POINTER(mslice_kernel_time), ctypes.c_int],
                                        ctypes.c_int),
                "mslice_nn_gemm_workspace": ([ctypes.c_int] * 3, sz),
                "mslice_nn_gemm": ([ctypes.c_int] * 3 + [vp, ll, ll, vp, ll, ll, vp, ll, vp, ctypes.c_int,
                                                         ctypes.c_float, vp, sz, vp], ctypes.c_int),
                "mslice_nn_space_to_depth": ([vp, vp] + [ctypes.c_int] * 6 + [vp], ctypes.c_int),
                "mslice_nn_pack_bf16": ([vp, ll, ll, ctypes.c_int, ctypes.c_int, vp, ll, vp], ctypes.c_int),
                "mslice_nn_gemm_bf16": ([ctypes.c_int] * 3 + [vp, ll, vp, ll, vp, ll, vp, ctypes.c_int,
                                                              ctypes.c_float, vp], ctypes.c_int),
                "mslice_nn_gemm_bf16_status": ([vp], ctypes.c_int),
                "mslice_nn_relu_backward": ([vp, vp, vp, sz, vp], ctypes.c_int),
                "mslice_nn_sigmoid_mse": ([vp, vp, vp, vp, vp, ctypes.c_int, ctypes.c_int, ctypes.c_float, vp],
                                          ctypes.c_int),
                "mslice_nn_detector_features": ([vp, vp, vp, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                 ctypes.c_float, ctypes.c_float, vp], ctypes.c_int),
                "mslice_nn_rasterize_boxes": ([vp] + [ctypes.c_int] * 5 + [ctypes.c_float, vp, vp],
                                              ctypes.c_int),
            }
            for name, (args, res) in sig.items():
                f = getattr(lib, name)
                f.argtypes, f.restype = args, res
            _lib = lib
    return _lib


def library_path() -> str:
    return _build.LIB


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _ptr(t, dtype=None, numel=None, what="tensor"):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("%s must be a CUDA tensor" % what)
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % what)
    if dtype is not None and t.dtype != dtype:
        raise TypeError("%s must be %s, got %s" % (what, dtype, t.dtype))
    if numel is not None and t.numel() != numel:
        raise ValueError("%s must have %d elements, got %d" % (what, numel, t.numel()))
    return ctypes.c_void_p(t.data_ptr())


def _check(rc, what):
    if rc != 0:
        raise MsliceError(rc, what)


def mslice_strerror(code: int) -> str:
    return _load().mslice_strerror(int(code)).decode()


def mslice_workspace_size(p: mslice_params, op: int) -> int:
    n = _load().mslice_workspace_size(ctypes.byref(p), int(op))
    if n == 0:
        raise MsliceError(-1, "mslice_workspace_size")
    return int(n)


def workspace(p: mslice_params, op: int, device=None) -> torch.Tensor:
    """A workspace tensor of mslice_workspace_size(p, op) bytes."""
    return torch.empty(mslice_workspace_size(p, op), dtype=torch.uint8,
                       device=device or torch.device("cuda"))


def _sizes(p):
    npx = p.ny * p.nz
    nvol = p.ns * npx * (p.nw if p.flags & MSLICE_PER_STRUCTURE else 1)
    return nvol, p.nw * npx


def mslice_forward(p, vol, probe, intensity, field_out, ws, stream=None):
    nvol, nfield = _sizes(p)
    _check(_load().mslice_forward(
        ctypes.byref(p), _ptr(vol, torch.complex64, nvol, "vol"),
        _ptr(probe, torch.complex64, nfield, "probe"),
        _ptr(intensity, torch.float32, nfield, "intensity"),
        _ptr(field_out, torch.complex64, nfield, "field_out"),
        _ptr(ws, torch.uint8, None, "ws"), ws.numel(), _stream(stream)), "mslice_forward")


def mslice_forward_static(p, vol, probe, intensity, field_out, stream=None):
    """mslice_forward with the library's fixed 32 MiB device workspace (no allocation;
    overlapping calls race)."""
    nvol, nfield = _sizes(p)
    _check(_load().mslice_forward_static(
        ctypes.byref(p), _ptr(vol, torch.complex64, nvol, "vol"),
        _ptr(probe, torch.complex64, nfield, "probe"),
        _ptr(intensity, torch.float32, nfield, "intensity"),
        _ptr(field_out, torch.complex64, nfield, "field_out"), _stream(stream)), "mslice_forward_static")


def mslice_forward_static_status(stream=None) -> int:
    """0, or a negative code (-4 = MSLICE_ETIMEDOUT) recorded by a device-side
    wait of the last mslice_forward_static call on the current device."""
    return int(_load().mslice_forward_static_status(_stream(stream)))


def mslice_adjoint(p, vol, probe, g_psi, grad_vol, ws, stream=None):
    nvol, nfield = _sizes(p)
    _check(_load().mslice_adjoint(
        ctypes.byref(p), _ptr(vol, torch.complex64, nvol, "vol"),
        _ptr(probe, torch.complex64, nfield, "probe"),
        _ptr(g_psi, torch.complex64, nfield, "g_psi"),
        _ptr(grad_vol, torch.complex64, nvol, "grad_vol"),
        _ptr(ws, torch.uint8, None, "ws"), ws.numel(), _stream(stream)), "mslice_adjoint")


def mslice_loss_grad(p, vol, probe, meas_amp, scale, loss_out, grad_vol, intensity, ws, stream=None):
    nvol, nfield = _sizes(p)
    _check(_load().mslice_loss_grad(
        ctypes.byref(p), _ptr(vol, torch.complex64, nvol, "vol"),
        _ptr(probe, torch.complex64, nfield, "probe"),
        _ptr(meas_amp, torch.float32, nfield, "meas_amp"), ctypes.c_float(scale),
        _ptr(loss_out, torch.float64, 1, "loss_out"),
        _ptr(grad_vol, torch.complex64, nvol, "grad_vol"),
        _ptr(intensity, torch.float32, nfield, "intensity"),
        _ptr(ws, torch.uint8, None, "ws"), ws.numel(), _stream(stream)), "mslice_loss_grad")


def mslice_batched_workspace_size(common, jobs, op, lanes=1) -> int:
    """jobs: the ctypes array of make_jobs()."""
    n = _load().mslice_batched_workspace_size(ctypes.byref(common), ctypes.cast(jobs, ctypes.c_void_p), len(jobs),
                                              int(op), int(lanes))
    if n == 0:
        raise MsliceError(-1, "mslice_batched_workspace_size")
    return int(n)


def mslice_loss_grad_batched(common, jobs, lanes, loss_total, ws, stream=None):
    _check(_load().mslice_loss_grad_batched(
        ctypes.byref(common), ctypes.cast(jobs, ctypes.c_void_p), len(jobs), int(lanes),
        _ptr(loss_total, torch.float64, 1, "loss_total"), _ptr(ws, torch.uint8, None, "ws"), ws.numel(),
        _stream(stream)), "mslice_loss_grad_batched")


def mslice_forward_batched(common, jobs, lanes, ws, stream=None):
    _check(_load().mslice_forward_batched(
        ctypes.byref(common), ctypes.cast(jobs, ctypes.c_void_p), len(jobs), int(lanes),
        _ptr(ws, torch.uint8, None, "ws"), ws.numel(), _stream(stream)), "mslice_forward_batched")


def mslice_batched_plan(common, jobs, op, lanes=1, blocks=False):
    """(group of each job, lane of each group[, blocks of each group]) of a
    batched call (host only)."""
    n = len(jobs)
    gj, lg, bg, ng = (ctypes.c_int * n)(), (ctypes.c_int * n)(), (ctypes.c_int * n)(), ctypes.c_int(0)
    _check(_load().mslice_batched_plan(ctypes.byref(common), ctypes.cast(jobs, ctypes.c_void_p), n, int(op),
                                       int(lanes), ctypes.cast(gj, ctypes.c_void_p), ctypes.cast(lg, ctypes.c_void_p),
                                       ctypes.cast(bg, ctypes.c_void_p), ctypes.byref(ng)), "mslice_batched_plan")
    if blocks:
        return list(gj), list(lg)[:ng.value], list(bg)[:ng.value]
    return list(gj), list(lg)[:ng.value]


def mslice_batched_status(common, jobs, op, lanes, ws, stream=None) -> int:
    return int(_load().mslice_batched_status(ctypes.byref(common), ctypes.cast(jobs, ctypes.c_void_p), len(jobs),
                                             int(op), int(lanes), _ptr(ws, torch.uint8, None, "ws"),
                                             _stream(stream)))


def mslice_loss_grad_multi(p, vols, probe, meas_amp, scales, loss_out, grad_vol, intensity, ws, stream=None):
    """Loss (summed) and per-structure gradients of nw structures; p.flags must
    carry MSLICE_PER_STRUCTURE so that the array sizes are per structure."""
    if not p.flags & MSLICE_PER_STRUCTURE:
        raise ValueError("set MSLICE_PER_STRUCTURE in p.flags")
    nvol, nfield = _sizes(p)
    sc = (ctypes.c_float * p.nw)(*[float(x) for x in scales])
    _check(_load().mslice_loss_grad_multi(
        ctypes.byref(p), _ptr(vols, torch.complex64, nvol, "vols"),
        _ptr(probe, torch.complex64, nfield, "probe"),
        _ptr(meas_amp, torch.float32, nfield, "meas_amp"), ctypes.cast(sc, ctypes.c_void_p),
        _ptr(loss_out, torch.float64, 1, "loss_out"),
        _ptr(grad_vol, torch.complex64, nvol, "grad_vol"),
        _ptr(intensity, torch.float32, nfield, "intensity"),
        _ptr(ws, torch.uint8, None, "ws"), ws.numel(), _stream(stream)), "mslice_loss_grad_multi")


def mslice_plan_tables(p, py, pz, probe_z, ws, stream=None):
    _check(_load().mslice_plan_tables(
        ctypes.byref(p), _ptr(py, torch.complex64, p.ny, "py"),
        _ptr(pz, torch.complex64, p.nz, "pz"),
        _ptr(probe_z, torch.complex64, p.nw * p.nz, "probe_z"),
        _ptr(ws, torch.uint8, None, "ws"), ws.numel(), _stream(stream)), "mslice_plan_tables")


def mslice_transmission(p, vol, t_out, stream=None):
    nvol, _ = _sizes(p)
    _check(_load().mslice_transmission(
        ctypes.byref(p), _ptr(vol, torch.complex64, nvol, "vol"),
        _ptr(t_out, torch.complex64, nvol, "t_out"), _stream(stream)), "mslice_transmission")


def mslice_intensity_vjp(psi, dI, g_psi, stream=None):
    n = psi.numel()
    _check(_load().mslice_intensity_vjp(
        _ptr(psi, torch.complex64, n, "psi"), _ptr(dI, torch.float32, n, "dI"),
        _ptr(g_psi, torch.complex64, n, "g_psi"), n, _stream(stream)), "mslice_intensity_vjp")


def mslice_status(ws, stream=None) -> int:
    """0, or a negative code (-4 = MSLICE_ETIMEDOUT) recorded by a device-side wait."""
    return int(_load().mslice_status(_ptr(ws, torch.uint8, None, "ws"), _stream(stream)))


def mslice_debug_wait(nblocks, withhold, timeout_ns, ws, stream=None):
    _check(_load().mslice_debug_wait(int(nblocks), int(withhold), int(timeout_ns),
                                     _ptr(ws, torch.uint8, None, "ws"), ws.numel(),
                                     _stream(stream)), "mslice_debug_wait")


def mslice_profile_enable(on: bool = True):
    """Start (and reset) or stop the per-launch event timing of the library."""
    _check(_load().mslice_profile_enable(int(bool(on))), "mslice_profile_enable")


def mslice_profile_read():
    """{kernel name: (launches, total_ms, units)} since the last enable."""
    buf = (mslice_kernel_time * 16)()
    n = _load().mslice_profile_read(buf, 16)
    if n < 0:
        raise MsliceError(n, "mslice_profile_read")
    return {buf[i].name.decode(): (int(buf[i].launches), float(buf[i].total_ms), float(buf[i].units))
            for i in range(n)}


def mslice_coarse_to_fine(p, c, theta, vol, stream=None):
    nvol, _ = _sizes(p)
    _check(_load().mslice_coarse_to_fine(
        ctypes.byref(p), ctypes.byref(c), _ptr(theta, torch.float32, c.cx * c.cz * c.cy, "theta"),
        _ptr(vol, torch.complex64, nvol, "vol"), _stream(stream)), "mslice_coarse_to_fine")


def mslice_fine_to_coarse(p, c, grad_vol, g_theta, stream=None):
    nvol, _ = _sizes(p)
    _check(_load().mslice_fine_to_coarse(
        ctypes.byref(p), ctypes.byref(c), _ptr(grad_vol, torch.complex64, nvol, "grad_vol"),
        _ptr(g_theta, torch.float32, c.cx * c.cz * c.cy, "g_theta"), _stream(stream)),
        "mslice_fine_to_coarse")


def mslice_adam_step(theta, m, v, grad, lr, b1, b2, eps, t, lo, hi, stream=None):
    n = theta.numel()
    _check(_load().mslice_adam_step(
        _ptr(theta, torch.float32, n, "theta"), _ptr(m, torch.float32, n, "m"),
        _ptr(v, torch.float32, n, "v"), _ptr(grad, torch.float32, n, "grad"), n, float(lr), float(b1),
        float(b2), float(eps), int(t), float(lo), float(hi), _stream(stream)), "mslice_adam_step")


# --- learned initialiser kernels --------------------------------------------------

def _span_ok(t, offsets, what):
    """The largest element offset a strided access touches must lie inside t."""
    if max(offsets) >= t.numel() or min(offsets) < 0:
        raise ValueError("%s: strided access outside the tensor (%d elements)" % (what, t.numel()))


def mslice_nn_gemm_workspace(M, N, K) -> int:
    return int(_load().mslice_nn_gemm_workspace(int(M), int(N), int(K)))


def mslice_nn_gemm(M, N, K, A, sam, sak, B, sbn, sbk, C, ldc, bias=None, relu=False, beta=0.0, ws=None,
                   stream=None):
    """C[m][n] = beta C[m][n] + sum_k A[m*sam + k*sak] B[n*sbn + k*sbk] (+ bias[n]) (ReLU);
    BF16 operands, FP32 accumulation (tensor cores)."""
    for t, w in ((A, "A"), (B, "B"), (C, "C"), (bias, "bias")):
        if t is not None and (not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float32
                              or not t.is_contiguous()):
            raise TypeError("%s must be a contiguous float32 CUDA tensor" % w)
    _span_ok(A, [(M - 1) * sam + (K - 1) * sak, 0], "A")
    _span_ok(B, [(N - 1) * sbn + (K - 1) * sbk, 0], "B")
    _span_ok(C, [(M - 1) * ldc + N - 1], "C")
    if bias is not None and bias.numel() < N:
        raise ValueError("bias must have N elements")
    need = mslice_nn_gemm_workspace(M, N, K)
    if need and (ws is None or ws.numel() * ws.element_size() < need):
        raise ValueError("gemm %dx%dx%d needs a %d-byte workspace" % (M, N, K, need))
    wsp = ctypes.c_void_p(ws.data_ptr()) if ws is not None else None
    wsb = ws.numel() * ws.element_size() if ws is not None else 0
    _check(_load().mslice_nn_gemm(
        int(M), int(N), int(K), ctypes.c_void_p(A.data_ptr()), int(sam), int(sak), ctypes.c_void_p(B.data_ptr()),
        int(sbn), int(sbk), ctypes.c_void_p(C.data_ptr()), int(ldc),
        ctypes.c_void_p(bias.data_ptr()) if bias is not None else None, int(bool(relu)), float(beta), wsp, wsb,
        _stream(stream)), "mslice_nn_gemm")


def mslice_nn_pack_bf16(src, s_row, s_k, rows, K, dst, ld, stream=None):
    """dst[r][k] = BF16(src[r*s_row + k*s_k]) for k < K, 0 for K <= k < ld (dst: int16/bfloat16 CUDA tensor)."""
    if not isinstance(src, torch.Tensor) or src.dtype != torch.float32 or not src.is_cuda:
        raise TypeError("src must be a float32 CUDA tensor")
    if not isinstance(dst, torch.Tensor) or dst.element_size() != 2 or not dst.is_cuda or dst.numel() < rows * ld:
        raise TypeError("dst must be a 2-byte CUDA tensor of at least rows * ld elements")
    _span_ok(src, [(rows - 1) * s_row + (K - 1) * s_k, 0], "src")
    _check(_load().mslice_nn_pack_bf16(ctypes.c_void_p(src.data_ptr()), int(s_row), int(s_k), int(rows), int(K),
                                       ctypes.c_void_p(dst.data_ptr()), int(ld), _stream(stream)),
           "mslice_nn_pack_bf16")


def mslice_nn_gemm_bf16(M, N, K, A, lda, B, ldb, C, ldc, bias=None, relu=False, beta=0.0, stream=None):
    """C[m][n] = beta C[m][n] + sum_k A[m][k] B[n][k] (+ bias[n]) (ReLU) on the tcgen05 tensor cores:
    A [M][lda] and B [N][ldb] BF16 (K contiguous, lda and ldb multiples of 8), C float32 [M][ldc]."""
    for t, w, rows, ld in ((A, "A", M, lda), (B, "B", N, ldb)):
        if not isinstance(t, torch.Tensor) or t.element_size() != 2 or not t.is_cuda or t.numel() < rows * ld:
            raise TypeError("%s must be a 2-byte CUDA tensor of at least %d x %d elements" % (w, rows, ld))
    if not isinstance(C, torch.Tensor) or C.dtype != torch.float32 or not C.is_cuda:
        raise TypeError("C must be a float32 CUDA tensor")
    _span_ok(C, [(M - 1) * ldc + N - 1], "C")
    if bias is not None and (bias.dtype != torch.float32 or bias.numel() < N):
        raise ValueError("bias must have N float32 elements")
    _check(_load().mslice_nn_gemm_bf16(
        int(M), int(N), int(K), ctypes.c_void_p(A.data_ptr()), int(lda), ctypes.c_void_p(B.data_ptr()), int(ldb),
        ctypes.c_void_p(C.data_ptr()), int(ldc), ctypes.c_void_p(bias.data_ptr()) if bias is not None else None,
        int(bool(relu)), float(beta), _stream(stream)), "mslice_nn_gemm_bf16")


def mslice_nn_gemm_bf16_status(stream=None) -> int:
    return int(_load().mslice_nn_gemm_bf16_status(_stream(stream)))


def mslice_nn_space_to_depth(x, out, B, H, W, C, p, inverse=False, stream=None):
    n = B * H * W * C
    _check(_load().mslice_nn_space_to_depth(
        _ptr(x, torch.float32, n, "in"), _ptr(out, torch.float32, n, "out"), int(B), int(H), int(W), int(C),
        int(p), int(bool(inverse)), _stream(stream)), "mslice_nn_space_to_depth")


def mslice_nn_relu_backward(y, dy, dz, stream=None):
    n = y.numel()
    _check(_load().mslice_nn_relu_backward(
        _ptr(y, torch.float32, n, "y"), _ptr(dy, torch.float32, n, "dy"), _ptr(dz, torch.float32, n, "dz"), n,
        _stream(stream)), "mslice_nn_relu_backward")


def mslice_nn_sigmoid_mse(z, target, y, dz, row_loss, rows, cols, hi=1.0, stream=None):
    n = rows * cols
    _check(_load().mslice_nn_sigmoid_mse(
        _ptr(z, torch.float32, n, "z"), _ptr(target, torch.float32, n, "target"), _ptr(y, torch.float32, n, "y"),
        _ptr(dz, torch.float32, n, "dz"), _ptr(row_loss, torch.float64, rows, "row_loss"), int(rows), int(cols),
        float(hi), _stream(stream)), "mslice_nn_sigmoid_mse")


def mslice_nn_detector_features(intensity, noise, x, nimg, nz, ny, counts, gain=1.0, stream=None):
    n = nimg * nz * ny
    _check(_load().mslice_nn_detector_features(
        _ptr(intensity, torch.float32, n, "intensity"), _ptr(noise, torch.float32, n, "noise"),
        _ptr(x, torch.float32, n, "x"), int(nimg), int(nz), int(ny), float(counts), float(gain),
        _stream(stream)), "mslice_nn_detector_features")


def mslice_nn_rasterize_boxes(boxes, out, shape, value, stream=None):
    """boxes int32 [nsamples][nboxes][6] -> out float32 [nsamples][shape]."""
    ns_, nb_ = int(boxes.shape[0]), int(boxes.shape[1])
    d0, d1, d2 = (int(v) for v in shape)
    _check(_load().mslice_nn_rasterize_boxes(
        _ptr(boxes, torch.int32, ns_ * nb_ * 6, "boxes"), nb_, ns_, d0, d1, d2, float(value),
        _ptr(out, torch.float32, ns_ * d0 * d1 * d2, "out"), _stream(stream)), "mslice_nn_rasterize_boxes")


def mslice_rotate(p, alpha_rad, psi_rad, center_nm, vol_sample, vol_lab, stream=None):
    """vol_lab = R vol_sample: the sample-frame volume rotated into the lab frame
    (pitch alpha after yaw psi about center_nm = (x, z, y) in nm)."""
    n = p.ns * p.nz * p.ny
    c = (ctypes.c_double * 3)(*[float(v) for v in center_nm])
    _check(_load().mslice_rotate(ctypes.byref(p), float(alpha_rad), float(psi_rad), c,
                                 _ptr(vol_sample, torch.complex64, n, "vol_sample"),
                                 _ptr(vol_lab, torch.complex64, n, "vol_lab"), _stream(stream)), "mslice_rotate")


def mslice_rotate_adjoint(p, alpha_rad, psi_rad, center_nm, g_lab, g_sample, stream=None):
    """g_sample = R^T g_lab (overwritten)."""
    n = p.ns * p.nz * p.ny
    c = (ctypes.c_double * 3)(*[float(v) for v in center_nm])
    _check(_load().mslice_rotate_adjoint(ctypes.byref(p), float(alpha_rad), float(psi_rad), c,
                                         _ptr(g_lab, torch.complex64, n, "g_lab"),
                                         _ptr(g_sample, torch.complex64, n, "g_sample"), _stream(stream)),
           "mslice_rotate_adjoint")


def mslice_shrinkwrap(theta, sigma, threshold, kept=None, ws=None, stream=None):
    """In place on theta [cx][cz][cy] (float32, CUDA): zero outside the
    shrink-wrap support (Gaussian blur of width sigma, threshold * its max)."""
    if theta.dim() != 3:
        raise ValueError("theta must be [cx][cz][cy]")
    cx, cz, cy = theta.shape
    need = _load().mslice_shrinkwrap_workspace(theta.numel())
    if ws is None:
        ws = torch.empty(need, dtype=torch.uint8, device=theta.device)
    _check(_load().mslice_shrinkwrap(_ptr(theta, torch.float32, None, "theta"), cx, cz, cy, float(sigma),
                                     float(threshold), _ptr(kept, torch.int32, 1, "kept"),
                                     _ptr(ws, torch.uint8, None, "ws"), ws.numel(), _stream(stream)),
           "mslice_shrinkwrap")


def mslice_snap(theta, levels, stream=None):
    """In place: every parameter becomes the nearest of ``levels`` (1..8 floats)."""
    lv = (ctypes.c_float * len(levels))(*[float(v) for v in levels])
    _check(_load().mslice_snap(_ptr(theta, torch.float32, None, "theta"), theta.numel(), lv, len(levels),
                               _stream(stream)), "mslice_snap")
