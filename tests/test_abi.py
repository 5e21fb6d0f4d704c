"""The C-ABI library loads and exports every symbol include/mslice.h declares
(host-only checks: no GPU compute)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "mslice.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(mslice_\w+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_2212_01253_gb300 import build
    return ctypes.CDLL(build.build())


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("mslice_forward", "mslice_adjoint", "mslice_loss_grad", "mslice_workspace_size",
              "mslice_strerror", "mslice_status"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_workspace_size_and_validation_on_host():
    from paper_2212_01253_gb300 import binding as B
    p = B.make_params(64, 64, 32)
    fwd = B.mslice_workspace_size(p, B.MSLICE_OP_FORWARD)
    lg = B.mslice_workspace_size(p, B.MSLICE_OP_LOSS_GRAD)
    # forward holds at least the transmission volume and one field
    assert fwd >= 64 * 64 * 32 * 8 + 64 * 64 * 8
    # gradient adds checkpoints (1 of 32 slices) and the 32-slice segment buffer
    assert lg >= fwd + 33 * 64 * 64 * 8
    for bad in (dict(ny=48), dict(nz=2048), dict(ns=0)):
        kw = dict(ny=64, nz=64, ns=32)
        kw.update(bad)
        with pytest.raises(B.MsliceError):
            B.mslice_workspace_size(B.make_params(**kw), 0)
    assert B.mslice_strerror(-4).startswith("a bounded")


def test_option_flags_size_their_buffers_and_reject_bad_combinations():
    """Host-only: the symmetric splitting adds the half-step tables, the probe
    copy and a zero slice; the angular spectrum adds its 2-D table; the angular
    spectrum with the symmetric splitting adds its half-step 2-D table."""
    from paper_2212_01253_gb300 import binding as B
    ny = nz = 64
    ns, nw = 8, 3
    base = B.mslice_workspace_size(B.make_params(ny, nz, ns, (0.2, 0.3, 0.4)), B.MSLICE_OP_FORWARD)
    strang = B.mslice_workspace_size(B.make_params(ny, nz, ns, (0.2, 0.3, 0.4), flags=B.MSLICE_STRANG),
                                     B.MSLICE_OP_FORWARD)
    angular = B.mslice_workspace_size(B.make_params(ny, nz, ns, (0.2, 0.3, 0.4), flags=B.MSLICE_ANGULAR),
                                      B.MSLICE_OP_FORWARD)
    both = B.mslice_workspace_size(B.make_params(ny, nz, ns, (0.2, 0.3, 0.4),
                                                 flags=B.MSLICE_ANGULAR | B.MSLICE_STRANG), B.MSLICE_OP_FORWARD)
    assert strang >= base + (nw + 1) * ny * nz * 8 + 2 * (ny + nz) * 8
    assert angular >= base + ny * nz * 8
    assert both >= strang + 2 * ny * nz * 8
    exit_wave = B.mslice_workspace_size(B.make_params(ny, nz, ns, flags=B.MSLICE_ANGULAR | B.MSLICE_EXIT_WAVE), 0)
    assert exit_wave > 0
    with pytest.raises(B.MsliceError):
        B.mslice_workspace_size(B.make_params(ny, nz, ns, flags=1 << 10), 0)


def test_shrinkwrap_workspace_size_on_host(lib):
    lib.mslice_shrinkwrap_workspace.restype = ctypes.c_size_t
    lib.mslice_shrinkwrap_workspace.argtypes = [ctypes.c_size_t]
    assert lib.mslice_shrinkwrap_workspace(216) >= 2 * 216 * 4


def test_tensor_core_gemm_validates_arguments_on_host(lib):
    """mslice_nn_gemm_bf16 and mslice_nn_pack_bf16 refuse bad sizes, strides
    and alignments before any device work (the pointers are never read)."""
    vp, ll, ci = ctypes.c_void_p, ctypes.c_longlong, ctypes.c_int
    f = lib.mslice_nn_gemm_bf16
    f.argtypes = [ci, ci, ci, vp, ll, vp, ll, vp, ll, vp, ci, ctypes.c_float, vp]
    f.restype = ci
    A, Bm, C = 0x100000, 0x200000, 0x300000     # 16-byte aligned, never dereferenced
    assert f(0, 256, 64, A, 64, Bm, 64, C, 256, None, 0, 0.0, None) == -1        # M < 1
    assert f(128, 256, 64, A, 60, Bm, 64, C, 256, None, 0, 0.0, None) == -1      # lda < K
    assert f(128, 256, 64, A, 68, Bm, 64, C, 256, None, 0, 0.0, None) == -1      # lda not a multiple of 8
    assert f(128, 256, 64, A + 8, 64, Bm, 64, C, 256, None, 0, 0.0, None) == -1  # A not 16-byte aligned
    assert f(128, 256, 64, A, 64, Bm, 64, C, 200, None, 0, 0.0, None) == -1      # ldc < N
    assert f(128, 256, 64, A, 64, None, 64, C, 256, None, 0, 0.0, None) == -1    # null B
    g = lib.mslice_nn_pack_bf16
    g.argtypes = [vp, ll, ll, ci, ci, vp, ll, vp]
    g.restype = ci
    assert g(A, 64, 1, 128, 64, Bm, 60, None) == -1      # ld < K
    assert g(None, 64, 1, 128, 64, Bm, 64, None) == -1   # null source
    assert g(A, 64, 1, 128, 64, Bm + 1, 64, None) == -1  # odd destination
