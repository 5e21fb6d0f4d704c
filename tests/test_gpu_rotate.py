"""Frame rotation of Eq. 2-3 on the GPU (mslice_rotate, mslice_rotate_adjoint)
against the FP64 oracle, and the lab-frame / sample-frame equivalence run
through the GPU slice loop."""
import numpy as np
import pytest
import torch

import cssi_inputs as ci
import oracle
from oracle import rotate as R
from tests import _gpu as G

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2212_01253_gb300 import build
    build.build()
    oracle.build()


def _params(ns, nz, ny, sp):
    from paper_2212_01253_gb300 import binding as B
    return B.make_params(ny, nz, ns, (0.3,), slice_nm=sp[0], dz_nm=sp[1], dy_nm=sp[2])


def _volume(kind, shape, seed):
    if kind == "pillars":
        ns, nz, ny = shape
        return ci.pillars_small(seed, ny=ny, nz=nz, ns=ns)
    return ci.random_volume(seed, shape[2], shape[1], shape[0], scale=1.0)


CASES = [
    ((24, 40, 36), (20.0, 2.0, 2.0), 2.5, -4.0, (230.0, 41.0, 33.0), "random"),
    ((32, 64, 64), (20.0, 2.0, 2.0), 0.3, 0.0, (0.0, 63.0, 63.0), "pillars"),
    ((16, 128, 8), (10.0, 1.0, 3.0), -1.0, 6.0, (100.0, 120.0, 5.0), "random"),
    ((3, 1, 1024), (20.0, 2.0, 2.0), 0.5, 2.0, (20.0, 0.0, 1000.0), "random"),
    ((40, 96, 24), (20.0, 2.0, 2.0), 20.0, -15.0, (400.0, 90.0, 20.0), "random"),
]


@pytest.mark.parametrize("shape,sp,alpha,psi,c,kind", CASES)
def test_rotate_vs_oracle(shape, sp, alpha, psi, c, kind):
    from paper_2212_01253_gb300 import binding as B
    v = _volume(kind, shape, sum(shape))
    p = _params(*shape, sp)
    out = torch.empty(shape, dtype=torch.complex64, device="cuda")
    B.mslice_rotate(p, np.deg2rad(alpha), np.deg2rad(psi), c, G.dev(v, np.complex64), out)
    torch.cuda.synchronize()
    ref = R.rotate(v.astype(np.complex64), sp, np.deg2rad(alpha), np.deg2rad(psi), c)
    got = out.cpu().numpy()
    assert G.rel(got, ref) <= 1e-6
    assert np.abs(got - ref).max() <= 1e-6 * np.abs(v).max()


@pytest.mark.parametrize("shape,sp,alpha,psi,c,kind", CASES[:4])
def test_rotate_adjoint_vs_oracle(shape, sp, alpha, psi, c, kind):
    from paper_2212_01253_gb300 import binding as B
    g = ci.random_volume(7 + sum(shape), shape[2], shape[1], shape[0], scale=1.0)
    p = _params(*shape, sp)
    out = torch.empty(shape, dtype=torch.complex64, device="cuda")
    B.mslice_rotate_adjoint(p, np.deg2rad(alpha), np.deg2rad(psi), c, G.dev(g, np.complex64), out)
    torch.cuda.synchronize()
    ref = R.rotate_adjoint(g.astype(np.complex64), sp, np.deg2rad(alpha), np.deg2rad(psi), c)
    assert G.rel(out.cpu().numpy(), ref) <= 1e-6


def test_rotate_adjoint_without_yaw_collapsed_faces_vs_oracle():
    """psi = 0 (the row-wise transpose) at 5 deg pitch over 64 slices: the
    lab rows shift by ~56 rows along z, so the sample rows on the z faces take
    dozens of collapsed lab rows (the transpose's long path), the others 2-4."""
    from paper_2212_01253_gb300 import binding as B
    shape, sp, alpha, psi, c = (64, 64, 40), (20.0, 2.0, 2.0), 5.0, 0.0, (600.0, 63.0, 39.0)
    g = ci.random_volume(99, shape[2], shape[1], shape[0], scale=1.0)
    p = _params(*shape, sp)
    out = torch.empty(shape, dtype=torch.complex64, device="cuda")
    B.mslice_rotate_adjoint(p, np.deg2rad(alpha), np.deg2rad(psi), c, G.dev(g, np.complex64), out)
    torch.cuda.synchronize()
    ref = R.rotate_adjoint(g.astype(np.complex64), sp, np.deg2rad(alpha), np.deg2rad(psi), c)
    got = out.cpu().numpy()
    assert G.rel(got, ref) <= 1e-6
    # the face rows carry the collapsed rows' sums
    assert G.rel(got[:, 0, :], ref[:, 0, :]) <= 1e-6 and G.rel(got[:, -1, :], ref[:, -1, :]) <= 1e-6


def test_rotate_adjoint_is_bitwise_reproducible_and_a_transpose():
    """The transpose is a gather in a fixed order: two calls agree bit for bit;
    and <R x, y> = <x, R^T y> to FP32 rounding."""
    from paper_2212_01253_gb300 import binding as B
    shape, sp, alpha, psi, c, _ = CASES[0]
    p = _params(*shape, sp)
    g = G.dev(ci.random_volume(41, shape[2], shape[1], shape[0], scale=1.0), np.complex64)
    x = G.dev(ci.random_volume(42, shape[2], shape[1], shape[0], scale=1.0), np.complex64)
    a1 = torch.empty(shape, dtype=torch.complex64, device="cuda")
    a2 = torch.empty_like(a1)
    rx = torch.empty_like(a1)
    B.mslice_rotate_adjoint(p, np.deg2rad(alpha), np.deg2rad(psi), c, g, a1)
    B.mslice_rotate_adjoint(p, np.deg2rad(alpha), np.deg2rad(psi), c, g, a2)
    B.mslice_rotate(p, np.deg2rad(alpha), np.deg2rad(psi), c, x, rx)
    torch.cuda.synchronize()
    assert torch.equal(a1, a2)
    lhs = torch.vdot(rx.flatten().to(torch.complex128), g.flatten().to(torch.complex128))
    rhs = torch.vdot(x.flatten().to(torch.complex128), a1.flatten().to(torch.complex128))
    assert abs(complex(lhs) - complex(rhs)) <= 1e-6 * abs(complex(lhs))


def test_zero_rotation_is_the_identity_bit_for_bit():
    from paper_2212_01253_gb300 import binding as B
    v = ci.random_volume(3, 48, 32, 10, scale=1.0)
    p = _params(10, 32, 48, (20.0, 2.0, 2.0))
    out = torch.empty(v.shape, dtype=torch.complex64, device="cuda")
    B.mslice_rotate(p, 0.0, 0.0, (100.0, 31.0, 47.0), G.dev(v, np.complex64), out)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(out.cpu().numpy(), v.astype(np.complex64))


def test_rotate_rejects_bad_arguments():
    from paper_2212_01253_gb300 import binding as B
    p = _params(4, 8, 8, (20.0, 2.0, 2.0))
    a = torch.zeros((4, 8, 8), dtype=torch.complex64, device="cuda")
    with pytest.raises(RuntimeError):
        B.mslice_rotate(p, 0.1, 0.0, (0.0, 0.0, 0.0), a, a)          # in place
    with pytest.raises(RuntimeError):
        B.mslice_rotate(p, float("nan"), 0.0, (0.0, 0.0, 0.0), a, torch.zeros_like(a))


@pytest.mark.parametrize("psi_deg", [0.0, 0.5])
def test_rotate_full_size_sampled_against_the_oracle(psi_deg):
    """512 x 512 x 1024, the headline volume, at the paper's 0.3 deg pitch,
    without yaw (row-wise x and z stencils) and with a 0.5 deg yaw: 20000
    sampled lab voxels against the oracle."""
    from paper_2212_01253_gb300 import binding as B
    shape, sp = (1024, 512, 512), (20.0, 2.0, 2.0)
    v = ci.pillars_large(0)
    c = (0.0, 511.0, 511.0)
    a, ps = np.deg2rad(0.3), np.deg2rad(psi_deg)
    out = torch.empty(shape, dtype=torch.complex64, device="cuda")
    B.mslice_rotate(_params(*shape, sp), a, ps, c, G.dev(v, np.complex64), out)
    torch.cuda.synchronize()
    rng = np.random.default_rng(11)
    idx = np.stack([rng.integers(0, n, 20000) for n in shape], axis=1)
    ti = torch.from_numpy(idx).cuda()
    got = out[ti[:, 0], ti[:, 1], ti[:, 2]].cpu().numpy()
    ref = R.rotate_at(v, sp, a, ps, c, idx)
    assert G.rel(got, ref) <= 1e-6


def test_lab_frame_matches_the_sample_frame_through_the_gpu_slice_loop():
    """The lab frame of Eq. 2-3 (GPU-rotated volume, straight beam) against the
    sample frame (tilted probe), both through the GPU forward: the far fields
    agree after a shift of k sin(alpha) = 34 bins along k_z (the FP64 oracle
    gives 5.4e-4 on this case)."""
    from paper_2212_01253_gb300 import binding as B
    ny, nz, ns, dz, delta, m = 64, 512, 1024, 2.0, 20.0, 34
    alpha = np.arcsin(m * ci.WAVELENGTH_NM / (nz * dz))
    vol = ci.pillars_large(3, ny=ny, nz=nz, ns=ns, count=8).astype(np.complex128)
    ramp = np.zeros(nz)
    ramp[:48] = np.linspace(1, 0, 48) ** 2
    ramp[-48:] = np.linspace(0, 1, 48) ** 2
    vol += 2e-5j * ramp[None, :, None]
    I_s = G.forward(oracle.Geometry(ny, nz, ns, slice_nm=delta, dz_nm=dz, alpha_i_deg=(np.rad2deg(alpha),)),
                    vol)[0]
    lab = torch.empty((ns, nz, ny), dtype=torch.complex64, device="cuda")
    B.mslice_rotate(_params(ns, nz, ny, (delta, dz, 2.0)), alpha, 0.0, (0.0, (nz / 2 - 0.5) * dz, (ny - 1.0)),
                    G.dev(vol, np.complex64), lab)
    torch.cuda.synchronize()
    geo_l = oracle.Geometry(ny, nz, ns, slice_nm=delta, dz_nm=dz, alpha_i_deg=(0.0,))
    I_l = G.forward(geo_l, lab.cpu().numpy())[0]
    assert G.rel(I_l, np.roll(I_s, m, axis=0)) < 2e-3
