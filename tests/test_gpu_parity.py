"""CUDA path (through the C ABI) against the FP64 oracle, element by element.

Tolerances: relative L2 <= 1e-4 on intensities (FP32 path), <= 1e-6 on the
FP64-built tables, <= 1e-3 on gradients.
"""
import numpy as np
import pytest
import torch

import cssi_inputs as ci
import oracle
from tests import _gpu as G

pytestmark = pytest.mark.gpu

TOL_I = 1e-4
TOL_GRAD = 1e-3


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2212_01253_gb300 import build
    build.build()
    oracle.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


# --------------------------------------------------------------------------
# plan tables and transmission (the FP64 steps)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("ny,nz", [(64, 64), (512, 256), (1, 1024), (1024, 8)])
def test_plan_tables_fp64(ny, nz):
    from paper_2212_01253_gb300 import binding as B
    geo = oracle.Geometry(ny, nz, 3, alpha_i_deg=(0.1, 0.3, 0.5))
    p = G.params(geo)
    ws = B.workspace(p, B.MSLICE_OP_FORWARD)
    py = torch.empty(ny, dtype=torch.complex64, device="cuda")
    pz = torch.empty(nz, dtype=torch.complex64, device="cuda")
    prz = torch.empty((3, nz), dtype=torch.complex64, device="cuda")
    B.mslice_plan_tables(p, py, pz, prz, ws)
    ref_y, ref_z = oracle.propagator_1d(geo)
    assert np.abs(py.cpu().numpy() - ref_y).max() < 1e-6
    assert np.abs(pz.cpu().numpy() - ref_z).max() < 1e-6
    # default probe rows: the oracle's plane wave, read back from a one-slice
    # vacuum exit wave would mix in the FFT; compare with the plain definition
    z = np.arange(nz) * geo.dz_nm
    k = 2 * np.pi / geo.wavelength_nm
    ref_p = np.exp(-1j * k * np.sin(geo.alpha_i_rad)[:, None] * z[None, :])
    assert np.abs(prz.cpu().numpy() - ref_p).max() < 1e-6


def test_transmission_fp64():
    from paper_2212_01253_gb300 import binding as B
    geo = oracle.Geometry(32, 64, 8)
    vol = ci.random_volume(3, 32, 64, 8, scale=100)
    p = G.params(geo)
    t = torch.empty(vol.shape, dtype=torch.complex64, device="cuda")
    B.mslice_transmission(p, G.dev(vol, np.complex64), t)
    kd = 2 * np.pi / geo.wavelength_nm * geo.slice_nm
    ref = np.exp(-1j * kd * np.conj(vol.astype(np.complex128)))
    assert np.abs(t.cpu().numpy() - ref).max() < 1e-6


@pytest.mark.parametrize("psi_deg", [0.35, -0.5])
def test_in_plane_angle_vs_oracle(psi_deg):
    """psi != 0: the default probe tilted in y as well; forward and gradient."""
    geo = oracle.Geometry(128, 64, 20, alpha_i_deg=(0.2, 0.4), psi_deg=psi_deg)
    vol = ci.random_volume(23, 128, 64, 20, scale=40)
    I_ref = oracle.forward(geo, vol)
    assert G.rel(G.forward(geo, vol), I_ref) <= TOL_I
    meas = (np.sqrt(I_ref) * 1.07).astype(np.float32)
    L_ref, g_ref = oracle.loss_grad(geo, vol, meas, 0.9)
    L, g = G.loss_grad(geo, vol, meas, 0.9, checkpoint_every=6)
    assert abs(L - L_ref) <= 1e-4 * abs(L_ref)
    assert G.rel(g, g_ref) <= TOL_GRAD


@pytest.mark.parametrize("ny,nz,ns,K", [(128, 64, 20, 6), (64, 128, 13, 13)])
def test_per_view_in_plane_angles_vs_oracle(ny, nz, ns, K):
    """Several views, each with its own (alpha, psi) pair (Eq. 2-3 per view):
    forward, loss and gradient summed over the views, against the oracle; and
    each view's intensity equals the single-view call's."""
    alphas, psis = (0.15, 0.3, 0.45, 0.25), (-0.5, 0.2, 0.0, 0.4)
    geo = oracle.Geometry(ny, nz, ns, alpha_i_deg=alphas, psi_deg=psis)
    vol = ci.random_volume(29 + ny, ny, nz, ns, scale=40)
    I_ref = oracle.forward(geo, vol)
    I = G.forward(geo, vol)
    assert G.rel(I, I_ref) <= TOL_I
    for w in range(len(alphas)):
        g1 = oracle.Geometry(ny, nz, ns, alpha_i_deg=(alphas[w],), psi_deg=psis[w])
        assert np.array_equal(G.forward(g1, vol)[0], I[w])
    meas = (np.sqrt(I_ref) * 1.07).astype(np.float32)
    L_ref, g_ref = oracle.loss_grad(geo, vol, meas, 0.9)
    L, g = G.loss_grad(geo, vol, meas, 0.9, checkpoint_every=K)
    assert abs(L - L_ref) <= 1e-4 * abs(L_ref)
    assert G.rel(g, g_ref) <= TOL_GRAD


def test_exact_transmission_fp64():
    """MSLICE_EXACT_TRANSMISSION: exp((k/2i) Delta (1 - n^2)), n = 1 - delta + i beta,
    evaluated in FP64 from n."""
    from paper_2212_01253_gb300 import binding as B
    geo = oracle.Geometry(32, 64, 8, exact_transmission=True)
    vol = ci.random_volume(4, 32, 64, 8, scale=100)
    p = G.params(geo)
    t = torch.empty(vol.shape, dtype=torch.complex64, device="cuda")
    B.mslice_transmission(p, G.dev(vol, np.complex64), t)
    k = 2 * np.pi / geo.wavelength_nm
    n = 1 - vol.astype(np.complex64).astype(np.complex128).conj()
    ref = np.exp(k / 2j * geo.slice_nm * (1 - n * n))
    assert np.abs(t.cpu().numpy() - ref).max() < 1e-6
    lin = np.exp(-1j * k * geo.slice_nm * np.conj(vol.astype(np.complex128)))
    assert np.abs(ref - lin).max() > 1e-5       # the flag changes the result


@pytest.mark.parametrize("ny,nz,ns,nw,K", [(64, 64, 24, 1, 5), (32, 64, 13, 3, 4), (512, 256, 20, 2, 20)])
def test_exact_transmission_loss_grad_vs_oracle(ny, nz, ns, nw, K):
    geo = oracle.Geometry(ny, nz, ns, alpha_i_deg=np.linspace(0.15, 0.45, nw), exact_transmission=True)
    vol = ci.random_volume(ny + ns, ny, nz, ns, scale=60)
    meas = _target(geo, vol.astype(np.complex128) * 1.1, 4)
    L_ref, g_ref, I_ref = oracle.loss_grad(geo, vol, meas, 0.7, return_intensity=True)
    L, g, I = G.loss_grad(geo, vol, meas, 0.7, checkpoint_every=K, return_intensity=True)
    assert G.rel(I, I_ref) <= TOL_I
    assert abs(L - L_ref) <= 1e-4 * abs(L_ref)
    assert G.rel(g, g_ref) <= TOL_GRAD
    # and it is not the linearised gradient
    lin = oracle.Geometry(ny, nz, ns, alpha_i_deg=np.linspace(0.15, 0.45, nw))
    _, g_lin = oracle.loss_grad(lin, vol, meas, 0.7)
    assert G.rel(g_lin, g_ref) > 10 * G.rel(g, g_ref)


# --------------------------------------------------------------------------
# symmetric splitting (MSLICE_STRANG): half steps of propagation at both ends
# --------------------------------------------------------------------------
@pytest.mark.parametrize("ny,nz,ns,nw,user_probe", [(64, 64, 12, 2, False), (32, 128, 1, 1, True),
                                                     (256, 64, 7, 3, False), (64, 32, 5, 1, True)])
def test_strang_forward_and_exit_wave_vs_oracle(ny, nz, ns, nw, user_probe):
    angles = np.linspace(0.15, 0.45, nw)
    geo = oracle.Geometry(ny, nz, ns, alpha_i_deg=angles, strang=True)
    vol = ci.random_volume(ny + 3 * ns, ny, nz, ns, scale=60)
    probe = ci.random_probe(ny + ns, nw, ny, nz) if user_probe else None
    I_ref = oracle.forward(geo, vol, probe=probe)
    I = G.forward(geo, vol, probe=probe)
    assert G.rel(I, I_ref) <= TOL_I
    ex_ref = oracle.forward(geo, vol, probe=probe, exit_wave=True)
    ex = G.forward(geo, vol, probe=probe, exit_wave=True)
    assert G.rel(ex, ex_ref) <= TOL_I
    # the transmission-first result is far outside the tolerance
    lie = oracle.Geometry(ny, nz, ns, alpha_i_deg=angles)
    assert G.rel(I, oracle.forward(lie, vol, probe=probe)) > 10 * TOL_I
    assert G.rel(ex, oracle.forward(lie, vol, probe=probe, exit_wave=True)) > 10 * TOL_I


@pytest.mark.parametrize("ny,nz,ns,nw,K,schedule", [(64, 64, 24, 1, 5, 0), (32, 64, 13, 3, 4, 0),
                                                    (64, 128, 16, 4, 16, 2)])
def test_strang_loss_grad_vs_oracle(ny, nz, ns, nw, K, schedule):
    geo = oracle.Geometry(ny, nz, ns, alpha_i_deg=np.linspace(0.15, 0.45, nw), strang=True)
    vol = ci.random_volume(2 * ny + ns, ny, nz, ns, scale=60)
    meas = _target(geo, vol.astype(np.complex128) * 1.1, 5)
    L_ref, g_ref, I_ref = oracle.loss_grad(geo, vol, meas, 0.7, return_intensity=True)
    L, g, I = G.loss_grad(geo, vol, meas, 0.7, checkpoint_every=K, return_intensity=True, schedule=schedule)
    assert G.rel(I, I_ref) <= TOL_I
    assert abs(L - L_ref) <= 1e-4 * abs(L_ref)
    assert G.rel(g, g_ref) <= TOL_GRAD


def test_strang_per_structure_vs_oracle():
    """mslice_loss_grad_multi with MSLICE_STRANG: each structure's half-step
    probe is its own default probe propagated by Delta/2."""
    from paper_2212_01253_gb300 import binding as B
    ny, nz, ns, nw = 64, 64, 9, 3
    angles = (0.2, 0.3, 0.4)
    vols = [ci.random_volume(300 + i, ny, nz, ns, scale=60) for i in range(nw)]
    geos = [oracle.Geometry(ny, nz, ns, alpha_i_deg=(a,), strang=True) for a in angles]
    meas = [_target(g, v.astype(np.complex128) * 1.1, 7 + i) for i, (g, v) in enumerate(zip(geos, vols))]
    scales = [0.7, 1.1, 0.9]
    p = B.make_params(ny, nz, ns, angles, checkpoint_every=4, flags=B.MSLICE_PER_STRUCTURE | B.MSLICE_STRANG)
    ws = B.workspace(p, B.MSLICE_OP_LOSS_GRAD)
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    grad = torch.empty((nw, ns, nz, ny), dtype=torch.complex64, device="cuda")
    B.mslice_loss_grad_multi(p, G.dev(np.stack(vols), np.complex64), None,
                             G.dev(np.concatenate(meas), np.float32), scales, loss, grad, None, ws)
    torch.cuda.synchronize()
    assert B.mslice_status(ws) == 0
    L_ref = 0.0
    for i in range(nw):
        Li, gi = oracle.loss_grad(geos[i], vols[i], meas[i], scales[i])
        L_ref += Li
        assert G.rel(grad[i].cpu().numpy(), gi) <= TOL_GRAD
    assert abs(float(loss.item()) - L_ref) <= 1e-4 * abs(L_ref)


# --------------------------------------------------------------------------
# angular-spectrum propagator (MSLICE_ANGULAR)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("ny,nz,ns,nw,user_probe", [(64, 64, 12, 2, False), (32, 128, 5, 1, True),
                                                     (128, 64, 7, 3, False), (32, 32, 1, 1, True),
                                                     (512, 256, 16, 2, False)])
def test_angular_forward_vs_oracle(ny, nz, ns, nw, user_probe):
    """1 nm pixels, where the angular spectrum and the paraxial propagator
    differ by 0.4-1.4 % in I."""
    angles = np.linspace(0.15, 0.45, nw)
    geo = oracle.Geometry(ny, nz, ns, dy_nm=1.0, dz_nm=1.0, alpha_i_deg=angles, angular=True)
    vol = ci.random_volume(ny + 5 * ns, ny, nz, ns, scale=60)
    probe = ci.random_probe(ny + ns, nw, ny, nz) if user_probe else None
    I_ref = oracle.forward(geo, vol, probe=probe)
    I = G.forward(geo, vol, probe=probe)
    assert G.rel(I, I_ref) <= TOL_I
    if ns > 1:
        par = oracle.Geometry(ny, nz, ns, dy_nm=1.0, dz_nm=1.0, alpha_i_deg=angles)
        assert G.rel(I, oracle.forward(par, vol, probe=probe)) > 10 * TOL_I


@pytest.mark.parametrize("ny,nz,ns,nw,K,schedule", [(64, 64, 24, 1, 5, 0), (32, 64, 13, 3, 4, 0),
                                                    (64, 128, 16, 4, 16, 2), (64, 64, 9, 2, 9, 0)])
def test_angular_loss_grad_vs_oracle(ny, nz, ns, nw, K, schedule):
    geo = oracle.Geometry(ny, nz, ns, dy_nm=1.0, dz_nm=1.0, alpha_i_deg=np.linspace(0.15, 0.45, nw),
                          angular=True)
    vol = ci.random_volume(3 * ny + ns, ny, nz, ns, scale=60)
    meas = _target(geo, vol.astype(np.complex128) * 1.1, 6)
    L_ref, g_ref, I_ref = oracle.loss_grad(geo, vol, meas, 0.7, return_intensity=True)
    L, g, I = G.loss_grad(geo, vol, meas, 0.7, checkpoint_every=K, return_intensity=True, schedule=schedule)
    assert G.rel(I, I_ref) <= TOL_I
    assert abs(L - L_ref) <= 1e-4 * abs(L_ref)
    assert G.rel(g, g_ref) <= TOL_GRAD


def test_angular_per_structure_vs_oracle():
    from paper_2212_01253_gb300 import binding as B
    ny, nz, ns, nw = 64, 64, 9, 3
    angles = (0.2, 0.3, 0.4)
    vols = [ci.random_volume(500 + i, ny, nz, ns, scale=60) for i in range(nw)]
    geos = [oracle.Geometry(ny, nz, ns, dy_nm=1.0, dz_nm=1.0, alpha_i_deg=(a,), angular=True) for a in angles]
    meas = [_target(g, v.astype(np.complex128) * 1.1, 9 + i) for i, (g, v) in enumerate(zip(geos, vols))]
    scales = [0.7, 1.1, 0.9]
    p = B.make_params(ny, nz, ns, angles, dy_nm=1.0, dz_nm=1.0, checkpoint_every=4,
                      flags=B.MSLICE_PER_STRUCTURE | B.MSLICE_ANGULAR)
    ws = B.workspace(p, B.MSLICE_OP_LOSS_GRAD)
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    grad = torch.empty((nw, ns, nz, ny), dtype=torch.complex64, device="cuda")
    B.mslice_loss_grad_multi(p, G.dev(np.stack(vols), np.complex64), None,
                             G.dev(np.concatenate(meas), np.float32), scales, loss, grad, None, ws)
    torch.cuda.synchronize()
    assert B.mslice_status(ws) == 0
    L_ref = 0.0
    for i in range(nw):
        Li, gi = oracle.loss_grad(geos[i], vols[i], meas[i], scales[i])
        L_ref += Li
        assert G.rel(grad[i].cpu().numpy(), gi) <= TOL_GRAD
    assert abs(float(loss.item()) - L_ref) <= 1e-4 * abs(L_ref)


@pytest.mark.parametrize("opts", [dict(exact_transmission=True, strang=True, psi_deg=0.35),
                                  dict(exact_transmission=True, angular=True, psi_deg=-0.5),
                                  dict(strang=True, psi_deg=0.2)])
def test_option_combinations_loss_grad_vs_oracle(opts):
    """The options together: each changes its own step, and none disturbs
    another (the half-step probe of the symmetric splitting starts from the
    psi-tilted default probe; the angular spectrum keeps the exact
    transmission's gradient factor)."""
    ny, nz, ns, nw = 64, 64, 12, 2
    geo = oracle.Geometry(ny, nz, ns, dy_nm=1.0, dz_nm=1.0, alpha_i_deg=(0.2, 0.4), **opts)
    vol = ci.random_volume(77, ny, nz, ns, scale=60)
    meas = _target(geo, vol.astype(np.complex128) * 1.1, 3)
    L_ref, g_ref, I_ref = oracle.loss_grad(geo, vol, meas, 0.8, return_intensity=True)
    L, g, I = G.loss_grad(geo, vol, meas, 0.8, checkpoint_every=5, return_intensity=True)
    assert G.rel(I, I_ref) <= TOL_I
    assert abs(L - L_ref) <= 1e-4 * abs(L_ref)
    assert G.rel(g, g_ref) <= TOL_GRAD


@pytest.mark.parametrize("ny,nz,ns,nw,K,schedule", [(64, 64, 12, 2, 5, 0), (32, 64, 9, 3, 4, 2),
                                                    (64, 128, 1, 2, 1, 0)])
def test_angular_with_symmetric_splitting_vs_oracle(ny, nz, ns, nw, K, schedule):
    """Angular spectrum and the symmetric splitting together: the half step
    before the first slice is the angular-spectrum propagator over Delta/2;
    forward, loss and gradient (checkpointed), one slice included."""
    geo = oracle.Geometry(ny, nz, ns, dy_nm=1.0, dz_nm=1.0, alpha_i_deg=np.linspace(0.15, 0.45, nw),
                          angular=True, strang=True, psi_deg=0.3)
    vol = ci.random_volume(5 * ny + ns, ny, nz, ns, scale=60)
    I_ref = oracle.forward(geo, vol)
    assert G.rel(G.forward(geo, vol, schedule=schedule), I_ref) <= TOL_I
    meas = _target(geo, vol.astype(np.complex128) * 1.1, 8)
    L_ref, g_ref, I2 = oracle.loss_grad(geo, vol, meas, 0.7, return_intensity=True)
    L, g, I = G.loss_grad(geo, vol, meas, 0.7, checkpoint_every=K, return_intensity=True, schedule=schedule)
    assert G.rel(I, I2) <= TOL_I
    assert abs(L - L_ref) <= 1e-4 * abs(L_ref)
    assert G.rel(g, g_ref) <= TOL_GRAD


@pytest.mark.parametrize("strang", [False, True])
@pytest.mark.parametrize("ny,nz,ns", [(64, 64, 10), (128, 64, 1)])
def test_angular_exit_wave_vs_oracle(ny, nz, ns, strang):
    """The exit wave phi_Ns with the angular spectrum (back from (k_y, z) after
    the last propagation; a half step with the symmetric splitting), user probe
    and default probe."""
    geo = oracle.Geometry(ny, nz, ns, dy_nm=1.0, dz_nm=1.0, alpha_i_deg=(0.2, 0.35), angular=True,
                          strang=strang)
    vol = ci.random_volume(9 * ny + ns, ny, nz, ns, scale=60)
    for probe in (None, ci.random_probe(ny + nz, 2, ny, nz)):
        ref = oracle.forward(geo, vol, probe=probe, exit_wave=True)
        got = G.forward(geo, vol, probe=probe, exit_wave=True)
        assert G.rel(got, ref) <= TOL_I


# --------------------------------------------------------------------------
# forward parity
# --------------------------------------------------------------------------
@pytest.mark.parametrize("seed", range(10))
def test_forward_small_pillars(seed):
    """64x64 at 2 nm, 32 slices of 20 nm, 0.3 deg, Si + 1-3 Au pillars."""
    geo = oracle.Geometry(64, 64, 32, alpha_i_deg=(0.3,))
    vol = ci.pillars_small(seed)
    ref = oracle.forward(geo, vol)
    got = G.forward(geo, vol)
    assert G.rel(got, ref) <= TOL_I


@pytest.mark.parametrize("ny,nz,ns,nw", [
    (8, 8, 3, 1), (16, 32, 5, 1), (32, 16, 7, 2), (1, 64, 4, 1), (64, 1, 4, 1), (2, 2, 2, 1),
    (1, 1, 3, 1), (128, 64, 9, 3), (64, 256, 6, 2), (256, 64, 5, 1), (4, 512, 3, 1),
    (512, 4, 3, 1), (33 - 1, 1024, 2, 1), (1024, 32, 2, 1),
])
def test_forward_shapes(ny, nz, ns, nw):
    """Ragged and degenerate grids, several tiles, several wavefields."""
    angles = np.linspace(0.1, 0.5, nw)
    geo = oracle.Geometry(ny, nz, ns, alpha_i_deg=angles)
    vol = ci.random_volume(ny * 7 + nz, ny, nz, ns, scale=50)
    ref = oracle.forward(geo, vol)
    got = G.forward(geo, vol)
    assert G.rel(got, ref) <= TOL_I


def test_forward_user_probe_and_field():
    geo = oracle.Geometry(64, 128, 12, alpha_i_deg=(0.2, 0.4))
    vol = ci.random_volume(5, 64, 128, 12, scale=50)
    probe = ci.random_probe(5, 2, 64, 128)
    ref_I, ref_psi = oracle.forward(geo, vol, probe=probe, return_field=True)
    I, psi = G.forward(geo, vol, probe=probe, return_field=True)
    assert G.rel(I, ref_I) <= TOL_I
    assert G.rel(psi, ref_psi) <= TOL_I


def test_forward_max_size():
    geo = oracle.Geometry(1024, 1024, 3, alpha_i_deg=(0.25,))
    vol = ci.random_volume(17, 1024, 1024, 3, scale=40)
    assert G.rel(G.forward(geo, vol), oracle.forward(geo, vol)) <= TOL_I


def test_exit_wave_gaussian_free_space():
    """Near field: Gaussian beam against the analytic Fresnel solution."""
    ny = nz = 64
    ns, delta, w0 = 32, 20.0, 10.0
    geo = oracle.Geometry(ny, nz, ns, slice_nm=delta, alpha_i_deg=(0.0,))
    probe = ci.gaussian_probe(ny, nz, 2.0, 2.0, w0)[None]
    out = G.forward(geo, np.zeros((ns, nz, ny)), probe=probe, exit_wave=True)[0]
    k = 2 * np.pi / geo.wavelength_nm
    z = (np.arange(nz) - nz // 2) * 2.0
    zz, yy = np.meshgrid(z, z, indexing="ij")
    W2 = w0 ** 2 + 2j * ns * delta / k
    ref = (w0 ** 2 / W2) * np.exp(-(zz ** 2 + yy ** 2) / W2)
    assert np.abs(out - ref).max() < 1e-5


def test_norm_conservation():
    geo = oracle.Geometry(128, 128, 40, alpha_i_deg=(0.3,))
    vol = ci.random_volume(8, 128, 128, 40, scale=30).real.astype(np.complex64)
    probe = ci.random_probe(8, 1, 128, 128)
    I = G.forward(geo, vol, probe=probe)
    assert abs(I.sum(dtype=np.float64) / (np.abs(probe.astype(np.complex128)) ** 2).sum() - 1) < 1e-5


def test_forward_deterministic():
    geo = oracle.Geometry(256, 256, 16, alpha_i_deg=(0.1, 0.2, 0.3))
    vol = ci.random_volume(2, 256, 256, 16)
    a = G.forward(geo, vol)
    b = G.forward(geo, vol)
    assert np.array_equal(a, b)


# --------------------------------------------------------------------------
# gradient parity
# --------------------------------------------------------------------------
def _target(geo, vol, seed):
    I = oracle.forward(geo, vol)
    rng = np.random.default_rng(seed)
    return (np.sqrt(I) * rng.uniform(0.7, 1.3, I.shape)).astype(np.float32)


@pytest.mark.parametrize("ny,nz,ns,nw,K", [(64, 64, 32, 1, 32), (64, 64, 32, 1, 5), (32, 64, 13, 3, 4),
                                           (128, 32, 20, 2, 7), (16, 16, 1, 1, 32), (8, 256, 9, 1, 1),
                                           (1024, 64, 3, 1, 3), (64, 1024, 3, 2, 2), (1, 64, 5, 1, 2),
                                           (64, 1, 5, 1, 5), (2, 2, 4, 1, 2), (32, 32, 4, 16, 3)])
def test_loss_grad_vs_oracle(ny, nz, ns, nw, K):
    geo = oracle.Geometry(ny, nz, ns, alpha_i_deg=np.linspace(0.15, 0.45, nw))
    vol = ci.random_volume(ny + nz + ns, ny, nz, ns, scale=40)
    meas = _target(geo, vol.astype(np.complex128) * 1.1, 1)
    s = 0.8
    L_ref, g_ref, I_ref = oracle.loss_grad(geo, vol, meas, s, return_intensity=True)
    L, g, I = G.loss_grad(geo, vol, meas, s, checkpoint_every=K, return_intensity=True)
    assert G.rel(I, I_ref) <= TOL_I
    assert abs(L - L_ref) <= 1e-4 * abs(L_ref)
    assert G.rel(g, g_ref) <= TOL_GRAD


def test_checkpoint_interval_does_not_change_the_gradient():
    geo = oracle.Geometry(64, 64, 24, alpha_i_deg=(0.3,))
    vol = ci.pillars_small(4, ns=24)
    meas = _target(geo, vol, 2)
    ref = G.loss_grad(geo, vol, meas, 1.0, checkpoint_every=24)
    for K in (1, 5, 8):
        L, g = G.loss_grad(geo, vol, meas, 1.0, checkpoint_every=K)
        assert L == ref[0]
        assert np.array_equal(g, ref[1])


@pytest.mark.parametrize("ny,nz,ns,nw,K", [(64, 64, 24, 2, 5), (128, 64, 17, 3, 4), (512, 512, 40, 9, 32),
                                           (32, 32, 9, 5, 2)])
def test_split_phase_schedule_is_bitwise_identical(ny, nz, ns, nw, K):
    """Schedule 2 of the angular-spectrum slice loop (two wavefield groups,
    split-phase barriers) reorders only which blocks run which rows and columns
    when: every value is computed by the same arithmetic, so intensities, loss
    and gradient equal schedule 1's.  (The paraxial loop ignores the field.)"""
    geo = oracle.Geometry(ny, nz, ns, alpha_i_deg=np.linspace(0.1, 0.5, nw), angular=True)
    vol = ci.random_volume(ny + ns + nw, ny, nz, ns, scale=40)
    I1 = G.forward(geo, vol, schedule=1)
    I2 = G.forward(geo, vol, schedule=2)
    assert np.array_equal(I1, I2)
    meas = (np.sqrt(I1) * 1.05).astype(np.float32)
    L1, g1, J1 = G.loss_grad(geo, vol, meas, 0.9, checkpoint_every=K, return_intensity=True, schedule=1)
    L2, g2, J2 = G.loss_grad(geo, vol, meas, 0.9, checkpoint_every=K, return_intensity=True, schedule=2)
    assert L1 == L2 and np.array_equal(g1, g2) and np.array_equal(J1, J2)


@pytest.mark.parametrize("opts", [dict(), dict(angular=True, dy_nm=1.0, dz_nm=1.0), dict(strang=True),
                                  dict(exact_transmission=True, psi_deg=0.3)])
def test_adjoint_vs_oracle(opts):
    """mslice_adjoint for a given detector gradient (the autograd path), with
    each propagator and splitting option."""
    geo = oracle.Geometry(64, 32, 10, alpha_i_deg=(0.2, 0.35), **opts)
    vol = ci.random_volume(31, 64, 32, 10, scale=40)
    rng = np.random.default_rng(31)
    gpsi = (rng.normal(size=(2, 32, 64)) + 1j * rng.normal(size=(2, 32, 64))).astype(np.complex64)
    probe = ci.random_probe(31, 2, 64, 32)
    ref = oracle.adjoint(geo, vol, gpsi, probe=probe)
    got = G.adjoint(geo, vol, gpsi, probe=probe, checkpoint_every=3)
    assert G.rel(got, ref) <= TOL_GRAD


def test_reconstruction_gradient_subvolume():
    """256x256x512 Poisson-target reconstruction case (1e6 counts): the CUDA
    gradient on a 16x16x8 sub-volume and overall against the FP64 oracle."""
    geo = oracle.Geometry(256, 256, 512, alpha_i_deg=(0.3,))
    truth = ci.pillar_array(0)
    I_gt = oracle.forward(geo, truth)
    meas, s = ci.poisson_target(I_gt, 1e6, seed=0)
    start = ci.substrate(256, 256, 512)
    L_ref, g_ref = oracle.loss_grad(geo, start, meas, s)
    L, g = G.loss_grad(geo, start, meas, s, checkpoint_every=32)
    assert abs(L - L_ref) <= 1e-4 * abs(L_ref)
    sub = (slice(200, 208), slice(128, 144), slice(120, 136))
    assert G.rel(g[sub], g_ref[sub]) <= TOL_GRAD
    assert G.rel(g, g_ref) <= TOL_GRAD


# --------------------------------------------------------------------------
# errors and the bounded device wait
# --------------------------------------------------------------------------
def test_argument_errors():
    from paper_2212_01253_gb300 import binding as B
    geo = oracle.Geometry(16, 16, 2)
    p = G.params(geo)
    ws = B.workspace(p, B.MSLICE_OP_FORWARD)
    vol = torch.zeros((2, 16, 16), dtype=torch.complex64, device="cuda")
    I = torch.empty((1, 16, 16), dtype=torch.float32, device="cuda")
    with pytest.raises(B.MsliceError) as e:
        B.mslice_forward(p, vol, None, I, None, ws[: ws.numel() // 2])
    assert e.value.code == -5
    p2 = G.params(geo)
    p2.psi_rad[0] = 0.2                             # in-plane angle beyond the paraxial range
    with pytest.raises(B.MsliceError) as e:
        B.mslice_forward(p2, vol, None, I, None, ws)
    assert e.value.code == -1
    p3 = G.params(geo)
    p3.ny = 24                                      # not a power of two
    vol3 = torch.zeros((2, 16, 24), dtype=torch.complex64, device="cuda")
    I3 = torch.empty((1, 16, 24), dtype=torch.float32, device="cuda")
    with pytest.raises(B.MsliceError) as e:
        B.mslice_forward(p3, vol3, None, I3, None, ws)
    assert e.value.code == -1
    with pytest.raises(B.MsliceError) as e:
        B.mslice_forward(p, vol, None, I, None, ws[1:])   # misaligned workspace
    assert e.value.code == -1


def test_bounded_wait_times_out_and_recovers():
    """A grid wait that can never complete gives up after its limit, records
    MSLICE_ETIMEDOUT, and the context stays usable."""
    from paper_2212_01253_gb300 import binding as B
    ws = torch.empty(1 << 20, dtype=torch.uint8, device="cuda")
    B.mslice_debug_wait(4, 0, 200_000_000, ws)
    assert B.mslice_status(ws) == 0
    B.mslice_debug_wait(4, 1, 50_000_000, ws)
    assert B.mslice_status(ws) == -4
    # next call resets the control block; work proceeds normally
    geo = oracle.Geometry(32, 32, 4)
    vol = ci.random_volume(1, 32, 32, 4)
    assert G.rel(G.forward(geo, vol), oracle.forward(geo, vol)) <= TOL_I


# --------------------------------------------------------------------------
# torch.autograd.Function over the C ABI
# --------------------------------------------------------------------------
def test_autograd_function_matches_oracle_adjoint():
    from paper_2212_01253_gb300.autograd import multislice_intensity
    geo = oracle.Geometry(64, 32, 9, alpha_i_deg=(0.2, 0.4))
    vol = ci.random_volume(41, 64, 32, 9, scale=40)
    rng = np.random.default_rng(41)
    wts = rng.uniform(-1, 1, (2, 32, 64)).astype(np.float32)
    v = torch.from_numpy(vol).cuda().requires_grad_(True)
    I = multislice_intensity(v, G.params(geo, checkpoint_every=4))
    loss = (I * torch.from_numpy(wts).cuda()).sum()
    loss.backward()
    # oracle: L = sum w I, dL/dPsi -> g = 2 w Psi
    I_ref, psi_ref = oracle.forward(geo, vol, return_field=True)
    g_ref = oracle.adjoint(geo, vol, 2 * wts * psi_ref)
    assert G.rel(I.detach().cpu().numpy(), I_ref) <= TOL_I
    assert G.rel(v.grad.cpu().numpy(), g_ref) <= TOL_GRAD
