"""Pins of the FP64 oracle against what the physics and mathematics fix.

None of these re-types the oracle's own formula: each compares it with an
independent closed form, a library routine on a special case, brute force, or
a finite-difference / transpose identity, chosen so that a dropped term, a
wrong sign, a wrong scale or a transposed axis fails at least one of them.
"""
import numpy as np
import pytest

import cssi_inputs as ci

pytestmark = pytest.mark.filterwarnings("ignore")

LAM = 0.155
K = 2 * np.pi / LAM


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a - b)) / np.linalg.norm(np.ravel(b)))


# --------------------------------------------------------------------------
# DFT: brute force and library special cases
# --------------------------------------------------------------------------
@pytest.mark.parametrize("n", [1, 2, 4, 8, 16, 32, 64, 128, 256, 512, 1024])
def test_fft_equals_naive_dft(oracle_lib, n):
    rng = np.random.default_rng(n)
    x = rng.normal(size=n) + 1j * rng.normal(size=n)
    for sign in (-1, 1):
        a = oracle_lib.dft1d(x, sign=sign, naive=False)
        b = oracle_lib.dft1d(x, sign=sign, naive=True)
        assert np.abs(a - b).max() <= 1e-13 * max(1.0, np.abs(b).max())


@pytest.mark.parametrize("n", [2, 8, 64, 512])
def test_dft_matches_numpy(oracle_lib, n):
    """Library special case: forward kernel e^{-i}, unnormalised; backward e^{+i}."""
    rng = np.random.default_rng(7 + n)
    x = rng.normal(size=n) + 1j * rng.normal(size=n)
    assert np.abs(oracle_lib.dft1d(x, -1) - np.fft.fft(x)).max() < 1e-12 * n
    assert np.abs(oracle_lib.dft1d(x, +1) - n * np.fft.ifft(x)).max() < 1e-12 * n


@pytest.mark.parametrize("shape", [(4, 8), (32, 32), (16, 64), (64, 16)])
def test_dft2_naive_vs_fft_and_numpy(oracle_lib, shape):
    rng = np.random.default_rng(sum(shape))
    x = rng.normal(size=shape) + 1j * rng.normal(size=shape)
    a = oracle_lib.dft2d(x, naive=False)
    b = oracle_lib.dft2d(x, naive=True)
    assert rel(a, b) < 1e-13
    assert rel(a, np.fft.fft2(x)) < 1e-13


def test_single_vacuum_slice_is_unitary_fft2(oracle_lib):
    """Ns=1, empty volume: Psi = fft2(probe, norm='ortho'), natural order."""
    ny, nz = 32, 16
    geo = oracle_lib.Geometry(ny, nz, 1)
    probe = ci.random_probe(3, 1, ny, nz).astype(np.complex128)
    vol = np.zeros((1, nz, ny), np.complex128)
    I, psi = oracle_lib.forward(geo, vol, probe=probe, return_field=True)
    ref = np.fft.fft2(probe[0], norm="ortho")
    assert np.abs(psi[0] - ref).max() < 1e-13
    assert np.abs(I[0] - np.abs(ref) ** 2).max() < 1e-13


# --------------------------------------------------------------------------
# Free-space Gaussian beam against the analytic paraxial solution
# --------------------------------------------------------------------------
@pytest.mark.parametrize("ny,nz,dy,dz", [(64, 64, 2.0, 2.0), (64, 128, 2.0, 1.0), (1, 128, 2.0, 1.0)])
def test_gaussian_free_space(oracle_lib, ny, nz, dy, dz):
    """phi0 = exp(-r^2/w0^2) propagates over L = Ns*Delta to
    (w0^2/W^2)^{d/2} exp(-r^2/W^2), W^2 = w0^2 + 2iL/k (d = number of transverse axes).

    Checked on the complex exit wave, so the propagator's scale Delta/2k, its
    sign, the k-grid of each axis (dy vs dz) and the FFT normalisation all
    enter."""
    ns, delta, w0 = 32, 20.0, 10.0
    L = ns * delta
    geo = oracle_lib.Geometry(ny, nz, ns, slice_nm=delta, dy_nm=dy, dz_nm=dz, alpha_i_deg=(0.0,))
    probe = ci.gaussian_probe(ny, nz, dy, dz, w0)[None]
    vol = np.zeros((ns, nz, ny), np.complex128)
    out = oracle_lib.forward(geo, vol, probe=probe, exit_wave=True)[0]
    z = (np.arange(nz) - nz // 2) * dz
    y = (np.arange(ny) - ny // 2) * dy
    zz, yy = np.meshgrid(z, y, indexing="ij")
    W2 = w0 ** 2 + 2j * L / K
    d = 1 if ny == 1 else 2
    r2 = zz ** 2 + (0 if ny == 1 else yy ** 2)
    ref = (w0 ** 2 / W2) ** (d / 2) * np.exp(-r2 / W2)
    assert np.abs(out - ref).max() < 1e-10
    # and the wrong-sign solution is far away (the pin can fail)
    bad = (w0 ** 2 / np.conj(W2)) ** (d / 2) * np.exp(-r2 / np.conj(W2))
    assert np.abs(out - bad).max() > 1e-2


# --------------------------------------------------------------------------
# Invariants and uniform media
# --------------------------------------------------------------------------
def test_norm_conservation_without_absorption(oracle_lib):
    ny, nz, ns = 32, 64, 12
    geo = oracle_lib.Geometry(ny, nz, ns, alpha_i_deg=(0.2, 0.4))
    vol = ci.random_volume(1, ny, nz, ns).real.astype(np.complex128) * 20  # beta = 0
    probe = ci.random_probe(2, 2, ny, nz).astype(np.complex128)
    I = oracle_lib.forward(geo, vol, probe=probe)
    for w in range(2):
        assert abs(I[w].sum() / (np.abs(probe[w]) ** 2).sum() - 1) < 1e-12
    # absorption removes power
    vol2 = vol + 1j * 1e-5
    I2 = oracle_lib.forward(geo, vol2, probe=probe)
    assert I2.sum() < I.sum() * (1 - 1e-3)


def test_uniform_medium(oracle_lib):
    """Uniform delta: only a global phase, I unchanged.  Uniform beta:
    I scales by exp(-2 k Delta beta Ns)."""
    ny, nz, ns, delta = 32, 32, 10, 20.0
    geo = oracle_lib.Geometry(ny, nz, ns, slice_nm=delta)
    probe = ci.random_probe(5, 1, ny, nz).astype(np.complex128)
    vac = oracle_lib.forward(geo, np.zeros((ns, nz, ny)), probe=probe)
    d = oracle_lib.forward(geo, np.full((ns, nz, ny), 3e-5 + 0j), probe=probe)
    assert rel(d, vac) < 1e-12
    beta = 2e-6
    b = oracle_lib.forward(geo, np.full((ns, nz, ny), 1j * beta), probe=probe)
    assert rel(b, vac * np.exp(-2 * K * delta * beta * ns)) < 1e-12


def test_periodic_shift_and_mirror_in_y(oracle_lib):
    ny, nz, ns = 32, 32, 8
    geo = oracle_lib.Geometry(ny, nz, ns)
    vol = ci.random_volume(9, ny, nz, ns, scale=30).astype(np.complex128)
    probe = ci.random_probe(9, 1, ny, nz).astype(np.complex128)
    I = oracle_lib.forward(geo, vol, probe=probe)[0]
    Is = oracle_lib.forward(geo, np.roll(vol, 5, axis=2), probe=np.roll(probe, 5, axis=2))[0]
    assert rel(Is, I) < 1e-12
    # mirror y -> m' = -m mod ny; intensity mirrored in k_y
    mirror = lambda a: np.roll(a[..., ::-1], 1, axis=-1)
    Im = oracle_lib.forward(geo, mirror(vol), probe=mirror(probe))[0]
    assert rel(Im, mirror(I)) < 1e-12
    # but a shift along z with a fixed probe is not an invariant (the pin can fail)
    Iz = oracle_lib.forward(geo, np.roll(vol, 5, axis=1), probe=probe)[0]
    assert rel(Iz, I) > 1e-6


# --------------------------------------------------------------------------
# Kinematic (Born) limit of one weak slice
# --------------------------------------------------------------------------
def test_born_single_weak_slice(oracle_lib):
    """t = 1 - i k Delta (delta - i beta) + O((k Delta |v|)^2): away from the
    zero order Psi = F_u((-i k Delta delta - k Delta beta) phi0) for a plane wave."""
    ny, nz, delta = 32, 64, 20.0
    kd = K * delta
    geo = oracle_lib.Geometry(ny, nz, 1, slice_nm=delta, alpha_i_deg=(0.0,))
    rng = np.random.default_rng(4)
    eps = 1e-4
    v = (rng.uniform(0, 1, (1, nz, ny)) + 1j * rng.uniform(0, 0.3, (1, nz, ny))) * eps / kd
    I, psi = oracle_lib.forward(geo, v, return_field=True)
    born = np.fft.fft2(-1j * kd * v[0].real - kd * v[0].imag, norm="ortho")
    mask = np.ones((nz, ny), bool)
    mask[0, 0] = False
    vmax = kd * np.abs(v).max()
    assert rel(psi[0][mask], born[mask]) < 3 * vmax
    # the opposite phase convention is far outside that band
    wrong = np.fft.fft2(1j * kd * v[0].real - kd * v[0].imag, norm="ortho")
    assert rel(psi[0][mask], wrong[mask]) > 0.1
    # zero order: sqrt(N) * mean transmission
    assert abs(psi[0][0, 0] - np.sqrt(nz * ny) * np.exp(-1j * kd * np.conj(v[0])).mean()) < 1e-12


# --------------------------------------------------------------------------
# Fresnel reflectivity of a flat Si substrate across the critical angle
# --------------------------------------------------------------------------
D_SI, B_SI = 7.6e-6, 1.75e-7


def _reflectivity(oracle_lib, adeg, delta=20.0, dz=2.0, nz=1024, w0=50.0, h0=250.0):
    a = np.deg2rad(adeg)
    surf = nz // 2
    ns = int(np.ceil((2.2 * h0 / np.tan(a) + 4 * w0 / np.sin(a)) / delta))
    geo = oracle_lib.Geometry(1, nz, ns, slice_nm=delta, dz_nm=dz, alpha_i_deg=(adeg,))
    one = np.zeros((1, nz, 1), np.complex128)
    one[:, :surf, :] = D_SI + 1j * B_SI
    one = ci.sponge(one, nz // 10, K * delta, strength=0.02 * delta / 20.0)
    vol = np.broadcast_to(one, (ns, nz, 1))
    probe = ci.gaussian_probe(1, nz, 2.0, dz, w0, z0_nm=surf * dz + h0, kz=-K * np.sin(a))[None]
    I = oracle_lib.forward(geo, vol, probe=probe)
    kz = 2 * np.pi * np.fft.fftfreq(nz, dz)
    r_sim = I[0, kz > 0, 0].sum() / (np.abs(probe) ** 2).sum()
    # closed form, weighted by the probe's angular spectrum (downward part)
    A = np.abs(np.fft.fft(probe[0, :, 0])) ** 2
    ap = -kz / K
    m = ap > 0
    q = np.sqrt(ap[m] ** 2 - 2 * D_SI + 2j * B_SI + 0j)
    r = (ap[m] - q) / (ap[m] + q)
    r_exp = (A[m] * np.abs(r) ** 2).sum() / A.sum()
    return r_sim, r_exp


@pytest.mark.slow
@pytest.mark.parametrize("adeg", [0.15, 0.2, 0.25, 0.3, 0.4, 0.5])
def test_fresnel_reflectivity(oracle_lib, adeg):
    """Specular reflectivity r = (a - sqrt(a^2 - 2 delta + 2 i beta)) / (a + ...)
    across alpha_c = sqrt(2 delta) ~ 0.223 deg (R falls from ~0.95 to ~0.003)."""
    r_sim, r_exp = _reflectivity(oracle_lib, adeg)
    assert abs(r_sim - r_exp) < 0.01, (r_sim, r_exp)


@pytest.mark.slow
def test_fresnel_reflectivity_small_angle(oracle_lib):
    """0.1 deg needs a wider beam so that its angular spread stays well below alpha."""
    r_sim, r_exp = _reflectivity(oracle_lib, 0.1, nz=2048, w0=100.0, h0=400.0)
    assert abs(r_sim - r_exp) < 0.01, (r_sim, r_exp)


def test_fresnel_total_reflection_needs_the_substrate(oracle_lib):
    """Without delta in the substrate nothing comes back up."""
    nz, dz, delta, adeg = 512, 2.0, 20.0, 0.2
    a = np.deg2rad(adeg)
    ns = int(2.2 * 200 / np.tan(a) / delta)
    geo = oracle_lib.Geometry(1, nz, ns, slice_nm=delta, dz_nm=dz, alpha_i_deg=(adeg,))
    probe = ci.gaussian_probe(1, nz, 2.0, dz, 50.0, z0_nm=nz // 2 * dz + 150, kz=-K * np.sin(a))[None]
    one = np.zeros((1, nz, 1), np.complex128)
    one[:, : nz // 2, :] = 1j * B_SI
    vol = np.broadcast_to(ci.sponge(one, 48, K * delta, 0.02), (ns, nz, 1))
    I = oracle_lib.forward(geo, vol, probe=probe)
    kz = 2 * np.pi * np.fft.fftfreq(nz, dz)
    assert I[0, kz > 0, 0].sum() / (np.abs(probe) ** 2).sum() < 1e-3


# --------------------------------------------------------------------------
# Slice-thickness convergence (Sec. 3: finer Delta changes little)
# --------------------------------------------------------------------------
def test_slice_thickness_convergence(oracle_lib):
    ny, nz, length = 32, 64, 640.0
    vol_coarse = ci.pillars_small(3, ny=ny, nz=nz, ns=8)
    diffs = []
    prev = None
    for rep in (1, 2, 4, 8):
        ns = 8 * rep
        geo = oracle_lib.Geometry(ny, nz, ns, slice_nm=length / ns)
        vol = np.repeat(vol_coarse, rep, axis=0)
        I = oracle_lib.forward(geo, vol)[0]
        if prev is not None:
            diffs.append(rel(I, prev))
        prev = I
    # first-order splitting: successive changes shrink
    assert diffs[1] < diffs[0] and diffs[2] < diffs[1]


def _paraxial_exact(nz, dz, w, probe, length):
    """exp(L (K + V)) phi0 for a medium uniform along the beam (ny = 1): the
    paraxial equation's generator is K = F^-1 diag(-i k_z^2 / 2k) F plus
    V = diag(-i k (delta - i beta)), exponentiated as a dense matrix."""
    import scipy.linalg
    kz = 2 * np.pi * np.fft.fftfreq(nz, dz)
    F = np.fft.fft(np.eye(nz), axis=0)
    Kop = np.linalg.solve(F, np.diag(-1j * kz ** 2 / (2 * K)) @ F)
    Vop = np.diag(-1j * K * np.conj(w))
    return scipy.linalg.expm(length * (Kop + Vop)) @ probe


@pytest.mark.parametrize("strang,order", [(False, 1), (True, 2)])
def test_splitting_order_against_the_matrix_exponential(oracle_lib, strang, order):
    """In a medium uniform along the beam the slices are exact, so the exit
    wave differs from exp(L (K + V)) phi0 only by the splitting: halving Delta
    halves the error of the transmission-first form and quarters that of the
    symmetric form.  A half step put in the wrong place or left out drops the
    symmetric form back to first order."""
    nz, dz, length = 32, 2.0, 2560.0
    z = np.arange(nz) * dz
    bump = np.exp(-((z - 32.0) / 10.0) ** 2)
    w = 4e-5 * bump + 2e-6j * bump
    probe = np.exp(-((z - 24.0) / 8.0) ** 2).astype(np.complex128)
    exact = _paraxial_exact(nz, dz, w, probe, length)
    errs = []
    for ns in (8, 16, 32, 64):
        geo = oracle_lib.Geometry(1, nz, ns, slice_nm=length / ns, dz_nm=dz, alpha_i_deg=(0.0,), strang=strang)
        vol = np.broadcast_to(w[None, :, None], (ns, nz, 1)).copy()
        out = oracle_lib.forward(geo, vol, probe=probe.reshape(1, nz, 1), exit_wave=True)[0, :, 0]
        errs.append(rel(out, exact))
    ratios = np.array(errs[:-1]) / np.array(errs[1:])
    assert np.all(np.abs(ratios - 2 ** order) < 0.1), ratios
    assert errs[-1] < (1e-4 if strang else 2e-2)


def _mode(ny, nz, a, b):
    """The DFT basis vector of bin (k_z index b, k_y index a) on an nz x ny grid."""
    l, m = np.meshgrid(np.arange(nz), np.arange(ny), indexing="ij")
    return np.exp(2j * np.pi * (a * m / ny + b * l / nz))


def test_angular_spectrum_propagates_a_plane_wave_by_its_exact_phase(oracle_lib):
    """One Fourier mode through vacuum gains exp(i L (sqrt(k^2 - k_perp^2) - k)),
    the Helmholtz phase, at a transverse frequency where the paraxial phase
    is off by 0.15 rad."""
    ny, nz, ns, d, delta = 16, 32, 40, 0.5, 20.0
    a, b = 3, -5
    ky, kz = 2 * np.pi * a / (ny * d), 2 * np.pi * b / (nz * d)
    kp2 = ky * ky + kz * kz
    L = ns * delta
    probe = _mode(ny, nz, a, b)[None]
    vol = np.zeros((ns, nz, ny), np.complex128)
    out = {}
    for angular in (False, True):
        geo = oracle_lib.Geometry(ny, nz, ns, slice_nm=delta, dy_nm=d, dz_nm=d, alpha_i_deg=(0.0,), angular=angular)
        out[angular] = oracle_lib.forward(geo, vol, probe=probe, exit_wave=True)[0]
    exact = probe[0] * np.exp(1j * L * (np.sqrt(K * K - kp2) - K))
    assert np.abs(out[True] - exact).max() < 1e-10
    paraxial = probe[0] * np.exp(-1j * L * kp2 / (2 * K))
    assert np.abs(out[False] - paraxial).max() < 1e-10
    assert np.abs(exact - paraxial).max() > 0.1


def test_angular_spectrum_damps_an_evanescent_mode(oracle_lib):
    """A mode with k_perp > k decays as exp(-L sqrt(k_perp^2 - k^2)) (times the
    carrier phase exp(-i L k) of the propagator's convention)."""
    ny, nz, ns, delta = 16, 4, 4, 0.05
    a = 7
    ky = 2 * np.pi * a / (ny * 0.05)
    assert ky > K
    probe = _mode(ny, nz, a, 0)[None]
    geo = oracle_lib.Geometry(ny, nz, ns, slice_nm=delta, dy_nm=0.05, dz_nm=0.05, alpha_i_deg=(0.0,),
                              angular=True)
    out = oracle_lib.forward(geo, np.zeros((ns, nz, ny)), probe=probe, exit_wave=True)[0]
    L = ns * delta
    exact = probe[0] * np.exp(-L * np.sqrt(ky * ky - K * K)) * np.exp(-1j * L * K)
    assert np.abs(exact).max() < 1e-2
    assert np.abs(out - exact).max() < 1e-13


def test_symmetric_splitting_in_free_space_is_the_full_propagation(oracle_lib):
    """With delta = beta = 0 both splittings propagate the exit wave over
    Ns Delta exactly: the symmetric form's two half steps make one full step."""
    ny, nz, ns = 16, 32, 5
    probe = ci.gaussian_probe(ny, nz, 2.0, 2.0, 6.0)[None]
    vol = np.zeros((ns, nz, ny), np.complex128)
    outs = [oracle_lib.forward(oracle_lib.Geometry(ny, nz, ns, alpha_i_deg=(0.0,), strang=st), vol,
                               probe=probe, exit_wave=True) for st in (False, True)]
    assert np.abs(outs[0] - outs[1]).max() < 1e-13


# --------------------------------------------------------------------------
# Gradient: central finite differences and the transpose identity
# --------------------------------------------------------------------------
def _loss_only(oracle_lib, geo, vol, meas, s, probe):
    I = oracle_lib.forward(geo, vol, probe=probe)
    return float(((np.sqrt(s * I) - meas) ** 2).sum())


def test_loss_matches_forward(oracle_lib):
    ny, nz, ns = 16, 32, 6
    geo = oracle_lib.Geometry(ny, nz, ns, alpha_i_deg=(0.3,))
    vol = ci.random_volume(2, ny, nz, ns, scale=40).astype(np.complex128)
    meas = np.random.default_rng(2).uniform(0.5, 2.0, (1, nz, ny))
    L, g, I = oracle_lib.loss_grad(geo, vol, meas, 0.7, return_intensity=True)
    assert abs(L - _loss_only(oracle_lib, geo, vol, meas, 0.7, None)) < 1e-10 * L
    assert rel(I, oracle_lib.forward(geo, vol)) < 1e-14


def test_exact_transmission_from_refractive_index(oracle_lib):
    """Eq. 1's transmission exp((k/2i) Delta (1 - n^2)) with n = 1 - delta + i beta,
    evaluated directly from n, against the oracle's exact form; the linearised
    form against exp(-i k Delta (delta - i beta)).  One uniform slice and an
    untilted plane wave: the exit wave is the transmission itself."""
    ny, nz = 8, 8
    delta, beta = 3e-3, 4e-4            # large enough that 1 - n^2 differs visibly from 2(delta - i beta)
    vol = np.full((1, nz, ny), delta + 1j * beta)
    k = 2 * np.pi / 0.155
    n = 1 - delta + 1j * beta
    for exact, ref in ((True, np.exp(k / 2j * 20.0 * (1 - n * n))),
                       (False, np.exp(-1j * k * 20.0 * (delta - 1j * beta)))):
        geo = oracle_lib.Geometry(ny, nz, 1, alpha_i_deg=(0.0,), exact_transmission=exact)
        phi = oracle_lib.forward(geo, vol, exit_wave=True)
        assert np.abs(phi - ref).max() < 1e-12
    # the two forms differ by k Delta |w|^2 / 2 in phase (about 3.7e-3 rad here)
    assert abs(np.angle(np.exp(k / 2j * 20.0 * (1 - n * n)) / np.exp(-1j * k * 20.0 * (delta - 1j * beta)))) > 1e-3


@pytest.mark.parametrize("exact,strang,angular", [(False, False, False), (True, False, False),
                                                   (False, True, False), (False, False, True)])
def test_gradient_central_differences(oracle_lib, exact, strang, angular):
    """dL/ddelta and dL/dbeta on a 16x16x8 sub-volume of a 32x32x16 grid."""
    ny, nz, ns = 32, 32, 16
    geo = oracle_lib.Geometry(ny, nz, ns, alpha_i_deg=(0.3,), exact_transmission=exact, strang=strang,
                              angular=angular)
    vol = ci.random_volume(11, ny, nz, ns, scale=40).astype(np.complex128)
    probe = ci.random_probe(11, 1, ny, nz).astype(np.complex128)
    I0 = oracle_lib.forward(geo, vol, probe=probe)
    meas = np.sqrt(I0) * np.random.default_rng(3).uniform(0.5, 1.5, I0.shape)
    s = 1.3
    L, g = oracle_lib.loss_grad(geo, vol, meas, s, probe=probe)
    h = 1e-4 * np.abs(vol).max()
    rng = np.random.default_rng(5)
    # every voxel of the sub-volume for delta would be 2048 x 4 evaluations;
    # a seeded random sample of 96 voxels keeps the CPU suite short
    idx = [(int(rng.integers(4, 12)), int(rng.integers(8, 24)), int(rng.integers(8, 24)))
           for _ in range(96)]
    fd, an = [], []
    for (x, z, y) in idx:
        for part, unit in ((0, 1.0), (1, 1j)):
            vp = vol.copy(); vp[x, z, y] += h * unit
            vm = vol.copy(); vm[x, z, y] -= h * unit
            d = (_loss_only(oracle_lib, geo, vp, meas, s, probe)
                 - _loss_only(oracle_lib, geo, vm, meas, s, probe)) / (2 * h)
            fd.append(d)
            an.append(g[x, z, y].real if part == 0 else g[x, z, y].imag)
    fd, an = np.array(fd), np.array(an)
    assert np.linalg.norm(fd - an) / np.linalg.norm(fd) < 1e-6


def test_adjoint_transpose_identity(oracle_lib):
    """<g, J w>_R = <J^T g, w> with J w the directional derivative of Psi."""
    ny, nz, ns = 16, 16, 10
    geo = oracle_lib.Geometry(ny, nz, ns, alpha_i_deg=(0.25, 0.35))
    vol = ci.random_volume(21, ny, nz, ns, scale=40).astype(np.complex128)
    rng = np.random.default_rng(21)
    w = rng.normal(size=vol.shape) + 1j * rng.normal(size=vol.shape)
    gpsi = rng.normal(size=(2, nz, ny)) + 1j * rng.normal(size=(2, nz, ny))
    h = 1e-3 * np.abs(vol).max() / np.abs(w).max()
    _, pp = oracle_lib.forward(geo, vol + h * w, return_field=True)
    _, pm = oracle_lib.forward(geo, vol - h * w, return_field=True)
    jw = (pp - pm) / (2 * h)
    lhs = float(np.real(np.vdot(gpsi, jw)))
    grad = oracle_lib.adjoint(geo, vol, gpsi)
    rhs = float((grad.real * w.real + grad.imag * w.imag).sum())
    assert abs(lhs - rhs) < 1e-6 * abs(lhs)


def test_loss_seed_zero_amplitude(oracle_lib):
    """Where the model amplitude vanishes the seed is 0 (the sqrt is singular)."""
    ny, nz, ns = 8, 8, 2
    geo = oracle_lib.Geometry(ny, nz, ns)
    probe = np.zeros((1, nz, ny), np.complex128)
    L, g = oracle_lib.loss_grad(geo, np.zeros((ns, nz, ny)), np.ones((1, nz, ny)), 1.0, probe=probe)
    assert L == pytest.approx(nz * ny)
    assert np.all(g == 0)


# --------------------------------------------------------------------------
# Reconstruction helpers: coarse-to-fine map and ADAM
# --------------------------------------------------------------------------
def test_coarse_map_transpose_identity(oracle_lib):
    """<E theta, g>_R = <theta, E^T g> with <u, g>_R = sum Re(u) Re(g) + Im(u) Im(g)."""
    rng = np.random.default_rng(7)
    shape, block, off = (3, 2, 4), (2, 3, 2), (1, 2, 0)
    fine = (8, 9, 9)
    theta = rng.normal(size=shape)
    g = rng.normal(size=fine) + 1j * rng.normal(size=fine)
    Et = oracle_lib.coarse_to_fine(theta, fine, block, off, beta_ratio=0.3)
    lhs = float((Et.real * g.real + Et.imag * g.imag).sum())
    rhs = float((theta * oracle_lib.fine_to_coarse(g, shape, block, off, beta_ratio=0.3)).sum())
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)
    # a constant theta fills exactly its block
    one = oracle_lib.coarse_to_fine(np.ones(shape), fine, block, off, beta_ratio=0.3)
    assert np.count_nonzero(one) == np.prod(shape) * np.prod(block)
    assert np.allclose(one[one != 0], 1 + 0.3j)


def test_adam_first_step_and_convergence(oracle_lib):
    """First step: m_hat = g, v_hat = g^2, so the step is lr * g / (|g| + eps);
    on f = sum (theta - c)^2 ADAM reaches the minimum."""
    g = np.array([2.0, -0.5, 1e-3])
    th, m, v = oracle_lib.adam_step(np.zeros(3), np.zeros(3), np.zeros(3), g, 0.1, 0.9, 0.999, 1e-8, 1)
    assert np.allclose(th, -0.1 * g / (np.abs(g) + 1e-8))
    c = np.array([0.3, -1.2, 2.0])
    th, m, v = np.zeros(3), np.zeros(3), np.zeros(3)
    for t in range(1, 3001):
        th, m, v = oracle_lib.adam_step(th, m, v, 2 * (th - c), 0.01, 0.9, 0.999, 1e-8, t)
    assert np.abs(th - c).max() < 1e-3
    # clamping to [lo, hi]
    th, _, _ = oracle_lib.adam_step(np.zeros(1), np.zeros(1), np.zeros(1), np.array([-1.0]), 1.0, 0.9, 0.999,
                                    1e-8, 1, lo=0.0, hi=0.5)
    assert th[0] == 0.5


def test_coarse_map_block_index_and_snapping(oracle_lib):
    """E with a host material: theta = 0 gives exactly the host index, the map is
    affine in theta with slope 1 + i beta_ratio; snapping picks the nearest level
    and the lower one on a tie."""
    th = np.array([[[0.0, 2.0]], [[1.0, -1.0]]])               # (cx, cz, cy) = (2, 1, 2)
    host = 7.6e-6 + 1.75e-7j
    vol = oracle_lib.coarse_to_fine(th, (4, 3, 4), (2, 1, 2), (0, 1, 0), beta_ratio=0.5, block_index=host)
    assert vol[0, 1, 0] == host and vol[1, 1, 1] == host          # theta = 0
    assert vol[0, 1, 2] == host + 2.0 + 1.0j                       # theta = 2
    assert vol[3, 1, 3] == host - 1.0 - 0.5j                       # theta = -1
    assert vol[0, 0, 0] == 0 and vol[0, 2, 0] == 0                 # outside the block
    got = oracle_lib.snap([0.2, 0.5, 0.51, -3.0, 7.0, 4.0], [0.0, 1.0, 4.0])
    np.testing.assert_array_equal(got, [0.0, 0.0, 1.0, 0.0, 4.0, 4.0])


def test_in_plane_angle_plane_wave_lands_in_one_bin(oracle_lib):
    """A default probe tilted in y by psi with sin(psi) = m lambda / (ny dy) is the
    DFT basis vector of bin -m: through vacuum its far field puts all of the
    intensity, ny nz, into detector column (ny - m) mod ny of row 0."""
    ny, nz, m = 64, 16, 5
    sin_psi = m * 0.155 / (ny * 2.0)
    geo = oracle_lib.Geometry(ny, nz, 3, alpha_i_deg=(0.0,), psi_deg=np.rad2deg(np.arcsin(sin_psi)))
    I = oracle_lib.forward(geo, np.zeros((3, nz, ny)))
    assert I[0, 0, ny - m] == pytest.approx(ny * nz, rel=1e-12)
    assert I.sum() == pytest.approx(ny * nz, rel=1e-12)
    assert I[0, 0, m] < 1e-20


# --------------------------------------------------------------------------
# The 1-D propagator tables P_y, P_z (Eq. 1's "C" of Fig. 1)
# --------------------------------------------------------------------------
def test_propagator_tables_move_a_basis_mode_by_their_product(oracle_lib):
    """Eq. 1: one DFT basis mode exp(2 pi i (a m / ny + b l / nz)) through one
    vacuum slice (exit wave, so the propagation is applied once) comes back as
    itself times P(k_y[a], k_z[b]) = exp(-i Delta (k_y^2 + k_z^2) / 2k).  The
    slice loop builds its own 2-D table (pinned to the analytic Fresnel beam
    above), so the mode's phase fixes P_y[a] P_z[b] from separate code.  The
    axes have different lengths and pixel sizes (ny != nz, dy != dz), so a
    swapped axis or spacing, a missing factor 2 or a sign error fails."""
    ny, nz, dy, dz, delta = 32, 8, 2.0, 0.5, 300.0
    geo = oracle_lib.Geometry(ny, nz, 1, slice_nm=delta, dy_nm=dy, dz_nm=dz, alpha_i_deg=(0.0,))
    py, pz = oracle_lib.propagator_1d(geo)
    assert py.shape == (ny,) and pz.shape == (nz,)
    # unit modulus, even in k (P[f] = P[-f]), 1 at k = 0
    assert np.abs(np.abs(py) - 1).max() < 1e-14 and np.abs(np.abs(pz) - 1).max() < 1e-14
    assert py[0] == 1 and pz[0] == 1
    assert np.abs(py[1:] - py[1:][::-1]).max() < 1e-14
    assert np.abs(pz[1:] - pz[1:][::-1]).max() < 1e-14
    m = np.arange(ny)[None, :]
    l = np.arange(nz)[:, None]
    for a, b in [(1, 0), (0, 1), (3, 2), (ny - 5, nz - 3), (ny // 2, nz // 2), (7, 0), (0, nz - 1)]:
        mode = np.exp(2j * np.pi * (a * m / ny + b * l / nz))
        out = oracle_lib.forward(geo, np.zeros((1, nz, ny)), probe=mode[None], exit_wave=True)[0]
        # the frequency of bin a in cycles per nm, with the sign numpy's fftfreq gives
        fy = (a if a < ny / 2 else a - ny) / (ny * dy)
        fz = (b if b < nz / 2 else b - nz) / (nz * dz)
        closed = np.exp(-1j * delta * LAM * np.pi * (fy * fy + fz * fz))   # Delta (2 pi f)^2 / 2k
        assert np.abs(out - closed * mode).max() < 1e-12, (a, b)
        assert abs(py[a] * pz[b] - closed) < 1e-13, (a, b)
        assert abs(py[a] - np.exp(-1j * delta * LAM * np.pi * fy * fy)) < 1e-13
        assert abs(pz[b] - np.exp(-1j * delta * LAM * np.pi * fz * fz)) < 1e-13


def test_per_view_in_plane_angles_land_in_their_own_bins(oracle_lib):
    """Eq. 2-3 with one in-plane angle per view: view w's default probe with
    sin(psi_w) = m_w lambda / (ny dy) is the DFT basis vector of bin -m_w, so
    through vacuum all of view w's intensity lands in column (ny - m_w) mod ny
    of row 0, whatever the other views' angles."""
    ny, nz = 64, 16
    ms = (5, -3, 0)
    psi = [np.rad2deg(np.arcsin(m * 0.155 / (ny * 2.0))) for m in ms]
    geo = oracle_lib.Geometry(ny, nz, 2, alpha_i_deg=(0.0, 0.0, 0.0), psi_deg=psi)
    I = oracle_lib.forward(geo, np.zeros((2, nz, ny)))
    for w, m in enumerate(ms):
        assert I[w, 0, (ny - m) % ny] == pytest.approx(ny * nz, rel=1e-12)
        assert I[w].sum() == pytest.approx(ny * nz, rel=1e-12)
    # the same views one at a time agree bit for bit
    for w in range(3):
        g1 = oracle_lib.Geometry(ny, nz, 2, alpha_i_deg=(0.0,), psi_deg=psi[w])
        assert np.array_equal(oracle_lib.forward(g1, np.zeros((2, nz, ny)))[0], I[w])
