"""Pins of the frame-rotation oracle (Eq. 2-3) on the CPU.

Each test ties ``oracle.rotate`` to something other than its own formula: the
geometry of a tilted surface, numpy's rot90, a rotation built by scipy from
axis-angle vectors, and the transpose identity with the separately written
scatter."""
import numpy as np
import pytest

from oracle import rotate as R

SP = (20.0, 2.0, 2.0)          # Delta, dz, dy in nm


def _crossing(profile, half):
    """Fractional index where a monotone profile crosses `half` (linear interpolation)."""
    k = int(np.nonzero((profile[:-1] - half) * (profile[1:] - half) <= 0)[0][0])
    return k + (half - profile[k]) / (profile[k + 1] - profile[k])


def test_zero_angles_are_the_identity():
    rng = np.random.default_rng(0)
    v = rng.standard_normal((6, 8, 5)) + 1j * rng.standard_normal((6, 8, 5))
    np.testing.assert_array_equal(R.rotate(v, SP, 0.0, 0.0, (50.0, 7.0, 4.0)), v)


@pytest.mark.parametrize("alpha_deg", [0.3, 1.0, -2.0])
def test_pitch_tilts_the_surface_by_alpha_rising_along_the_beam(alpha_deg):
    """A flat substrate seen in the lab frame: in slice J the surface sits at
    z_c + tan(alpha) (x_J - x_c), from the geometry of a plane tilted by
    alpha.  The substrate's edge is a linear ramp over 8 rows, so that the
    half-value level is found exactly by linear interpolation."""
    ns, nz, ny = 48, 64, 2
    c = (ns / 2 * SP[0], (nz / 2 - 0.5) * SP[1], 0.0)      # centre on the surface plane
    ramp = np.clip(0.5 - (np.arange(nz) * SP[1] - c[1]) / (8 * SP[1]), 0.0, 1.0)
    v = np.broadcast_to(ramp[None, :, None], (ns, nz, ny)).copy()
    a = np.deg2rad(alpha_deg)
    lab = R.rotate(v, SP, a, 0.0, c).real
    for J in range(0, ns, 7):
        z = _crossing(lab[J, :, 0], 0.5) * SP[1]
        expect = c[1] + np.tan(a) * (J * SP[0] - c[0])
        assert abs(z - expect) < 1e-9, (J, z, expect)


@pytest.mark.parametrize("psi_deg", [0.5, -3.0])
def test_yaw_moves_a_feature_toward_plus_y_along_the_beam(psi_deg):
    ns, nz, ny = 40, 2, 64
    c = (ns / 2 * SP[0], 0.0, (ny / 2 - 0.5) * SP[2])
    ramp = np.clip(0.5 - (np.arange(ny) * SP[2] - c[2]) / (8 * SP[2]), 0.0, 1.0)
    v = np.broadcast_to(ramp[None, None, :], (ns, nz, ny)).copy()
    p = np.deg2rad(psi_deg)
    lab = R.rotate(v, SP, 0.0, p, c).real
    for J in range(0, ns, 6):
        y = _crossing(lab[J, 0, :], 0.5) * SP[2]
        assert abs(y - (c[2] + np.tan(p) * (J * SP[0] - c[0]))) < 1e-9


def test_quarter_turn_on_a_cube_is_numpy_rot90():
    n = 9
    rng = np.random.default_rng(1)
    v = rng.standard_normal((n, n, 3))
    c = ((n - 1) / 2, (n - 1) / 2, 1.0)
    lab = R.rotate(v, (1.0, 1.0, 1.0), np.pi / 2, 0.0, c).real
    np.testing.assert_allclose(lab, np.rot90(v, 1, axes=(0, 1)), atol=1e-12)


def test_linear_field_is_rotated_exactly():
    """Trilinear interpolation reproduces a linear field, so inside the volume
    the lab value is the field at the rotated point; the rotation here comes
    from scipy's axis-angle construction (pitch about the third axis of the
    right-handed (x, z, y) frame, yaw about the second)."""
    from scipy.spatial.transform import Rotation
    ns, nz, ny = 24, 40, 36
    a, p = np.deg2rad(2.5), np.deg2rad(-4.0)
    M = Rotation.from_rotvec([0.0, 0.0, a]) * Rotation.from_rotvec([0.0, -p, 0.0])
    grad = np.array([0.013 + 0.002j, -0.07 + 0.01j, 0.031 - 0.005j])
    J, L, Mc = np.meshgrid(np.arange(ns), np.arange(nz), np.arange(ny), indexing="ij")
    pos = np.stack([J * SP[0], L * SP[1], Mc * SP[2]], axis=-1)
    v = pos @ grad + (0.5 - 0.25j)
    c = np.array([230.0, 41.0, 33.0])
    lab = R.rotate(v, SP, a, p, c)
    s = c + M.inv().apply((pos - c).reshape(-1, 3)).reshape(pos.shape)
    f = s / np.array(SP)
    inside = np.all((f >= 0) & (f <= np.array([ns, nz, ny]) - 1), axis=-1)
    assert inside.mean() > 0.5
    expect = s @ grad + (0.5 - 0.25j)
    assert np.abs(lab - expect)[inside].max() < 1e-11


@pytest.mark.parametrize("shape,alpha_deg,psi_deg", [((7, 9, 5), 3.0, 0.0), ((6, 8, 10), -1.5, 6.0),
                                                      ((1, 8, 4), 2.0, 1.0)])
def test_adjoint_is_the_transpose(shape, alpha_deg, psi_deg):
    rng = np.random.default_rng(2)
    v = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    u = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    c = (shape[0] * 10.0, shape[1] * 0.7, shape[2] * 1.1)
    a, p = np.deg2rad(alpha_deg), np.deg2rad(psi_deg)
    lhs = np.vdot(R.rotate(v, SP, a, p, c), u)
    rhs = np.vdot(v, R.rotate_adjoint(u, SP, a, p, c))
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def _equivalence_case():
    """Si substrate with four Au boxes and absorbing beta ramps in the top and
    bottom 24 rows; alpha chosen so that k sin(alpha) is m = 17 detector bins."""
    import cssi_inputs as ci
    ny, nz, ns, dz, delta, m = 32, 256, 256, 2.0, 20.0, 17
    alpha = np.arcsin(m * ci.WAVELENGTH_NM / (nz * dz))
    vol = ci.substrate(ny, nz, ns).astype(np.complex128)
    rng = np.random.default_rng(0)
    for _ in range(4):
        x0, lx = rng.integers(0, ns - 60), rng.integers(20, 60)
        y0, h = rng.integers(0, ny - 8), rng.integers(5, 20)
        vol[x0:x0 + lx, nz // 2:nz // 2 + h, y0:y0 + 8] = ci.AU
    ramp = np.zeros(nz)
    ramp[:24] = np.linspace(1, 0, 24) ** 2
    ramp[-24:] = np.linspace(0, 1, 24) ** 2
    vol += 2e-5j * ramp[None, :, None]
    return vol, (ny, nz, ns, dz, delta, m, alpha)


def test_lab_frame_equals_sample_frame_with_a_tilted_probe(oracle_lib):
    """The paper's lab frame (volume rotated by Eq. 2-3, straight beam) and the
    sample frame of the slice loops (probe tilted by alpha) are related by a
    Galilean boost of the paraxial equation: their far fields agree after a
    shift of k sin(alpha) along k_z.  The frames coincide at the entrance
    face (rotation centre x = 0 on the surface)."""
    vol, (ny, nz, ns, dz, delta, m, alpha) = _equivalence_case()
    geo_s = oracle_lib.Geometry(ny, nz, ns, slice_nm=delta, dz_nm=dz, alpha_i_deg=(np.rad2deg(alpha),))
    I_s = oracle_lib.forward(geo_s, vol)[0]
    c = (0.0, (nz / 2 - 0.5) * dz, (ny - 1) / 2 * 2.0)
    geo_l = oracle_lib.Geometry(ny, nz, ns, slice_nm=delta, dz_nm=dz, alpha_i_deg=(0.0,))
    I_l = oracle_lib.forward(geo_l, R.rotate(vol, (delta, dz, 2.0), alpha, 0.0, c))[0]
    shifted = np.roll(I_s, m, axis=0)
    err = np.linalg.norm(I_l - shifted) / np.linalg.norm(I_l)
    assert err < 5e-3
    # the opposite pitch (surface falling away from the beam) is far off
    I_bad = oracle_lib.forward(geo_l, R.rotate(vol, (delta, dz, 2.0), -alpha, 0.0, c))[0]
    assert np.linalg.norm(I_bad - shifted) / np.linalg.norm(I_bad) > 5 * err
    # and without the shift the two frames disagree entirely
    assert np.linalg.norm(I_l - I_s) / np.linalg.norm(I_l) > 0.5


def test_pointwise_evaluation_matches_the_whole_volume():
    rng = np.random.default_rng(4)
    shape = (9, 12, 10)
    v = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    args = (SP, np.deg2rad(1.7), np.deg2rad(-2.2), (60.0, 9.0, 8.0))
    full = R.rotate(v, *args)
    idx = np.stack([rng.integers(0, n, 50) for n in shape], axis=1)
    np.testing.assert_allclose(R.rotate_at(v, *args, idx), full[idx[:, 0], idx[:, 1], idx[:, 2]], rtol=0,
                               atol=1e-14)
