"""FP64 oracle of the frame rotation of Eq. 2-3 (sample frame -> lab frame).

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle``: imported by ``tests/``
and nothing in the product path.  Plain numpy in double precision; shares no
code with the CUDA kernels.

Eq. 2 gives the index of refraction in the lab frame as the sample-frame index
under a pitch rotation by the incidence angle alpha_i after a yaw rotation by
the in-plane angle psi (Eq. 3).  Here the axes are (x, z, y): x along the beam
(the slice index j, x = j Delta), z the surface normal (row l, z = l dz), y in
plane (column m, y = m dy).  Both volumes live on that same lattice.

  lab point r = c + M (s - c),   M = R_pitch(alpha) R_yaw(psi)
  R_pitch(alpha): x' = cos(a) x - sin(a) z,  z' = sin(a) x + cos(a) z
  R_yaw(psi):     x' = cos(p) x - sin(p) y,  y' = sin(p) x + cos(p) y

Signs: the pitch makes the sample surface rise along +x in the lab frame, so a
straight beam travelling along +x meets it at alpha from above, which is the
geometry of the tilted probe exp(-i k sin(alpha) z) in the sample frame; the
yaw moves a sample feature toward +y along +x, as the probe
exp(-i k sin(psi) y) moves toward -y.  (The paper prints the matrices but no
axis orientation, so the orientation is fixed by that physics.)

The lab volume at r is the sample volume at s = c + M^T (r - c), by trilinear
interpolation on the sample lattice in index units, with the index clamped to
[0, n-1] per axis (the volume extends beyond its faces by its edge values:
substrate below, vacuum above).  The adjoint scatters each lab value back with
the same weights.
"""
from __future__ import annotations

import numpy as np


def rotation(alpha_rad, psi_rad):
    """M = R_pitch(alpha) R_yaw(psi) on (x, z, y) vectors (Eq. 3)."""
    ca, sa = np.cos(alpha_rad), np.sin(alpha_rad)
    cp, sp = np.cos(psi_rad), np.sin(psi_rad)
    pitch = np.array([[ca, -sa, 0.0], [sa, ca, 0.0], [0.0, 0.0, 1.0]])
    yaw = np.array([[cp, 0.0, -sp], [0.0, 1.0, 0.0], [sp, 0.0, cp]])
    return pitch @ yaw


def _sample_index(shape, spacing, alpha_rad, psi_rad, center_nm):
    """Fractional sample-lattice index (x, z, y) of every lab voxel."""
    ns, nz, ny = shape
    J, Lr, Mc = np.meshgrid(np.arange(ns), np.arange(nz), np.arange(ny), indexing="ij")
    r = np.stack([J * spacing[0], Lr * spacing[1], Mc * spacing[2]], axis=-1).astype(np.float64)
    c = np.asarray(center_nm, dtype=np.float64)
    s = c + (r - c) @ rotation(alpha_rad, psi_rad)      # row vector times M = (M^T (r - c))^T
    return s / np.asarray(spacing, dtype=np.float64)


def _stencil(f, n):
    """Clamped lower index and weight of the upper neighbour along one axis."""
    fc = np.clip(f, 0.0, n - 1.0)
    if n == 1:
        return np.zeros(f.shape, np.int64), np.zeros(f.shape), np.zeros(f.shape, np.int64)
    i0 = np.minimum(np.floor(fc).astype(np.int64), n - 2)
    return i0, fc - i0, i0 + 1


def _weights(shape, spacing, alpha_rad, psi_rad, center_nm):
    f = _sample_index(shape, spacing, alpha_rad, psi_rad, center_nm)
    axes = [_stencil(f[..., a], shape[a]) for a in range(3)]
    for bx in (0, 1):
        for bz in (0, 1):
            for by in (0, 1):
                ix = axes[0][2] if bx else axes[0][0]
                iz = axes[1][2] if bz else axes[1][0]
                iy = axes[2][2] if by else axes[2][0]
                w = ((axes[0][1] if bx else 1 - axes[0][1]) * (axes[1][1] if bz else 1 - axes[1][1])
                     * (axes[2][1] if by else 1 - axes[2][1]))
                yield ix, iz, iy, w


def rotate(vol, spacing, alpha_rad, psi_rad, center_nm):
    """Lab-frame volume [ns][nz][ny] from the sample-frame one (Eq. 2).

    spacing = (Delta, dz, dy) in nm; center_nm = (x, z, y) of the rotation
    centre."""
    vol = np.asarray(vol, dtype=np.complex128)
    out = np.zeros(vol.shape, np.complex128)
    for ix, iz, iy, w in _weights(vol.shape, spacing, alpha_rad, psi_rad, center_nm):
        out += w * vol[ix, iz, iy]
    return out


def rotate_adjoint(g, spacing, alpha_rad, psi_rad, center_nm):
    """Transpose of `rotate`: a lab-frame gradient scattered to the sample frame."""
    g = np.asarray(g, dtype=np.complex128)
    out = np.zeros(g.shape, np.complex128)
    for ix, iz, iy, w in _weights(g.shape, spacing, alpha_rad, psi_rad, center_nm):
        np.add.at(out, (ix, iz, iy), w * g)
    return out


def rotate_at(vol, spacing, alpha_rad, psi_rad, center_nm, idx):
    """`rotate` evaluated only at the lab voxels idx[k] = (j, l, m), for volumes
    too large to resample whole on the host."""
    idx = np.asarray(idx, dtype=np.int64).reshape(-1, 3)
    sp = np.asarray(spacing, dtype=np.float64)
    c = np.asarray(center_nm, dtype=np.float64)
    f = (c + (idx * sp - c) @ rotation(alpha_rad, psi_rad)) / sp
    axes = [_stencil(f[:, a], vol.shape[a]) for a in range(3)]
    out = np.zeros(len(idx), np.complex128)
    for bx in (0, 1):
        for bz in (0, 1):
            for by in (0, 1):
                w = ((axes[0][1] if bx else 1 - axes[0][1]) * (axes[1][1] if bz else 1 - axes[1][1])
                     * (axes[2][1] if by else 1 - axes[2][1]))
                out += w * vol[axes[0][2] if bx else axes[0][0], axes[1][2] if bz else axes[1][0],
                               axes[2][2] if by else axes[2][0]].astype(np.complex128)
    return out
