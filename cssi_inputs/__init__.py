"""Seeded synthetic inputs for the multislice CSSI workloads.

This module only builds inputs: index volumes, probes and noisy targets.  It
holds none of the multislice arithmetic, and both the CUDA path (bench,
tests) and the FP64 oracle (tests) consume what it returns.

Conventions
-----------
* Volume ``vol[x][z][y]`` complex64 = delta + i*beta; x is the slice index
  along the beam, z the surface normal (z index 0 = bottom, substrate), y the
  in-plane transverse axis.  The substrate fills rows ``[0, nz // 2)``.
* Materials are the ones of the paper's samples at 8 keV: Si substrate
  (delta = 7.6e-6, beta = 1.75e-7) and Au structures (delta = 4.7e-5,
  beta = 4.9e-6); vacuum is 0.
* Structures are rectangular Au boxes standing on the Si surface (Table 1
  lists elongated rods and two-layer FIB structures; the footprints used here
  are a stated reading, not the paper's samples, whose data is not public).
"""
from __future__ import annotations

import numpy as np

SI = complex(7.6e-6, 1.75e-7)
AU = complex(4.7e-5, 4.9e-6)

WAVELENGTH_NM = 0.155


def _place(rng, vol, count, h_rows, w_range, l_range, line_frac=0.0, line_range=None,
           max_tries=200):
    """Place up to ``count`` non-overlapping Au boxes on the substrate surface."""
    ns, nz, ny = vol.shape
    surf = nz // 2
    taken = np.zeros((ns, ny), dtype=bool)
    boxes = []
    for _ in range(count):
        for _try in range(max_tries):
            if line_range is not None and rng.random() < line_frac:
                length = int(rng.integers(line_range[0], line_range[1] + 1))
            else:
                length = int(rng.integers(l_range[0], l_range[1] + 1))
            width = int(rng.integers(w_range[0], w_range[1] + 1))
            height = int(rng.integers(h_rows[0], h_rows[1] + 1))
            length, width = min(length, ns), min(width, ny)
            height = min(height, nz - surf)
            x0 = int(rng.integers(0, ns - length + 1))
            y0 = int(rng.integers(0, ny - width + 1))
            if taken[x0:x0 + length, y0:y0 + width].any():
                continue
            taken[x0:x0 + length, y0:y0 + width] = True
            vol[x0:x0 + length, surf:surf + height, y0:y0 + width] = AU
            boxes.append((x0, length, y0, width, height))
            break
    return boxes


def substrate(ny, nz, ns, dtype=np.complex64):
    """Flat Si half-space (rows [0, nz//2)) with vacuum above."""
    vol = np.zeros((ns, nz, ny), dtype=dtype)
    vol[:, : nz // 2, :] = SI
    return vol


def pillars_small(seed, ny=64, nz=64, ns=32, dz_nm=2.0):
    """64x64 grid, 32 slices: Si substrate plus 1-3 Au pillars 10-40 nm tall.

    Footprints: y-width and x-length uniform in [4, 16] pixels / slices."""
    rng = np.random.default_rng(seed)
    vol = substrate(ny, nz, ns)
    n = int(rng.integers(1, 4))
    h = (int(round(10.0 / dz_nm)), int(round(40.0 / dz_nm)))
    _place(rng, vol, n, h, (4, 16), (4, 16))
    return vol


def pillars_large(seed, ny=512, nz=512, ns=1024, dz_nm=2.0, count=50):
    """512x512 grid, 1024 slices: 50 Au pillars or lines 5-60 nm tall on Si.

    Footprints: y-width in [2, 64] px; x-length in [2, 64] slices for pillars,
    [64, ns] for lines (30 % of the structures)."""
    rng = np.random.default_rng(seed)
    vol = substrate(ny, nz, ns)
    h = (max(1, int(round(5.0 / dz_nm))), int(round(60.0 / dz_nm)))
    _place(rng, vol, count, h, (2, 64), (2, 64), line_frac=0.3, line_range=(min(64, ns), ns))
    return vol


def pillar_array(seed, ny=256, nz=256, ns=512, dz_nm=2.0, count=16):
    """Ground-truth structure for reconstruction: ``count`` Au pillars 5-60 nm tall."""
    rng = np.random.default_rng(seed)
    vol = substrate(ny, nz, ns)
    h = (max(1, int(round(5.0 / dz_nm))), int(round(60.0 / dz_nm)))
    _place(rng, vol, count, h, (4, 48), (8, 128))
    return vol


def random_volume(seed, ny, nz, ns, scale=1.0, dtype=np.complex64):
    """Dense random delta/beta in the range of the materials (for parity tests)."""
    rng = np.random.default_rng(seed)
    d = rng.uniform(0.0, 5e-5, size=(ns, nz, ny)) * scale
    b = rng.uniform(0.0, 5e-6, size=(ns, nz, ny)) * scale
    return (d + 1j * b).astype(dtype)


def random_probe(seed, nw, ny, nz, dtype=np.complex64):
    """Random complex probe of unit mean intensity."""
    rng = np.random.default_rng(seed)
    p = rng.normal(size=(nw, nz, ny)) + 1j * rng.normal(size=(nw, nz, ny))
    return (p / np.sqrt(2.0)).astype(dtype)


def gaussian_probe(ny, nz, dy_nm, dz_nm, w0_nm, z0_nm=None, y0_nm=None, ky=0.0, kz=0.0,
                   dtype=np.complex128):
    """exp(-((y-y0)^2 + (z-z0)^2) / w0^2) * exp(i (ky y + kz z)) on the grid y=m dy, z=l dz.

    With ``ny == 1`` the profile is along z only."""
    z = np.arange(nz) * dz_nm
    y = np.arange(ny) * dy_nm
    z0 = (nz // 2) * dz_nm if z0_nm is None else z0_nm
    y0 = (ny // 2) * dy_nm if y0_nm is None else y0_nm
    zz, yy = np.meshgrid(z, y, indexing="ij")
    r2 = (zz - z0) ** 2 + (0.0 if ny == 1 else (yy - y0) ** 2)
    p = np.exp(-r2 / w0_nm ** 2) * np.exp(1j * (ky * yy + kz * zz))
    return p.astype(dtype)


def sponge(vol, rows, kd, strength=0.05, top=True, bottom=True):
    """Add an absorbing beta ramp (quadratic) over ``rows`` rows at the top and bottom.

    ``strength`` is the per-slice amplitude attenuation exponent k*Delta*beta at
    the outermost row; ``kd`` = k*Delta of the geometry."""
    ns, nz, ny = vol.shape
    ramp = (np.arange(1, rows + 1) / rows) ** 2 * strength / kd
    out = vol.astype(np.complex128, copy=True)
    if top:
        out[:, nz - rows:, :] += 1j * ramp[:, None]
    if bottom:
        out[:, :rows, :] += 1j * ramp[::-1][:, None]
    return out.astype(vol.dtype)


def poisson_target(intensity, total_counts=1e6, seed=0):
    """Detector emulation: scale s = total/sum(I), counts ~ Poisson(s I).

    Returns (meas_amp = sqrt(counts) as float32, s)."""
    rng = np.random.default_rng(seed)
    intensity = np.asarray(intensity, dtype=np.float64)
    s = float(total_counts) / float(intensity.sum())
    counts = rng.poisson(s * intensity)
    return np.sqrt(counts).astype(np.float32), s


def batched_jobs(seed, njobs=64):
    """Uneven job list: grids 128..512 (independently per axis), 128-1024 slices,
    incidence 0.1-0.5 deg.  Returns a list of dicts (shapes and angle only)."""
    rng = np.random.default_rng(seed)
    jobs = []
    for _ in range(njobs):
        jobs.append(dict(ny=int(rng.choice([128, 256, 512])), nz=int(rng.choice([128, 256, 512])),
                         ns=int(rng.choice([128, 256, 512, 1024])),
                         alpha_deg=float(rng.uniform(0.1, 0.5)), seed=int(rng.integers(1 << 30))))
    return jobs


def sweep_angles_deg(n=9, lo=0.1, hi=0.5):
    """Incidence angles swept across the Si critical angle (~0.22 deg)."""
    return np.linspace(lo, hi, n)


def boxes_nm(seed, ny, nz, length_nm, dz_nm=2.0, count=20):
    """Au boxes standing on the Si surface, with their extent along the beam in
    nm rather than in slices, so that one structure can be sliced at any
    thickness.  Returns rows (x0_nm, x1_nm, y0, y1, height_rows): x-length
    uniform in [2, 32] % of length_nm, y-width in [2, ny/8] pixels, height
    5-60 nm; footprints do not overlap."""
    rng = np.random.default_rng(seed)
    h = (max(1, int(round(5.0 / dz_nm))), int(round(60.0 / dz_nm)))
    boxes = []
    for _ in range(count):
        for _try in range(200):
            lx = float(rng.uniform(0.02, 0.32)) * length_nm
            x0 = float(rng.uniform(0.0, length_nm - lx))
            wy = int(rng.integers(2, max(3, ny // 8) + 1))
            y0 = int(rng.integers(0, ny - wy + 1))
            ok = all(x0 >= b[1] or x0 + lx <= b[0] or y0 >= b[3] or y0 + wy <= b[2] for b in boxes)
            if ok:
                boxes.append((x0, x0 + lx, y0, y0 + wy, min(int(rng.integers(h[0], h[1] + 1)), nz - nz // 2)))
                break
    return boxes


def slice_boxes(boxes, ny, nz, length_nm, slice_nm, dtype=np.complex64):
    """Si substrate plus the boxes of `boxes_nm`, cut into round(length/slice)
    slices of thickness slice_nm.  A slice's voxel is the box's occupancy
    averaged over the slice's thickness (the fraction of [j D, (j+1) D] that
    the box covers), times the Au index."""
    ns = int(round(length_nm / slice_nm))
    vol = substrate(ny, nz, ns, dtype=np.complex128)
    surf = nz // 2
    edges = np.arange(ns + 1) * slice_nm
    for x0, x1, y0, y1, hgt in boxes:
        frac = np.clip(np.minimum(edges[1:], x1) - np.maximum(edges[:-1], x0), 0.0, None) / slice_nm
        vol[:, surf:surf + hgt, y0:y1] += frac[:, None, None] * AU
    return vol.astype(dtype)
