"""Launch-shape autotuner for the persistent slice-loop kernels.

For a grid shape (ny, nz) and a number of wavefields nw it times the forward
slice loop over a short synthetic volume for every candidate launch shape --
the number of persistent blocks and the column-group width of the column
passes (the number of adjacent columns whose z-FFTs one group of threads runs
together) -- and keeps the fastest.  The paraxial slice loop runs one pass per
slice with one grid barrier, so the split-phase schedule (an option of the
angular-spectrum kernels) is not a candidate.  Results are cached per device in a JSON
file next to the built library.  The shape changes only which threads do which
transform, never the arithmetic, so results are bitwise independent of it.
"""
from __future__ import annotations

import json
import os
import threading

import numpy as np
import torch

from . import binding as B
from . import build as _build

_lock = threading.Lock()
_cache = None
MS_THREADS = 256


def _cache_path():
    return os.path.join(_build.BUILD_DIR, "autotune.json")


def _load_cache():
    global _cache
    if _cache is None:
        try:
            _cache = json.load(open(_cache_path()))
        except (OSError, ValueError):
            _cache = {}
    return _cache


def _save_cache():
    try:
        os.makedirs(_build.BUILD_DIR, exist_ok=True)
        tmp = _cache_path() + ".tmp%d" % os.getpid()
        json.dump(_cache, open(tmp, "w"), indent=1, sort_keys=True)
        os.replace(tmp, _cache_path())
    except OSError:
        pass


def col_widths(nz):
    """Usable column-group widths for a column length nz (mirrors the library's check)."""
    T = nz // 32 if nz > 32 else 1
    out = []
    for cw in (2, 4, 8, 16, 32):
        lo = 4 if 32 // T > 4 else 32 // T
        if cw * T <= MS_THREADS and MS_THREADS % (cw * T) == 0 and cw >= lo and (T > 1 or cw == 32):
            out.append(cw)
    return out


def candidates(ny, nz, nw, sms):
    grids = sorted({0, sms, max(1, sms // 2), max(1, sms // 4)})
    return [(g, cw, 1) for g in grids for cw in col_widths(nz)]


def _time_forward(ny, nz, nw, grid, cw, sched, ns=16, reps=3, device="cuda"):
    rng = np.random.default_rng(0)
    vol = torch.from_numpy((rng.uniform(0, 5e-5, (ns, nz, ny)) + 1j * rng.uniform(0, 5e-6, (ns, nz, ny)))
                           .astype(np.complex64)).to(device)
    p = B.make_params(ny, nz, ns, np.linspace(0.1, 0.5, nw), grid_blocks=grid, col_width=cw, schedule=sched)
    ws = B.workspace(p, B.MSLICE_OP_FORWARD, device)
    inten = torch.empty((nw, nz, ny), dtype=torch.float32, device=device)
    B.mslice_forward(p, vol, None, inten, None, ws)
    torch.cuda.synchronize()
    best = float("inf")
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        B.mslice_forward(p, vol, None, inten, None, ws)
        e1.record()
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1))
    if B.mslice_status(ws) != 0:
        raise RuntimeError("device-side wait timed out while tuning")
    return best


def tune(ny, nz, nw, device="cuda", force=False):
    """(grid_blocks, col_width, schedule) for this shape, tuned on first use and cached."""
    dev = torch.device(device)
    key = "v3|%s|%d|%d|%d" % (torch.cuda.get_device_name(dev), ny, nz, nw)
    with _lock:
        cache = _load_cache()
        if not force and key in cache:
            return tuple(cache[key]["shape"])
        sms = torch.cuda.get_device_properties(dev).multi_processor_count
        results = []
        for g, cw, sc in candidates(ny, nz, nw, sms):
            results.append((_time_forward(ny, nz, nw, g, cw, sc, device=dev), g, cw, sc))
        results.sort()
        ms, g, cw, sc = results[0]
        cache[key] = {"shape": [g, cw, sc], "ms_16_slices": ms,
                      "tried": [[r[1], r[2], r[3], r[0]] for r in results]}
        _save_cache()
        return (g, cw, sc)


def apply(p, device="cuda"):
    """Set p.grid_blocks, p.col_width and p.schedule from the tuned shape of (p.ny, p.nz, p.nw)."""
    g, cw, sc = tune(p.ny, p.nz, p.nw, device)
    p.grid_blocks, p.col_width, p.schedule = int(g), int(cw), int(sc)
    return p
