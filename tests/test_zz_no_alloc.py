"""The allocation-free forward entry point (fixed device workspace inside the
library) gives the same detector images as mslice_forward with a caller
workspace, on two calls in a row; sizes beyond its capacity are refused.

Callers that cannot allocate device memory (inside a foreign graph capture,
real-time or plugin hosts) use this entry point.  The file sorts last so that
a run stopping at the first failure has run every other test first."""
import numpy as np
import pytest
import torch

import cssi_inputs as ci

pytestmark = pytest.mark.gpu

TOL_I = 1e-4


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2212_01253_gb300 import build
    build.build()


def _reference(B, p, vol):
    ws = B.workspace(p, B.MSLICE_OP_FORWARD)
    out = torch.empty((p.nw, p.nz, p.ny), dtype=torch.float32, device="cuda")
    B.mslice_forward(p, vol, None, out, None, ws)
    torch.cuda.synchronize()
    return out


def test_static_forward_matches_workspace_forward_twice():
    from paper_2212_01253_gb300 import binding as B
    cases = [(64, 64, 32, (0.3,), ci.pillars_small(2)),
             (128, 64, 9, (0.1, 0.3, 0.5), ci.random_volume(4, 128, 64, 9, scale=40))]
    for ny, nz, ns, ang, vol_h in cases:
        p = B.make_params(ny, nz, ns, ang)
        vol = torch.from_numpy(vol_h).cuda()
        ref = _reference(B, p, vol)
        for _ in range(2):
            out = torch.full((p.nw, nz, ny), float("nan"), dtype=torch.float32, device="cuda")
            B.mslice_forward_static(p, vol, None, out, None)
            torch.cuda.synchronize()
            err = float(torch.linalg.norm(out - ref) / torch.linalg.norm(ref))
            assert err <= TOL_I, err
            # the status word of the library-owned workspace: no wait ran out
            assert B.mslice_forward_static_status() == 0


def test_static_forward_refuses_oversized_problems():
    from paper_2212_01253_gb300 import binding as B
    p = B.make_params(512, 512, 64, (0.3,))          # 128 MiB of transmission alone
    vol = torch.zeros((64, 512, 512), dtype=torch.complex64, device="cuda")
    out = torch.empty((1, 512, 512), dtype=torch.float32, device="cuda")
    with pytest.raises(B.MsliceError) as e:
        B.mslice_forward_static(p, vol, None, out, None)
    assert e.value.code == -5
