"""Shrink-wrap support update on the GPU (mslice_shrinkwrap) against the
oracle: the support is an FP32 decision taken the same way on both sides, so
the result is compared bit for bit."""
import numpy as np
import pytest
import torch

from oracle import support as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2212_01253_gb300 import build
    build.build()


@pytest.mark.parametrize("shape,sigma,threshold", [((6, 6, 6), 1.0, 0.2), ((64, 64, 64), 1.5, 0.1),
                                                    ((9, 1, 17), 0.75, 0.3), ((1, 1, 1), 1.0, 0.5),
                                                    ((40, 12, 33), 5.0, 0.05)])
def test_shrinkwrap_vs_oracle_bit_for_bit(shape, sigma, threshold):
    from paper_2212_01253_gb300 import binding as B
    rng = np.random.default_rng(sum(shape))
    th = (rng.random(shape) ** 4 * 4.7e-5).astype(np.float32)      # mostly small, a few large
    ref, mask = S.shrinkwrap(th, sigma, threshold)
    t = torch.from_numpy(th).cuda()
    kept = torch.zeros(1, dtype=torch.int32, device="cuda")
    B.mslice_shrinkwrap(t, sigma, threshold, kept=kept)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(t.cpu().numpy(), ref)
    assert int(kept.item()) == int(mask.sum())


def test_shrinkwrap_rejects_bad_arguments():
    from paper_2212_01253_gb300 import binding as B
    t = torch.zeros((4, 4, 4), dtype=torch.float32, device="cuda")
    with pytest.raises(RuntimeError):
        B.mslice_shrinkwrap(t, 0.0, 0.2)
    with pytest.raises(RuntimeError):
        B.mslice_shrinkwrap(t, 1.0, 1.5)
    with pytest.raises(RuntimeError):
        B.mslice_shrinkwrap(t, 6.0, 0.2)          # radius 18 > 16


def test_reconstructor_applies_the_support_after_the_adam_step():
    """Reconstructor(shrinkwrap_every=2) equals plain steps with
    mslice_shrinkwrap called after every second ADAM step, bit for bit."""
    import cssi_inputs as ci
    import oracle
    from paper_2212_01253_gb300 import binding as B
    from paper_2212_01253_gb300.recon import Reconstructor
    from tests import _gpu as G
    oracle.build()
    ny = nz = 64
    ns = 32
    shape, block, off = (4, 8, 8), (8, 4, 8), (0, 32, 0)
    geo = oracle.Geometry(ny, nz, ns, alpha_i_deg=(0.3,))
    rng = np.random.default_rng(5)
    truth = (rng.random(shape) < 0.3).astype(np.float64) * 4.7e-5
    base = ci.substrate(ny, nz, ns)
    I_gt = oracle.forward(geo, oracle.coarse_to_fine(truth, (ns, nz, ny), block, off, base=base))
    meas, s = ci.poisson_target(I_gt, 1e6, seed=2)
    p = G.params(geo)
    c = B.make_coarse(shape, block, off)
    theta0 = torch.from_numpy((rng.random(shape) * 4.7e-5).astype(np.float32)).cuda()
    args = (p, c, G.dev(base, np.complex64), G.dev(meas, np.float32), s)
    R1 = Reconstructor(*args, theta0=theta0, lr=2e-6, shrinkwrap_every=2, shrinkwrap_sigma=1.0,
                       shrinkwrap_threshold=0.3)
    R2 = Reconstructor(*args, theta0=theta0, lr=2e-6)
    for t in range(1, 5):
        R1.step()
        R2.step()
        if t % 2 == 0:
            B.mslice_shrinkwrap(R2.theta.view(*shape), 1.0, 0.3)
    torch.cuda.synchronize()
    assert torch.equal(R1.theta, R2.theta)
    assert int((R1.theta == 0).sum()) > 0          # the support removed something
