"""Pins of the shrink-wrap support oracle (CPU): a library Gaussian filter,
the closed-form blur of a single voxel, and the behaviour the update exists
for (isolated weak voxels removed, a compact object kept)."""
import numpy as np
import pytest

from oracle import support as S


@pytest.mark.parametrize("sigma", [0.6, 1.0, 1.7])
def test_blur_is_a_truncated_gaussian_filter(sigma):
    import scipy.ndimage
    rng = np.random.default_rng(0)
    th = rng.random((9, 12, 10))
    ref = scipy.ndimage.gaussian_filter(th, sigma, mode="constant", cval=0.0, truncate=3.0)
    np.testing.assert_allclose(S.blur64(th, sigma), ref, rtol=0, atol=1e-12)
    # the FP32 blur is that filter to FP32 rounding
    np.testing.assert_allclose(S.blur(th, sigma), ref, rtol=0, atol=4e-7)


def test_blur_of_one_voxel_is_the_outer_product_of_the_taps():
    sigma = 1.3
    w = np.exp(-np.arange(-4, 5) ** 2 / (2 * sigma ** 2))
    w /= w.sum()
    th = np.zeros((11, 11, 11))
    th[5, 5, 5] = 1.0
    np.testing.assert_allclose(S.blur64(th, sigma)[1:10, 1:10, 1:10], np.einsum("i,j,k->ijk", w, w, w),
                               rtol=0, atol=1e-15)


def test_threshold_extremes():
    rng = np.random.default_rng(1)
    th = rng.random((6, 7, 8)).astype(np.float32)
    out, mask = S.shrinkwrap(th, 1.0, 0.0)
    assert mask.all() and np.array_equal(out, th)
    out, mask = S.shrinkwrap(th, 1.0, 1.0)
    b = S.blur(th, 1.0)
    assert mask.sum() >= 1 and np.all(b[mask] == b.max())


def test_isolated_weak_voxels_are_removed_and_the_object_kept():
    th = np.zeros((16, 16, 16), np.float32)
    th[6:9, 6:9, 6:9] = 1.0
    for p in [(1, 1, 1), (14, 2, 13), (2, 14, 3), (13, 13, 14)]:
        th[p] = 0.05
    out, mask = S.shrinkwrap(th, 1.0, 0.2)
    assert np.all(out[6:9, 6:9, 6:9] == 1.0)
    assert all(out[p] == 0 for p in [(1, 1, 1), (14, 2, 13), (2, 14, 3), (13, 13, 14)])
