"""The synthetic input generators (CPU): structures sliced at any thickness."""
import numpy as np

import cssi_inputs as ci


def test_sliced_boxes_keep_the_integral_along_the_beam():
    """Slice averaging keeps the integral of the index along x at every slice
    thickness, and never exceeds the Au index above the surface."""
    ny, nz, length = 64, 32, 4000.0
    boxes = ci.boxes_nm(3, ny, nz, length, count=8)
    assert len(boxes) == 8
    ref = None
    for d in (200.0, 50.0, 12.5):
        v = ci.slice_boxes(boxes, ny, nz, length, d).astype(np.complex128)
        assert v.shape == (int(round(length / d)), nz, ny)
        top = v[:, nz // 2:, :]
        assert np.all(top.real >= 0) and np.all(top.real <= ci.AU.real * (1 + 1e-6))
        integral = top.sum(axis=0) * d
        if ref is None:
            ref = integral
        assert np.abs(integral - ref).max() <= 1e-6 * np.abs(ref).max()
        np.testing.assert_array_equal(v[:, : nz // 2, :], np.complex64(ci.SI))


def test_box_footprints_do_not_overlap():
    boxes = ci.boxes_nm(1, 128, 64, 10000.0, count=20)
    for i, a in enumerate(boxes):
        for b in boxes[i + 1:]:
            assert a[1] <= b[0] or b[1] <= a[0] or a[3] <= b[2] or b[3] <= a[2]
