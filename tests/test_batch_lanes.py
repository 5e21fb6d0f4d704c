"""Host logic of the batched entry points (CPU, no device work): how the
library groups uneven jobs by grid shape, spreads the groups over lanes and
sizes the batch workspace (mslice_batched_plan, mslice_batched_workspace_size)."""
import itertools

import pytest

from paper_2212_01253_gb300 import binding as B


def _jobs(shapes, alphas=None):
    arr = (B.mslice_job * len(shapes))()
    for i, (ny, nz, ns) in enumerate(shapes):
        j = arr[i]
        j.ny, j.nz, j.ns = ny, nz, ns
        j.alpha_i_rad = 0.001 * (1 + i % 7) if alphas is None else alphas[i]
        j.scale = 1.0
        # planning never dereferences the buffers; any 16-byte aligned address
        j.vol = j.meas_amp = j.grad_vol = j.intensity = 0x100000 * (i + 1)
    return arr


SHAPES = [(128, 256, 512), (512, 512, 1024), (128, 256, 512), (256, 128, 128), (128, 128, 128),
          (512, 512, 1024), (128, 256, 512), (256, 256, 256), (128, 128, 128), (64, 64, 1)]


@pytest.mark.parametrize("lanes", [1, 2, 3, 4, 16])
def test_every_group_lands_on_one_lane(lanes):
    common = B.make_params(64, 64, 1)
    arr = _jobs(SHAPES)
    gj, lg = B.mslice_batched_plan(common, arr, B.MSLICE_OP_LOSS_GRAD, lanes)
    assert all(0 <= l < lanes for l in lg)
    if lanes == 1:
        assert set(lg) == {0}
    if lanes >= len(lg):
        # longest first onto the least loaded lane: while lanes are empty,
        # every group opens a new one
        assert sorted(lg) == list(range(len(lg)))


@pytest.mark.parametrize("lanes", [1, 2, 4, 16])
def test_group_grids_are_sized_by_their_tasks(lanes):
    """With lanes > 1 every group runs on the blocks its tasks fill (one row
    task per warp: 256 / (ny / 32) rows a block), at most half of the 152 SMs;
    with one lane on the default grid (0)."""
    common = B.make_params(64, 64, 1)
    arr = _jobs(SHAPES)
    gj, lg, bg = B.mslice_batched_plan(common, arr, B.MSLICE_OP_LOSS_GRAD, lanes, blocks=True)
    if lanes == 1:
        assert set(bg) == {0}
        return
    for g, b in enumerate(bg):
        members = [i for i in range(len(SHAPES)) if gj[i] == g]
        ny, nz, ns = SHAPES[members[0]]
        rows_per_block = 256 // max(1, ny // 32)
        need = -(-nz * len(members) // rows_per_block)
        assert 1 <= b <= 76 and b >= min(need, 76)
    # the 512 x 512 x 1024 pair: 1024 rows (and 1024 columns) of 512 points,
    # 16 rows a block: 64 blocks
    assert bg[gj[SHAPES.index((512, 512, 1024))]] == 64
    # (64, 64, 1): 64 rows of 64 points, 128 rows a block: one block
    assert bg[gj[SHAPES.index((64, 64, 1))]] == 1


def test_batch_workspace_is_the_sum_of_the_group_workspaces():
    common = B.make_params(64, 64, 1, checkpoint_every=32)
    arr = _jobs(SHAPES)
    gj, _ = B.mslice_batched_plan(common, arr, B.MSLICE_OP_LOSS_GRAD, 1)
    align = lambda x: (x + 255) // 256 * 256
    expect = align(8 * (max(gj) + 1))
    for g in range(max(gj) + 1):
        members = [i for i in range(len(SHAPES)) if gj[i] == g]
        ny, nz, ns = SHAPES[members[0]]
        p = B.make_params(ny, nz, ns, [0.1] * len(members), checkpoint_every=32, flags=B.MSLICE_PER_STRUCTURE)
        expect += align(B.mslice_workspace_size(p, B.MSLICE_OP_LOSS_GRAD))
    assert B.mslice_batched_workspace_size(common, arr, B.MSLICE_OP_LOSS_GRAD, 1) == expect


def test_invalid_batches_are_refused():
    common = B.make_params(64, 64, 1)
    with pytest.raises(B.MsliceError) as e:
        B.mslice_batched_plan(common, _jobs([(96, 64, 4)]), B.MSLICE_OP_FORWARD, 1)
    assert e.value.code == -1
    arr = _jobs([(64, 64, 4)])
    arr[0].vol = 0x100008                        # not 16-byte aligned
    with pytest.raises(B.MsliceError):
        B.mslice_batched_plan(common, arr, B.MSLICE_OP_FORWARD, 1)
    for lanes in (0, 17):
        with pytest.raises(B.MsliceError):
            B.mslice_batched_plan(common, _jobs([(64, 64, 4)]), B.MSLICE_OP_FORWARD, lanes)
    ang = B.make_params(64, 64, 1, flags=B.MSLICE_ANGULAR)
    with pytest.raises(B.MsliceError) as e:
        B.mslice_batched_plan(ang, _jobs([(64, 64, 4)]), B.MSLICE_OP_FORWARD, 1)
    assert e.value.code == -2
    arr = _jobs([(64, 64, 4)])
    arr[0].scale = 0.0                           # loss + gradient needs s > 0
    with pytest.raises(B.MsliceError):
        B.mslice_batched_plan(common, arr, B.MSLICE_OP_LOSS_GRAD, 1)
    assert B.mslice_batched_plan(common, arr, B.MSLICE_OP_FORWARD, 1)[0] == [0]    # the forward has no s
    arr[0].intensity = None                      # the forward needs the intensity buffer
    with pytest.raises(B.MsliceError):
        B.mslice_batched_plan(common, arr, B.MSLICE_OP_FORWARD, 1)
