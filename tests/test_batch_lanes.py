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


def _cost(shape, n):
    ny, nz, ns = shape
    return n * ny * nz * ns / 4e10 + ns * 2.5e-5


def test_groups_hold_one_shape_in_job_order():
    common = B.make_params(64, 64, 1)
    arr = _jobs(SHAPES)
    gj, lg = B.mslice_batched_plan(common, arr, B.MSLICE_OP_LOSS_GRAD, 1)
    # groups numbered by first appearance
    assert gj == [0, 1, 0, 2, 3, 1, 0, 4, 3, 5]
    assert lg == [0] * 6


def test_a_shape_with_more_jobs_than_one_run_holds_is_split():
    common = B.make_params(64, 64, 1)
    arr = _jobs([(64, 64, 4)] * (B.MSLICE_MAX_ANGLES + 3))
    gj, lg = B.mslice_batched_plan(common, arr, B.MSLICE_OP_FORWARD, 1)
    assert gj == [0] * B.MSLICE_MAX_ANGLES + [1] * 3 and len(lg) == 2


@pytest.mark.parametrize("lanes", [1, 2, 3, 4, 16])
def test_lanes_longest_first_onto_the_least_loaded(lanes):
    common = B.make_params(64, 64, 1)
    arr = _jobs(SHAPES)
    gj, lg = B.mslice_batched_plan(common, arr, B.MSLICE_OP_LOSS_GRAD, lanes)
    groups = sorted(set(gj))
    cost = [_cost(SHAPES[gj.index(g)], gj.count(g)) for g in groups]
    assert all(0 <= l < lanes for l in lg)
    loads = [sum(c for c, l in zip(cost, lg) if l == k) for k in range(lanes)]
    # greedy longest-first: the heaviest lane exceeds the lightest by at most one group
    assert max(loads) - min(loads) <= max(cost) + 1e-12
    # the most expensive group starts lane 0, the next ones the next empty lanes
    order = sorted(range(len(cost)), key=lambda k: (-cost[k], k))
    for rank, k in enumerate(order[:min(lanes, len(cost))]):
        assert lg[k] == rank


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
