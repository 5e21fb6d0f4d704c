"""Host logic of the N > 1 path on CPU: two gloo ranks.

Independent structures are split between the ranks by index, and the
whole-job rate is the units of all ranks over the slowest rank's time. Both
are checked here without a GPU, with world size 2 over 127.0.0.1."""
import socket

import pytest
import torch.multiprocessing as mp

from paper_2212_01253_gb300.shard import shard, whole_job_rate


@pytest.mark.parametrize("n,world", [(0, 1), (1, 2), (7, 2), (64, 3), (64, 8), (5, 8)])
def test_shard_is_a_balanced_partition(n, world):
    blocks = [shard(n, r, world) for r in range(world)]
    seen = [i for b in blocks for i in b]
    assert seen == list(range(n))                       # disjoint, covering, in order
    sizes = [len(b) for b in blocks]
    assert max(sizes) - min(sizes) <= 1 and sizes == sorted(sizes, reverse=True)


def test_shard_rejects_bad_rank():
    with pytest.raises(ValueError):
        shard(4, 2, 2)
    with pytest.raises(ValueError):
        shard(4, 0, 0)


def test_rate_without_process_group_is_local():
    assert whole_job_rate(1000, 2.0) == (5e5, 2.0)


def _rank(rank, world, port, jobs, out):
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=world)
    try:
        mine = list(shard(jobs, rank, world))
        units = 1000 * len(mine)                        # each structure: 1000 units
        ms = 10.0 * (rank + 1)                          # rank 1 is the slower one
        rate, ms_max = whole_job_rate(units, ms)
        dist.barrier()
        out.put((rank, mine, rate, ms_max))
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_ranks_split_the_batch_and_report_the_whole_job():
    world, jobs = 2, 9
    ctx = mp.get_context("spawn")
    out = ctx.SimpleQueue()
    mp.start_processes(_rank, args=(world, _free_port(), jobs, out), nprocs=world, join=True,
                       start_method="spawn")
    res = sorted(out.get() for _ in range(world))
    assert [r[1] for r in res] == [list(range(0, 5)), list(range(5, 9))]
    for _, _, rate, ms_max in res:
        assert ms_max == 20.0                           # the slowest rank's time
        assert rate == pytest.approx(9000 / 0.020)      # all ranks' units over it
