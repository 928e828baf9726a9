"""The whole-job figures of bench.py under several ranks (one replica per rank, weak scaling): the
slowest rank's time over all ranks, and the rate of all replicas in that time.  Two gloo ranks on
the CPU."""
import os

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        assert bench.dist_info() == (rank, world, rank)
        # rank r took (10 + r) ms for the stage loop and (50 - r) ms for the FP64 loop
        ms = bench.max_over_ranks([10.0 + rank, 50.0 - rank])
        out[rank] = (ms, bench.whole_job_rate(1000, 4, world, ms[0]))
    finally:
        dist.destroy_process_group()


def test_two_ranks_take_the_slowest_time():
    world = 2
    port = 29500 + os.getpid() % 1000
    with mp.Manager() as man:
        out = man.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        ms, rate = res[r]
        assert ms == [11.0, 50.0]
        assert rate == pytest.approx(1000 * 4 * world / 11e-3)


def test_one_process_is_its_own_maximum():
    import bench
    assert bench.max_over_ranks([3.0, 4.0]) == [3.0, 4.0]
    assert bench.whole_job_rate(1000, 4, 1, 2.0) == pytest.approx(2e6)
