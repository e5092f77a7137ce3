"""The multi-rank timing logic of bench.py on CPU: two gloo ranks, each with its
own replica time; the job reports the slowest rank and the summed work."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t = bench.max_over_ranks(10.0 + rank)
    out[rank] = (t, bench.whole_job_rate(1000, world, 5, t))
    dist.destroy_process_group()


def test_max_over_ranks_and_rate_gloo():
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.start_processes(_worker, args=(2, port, out), nprocs=2, start_method="spawn")
        res = dict(out)
    assert res[0][0] == res[1][0] == 11.0
    assert res[0][1] == pytest.approx(2 * 1000 * 5 / 0.011)


def test_single_rank_passthrough():
    import bench
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.whole_job_rate(100, 1, 10, 1000.0) == pytest.approx(1000.0)


def test_oracle_all_cores_leg():
    """The all-cores oracle leg: one spawned process per host core, each on its own
    cell range; every worker reports, and the rate is the cells over the slowest."""
    import bench
    import oracle
    oracle.build()
    rate, cores, wall = bench.oracle_rate_all_cores("poisson_q1_8", 512, 16)
    assert cores == len(os.sched_getaffinity(0))
    assert wall > 0 and rate == pytest.approx(cores * 16 / wall)
