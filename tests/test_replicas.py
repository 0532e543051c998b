"""Multi-process host logic of `bench.py --gpus N` on CPU (gloo, world size 2).

The solver does not shard: under torchrun every rank solves its own
right-hand sides (replicas), and the only collective is the max-over-ranks
reduction of the timings, after which rank 0 reports the whole-job rate.
These tests run that logic in two CPU processes.
"""
import os
import socket
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank-dependent timings: the job takes as long as its slowest rank
        ms = bench.max_over_ranks([10.0 + rank, 50.0 - rank, 0.5 * (rank + 1)], world, "cpu")
        seeds = sorted({bench.rhs_seed(rank, s, j) for s in range(40) for j in range(3)})
        gathered = [None] * world
        dist.all_gather_object(gathered, seeds)
        out[rank] = (ms, gathered)
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_distinct_seeds_world2():
    world = 2
    port = _free_port()
    with mp.get_context("spawn").Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        ms, gathered = res[rank]
        assert ms == [11.0, 50.0, 1.0]
        a, b = set(gathered[0]), set(gathered[1])
        assert len(a) == 120 and len(b) == 120 and not (a & b), "ranks must solve different problems"


def test_single_process_needs_no_collective():
    assert bench.max_over_ranks([3.0, 4.0], 1, "cpu") == [3.0, 4.0]


@pytest.mark.parametrize("world", [1, 2, 4, 8])
def test_job_rate_counts_every_rank(world):
    # three solves per step in 30 ms on each of `world` ranks
    assert bench.job_rate(world, 3, 0.030) == pytest.approx(100.0 * world)


def test_l_shape_sizes_match_the_paper():
    """The L-shape workload uses the paper's domains: (n-1)^2 - (n/2)^2 points
    (N = 12033 ... 784385 in the paper's L-shape table)."""
    from paper_1802_03770_gb300.workloads import l_shape_mask
    assert [int(l_shape_mask(n).sum()) for n in (128, 256, 512, 1024)] == [12033, 48641, 195585, 784385]


def test_octagon_sizes_match_the_paper():
    """The octagonal domain's sizes printed in Table tab:octagon2."""
    from paper_1802_03770_gb300.workloads import octagon_mask
    assert [int(octagon_mask(n).sum()) for n in (128, 256, 512, 1024)] == [14145, 56961, 228609, 915969]
    m = octagon_mask(128)
    assert (m == m[::-1]).all() and (m == m[:, ::-1]).all() and (m == m.T).all()
