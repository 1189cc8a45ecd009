"""The benchmark's multi-rank path on the CPU: two gloo ranks (world size 2,
127.0.0.1), as torchrun would start them.  Every rank runs an independent
replica (its own seed); the whole-job figure sums the units every rank
processed and divides by the slowest rank's time."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, lr = bench.rank_info()
        units, seconds = bench.aggregate_over_ranks(100.0 * (rank + 1), 0.5 + rank, None)
        out[rank] = (r, w, lr, units, seconds, bench.rank_seed(rank), bench.config_dict(w)["parallelism"])
    finally:
        dist.destroy_process_group()


@pytest.mark.timeout(120)
def test_two_gloo_ranks_aggregate_units_and_slowest_time():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        r, w, lr, units, seconds, seed, par = res[rank]
        assert (r, w, lr) == (rank, world, rank)
        assert units == 300.0 and seconds == 1.5  # 100 + 200 units, max(0.5, 1.5) s
        assert par == "replicas2"
    assert res[0][5] != res[1][5]  # independent circuits per rank


def test_single_rank_is_unchanged():
    assert bench.aggregate_over_ranks(7.0, 2.0) == (7.0, 2.0)
