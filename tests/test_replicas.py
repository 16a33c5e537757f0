"""Replica logic of multi-GPU runs, on CPU ranks over gloo (world size 2):
distinct seeds per rank, the maximum of the elapsed times on every rank,
and the aggregate throughput."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_1904_12228_gb300 import replicas  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, loc = replicas.rank_info()
        seeds = replicas.replica_seeds(1236, 1, r)
        mine = 10.0 + 7.5 * r            # this rank's elapsed milliseconds
        slowest = replicas.max_over_ranks(mine, dist, "cpu")
        dist.barrier()
        out[r] = (r, w, loc, seeds, slowest, replicas.aggregate_throughput(1000, w, slowest))
    finally:
        dist.destroy_process_group()


def test_two_replicas_over_gloo():
    world = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
        res = [out[r] for r in range(world)]
    assert [x[0] for x in res] == [0, 1] and all(x[1] == 2 for x in res) and [x[2] for x in res] == [0, 1]
    assert res[0][3] != res[1][3]                       # distinct scene and adjoint seeds
    assert res[0][4] == res[1][4] == 17.5               # every rank sees the slowest time
    assert res[0][5] == res[1][5] == pytest.approx(2 * 1000 / 0.0175)


def test_single_process_defaults(monkeypatch):
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    assert replicas.rank_info() == (0, 1, 0)
    assert replicas.max_over_ranks(3.0) == 3.0
    with pytest.raises(ValueError):
        replicas.aggregate_throughput(1, 1, 0.0)
