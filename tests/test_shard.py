"""Sharding of independent boxes and requests over ranks, and the combination
of per-rank timings, with world_size 2 over gloo on the CPU."""

import os
import socket

import pytest
import torch.multiprocessing as mp

from paper_1911_04712_gb300.shard import combine, gather_list, shard_boxes, shard_requests
from paper_1911_04712_gb300.workloads import box_mix


def test_box_partition_is_complete_and_balanced():
    specs = box_mix(512, master_seed=0)
    costs = [s.n * s.steps for s in specs]
    for world in (1, 2, 4, 8):
        parts = [shard_boxes(costs, r, world) for r in range(world)]
        flat = sorted(k for p in parts for k in p)
        assert flat == list(range(len(specs)))
        loads = [sum(costs[k] for k in p) for p in parts]
        assert max(loads) <= 1.01 * sum(costs) / world + max(costs)


def test_request_round_robin():
    parts = [shard_requests(10, r, 3) for r in range(3)]
    assert parts == [[0, 3, 6, 9], [1, 4, 7], [2, 5, 8]]


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    units, secs = combine(100.0 * (rank + 1), 2.0 + rank, dist)
    lat = gather_list([rank * 10 + k for k in range(rank + 1)], dist)
    costs = [5, 3, 3, 2, 1]
    mine = shard_boxes(costs, rank, world)
    allmine = gather_list(mine, dist)
    q.put((rank, units, secs, lat, sorted(allmine)))
    dist.destroy_process_group()


def test_two_rank_gloo_combination():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, units, secs, lat, allmine in out:
        assert units == pytest.approx(300.0)      # summed over ranks
        assert secs == pytest.approx(3.0)         # slowest rank
        assert sorted(lat) == [0, 10, 11]
        assert allmine == [0, 1, 2, 3, 4]          # every box owned exactly once
