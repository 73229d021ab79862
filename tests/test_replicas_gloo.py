"""The multi-GPU path is replicas only (no data-path collective); its host
logic - disjoint shards per rank and the barrier / max / sum reductions used
for timing - is exercised here with two gloo ranks on the CPU."""
import os
import socket

import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2005_02704_gb300 import replicas


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, lr = replicas.env()
    red = replicas.Reducer(w)
    red.barrier()
    # each rank "times" a different amount of work; the job is as slow as the slowest
    t = 10.0 + rank
    out = {"rank": r, "world": w, "max": red.max(t), "sum": red.sum(1000 * (rank + 1)),
           "seed0": replicas.shard_seed0(r, 512), "shard": list(replicas.shard_scans(7, r, w))}
    red.barrier()
    dist.destroy_process_group()
    q.put(out)


def test_two_gloo_ranks_reduce_and_shard():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted([q.get(timeout=120) for _ in range(world)], key=lambda d: d["rank"])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [d["max"] for d in res] == [11.0, 11.0]
    assert [d["sum"] for d in res] == [3000.0, 3000.0]
    assert res[0]["seed0"] == 2000 and res[1]["seed0"] == 2512
    assert res[0]["shard"] + res[1]["shard"] == list(range(7))


def test_single_process_is_identity():
    red = replicas.Reducer(1)
    red.barrier()
    assert red.max(3.5) == 3.5 and red.sum(2.0) == 2.0
    assert list(replicas.shard_scans(5, 0, 1)) == [0, 1, 2, 3, 4]
