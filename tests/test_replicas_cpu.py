"""The N > 1 path: slices shard over ranks with no data exchange, and the
timing reduction (max over ranks) works -- checked with world_size-2 gloo
process groups on CPU."""
import os
import socket

import pytest

from paper_2409_13344_gb300.replicas import shard


def test_shard_partitions_exactly():
    for n in (0, 1, 7, 64, 120):
        for world in (1, 2, 3, 4, 8):
            parts = [shard(n, r, world) for r in range(world)]
            flat = [i for p in parts for i in p]
            assert flat == list(range(n))
            sizes = [len(p) for p in parts]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        shard(4, 2, 2)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    from paper_2409_13344_gb300 import replicas
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, lr = replicas.dist_env()
    mine = replicas.shard(10, r, w)
    t = replicas.max_over_ranks(1.0 + r)
    total = replicas.sum_over_ranks(len(mine))
    dist.barrier()
    dist.destroy_process_group()
    q.put((r, mine, t, total))


def test_two_rank_gloo():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res[0][1] == [0, 1, 2, 3, 4] and res[1][1] == [5, 6, 7, 8, 9]
    assert res[0][2] == res[1][2] == 2.0          # max over ranks
    assert res[0][3] == res[1][3] == 10.0         # every slice counted once
