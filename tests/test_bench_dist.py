"""Host-side logic of multi-rank benchmark runs (replicas), on CPU with gloo:
ranks exchange only the timed duration (max) and the cells processed (sum)."""
import os

import pytest


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    r = bench.aggregate({"seconds": 1.0 + rank, "cells": 1000 * (rank + 1)}, world)
    rank_env = bench.dist_env()
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, r, rank_env))


def test_aggregate_two_ranks():
    mp = pytest.importorskip("torch.multiprocessing")
    import socket
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, r, env in res:
        assert r == {"max_s": 2.0, "cells": 3000.0}
        assert env[0] == rank and env[1] == 2


def test_aggregate_single_rank_is_local():
    import bench
    assert bench.aggregate({"seconds": 0.5, "cells": 7}, 1) == {"max_s": 0.5, "cells": 7}
