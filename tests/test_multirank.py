"""The N > 1 path of bench.py on CPU ranks (gloo, world size 2): ranks take
disjoint waves of the query pool (no data exchange) and the job time is the
maximum over ranks."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank(rank, world, port, q):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    n_waves, Q, steps = 16, 256, 12
    offs = [bench.wave_offset(s, rank, world, n_waves, Q) for s in range(steps)]
    got = [None] * world
    dist.all_gather_object(got, offs)
    t = bench.max_over_ranks(1.0 + rank, dist, torch.device("cpu"))
    q.put((rank, got, t))
    dist.destroy_process_group()


def test_two_cpu_ranks_shard_the_pool():
    import socket
    import torch.multiprocessing as mp
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, got, t in out:
        assert t == 2.0                       # max over ranks
        a, b = got
        first = set(a[:8]) | set(b[:8])       # 16 waves: the first 8 steps of 2 ranks cover all
        assert len(first) == 16
        assert all(x % 256 == 0 for x in a + b)
        assert set(a[:8]).isdisjoint(set(b[:8]))
