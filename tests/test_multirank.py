"""The N > 1 paths of bench.py on CPU ranks (gloo, world size 2): ranks take
disjoint waves of the query pool (no data exchange) and the job time is the
maximum over ranks; for a sliced count, ranks take disjoint shares of the
slice assignments, all-gather their partial sums and add them in the C
library."""
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


class _OracleSlicePlan:
    """Stands in, on a CPU rank, for a sliced plan: execute_slices(lo, hi)
    returns the partial sum over the slice assignments [lo, hi), each
    conditioned count (Thm 4.2: the other value of a sliced variable gets
    weight zero) from the oracle, the partial sum taken with the product's
    wmc_combine_results."""

    def __init__(self, cnf, wp, wn, sliced):
        self.cnf, self.wp, self.wn, self.sliced = cnf, wp, wn, sliced

    def info(self, Q):
        from types import SimpleNamespace
        return SimpleNamespace(n_slice_vars=len(self.sliced))

    def execute_slices(self, lo, hi, wq, wnq):
        import oracle
        from paper_2006_15512_b300 import Result, combine_results
        parts = []
        for eta in range(lo, hi):
            cwp, cwn = self.wp.copy(), self.wn.copy()
            for k, v in enumerate(self.sliced):
                if (eta >> k) & 1:
                    cwn[v] = 0.0
                else:
                    cwp[v] = 0.0
            b = oracle.brute_force(self.cnf, cwp, cwn)[0]
            parts.append(Result(b.mant, b.exp2, 0.0, 0, 0.0))
        return [combine_results(parts)]


def _slice_rank(rank, world, port, q):
    """One CPU rank of the sliced count through bench.py's multi-rank path:
    its share of the slice assignments (slice_range), the shares
    all-gathered over gloo and summed with wmc_combine_results."""
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    import oracle
    import wmcgen
    import paper_2006_15512_b300 as w
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    cnf = wmcgen.random_kcnf(14, 40, seed=4)
    wp, wn = wmcgen.weights_complementary(14, 4, 0.1, 0.9)
    plan = _OracleSlicePlan(cnf, wp, wn, [2, 5, 9])  # slice bit k fixes variable sliced[k]
    tot = bench.sliced_count(w, plan, None, None, rank, world, dist, torch.device("cpu"))
    full = oracle.brute_force(cnf, wp, wn)[0]
    q.put((rank, w.slice_range(8, rank, world), tot[0].mant, tot[0].exp2, full.mant, full.exp2))
    dist.destroy_process_group()


def test_two_cpu_ranks_shard_the_slices():
    """Index slicing across processes (Alg. 3, Thm 4.2): two gloo ranks take
    disjoint halves of the 2^3 slice assignments and the exponent-aligned
    sum of their shares equals the unsliced count."""
    import socket
    import torch.multiprocessing as mp
    from oracle import Big
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_slice_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    ranges = sorted(r for _, r, *_ in out)
    assert ranges == [(0, 4), (4, 8)]
    for rank, _, m, e, fm, fe in out:
        assert Big(m, e).rel_diff(Big(fm, fe)) <= 1e-14
