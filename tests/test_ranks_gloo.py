"""The multi-rank path of bench.py, on the host with gloo and two ranks.

The snap arm shards whole replicas (one system per rank, seed + rank) with no
data-path collective; what crosses ranks is the timing: a barrier, the max of
the per-rank times and the sum of the per-rank particle counts, so that the
reported throughput is every rank's particles over the slowest rank's time.
The reference arm runs on rank 0 alone; the other ranks exit without work.
"""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        g = bench.RankGroup(dist, world, "cpu")
        g.barrier()
        mx = g.max_all(1.5 * (rank + 1))
        sm = g.sum_all(10.0 * (rank + 1))
        thr = g.throughput(n_local=1000 * (rank + 1), steps=50, seconds_local=0.5 + rank)
        seeds = [None] * world
        dist.all_gather_object(seeds, bench.rank_seed(20260921, rank))
        g.barrier()
        q.put((rank, mx, sm, thr, seeds))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_reduce_and_shard():
    import torch.multiprocessing as mp
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
    for rank, mx, sm, thr, seeds in out:
        assert mx == 3.0                       # the slowest rank's number
        assert sm == 30.0                      # every rank's number
        assert thr == pytest.approx((1000 + 2000) * 50 / 1.5)
        assert seeds == [20260921, 20260922]   # one replica per rank, distinct seeds


def test_one_rank_is_the_identity():
    import bench

    class NoDist:
        class ReduceOp:
            MAX = SUM = None

        def barrier(self):
            raise AssertionError("no collective with one rank")

        def all_reduce(self, *a, **k):
            raise AssertionError("no collective with one rank")

    g = bench.RankGroup(NoDist(), 1, "cpu")
    g.barrier()
    assert g.max_all(2.5) == 2.5 and g.sum_all(4.0) == 4.0
    assert g.throughput(100, 10, 0.5) == 2000.0


def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    # a non-zero rank returns before touching its arguments or the oracle
    assert bench.run_reference(None) is None


def test_secondary_leg_failure_is_recorded_at_one_rank_and_raised_at_several():
    import bench

    def boom():
        raise RuntimeError("leg failed")

    out = {}
    bench.run_leg(out, "leg", 1, boom)
    assert out == {"leg": {"error": "RuntimeError: leg failed"}}
    bench.run_leg(out, "ok", 1, lambda: {"value": 1.0})
    assert out["ok"] == {"value": 1.0}
    with pytest.raises(RuntimeError):
        bench.run_leg({}, "leg", 2, boom)
