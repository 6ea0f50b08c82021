"""The benchmark's multi-process path on CPU: two gloo ranks reduce their
per-step times to the maximum and agree on the whole-job throughput (each
rank a replica of the workload; no data-path collective)."""
import os
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local_ms = 10.0 + 5.0 * rank                 # rank 1 is the slower replica
        ms = bench.max_over_ranks(local_ms, torch.device("cpu"))
        value = bench.job_throughput(1440, world, ms)
        q.put((rank, ms, value))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_rank_reduction():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + (os.getpid() % 1000)
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, ms, value in res:
        assert ms == 15.0
        assert value == pytest.approx(2 * 1440 / 15e-3)


def test_dist_env_defaults(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    assert bench.dist_env() == (0, 1, 0)
    monkeypatch.setenv("RANK", "1"); monkeypatch.setenv("WORLD_SIZE", "2"); monkeypatch.setenv("LOCAL_RANK", "1")
    assert bench.dist_env() == (1, 2, 1)


def test_oracle_baseline_sample():
    """The CPU baseline's samples (all host cores and one core): bounded, the
    vesicles they report timed, and the one-core rate the slower."""
    sys.path.insert(0, ROOT)
    import bench
    from paper_1812_04719_gb300 import scenegen as G
    sc = G.scene_small((2, 2, 1), p=4, seed=3)
    nv, secs, threads, desc, one = bench.oracle_sample(sc, 0.5)
    assert 1 <= nv <= sc.n and secs > 0 and threads >= 1 and "random vesicles" in desc
    nv1, secs1, desc1 = one
    assert 1 <= nv1 <= sc.n and secs1 > 0 and "random vesicles" in desc1
