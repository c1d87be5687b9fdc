"""The multi-process path of bench.py (independent replicas, one per rank) on CPU with the
gloo backend and two ranks: the timed region's reduction takes the slowest rank, the
whole-job rate counts every rank's units, and the oracle reference arm runs on rank 0
only (the other ranks return without work)."""
import os
import sys

import pytest

torch = pytest.importorskip("torch")
dist = pytest.importorskip("torch.distributed")
mp = pytest.importorskip("torch.multiprocessing")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t = bench.max_over_ranks(dist, 1.0 + rank, "cpu")
        rate = bench.whole_job_rate(62 * 10, world, t)
        skipped = bench.run_reference(None, rank, world) is None if rank != 0 else True
        out.put((rank, t, rate, skipped))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = 29500 + (os.getpid() % 2000)
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [2.0, 2.0]           # the slower rank's time on both
    assert all(abs(r[2] - 620.0) < 1e-12 for r in res)  # 2 ranks x 620 units / 2 s
    assert all(r[3] for r in res)


def test_single_process_helpers():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(None, 3.5, "cpu") == 3.5
    assert bench.whole_job_rate(10, 4, 2.0) == 20.0
