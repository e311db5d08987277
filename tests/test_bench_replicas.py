"""The benchmark's multi-rank path on CPU: two gloo ranks (replicas only --
the path has no exchange step), rendezvous on 127.0.0.1, max/sum over ranks,
the whole-job rate, and the reference arm's rank > 0 exit."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
mp = pytest.importorskip("torch.multiprocessing")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench
    w, r, local = bench.dist_init(world)
    assert (w, r, local) == (world, rank, rank)
    bench.barrier(w)
    mx = bench.max_over_ranks(float(rank + 1), w)
    sm = bench.sum_over_ranks(10.0 * (rank + 1), w)
    # rank k processed 1000 (k + 1) units in (k + 1) / 2 seconds
    rate = bench.job_rate(1000 * (rank + 1), 0.5 * (rank + 1), w)

    class A:  # the reference arm returns at once on ranks > 0
        seed, warmup, steps, cpu_bins, gpus = 1, 0, 1, 1, world

    ref = bench.run_reference(A, w, rank) if rank > 0 else None
    bench.barrier(w)
    import torch.distributed as dist
    dist.destroy_process_group()
    out.put((rank, mx, sm, rate, ref))


def test_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(k, 2, port, q)) for k in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, mx, sm, rate, ref in res:
        assert mx == 2.0 and sm == 30.0
        assert rate == pytest.approx(3000 / 1.0)
        assert ref is None
