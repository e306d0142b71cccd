"""Multi-rank path of the benchmark on CPU (gloo, world size 2).

Points of a phase-diagram scan are independent problems, so ranks share no
data: each rank runs its own point(s) and the job's only collective is the
final reduction of the timings (max over ranks) and of the work done (sum
over ranks).  These tests run that reduction between two processes and check
that the ranks draw different points.
"""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, root, q):
    sys.path.insert(0, root)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        secs, units = bench.aggregate_ranks(dist, 1.0 + 0.5 * rank, 10 * (rank + 1), device="cpu")
        q.put((rank, secs, units, bench.rank_tprime(rank), bench.rank_scan_seed(rank)))
    finally:
        dist.destroy_process_group()


def test_two_ranks_reduce_time_by_max_and_work_by_sum():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, ROOT, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, secs, units, _, _ in out:
        assert secs == 1.5 and units == 30.0  # max(1.0, 1.5), 10 + 20 on every rank
    assert out[0][3] != out[1][3]  # different production points (t')
    assert out[0][4] != out[1][4]  # different scan seeds


def test_single_rank_needs_no_collective():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.aggregate_ranks(None, 2.5, 7) == (2.5, 7.0)


def test_ranks_draw_disjoint_scan_points():
    sys.path.insert(0, ROOT)
    import bench
    import workloads as W
    a = W.batch_points(8, bench.rank_scan_seed(0))
    b = W.batch_points(8, bench.rank_scan_seed(1))
    key = lambda q: (q["tp"], q["density"], q["U"], q["shells"], q["nf"])
    assert not set(map(key, a)) & set(map(key, b))
    assert np.all(np.isfinite([q["tp"] for q in a + b]))


def test_ranks_run_different_points_of_the_large_workload():
    sys.path.insert(0, ROOT)
    import bench
    import workloads as W
    tps = [bench.rank_tprime(r, "cfg5") for r in range(8)]
    assert len(set(tps)) == 8 and tps[0] == W.config("cfg5")["tp"]
