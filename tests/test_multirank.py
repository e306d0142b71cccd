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


# --- loop rows of one point split over ranks -------------------------------
#
# The loop contraction of a single point shards over its loop rows (the paper
# distributes the bosonic momenta over MPI ranks, Sec. 3): rank r computes
# the rows of its range, one all-gather completes the row loops on every
# rank, and every rank expands them to all l.  Here the rows are computed by
# the oracle on each CPU rank and gathered over gloo; the expansion of the
# gathered rows must equal the oracle's loops at every l.

def _shard_worker(rank, world, port, root, q):
    sys.path.insert(0, root)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from oracle import loops
        from paper_1604_06296_gb300 import sharded
        from tests.conftest import make_problem
        prob = make_problem(shells=2, nc=6, nf=24, tp=-0.3)
        lam = 0.4
        rows = sharded.row_classes(prob.ncx, prob.ncy)
        par = prob.basis.parity
        pairs = [(m, n) for m in range(prob.nff) for n in range(m, prob.nff)
                 if par[m] * par[n] > 0]
        parts = sharded.row_partition(len(rows), world)
        r0, r1 = parts[rank]
        buf = torch.zeros((2, len(rows), len(pairs)), dtype=torch.float64)
        reps = [rows[r][0][0] for r in range(r0, r1)]
        pp, ph = loops.chi_dot(prob, lam, reps)
        for i, r in enumerate(range(r0, r1)):
            for q_, (m, n) in enumerate(pairs):
                buf[0, r, q_], buf[1, r, q_] = pp[i, m, n], ph[i, m, n]
        sharded.gather_rows(buf, parts, rank, dist)
        # expansion of every row to the l it serves, chi(g l) = C chi(l) C^T
        full = np.zeros((2, prob.nl, prob.nff, prob.nff))
        for r, images in enumerate(rows):
            X = np.zeros((2, prob.nff, prob.nff))
            for q_, (m, n) in enumerate(pairs):
                X[:, m, n] = X[:, n, m] = buf[:, r, q_].numpy()
            for l, g in images:
                C = prob.basis.rep_matrix(np.array(g).reshape(2, 2))
                full[:, l] = C @ X @ C.T
        ref = np.stack(loops.chi_dot(prob, lam))
        err = float(np.abs(full - ref).max() / np.abs(ref).max())
        q.put((rank, parts, err, sum(len(x) for x in rows)))
    finally:
        dist.destroy_process_group()


def test_two_ranks_split_loop_rows_and_gather_equals_oracle():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_shard_worker, args=(r, 2, port, ROOT, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (_, parts, err0, served), (_, _, err1, _) = out
    assert parts[0][0] == 0 and parts[0][1] == parts[1][0] and parts[0][1] > 0
    assert served == 36                       # every l of the 6 x 6 grid, once
    assert err0 < 1e-13 and err1 < 1e-13


def test_row_partition_and_classes():
    sys.path.insert(0, ROOT)
    from paper_1604_06296_gb300 import sharded
    import bench
    for world in (1, 2, 3, 8):
        parts = sharded.row_partition(325, world)
        assert parts[0][0] == 0 and parts[-1][1] == 325
        assert all(a[1] == b[0] for a, b in zip(parts, parts[1:]))
        assert max(b - a for a, b in parts) - min(b - a for a, b in parts) <= 1
    for nc in (8, 24, 48):
        rows = sharded.row_classes(nc, nc)
        assert len(rows) == bench.loop_rows(nc, nc, 4 * nc, 4 * nc)
        assert sorted(l for r in rows for l, _ in r) == list(range(nc * nc))
        assert all(r[0][1] == sharded.C4V[0] for r in rows)
