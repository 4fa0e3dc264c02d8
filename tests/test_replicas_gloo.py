"""The multi-process (replicas) path of bench.py, on CPU with the gloo backend and two ranks: each
rank gets its own pencil (a distinct shift), and the job's figures are the slowest rank's time and
every rank's eigenpairs."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, out):
    import torch.distributed as dist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        assert bench.dist_env() == (ws, rank, rank)
        spec, es, sigma = bench.workload("c1", rank)
        # rank-dependent inputs: times 10 + rank ms, eigenpairs 20 + rank
        res = bench.combine_ranks(10.0 + rank, 100.0 + 5 * rank, 20 + rank, 18 + rank, ws, "cpu")
        out[rank] = (res, sigma)
    finally:
        dist.destroy_process_group()


def test_two_rank_replicas_combine_max_time_and_summed_pairs():
    ws = 2
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank_main, args=(ws, port, out), nprocs=ws, join=True)
        res = dict(out)
    for rank in range(ws):
        (dev_ms, e2e_ms, good, e2e_good), _ = res[rank]
        assert dev_ms == 11.0 and e2e_ms == 105.0  # slowest rank
        assert good == 41.0 and e2e_good == 37.0    # all ranks' eigenpairs
    assert res[0][1] != res[1][1]                   # distinct shifts: independent problems


def _rank_solve(rank, ws, port, out):
    """One replica's real work on the host: its own shift (bench.workload's rule), the oracle's
    pencil, the nev eigenpairs nearest that shift and their explicit residuals; then the job's
    figures through bench.combine_ranks over gloo."""
    import time

    import numpy as np
    import torch.distributed as dist

    import bench
    from oracle import eig, gas, pencil
    from paper_2607_27440_b300 import workloads as wl
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        _, es, sigma = bench.workload("c1", rank)
        spec = wl.tiny(nx=9, qx=4, qy=2, mach=3.0).as_dict()
        t0 = time.perf_counter()
        d = gas.pencil_data(spec)
        A, B = pencil.assemble_dense(spec, d)
        lam, X, _ = eig.interior(A, pencil.boundary_rows(d))
        idx = eig.nearest(lam, sigma, 6)
        res = eig.residuals(spec, d, lam[idx], X[:, idx])
        good = int(np.sum(res <= 1e-10))
        ms = (time.perf_counter() - t0) * 1e3
        out[rank] = (bench.combine_ranks(ms, ms, good, good, ws, "cpu"), ms, good, sigma, tuple(np.sort_complex(lam[idx])))
    finally:
        dist.destroy_process_group()


def test_two_rank_replicas_each_solve_their_own_pencil():
    """Two gloo ranks each solve their own shifted problem on the host: the combined figures are the
    slowest rank's time and the sum of the ranks' verified eigenpairs, identical on every rank."""
    ws = 2
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank_solve, args=(ws, port, out), nprocs=ws, join=True)
        res = dict(out)
    times = [res[r][1] for r in range(ws)]
    goods = [res[r][2] for r in range(ws)]
    assert all(g == 6 for g in goods)                   # every pair verified on its own rank
    for r in range(ws):
        dev_ms, e2e_ms, good, e2e_good = res[r][0]
        assert abs(dev_ms - max(times)) < 1e-9 and abs(e2e_ms - max(times)) < 1e-9
        assert good == sum(goods) and e2e_good == sum(goods)
    assert res[0][3] != res[1][3]                       # distinct shifts


def test_single_rank_passes_through():
    import bench
    assert bench.combine_ranks(3.0, 4.0, 5, 6, 1, "cpu") == (3.0, 4.0, 5, 6)
