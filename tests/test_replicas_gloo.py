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


def test_single_rank_passes_through():
    import bench
    assert bench.combine_ranks(3.0, 4.0, 5, 6, 1, "cpu") == (3.0, 4.0, 5, 6)
