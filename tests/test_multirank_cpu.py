"""The multi-GPU path of bench.py is weak scaling over independent problems: each rank plans its own problem,
and only the timing crosses ranks (a barrier and the maximum over ranks).  Here two gloo ranks on the CPU run
that host logic."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, out):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "WORLD_SIZE": str(ws),
                       "RANK": str(rank), "LOCAL_RANK": str(rank)})
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        w, r, local = bench.dist_env()
        ms_local = 10.0 + 5.0 * rank          # rank 1 is the slower one
        dist.barrier()
        ms = bench.max_over_ranks(ms_local, torch.device("cpu"))
        rate = bench.job_rate(4096 * 10, w, ms)
        seeds = [None] * ws
        dist.all_gather_object(seeds, bench.rank_seed(r))
        out[rank] = (w, r, local, ms, rate, seeds)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_weak_scaling_timing():
    ws, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        procs = [ctx.Process(target=_rank_main, args=(r, ws, port, out)) for r in range(ws)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(timeout=120)
            assert p.exitcode == 0
        res = dict(out)
    for r in range(ws):
        w, rank, local, ms, rate, seeds = res[r]
        assert (w, rank, local) == (ws, r, r)
        assert ms == 15.0                      # every rank sees the slowest rank's time
        assert rate == pytest.approx(4096 * 10 * ws / 0.015)
        assert len(set(seeds)) == ws           # independent problems per rank
