"""The multi-process path of bench.py on CPU (gloo, two ranks): replicas take distinct PURSEs, the
whole-job step time is the slowest rank's and the executed evaluations add up."""
import os
import socket

import pytest
import torch.multiprocessing as mp

import bench


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t, e = bench.combine_ranks(0.5 + rank, 1000 * (rank + 1), dist, "cpu")
        p = bench.make_purse(rank)
        out.put((rank, t, e, float(p.obs[0, 0])))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_rank_combination_on_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for pr in procs:
        pr.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    assert all(r[1] == pytest.approx(1.5) for r in res)          # slowest rank's step time
    assert all(r[2] == pytest.approx(3000.0) for r in res)       # evaluations of both ranks
    assert res[0][3] != res[1][3]                                # each replica its own PURSE


def test_single_process_combination_is_identity():
    assert bench.combine_ranks(0.25, 7, None, "cpu") == (0.25, 7.0)
