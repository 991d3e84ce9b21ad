"""The multi-rank bench path on CPU (gloo, world size 2): each rank flags its
own units (weak scaling, no data-path collective); the job time is the
maximum over ranks and the throughput counts every rank's samples."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = [12.5, 20.0][rank]
    t = bench.max_over_ranks(ms, world, torch.device("cpu"))
    v = bench.job_msamples_per_s(1000, world, 4, t)
    q.put((rank, t, v))
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_and_job_throughput_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [20.0, 20.0]
    # 2 ranks x 1000 samples x 4 steps in 20 ms
    assert res[0][2] == pytest.approx(2 * 1000 * 4 / 0.020 / 1e6)


def test_single_rank_needs_no_process_group():
    assert bench.max_over_ranks(3.0, 1, torch.device("cpu")) == 3.0
    assert bench.dist_env() == (0, 1, 0) or os.environ.get("WORLD_SIZE")
