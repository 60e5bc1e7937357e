"""The multi-rank path of bench.py (N independent replicas, no data-path
collective): the whole-job aggregation across ranks and the per-rank
workload, on CPU with the gloo backend, world size 2."""
import os
import socket

import numpy as np
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t, nb = bench.reduce_ranks(1.0 + rank, 100.0 * (rank + 1), torch.device("cpu"))
    w, U, b = bench.build_workload("dwf_4x4x4x4_ls8", rank)
    q.put((rank, t, nb, float(np.abs(b).sum()), float(np.abs(U).sum())))
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_aggregate_max_time_and_summed_bytes():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, nb, _, _ in res:
        assert t == 2.0  # the slowest rank
        assert nb == 300.0  # all ranks' bytes
    # each replica solves its own source on the same gauge field
    assert res[0][3] != res[1][3]
    assert res[0][4] == res[1][4]
