"""The multi-GPU run is replicas only: each rank runs the whole step on its
own GPU and the single collective is the max (step time) / sum (launches)
over ranks.  That host logic runs here on two gloo ranks on CPU."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        assert bench.dist_env()[:2] == (ws, rank)
        mx = bench.reduce_over_ranks(10.0 + rank, ws, "max")
        sm = bench.reduce_over_ranks(100 + rank, ws, "sum")
        one = bench.reduce_over_ranks(3.0, 1, "max")
        out.put((rank, mx, sm, one))
    finally:
        dist.destroy_process_group()


def test_replica_reductions_over_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res == [(0, 11.0, 201.0, 3.0), (1, 11.0, 201.0, 3.0)]
