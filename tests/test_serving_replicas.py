"""Serving on several GPUs as replicas: operator placement by least committed
bytes, one Server (slots, ledger, cache) per device, disjoint request
streams per rank and the host-side gather of latencies.  Host logic with a
fake hierarchy: CPU only (one process with two device ledgers, and two gloo
ranks)."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2602_05686_gb300.serving import (MultiServer, Request, Server, gather_stats, merge_stats,  # noqa: E402
                                            partition, place_operators)


class Fake:
    def __init__(self, problem, stream=None, **kw):
        self.nb = problem["bytes"]

    def stats(self):
        return {"device_bytes": self.nb}

    def solve(self, b, tol=1e-8, check=False):
        return [v * 3 for v in b], {"status": 0, "iters": 2, "rel_res": 1e-9}

    def solve_batch(self, B, tol=1e-8, check=False):
        return [[v * 3 for v in b] for b in B], [{"status": 0, "iters": 2, "rel_res": 1e-9} for _ in B]

    def free(self):
        pass


SIZES = {0: 500, 1: 100, 2: 300, 3: 200, 4: 50, 5: 400}


def requests():
    # operators arrive in the order 0, 1, 2, 3, 4, 5 and come back later
    pattern = [0, 1, 2, 0, 3, 4, 1, 5, 2, 2, 0, 3, 5, 4, 1]
    return [Request(rid=i, op=op, arrival=0.001 * i, rhs=[float(i)]) for i, op in enumerate(pattern)]


def server(make_problem, options, slots=2, hbm_budget=10_000, device=None, **kw):
    s = Server(make_problem, options, slots=slots, hbm_budget=hbm_budget, hierarchy_factory=Fake,
               stream_factory=lambda: None, device=device)
    s._estimate = lambda op: SIZES[op]
    return s


def test_placement_takes_the_least_committed_device():
    place, committed = place_operators(requests(), lambda op: SIZES[op], 2)
    # first arrivals 0,1,2,3,4,5: 0->d0 (500), 1->d1 (100), 2->d1 (400),
    # 3->d1 (600), 4->d0 (550), 5->d0 (950)
    assert place == {0: 0, 1: 1, 2: 1, 3: 1, 4: 0, 5: 0}
    assert committed == [950, 600]
    # the same request list gives the same map (every rank computes it alone)
    assert place_operators(list(reversed(requests())), lambda op: SIZES[op], 2)[0] == place
    # one device takes everything
    assert set(place_operators(requests(), lambda op: SIZES[op], 1)[0].values()) == {0}


def test_multiserver_serves_each_operator_on_one_device():
    probs = {op: {"n": 4, "nnz": 8, "bytes": b} for op, b in SIZES.items()}
    ms = MultiServer(lambda op: probs[op], lambda op: {}, devices=[None, None], slots=2, hbm_budget=10_000,
                     server_factory=server)
    rs = requests()
    out = ms.serve(rs, realtime=False)
    assert out["requests"] == len(rs) and out["failed"] == 0 and out["devices"] == 2
    assert all(r.result == [3.0 * r.rid] for r in rs)
    assert sorted(out["per_device_requests"]) == sorted([sum(1 for r in rs if ms.placement[r.op] == d)
                                                         for d in (0, 1)])
    # one setup per operator: each operator lives on exactly one device
    assert out["setups"] == len(SIZES)
    assert out["p50_s"] <= out["p99_s"]
    for k, s in enumerate(ms.servers):
        assert set(s.cache) == {op for op, d in ms.placement.items() if d == k}
        assert s.stats["peak_committed"] <= 10_000
    ms.close()


def test_merge_stats_percentiles_over_all_requests():
    a = dict(requests=3, wall_s=2.0, latencies=[0.1, 0.2, 0.3], peak_committed=5, setups=1, failed=0)
    b = dict(requests=2, wall_s=4.0, latencies=[0.05, 0.9], peak_committed=7, setups=2, failed=1)
    m = merge_stats([a, b])
    assert m["requests"] == 5 and m["wall_s"] == 4.0 and m["throughput_rps"] == 1.25
    assert m["p50_s"] == 0.2 and m["p99_s"] == 0.9 and m["setups"] == 3 and m["failed"] == 1


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    from paper_2602_05686_gb300.serving import gather_stats, partition
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        rs = requests()
        mine, place = partition(rs, lambda op: SIZES[op], rank, ws)
        probs = {op: {"n": 4, "nnz": 8, "bytes": b} for op, b in SIZES.items()}
        s = server(lambda op: probs[op], lambda op: {})
        local = s.serve(mine, realtime=False)
        merged = gather_stats(local, ws)
        out.put((rank, sorted(r.rid for r in mine), sorted(set(r.op for r in mine)),
                 all(r.result == [3.0 * r.rid] for r in mine), merged["requests"], merged["setups"],
                 merged["per_device_requests"]))
        s.close()
    finally:
        dist.destroy_process_group()


def test_ranks_serve_disjoint_streams_and_gather_on_the_host():
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
    (r0, rids0, ops0, ok0, n0, s0, per0), (r1, rids1, ops1, ok1, n1, s1, per1) = res
    assert ok0 and ok1
    assert not set(rids0) & set(rids1) and sorted(rids0 + rids1) == list(range(len(requests())))
    assert ops0 == [0, 4, 5] and ops1 == [1, 2, 3]
    assert n0 == n1 == len(requests()) and s0 == s1 == len(SIZES)
    assert per0 == per1 == [len(rids0), len(rids1)]
