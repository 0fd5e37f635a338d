"""Host logic of the continuous-batching server (admission, cache, ledger,
eviction, latency bookkeeping) with a fake hierarchy: CPU only."""
import threading
import time

import pytest

from paper_2602_05686_gb300.serving import Request, Server


class FakeHierarchy:
    live = 0
    peak = 0
    batches = []
    lock = threading.Lock()

    def __init__(self, problem, stream=None, **kw):
        self.n = problem["n"]
        self.nb = problem["bytes"]
        with FakeHierarchy.lock:
            FakeHierarchy.live += 1
            FakeHierarchy.peak = max(FakeHierarchy.peak, FakeHierarchy.live)
        time.sleep(0.01)  # "setup"

    def stats(self):
        return {"device_bytes": self.nb}

    def solve(self, b, tol=1e-8, check=False):
        time.sleep(0.002)
        return [v * 2 for v in b], {"status": 0, "iters": 3, "rel_res": 1e-9}

    def solve_batch(self, B, tol=1e-8, check=False):
        FakeHierarchy.batches.append(len(B))
        time.sleep(0.002)
        return [[v * 2 for v in b] for b in B], [{"status": 0, "iters": 3, "rel_res": 1e-9} for _ in B]

    def free(self):
        with FakeHierarchy.lock:
            FakeHierarchy.live -= 1


def make_server(slots, budget, nops=4):
    probs = {op: {"n": 10, "nnz": 30, "bytes": 100 * (op + 1)} for op in range(nops)}
    s = Server(lambda op: probs[op], lambda op: {}, slots=slots, hbm_budget=budget,
               hierarchy_factory=FakeHierarchy, stream_factory=lambda: None)
    s._estimate = lambda op: probs[op]["bytes"]
    return s


def reqs(pattern, gap=0.0):
    return [Request(rid=i, op=op, arrival=i * gap, rhs=[float(i), 1.0]) for i, op in enumerate(pattern)]


def test_cache_hits_skip_setup():
    FakeHierarchy.live = FakeHierarchy.peak = 0
    s = make_server(slots=2, budget=10_000)
    rs = reqs([0, 0, 1, 0, 1, 1, 2])
    out = s.serve(rs, realtime=False)
    assert out["requests"] == 7 and out["failed"] == 0
    assert out["setups"] == 3 and out["hits"] + out["setups"] == 7
    assert all(r.result == [2.0 * r.rid, 2.0] for r in rs)
    assert out["p50_s"] <= out["p99_s"]
    s.close()
    assert FakeHierarchy.live == 0


def test_ledger_never_exceeds_budget_and_evicts_lru():
    FakeHierarchy.live = FakeHierarchy.peak = 0
    s = make_server(slots=2, budget=450, nops=4)  # op bytes 100, 200, 300, 400
    rs = reqs([0, 1, 2, 3, 0, 1, 2, 3])
    out = s.serve(rs, realtime=False)
    assert out["failed"] == 0
    assert out["peak_committed"] <= 450 or out["setups"] >= 1
    assert out["evictions"] >= 1
    s.close()


def test_poisson_like_arrivals_are_released_in_time():
    FakeHierarchy.live = FakeHierarchy.peak = 0
    s = make_server(slots=3, budget=10_000)
    rs = reqs([0, 1, 2, 0, 1, 2, 0, 1], gap=0.005)
    out = s.serve(rs, realtime=True)
    assert out["failed"] == 0
    for r in rs:
        assert r.start >= r.arrival - 1e-6 and r.done >= r.start
    assert out["wall_s"] >= rs[-1].arrival


def test_single_slot_serialises():
    FakeHierarchy.live = FakeHierarchy.peak = 0
    s = make_server(slots=1, budget=10_000)
    rs = reqs([0, 1, 2])
    s.serve(rs, realtime=False)
    spans = sorted((r.start, r.done) for r in rs)
    for (a0, a1), (b0, b1) in zip(spans, spans[1:]):
        assert b0 >= a1 - 1e-3
    assert FakeHierarchy.peak <= 3


@pytest.mark.parametrize("slots", [1, 4])
def test_results_identical_alone_and_in_the_mix(slots):
    FakeHierarchy.live = FakeHierarchy.peak = 0
    alone = {}
    for r in reqs([0, 1, 2, 3, 0, 1]):
        s = make_server(slots=1, budget=10_000)
        s.serve([r], realtime=False)
        alone[r.rid] = r.result
        s.close()
    s = make_server(slots=slots, budget=10_000)
    mix = reqs([0, 1, 2, 3, 0, 1])
    s.serve(mix, realtime=False)
    for r in mix:
        assert r.result == alone[r.rid]
    s.close()


def test_concurrent_requests_share_one_setup():
    FakeHierarchy.live = FakeHierarchy.peak = 0
    s = make_server(slots=4, budget=10_000)
    rs = reqs([0, 0, 0, 0, 1, 1, 1, 1])
    out = s.serve(rs, realtime=False)
    assert out["setups"] == 2 and out["hits"] == 6 and out["failed"] == 0
    s.close()


def test_failed_request_is_retired_with_status():
    class Failing(FakeHierarchy):
        def solve(self, b, tol=1e-8, check=False):
            if b[0] == 2.0:
                raise RuntimeError("injected failure")
            return super().solve(b, tol, check)

    probs = {0: {"n": 10, "nnz": 30, "bytes": 10}}
    s = Server(lambda op: probs[op], lambda op: {}, slots=2, hbm_budget=10_000, hierarchy_factory=Failing,
               stream_factory=lambda: None, batch=1)
    s._estimate = lambda op: 10
    rs = reqs([0, 0, 0, 0])
    out = s.serve(rs, realtime=False)
    assert out["failed"] == 1
    assert [r.status != 0 for r in rs] == [False, False, True, False]
    assert s.committed == 10  # only the cached hierarchy stays committed
    s.close()

    # a failing multi-right-hand-side job retires all of its requests
    class FailingBatch(FakeHierarchy):
        def solve_batch(self, B, tol=1e-8, check=False):
            raise RuntimeError("injected failure")

    s = Server(lambda op: probs[op], lambda op: {}, slots=1, hbm_budget=10_000, hierarchy_factory=FailingBatch,
               stream_factory=lambda: None, batch=4)
    s._estimate = lambda op: 10
    rs = reqs([0, 0, 0])
    out = s.serve(rs, realtime=False)
    assert out["failed"] == 3 and out["jobs"] == 1 and all(r.info.get("error") for r in rs)
    assert s.committed == 10
    s.close()


class StoredFake(FakeHierarchy):
    """a fake whose store is a small text file"""
    loads = 0

    def save(self, path):
        with open(path, "w") as f:
            f.write(f"{self.n} {self.nb}")

    @classmethod
    def load(cls, path, stream=None, **kw):
        with open(path) as f:
            n, nb = (int(x) for x in f.read().split())
        StoredFake.loads += 1
        return cls({"n": n, "bytes": nb})


def test_store_carries_setups_across_servers(tmp_path):
    """a second server (a restarted process) loads the stored hierarchies
    instead of running setups; a damaged store is rebuilt"""
    probs = {op: {"n": 10, "nnz": 30, "bytes": 100 * (op + 1)} for op in range(3)}

    def server():
        s = Server(lambda op: probs[op], lambda op: {"theta": 0.05}, slots=2, hbm_budget=10_000,
                   hierarchy_factory=StoredFake, stream_factory=lambda: None, store_dir=str(tmp_path),
                   hierarchy_loader=StoredFake.load)
        s._estimate = lambda op: probs[op]["bytes"]
        return s

    s1 = server()
    out1 = s1.serve(reqs([0, 1, 0, 2]), realtime=False)
    s1.close()
    assert out1["setups"] == 3 and out1["stores"] == 3 and out1["loads"] == 0
    assert len(list(tmp_path.glob("*.saamg"))) == 3 and not list(tmp_path.glob("*.tmp"))
    s2 = server()
    out2 = s2.serve(reqs([2, 1, 0, 0]), realtime=False)
    s2.close()
    assert out2["setups"] == 0 and out2["loads"] == 3 and out2["failed"] == 0
    # options are part of the store name: other options miss the store
    s3 = Server(lambda op: probs[op], lambda op: {"theta": 0.1}, slots=1, hbm_budget=10_000,
                hierarchy_factory=StoredFake, stream_factory=lambda: None, store_dir=str(tmp_path),
                hierarchy_loader=StoredFake.load)
    out3 = s3.serve(reqs([0]), realtime=False)
    s3.close()
    assert out3["setups"] == 1 and out3["loads"] == 0
    # a damaged store falls back to a setup
    for f in tmp_path.glob("op1-*.saamg"):
        f.write_text("garbage")
    s4 = server()
    out4 = s4.serve(reqs([1]), realtime=False)
    s4.close()
    assert out4["setups"] == 1 and out4["failed"] == 0


def test_same_operator_requests_share_one_job():
    """requests of one operator waiting together form one multi-right-hand-side
    job (at most `batch` columns); results match the one-by-one schedule"""
    FakeHierarchy.live = FakeHierarchy.peak = 0
    FakeHierarchy.batches = []
    probs = {op: {"n": 10, "nnz": 30, "bytes": 100} for op in range(2)}
    s = Server(lambda op: probs[op], lambda op: {}, slots=1, hbm_budget=10_000, hierarchy_factory=FakeHierarchy,
               stream_factory=lambda: None, batch=3)
    s._estimate = lambda op: probs[op]["bytes"]
    rs = reqs([0, 0, 0, 0, 1, 0, 1])
    out = s.serve(rs, realtime=False)
    s.close()
    assert out["failed"] == 0 and out["requests"] == 7
    assert all(r.result == [2.0 * r.rid, 2.0] for r in rs)
    assert max(FakeHierarchy.batches) <= 3 and sum(FakeHierarchy.batches) + (out["jobs"] - len(FakeHierarchy.batches)) == 7
    assert out["jobs"] < 7 and out["batched"] >= 2
    assert out["hits"] + out["setups"] == 7
    s1 = Server(lambda op: probs[op], lambda op: {}, slots=1, hbm_budget=10_000, hierarchy_factory=FakeHierarchy,
                stream_factory=lambda: None, batch=1)
    out1 = s1.serve(reqs([0, 0, 1]), realtime=False)
    s1.close()
    assert out1["jobs"] == 3 and out1["batched"] == 0


def test_group_executor_solves_distinct_operators_together():
    """group_solves: ready single-request jobs of different operators go to one
    group call (one request per operator per group)"""
    FakeHierarchy.live = FakeHierarchy.peak = 0
    calls = []

    def group_solver(hs, rhs, tol):
        calls.append(len(hs))
        assert len({id(h) for h in hs}) == len(hs)   # distinct operators
        time.sleep(0.01)
        return [[v * 2 for v in b] for b in rhs], [{"status": 0, "iters": 3, "rel_res": 1e-9} for _ in hs]

    probs = {op: {"n": 10, "nnz": 30, "bytes": 100} for op in range(6)}
    s = Server(lambda op: probs[op], lambda op: {}, slots=6, hbm_budget=10_000, hierarchy_factory=FakeHierarchy,
               stream_factory=lambda: None, group_solves=True, group_solver=group_solver, batch=1)
    s._estimate = lambda op: 100
    rs = reqs([0, 1, 2, 3, 4, 5, 0, 1, 2, 3])
    out = s.serve(rs, realtime=False)
    assert out["failed"] == 0 and out["requests"] == 10
    assert all(r.result == [2.0 * r.rid, 2.0] for r in rs)
    assert out["grouped"] == 10 and sum(calls) == 10 and max(calls) > 1 and out["groups"] == len(calls)
    s.close()
