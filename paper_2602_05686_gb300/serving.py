"""Continuous-batching solve service on one GPU.

Requests (operator id, right-hand side) arrive over time.  A fixed number of
slots run requests concurrently, each slot on its own CUDA stream and host
thread (the C library releases the GIL inside every call), so the setup and
solve kernels of different requests overlap on the device.  A request is
admitted when a slot is free and the device-memory ledger has room for its
hierarchy (if not cached) plus its Krylov vectors.  Hierarchies are cached on
the device by operator id, so successive right-hand sides of one operator
(load steps of one stack) skip setup; the least recently used idle
hierarchies are evicted when the ledger needs room.  Setup of an operator is
amortised over its right-hand sides, as the paper notes for repeated solves
(Sec. 4.3).  With a store directory the amortisation reaches across
processes and restarts: a built hierarchy is written there (sa_serialize)
and a later miss on the same operator and options loads it (sa_deserialize)
instead of running the setup.

Requests for the same operator that are waiting together are served as one
multi-right-hand-side job (up to `batch` columns, sa_solve_batch): every
operator product, V-cycle and vector update of the job is one launch for all
its columns.  With group_solves=True, single-request jobs of DIFFERENT
operators whose hierarchies are ready are solved together by one executor
thread (sa_solve_group): every operator product, V-cycle kernel (coarse
solves included) and CG update is one launch for all of them, which is where
small problems, whose launches are mostly empty, gain.  A group is formed
from whatever is ready when the executor is free; requests that become ready
during a group solve form the next one.  Every numerical step runs in the CUDA library; this module only
schedules.
Results do not depend on the schedule: every kernel of the library is
deterministic and a column of a multi-right-hand-side solve equals the
one-vector solve bitwise, so a request solved alone and in the mix gives
bit-identical solutions.

Several GPUs serve as replicas: each operator is placed on one device (the
one with the least committed bytes when the operator first arrives, by the
ledger's estimate), every device runs its own Server (slots, streams,
ledger, cache), and the requests of an operator always go to its device.
MultiServer does this in one process; under torch.distributed each rank
serves the operators placed on it (`partition`) and the latencies are
gathered on the host (`gather_stats`), the only exchange between replicas.
"""
from __future__ import annotations

import contextlib
import hashlib
import heapq
import os
import statistics
import threading
import time
from dataclasses import dataclass, field


def _pct(sorted_vals, q):
    if not sorted_vals:
        return 0.0
    return sorted_vals[min(len(sorted_vals) - 1, int(round(q * (len(sorted_vals) - 1))))]


@dataclass
class Request:
    rid: int
    op: int
    arrival: float                 # seconds since the start of the run
    rhs: object = None             # CUDA tensor (float64)
    result: object = None
    info: dict = field(default_factory=dict)
    start: float = 0.0
    done: float = 0.0
    cache_hit: bool = False
    status: int = 0


class _Entry:
    def __init__(self, h, nbytes):
        self.h = h
        self.nbytes = nbytes
        self.users = 0
        self.last = 0.0
        self.lock = threading.Lock()  # one solve at a time per hierarchy


class Server:
    """slots: concurrent requests; hbm_budget: bytes the ledger may commit.
    make_problem(op) -> problem dict; options(op) -> Hierarchy keyword args."""

    def __init__(self, make_problem, options, slots=4, hbm_budget=64 << 30, tol=1e-8, hierarchy_factory=None,
                 stream_factory=None, store_dir=None, store_key=None, hierarchy_loader=None, batch=8, device=None,
                 group_solves=False, group_solver=None, group_max=64):
        # device: the CUDA device this server's slots run on (made current in
        # every slot thread); None keeps the caller's current device
        self.device = device
        # group_solves: single-request jobs of different operators are solved
        # together (group_solver(hierarchies, rhs, tol) -> (xs, infos))
        self.group_solves = bool(group_solves)
        if self.group_solves and group_solver is None:
            from .api import solve_group

            def group_solver(hs, rhs, tol):
                return solve_group(hs, rhs, tol=tol, check=False)
        self.group_solver = group_solver
        self.group_max = max(1, min(64, int(group_max)))
        self._ready = []            # (entry, request, event) waiting for the group executor
        self._gcv = threading.Condition()
        self._gthread = None
        self._gstop = False
        if hierarchy_factory is None:
            from .api import Hierarchy as hierarchy_factory
        if hierarchy_loader is None and store_dir is not None:
            from .api import Hierarchy
            hierarchy_loader = Hierarchy.load
        self.loader = hierarchy_loader
        self.store_dir = store_dir
        # store_key(op) names an operator across processes (default: its id)
        self.store_key = store_key or (lambda op: f"op{op}")
        if stream_factory is None:
            import torch
            stream_factory = torch.cuda.Stream
        self.factory = hierarchy_factory
        self.make_problem = make_problem
        self.options = options
        self.slots = slots
        self.budget = int(hbm_budget)
        self.tol = tol
        self.cache = {}
        self.committed = 0
        self.cv = threading.Condition()
        self.streams = [stream_factory() for _ in range(slots)]
        self.free_slots = list(range(slots))
        self.batch = max(1, int(batch))
        self.stats = dict(admitted=0, setups=0, hits=0, evictions=0, peak_committed=0, loads=0, stores=0, jobs=0,
                          batched=0, groups=0, grouped=0, max_group=0)
        self._problems = {}
        self.building = {}  # op -> threading.Event of an in-flight setup

    # -- memory ledger -------------------------------------------------------
    def _estimate(self, op):
        """device bytes a new hierarchy of `op` will hold (ledger estimate:
        about 3x the fine matrix in CSR, plus vectors)"""
        p = self._problem(op)
        return int(3.0 * (12 * p["nnz"] + 8 * (p["n"] + 1)) + 40 * 8 * p["n"])

    def _problem(self, op):
        if op not in self._problems:
            self._problems[op] = self.make_problem(op)
        return self._problems[op]

    def _make_room(self, need):
        """evict idle cached hierarchies (least recently used first); caller holds cv"""
        while self.committed + need > self.budget:
            idle = [(e.last, k) for k, e in self.cache.items() if e.users == 0]
            if not idle:
                return False
            _, k = min(idle)
            e = self.cache.pop(k)
            e.h.free()
            self.committed -= e.nbytes
            self.stats["evictions"] += 1
        return True

    # -- hierarchy store ---------------------------------------------------------
    def _store_path(self, op):
        if self.store_dir is None:
            return None
        opts = self.options(op)
        tag = hashlib.sha256(repr(sorted((k, repr(v)) for k, v in opts.items() if k != "stream")).encode())
        return os.path.join(self.store_dir, f"{self.store_key(op)}-{tag.hexdigest()[:16]}.saamg")

    def _load_or_build(self, op, stream):
        """the stored hierarchy of op when one exists (a damaged store is
        rebuilt), else a new setup, which is then stored"""
        opts = self.options(op)
        path = self._store_path(op)
        if path is not None and os.path.exists(path):
            try:
                h = self.loader(path, stream=stream, precision=opts.get("precision", "fp64"),
                                maxit=opts.get("maxit", 500))
                with self.cv:
                    self.stats["loads"] += 1
                return h
            except Exception:
                pass
        h = self.factory(self._problem(op), stream=stream, **opts)
        with self.cv:
            self.stats["setups"] += 1
        if path is not None:
            os.makedirs(self.store_dir, exist_ok=True)
            tmp = f"{path}.{os.getpid()}.{threading.get_ident()}.tmp"
            h.save(tmp)
            os.replace(tmp, path)  # readers never see a partial store
            with self.cv:
                self.stats["stores"] += 1
        return h

    # -- one request on one slot ---------------------------------------------
    def _ctx(self, stream):
        if stream is None or not hasattr(stream, "cuda_stream"):
            return contextlib.nullcontext()
        import torch
        return torch.cuda.stream(stream)

    def _acquire(self, req, stream):
        """the cached hierarchy of req.op, building it if nobody else is; a
        request whose operator is being built by another slot waits for it"""
        while True:
            builder = False
            with self.cv:
                entry = self.cache.get(req.op)
                if entry is not None:
                    entry.users += 1
                    req.cache_hit = True
                    self.stats["hits"] += 1
                    self.committed -= req.info.pop("_reserved", 0)
                    return entry
                ev = self.building.get(req.op)
                if ev is None:
                    ev = threading.Event()
                    self.building[req.op] = ev
                    builder = True
            if not builder:
                ev.wait()
                continue  # cached now (or evicted again: retry)
            try:
                h = self._load_or_build(req.op, stream)
                nbytes = h.stats()["device_bytes"]
                with self.cv:
                    entry = _Entry(h, nbytes)
                    entry.users += 1
                    self.cache[req.op] = entry
                    # the measured size replaces the admission estimate
                    self.committed += nbytes - req.info.pop("_reserved", 0)
                return entry
            finally:
                with self.cv:
                    self.building.pop(req.op, None)
                    self.cv.notify_all()
                ev.set()

    def _run(self, job, slot, t0):
        """one job: requests of one operator, solved together"""
        if self.device is not None:
            import torch
            torch.cuda.set_device(self.device)
        stream = self.streams[slot]
        req = job[0]
        with self._ctx(stream):
            entry = None
            try:
                entry = self._acquire(req, stream)
                for r in job[1:]:
                    r.cache_hit = True
                if len(job) > 1:
                    with self.cv:
                        self.stats["hits"] += len(job) - 1
                rhs = [r.rhs for r in job]
                if hasattr(rhs[0], "to") and stream is not None and hasattr(stream, "cuda_stream"):
                    rhs = [v.to(device="cuda", non_blocking=True) for v in rhs]
                    stream.synchronize()  # the cached handle may run on another slot's stream
                if len(job) == 1 and self.group_solves:
                    results = [self._group_solve(entry, rhs[0])]
                else:
                    with entry.lock:
                        if len(job) == 1:
                            x, info = entry.h.solve(rhs[0], tol=self.tol, check=False)
                            results = [(x, info)]
                        else:
                            import torch
                            B = torch.stack(rhs) if hasattr(rhs[0], "to") else rhs
                            X, infos = entry.h.solve_batch(B, tol=self.tol, check=False)
                            results = [(X[c], infos[c]) for c in range(len(job))]
                for r, (x, info) in zip(job, results):
                    r.result = x
                    r.info.update(info)
                    r.status = info["status"]
            except Exception as e:  # a failed job retires its requests with the status
                for r in job:
                    r.status = getattr(e, "status", -1)
                    r.info["error"] = str(e)
            done = time.perf_counter() - t0
            with self.cv:
                for r in job:
                    r.done = done
                    self.committed -= r.info.pop("_reserved", 0)
                if entry is not None:
                    entry.users -= 1
                    entry.last = done
                self.free_slots.append(slot)
                self.cv.notify_all()

    # -- group solves -----------------------------------------------------------
    def _group_solve(self, entry, rhs):
        """hands (entry, rhs) to the group executor and waits for its result"""
        item = {"entry": entry, "rhs": rhs, "done": threading.Event(), "res": None, "err": None}
        with self._gcv:
            if self._gthread is None:
                self._gstop = False
                self._gthread = threading.Thread(target=self._group_loop, daemon=True)
                self._gthread.start()
            self._ready.append(item)
            self._gcv.notify_all()
        item["done"].wait()
        if item["err"] is not None:
            raise item["err"]
        return item["res"]

    def _group_loop(self):
        """the executor: solves everything ready (one request per operator) in
        one group solve, then the next group"""
        if self.device is not None:
            import torch
            torch.cuda.set_device(self.device)
        while True:
            with self._gcv:
                while not self._ready and not self._gstop:
                    self._gcv.wait(timeout=0.05)
                if self._gstop and not self._ready:
                    return
                group, rest, seen = [], [], set()
                for it in self._ready:
                    if id(it["entry"]) in seen or len(group) >= self.group_max:
                        rest.append(it)
                    else:
                        seen.add(id(it["entry"]))
                        group.append(it)
                self._ready = rest
            locks = [it["entry"].lock for it in group]
            for lk in locks:
                lk.acquire()
            try:
                xs, infos = self.group_solver([it["entry"].h for it in group], [it["rhs"] for it in group], self.tol)
                for it, x, info in zip(group, xs, infos):
                    it["res"] = (x, info)
            except Exception as e:  # every member of a failed group retires with the error
                for it in group:
                    it["err"] = e
            finally:
                for lk in locks:
                    lk.release()
            with self.cv:
                self.stats["groups"] += 1
                self.stats["grouped"] += len(group)
                self.stats["max_group"] = max(self.stats["max_group"], len(group))
            for it in group:
                it["done"].set()

    def _stop_group(self):
        with self._gcv:
            self._gstop = True
            self._gcv.notify_all()
        if self._gthread is not None:
            self._gthread.join(timeout=30)
        self._gthread = None

    # -- the loop -----------------------------------------------------------
    def serve(self, requests, realtime=True):
        """Runs the request list (sorted by arrival); returns latency stats.
        realtime: requests are released at their arrival times."""
        t0 = time.perf_counter()
        pending = list(requests)
        pending.sort(key=lambda r: r.arrival)
        threads = []
        queue = []  # arrived, not yet admitted (FIFO by arrival)
        k = 0
        while k < len(pending) or queue:
            now = time.perf_counter() - t0
            while k < len(pending) and (not realtime or pending[k].arrival <= now):
                heapq.heappush(queue, (pending[k].arrival, pending[k].rid, pending[k]))
                k += 1
            admitted = False
            with self.cv:
                if queue and self.free_slots:
                    req = queue[0][2]
                    need = 0 if (req.op in self.cache or req.op in self.building) else self._estimate(req.op)
                    busy = any(e.users for e in self.cache.values()) or len(self.free_slots) < self.slots
                    if self._make_room(need) or not busy:
                        heapq.heappop(queue)
                        # waiting requests of the same operator join this job
                        job = [req]
                        if self.batch > 1:
                            same = sorted(e for e in queue if e[2].op == req.op)[: self.batch - 1]
                            if same:
                                job += [e[2] for e in same]
                                ids = {id(e[2]) for e in same}
                                queue[:] = [e for e in queue if id(e[2]) not in ids]
                                heapq.heapify(queue)
                        slot = self.free_slots.pop()
                        self.committed += need
                        req.info["_reserved"] = need
                        self.stats["peak_committed"] = max(self.stats["peak_committed"], self.committed)
                        now2 = time.perf_counter() - t0
                        for r in job:
                            r.start = now2
                        self.stats["admitted"] += len(job)
                        self.stats["jobs"] += 1
                        if len(job) > 1:
                            self.stats["batched"] += len(job)
                        th = threading.Thread(target=self._run, args=(job, slot, t0), daemon=True)
                        th.start()
                        threads.append(th)
                        admitted = True
                if not admitted:
                    wait = 0.002
                    if k < len(pending) and realtime:
                        wait = max(0.0, min(wait, pending[k].arrival - (time.perf_counter() - t0)))
                    self.cv.wait(timeout=wait if wait > 0 else 0.0005)
        for th in threads:
            th.join()
        wall = time.perf_counter() - t0
        lat = [r.done - r.arrival for r in requests]
        lat.sort()

        def pct(q):
            return _pct(lat, q)

        return dict(requests=len(requests), wall_s=wall, throughput_rps=len(requests) / wall,
                    p50_s=pct(0.50), p99_s=pct(0.99), mean_s=statistics.mean(lat), **self.stats,
                    failed=sum(1 for r in requests if r.status not in (0,)), latencies=lat)

    def close(self):
        self._stop_group()
        for e in self.cache.values():
            e.h.free()
        self.cache.clear()
        self.committed = 0


# ---------------------------------------------------------------------------
# several GPUs: replicas with operator placement
# ---------------------------------------------------------------------------
def place_operators(requests, estimate, ndev):
    """Deterministic placement of operators on ndev devices: operators are
    taken in the order of their first arrival (ties by operator id) and each
    goes to the device with the least committed bytes so far (ties: lowest
    index), committing estimate(op) bytes there.  Every process that computes
    it from the same request list gets the same map.  Returns (op -> device,
    committed bytes per device)."""
    first = {}
    for r in sorted(requests, key=lambda r: (r.arrival, r.rid)):
        first.setdefault(r.op, r.arrival)
    committed = [0] * max(1, int(ndev))
    place = {}
    for op in sorted(first, key=lambda o: (first[o], o)):
        d = min(range(len(committed)), key=lambda k: (committed[k], k))
        place[op] = d
        committed[d] += int(estimate(op))
    return place, committed


def partition(requests, estimate, rank, world):
    """the requests this rank serves: those of the operators placed on it"""
    place, _ = place_operators(requests, estimate, world)
    return [r for r in requests if place[r.op] == rank], place


def merge_stats(parts):
    """one latency report from per-device serve() results (each with its
    `latencies`): percentiles over all requests, throughput over the slowest
    device's wall time, counters summed"""
    lat = sorted(x for p in parts for x in p["latencies"])
    wall = max(p["wall_s"] for p in parts)
    out = dict(requests=len(lat), wall_s=wall, throughput_rps=len(lat) / wall if wall > 0 else 0.0,
               p50_s=_pct(lat, 0.50), p99_s=_pct(lat, 0.99), mean_s=statistics.mean(lat) if lat else 0.0,
               devices=len(parts), per_device_requests=[p["requests"] for p in parts],
               per_device_peak_committed=[p["peak_committed"] for p in parts])
    for k in ("admitted", "setups", "hits", "evictions", "loads", "stores", "jobs", "batched", "failed"):
        out[k] = sum(p.get(k, 0) for p in parts)
    return out


def gather_stats(local, world):
    """the per-rank serve() results gathered on every rank (host objects over
    the default process group), merged"""
    if world <= 1:
        return merge_stats([local])
    import torch.distributed as dist
    parts = [None] * world
    dist.all_gather_object(parts, local)
    return merge_stats(parts)


class MultiServer:
    """Replicas on several devices in one process: operators are placed by
    place_operators on the ledgers' estimates, each device runs its own
    Server (own slots, streams, ledger of hbm_budget bytes and cache), and
    serve() runs the devices' request streams concurrently."""

    def __init__(self, make_problem, options, devices, slots=4, hbm_budget=64 << 30, server_factory=None, **kw):
        self.devices = list(devices)
        make = server_factory or Server
        self.servers = []
        for d in self.devices:
            extra = dict(kw)
            if "stream_factory" not in extra and d is not None:
                import torch
                extra["stream_factory"] = (lambda dev=d: torch.cuda.Stream(device=dev))
            self.servers.append(make(make_problem, options, slots=slots, hbm_budget=hbm_budget, device=d, **extra))
        self.placement = {}

    def serve(self, requests, realtime=True):
        place, committed = place_operators(requests, self.servers[0]._estimate, len(self.servers))
        self.placement = place
        per = [[r for r in requests if place[r.op] == k] for k in range(len(self.servers))]
        outs = [None] * len(self.servers)

        def run(k):
            outs[k] = self.servers[k].serve(per[k], realtime=realtime) if per[k] else dict(
                requests=0, wall_s=0.0, latencies=[], peak_committed=0)

        ths = [threading.Thread(target=run, args=(k,), daemon=True) for k in range(len(self.servers))]
        for t in ths:
            t.start()
        for t in ths:
            t.join()
        out = merge_stats(outs)
        out["placement_committed_estimate"] = committed
        return out

    def close(self):
        for s in self.servers:
            s.close()
