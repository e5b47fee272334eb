"""Continuous-batching solve server over the batched C ABI.

Requests (a body, a step count, an arrival time) arrive over time; the
server admits them first come, first served while their device memory fits
a budget, advances every admitted body together with lbm_batch_step in
chunks that end exactly when the next admitted request completes (so each
request gets exactly its step count), reads each finished request's
displacement back to the host, frees it, and admits the next ones.  The
batch is rebuilt whenever its membership changes.  Latency of a request =
completion (its result on the host) minus arrival.  A request that fails
(its body cannot be created, its batch's step fails, or its result cannot
be read) completes with the error's status while the others go on.

The GPU work goes through lbm.Body / lbm.Batch only; the scheduling logic
talks to a small backend interface, so it also runs on the host with a
simulated backend (tests)."""
from __future__ import annotations

import collections
import concurrent.futures
import dataclasses
import itertools
import math
import time
from typing import Callable, Dict, List, Optional

import numpy as np

from .lbm import LBM_E_UNSTABLE


@dataclasses.dataclass
class Record:
    index: int
    arrival: float
    admitted: float
    completed: float
    nodes: int
    steps: int
    status: int

    @property
    def latency(self) -> float:
        return self.completed - self.arrival


class GpuBackend:
    """lbm.Body / lbm.Batch on one device and stream.  scheme: the
    footnote's predictor by default, which stays stable over the trace's
    materials (Poisson ratio up to 0.44 in periodic bodies, where Algorithm
    1's explicit moment grows once lambda > mu)."""

    def __init__(self, storage: str = "f16", stream: int = 0, device: int = 0, scheme: Optional[int] = None):
        from . import lbm

        self.lbm = lbm
        self.scheme = lbm.LBM_SCHEME_PREDICTOR if scheme is None else int(scheme)
        self.storage = storage
        self.stream = stream
        self.device = device

    def estimate(self, prob) -> int:
        """Device bytes a body will hold: two state copies and the read-out
        fields over the padded planes (the layout lbm_create allocates)."""
        es = {"f64": 8, "f32": 4, "f16": 2, "bf16": 2}[self.storage]
        ec = 8 if self.storage == "f64" else 4
        ucp = 1 if self.storage in ("f64",) else 2
        pitch = (8 + prob.nx + 144 + 16 + 63) // 64 * 64
        plane = pitch * (prob.ny + 6)
        state = plane * (9 * es + 2 * ucp * ec + 2 * ec)
        return 2 * state + 5 * 8 * prob.nx * prob.ny + 2 * 16 * prob.nx * prob.ny

    def prepare(self, prob):
        """The request's initial fields built on the host (the server runs
        this in its loader threads when the request arrives, off the GPU
        loop's path)."""
        if getattr(prob, "make_initial", None) is None:
            return prob
        u0, v0 = prob.make_initial()
        if v0 is not None and not v0.any():
            v0 = None  # zero initial velocity: lbm_create sets it without a copy
        return dataclasses.replace(prob, u0=u0, v0=v0, make_initial=None)

    def create(self, prob):
        return self.lbm.Body(prob, storage=self.storage, scheme=self.scheme, stream=self.stream, device=self.device)

    def memory(self, body) -> int:
        return int(self.lbm.lbm_memory_info(body.ctx)[0])

    def batch(self, bodies):
        return self.lbm.Batch(bodies, stream=self.stream)

    def step(self, batch, n: int) -> None:
        batch.step(n)

    def sync(self, batch) -> List[int]:
        return batch.sync()

    def result(self, body) -> np.ndarray:
        return body.read(self.lbm.LBM_FIELD_U, allow_unstable=True)["u"]

    def close(self, body) -> None:
        body.close()

    def close_batch(self, batch) -> None:
        batch.close()


class Server:
    """FCFS admission against an HBM budget, continuous batching.

    target_chunk_s: wall time aimed at per lbm_batch_step call (bounds how
    long an arrival waits before it can be admitted); max_chunk: steps per
    call at most.

    loader_threads: threads that prepare the next `prefetch` requests in
    arrival order (the backend's prepare(), if it has one: their initial
    fields on the host) while the GPU works.  A request comes with its input
    data, so its preparation may start before its arrival time (the client's
    side of the exchange); admission takes the prepared problem.

    Arrivals join the batch at chunk boundaries, not inside a chunk: a chunk
    is one lbm_batch_step call, replayed as CUDA graphs over a fixed set of
    members, and admitting a member inside it would mean rebuilding the
    batch's graphs while they run.  With chunks of at most target_chunk_s
    (50 ms by default) an arrival waits at most that long for its turn, far
    below the solve times."""

    def __init__(self, backend, hbm_budget: float = 150e9, target_chunk_s: float = 0.05, max_chunk: int = 2048,
                 clock: Callable[[], float] = time.perf_counter, sleep: Callable[[float], None] = time.sleep,
                 keep_results: bool = False, loader_threads: int = 8, prefetch: int = 32):
        self.be = backend
        self.loader_threads = int(loader_threads)
        self.prefetch = int(prefetch)
        self.budget = float(hbm_budget)
        self.target_chunk_s = float(target_chunk_s)
        self.max_chunk = int(max_chunk)
        self.clock = clock
        self.sleep = sleep
        self.keep_results = keep_results
        self.results: Dict[int, np.ndarray] = {}

    def run(self, requests) -> dict:
        order = sorted(range(len(requests)), key=lambda i: requests[i].arrival)
        pending = collections.deque(order)
        waiting: collections.deque = collections.deque()
        active: List[dict] = []
        records: List[Record] = []
        rejected: List[int] = []
        t0 = self.clock()
        prepare = getattr(self.be, "prepare", None)
        pool = (concurrent.futures.ThreadPoolExecutor(self.loader_threads)
                if prepare is not None and self.loader_threads > 0 else None)
        prepared: Dict[int, concurrent.futures.Future] = {}
        try:
            return self._loop(requests, pending, waiting, active, records, rejected, t0, pool, prepare, prepared)
        finally:
            if pool is not None:
                pool.shutdown(wait=True, cancel_futures=True)

    def _loop(self, requests, pending, waiting, active, records, rejected, t0, pool, prepare, prepared):
        used = 0.0
        peak_used = 0.0
        batch = None
        dirty = False
        sec_per_step = None
        chunks = 0
        rebuilds = 0
        max_active = 0
        busy = 0.0
        # host time in each backend call outside the timed chunks
        host = {"create": 0.0, "batch": 0.0, "result": 0.0, "close": 0.0}
        while pending or waiting or active:
            now = self.clock() - t0
            while pending and requests[pending[0]].arrival <= now:
                waiting.append(pending.popleft())
            # the loader prepares the next requests while the GPU works
            self._prefetch(requests, waiting, pending, pool, prepare, prepared)
            # first come, first served: admit the head while it fits
            while waiting:
                i = waiting[0]
                need = float(self.be.estimate(requests[i].problem))
                if need > self.budget:  # can never fit
                    waiting.popleft()
                    rejected.append(i)
                    if i in prepared:
                        prepared.pop(i).cancel()
                    continue
                if used + need > self.budget:
                    break
                waiting.popleft()
                tc = self.clock()
                try:
                    self._prefetch(requests, waiting, pending, pool, prepare, prepared)
                    if i in prepared:
                        prob = prepared.pop(i).result()
                    else:  # admitted before the loader reached it
                        prob = prepare(requests[i].problem) if prepare is not None else requests[i].problem
                    body = self.be.create(prob)
                    mem = float(self.be.memory(body))
                except Exception as e:  # this request fails alone
                    records.append(self._failed(requests, i, t0, e))
                    continue
                finally:
                    host["create"] += self.clock() - tc
                used += mem
                peak_used = max(peak_used, used)
                active.append({"i": i, "body": body, "left": int(requests[i].steps), "mem": mem,
                               "admitted": self.clock() - t0})
                dirty = True
            if not active:
                if pending:
                    self.sleep(max(0.0, requests[pending[0]].arrival - (self.clock() - t0)))
                continue
            max_active = max(max_active, len(active))
            if dirty:
                tb = self.clock()
                if batch is not None:
                    self.be.close_batch(batch)
                batch = self.be.batch([a["body"] for a in active])
                dirty = False
                rebuilds += 1
                host["batch"] += self.clock() - tb
            n = min(a["left"] for a in active)
            if sec_per_step:
                n = min(n, max(16, int(self.target_chunk_s / sec_per_step)))
            n = max(1, min(n, self.max_chunk))
            ts = self.clock()
            try:
                self.be.step(batch, n)
                statuses = self.be.sync(batch)
            except Exception as e:
                # the batch is unusable: its members fail with its status,
                # the server goes on with the next requests
                for a in active:
                    records.append(self._failed(requests, a["i"], t0, e, a["admitted"]))
                    self._quiet(self.be.close, a["body"])
                    used -= a["mem"]
                self._quiet(self.be.close_batch, batch)
                batch, active, dirty = None, [], False
                continue
            dt = self.clock() - ts
            busy += dt
            chunks += 1
            sec_per_step = dt / n
            still = []
            for a, st in zip(active, statuses):
                a["left"] -= n
                if a["left"] > 0:
                    still.append(a)
                    continue
                tr = self.clock()
                try:
                    u = self.be.result(a["body"])  # the response reaches the host
                except Exception as e:
                    u, st = None, self._status(e)
                done_t = self.clock() - t0
                host["result"] += done_t + t0 - tr
                r = requests[a["i"]]
                records.append(Record(a["i"], r.arrival, a["admitted"], done_t, r.problem.nx * r.problem.ny,
                                      int(r.steps), int(st)))
                if self.keep_results and u is not None:
                    self.results[a["i"]] = u
                tq = self.clock()
                self._quiet(self.be.close, a["body"])
                host["close"] += self.clock() - tq
                used -= a["mem"]
                dirty = True
            active = still
        if batch is not None:
            self.be.close_batch(batch)
        makespan = self.clock() - t0
        out = self._stats(requests, records, rejected, makespan, busy, peak_used, chunks, rebuilds, max_active)
        out["host_s"] = host
        return out

    def _prefetch(self, requests, waiting, pending, pool, prepare, prepared) -> None:
        """Hands the next `prefetch` requests in arrival order to the loader."""
        if pool is None:
            return
        for i in itertools.islice(itertools.chain(waiting, pending), self.prefetch):
            if i not in prepared:
                prepared[i] = pool.submit(prepare, requests[i].problem)

    @staticmethod
    def _status(e) -> int:
        return int(getattr(e, "status", -1))

    @staticmethod
    def _quiet(fn, *args) -> None:
        try:
            fn(*args)
        except Exception:
            pass

    def _failed(self, requests, i, t0, e, admitted=None) -> Record:
        now = self.clock() - t0
        r = requests[i]
        return Record(i, r.arrival, now if admitted is None else admitted, now, r.problem.nx * r.problem.ny,
                      int(r.steps), self._status(e))

    def _stats(self, requests, records, rejected, makespan, busy, peak_used, chunks, rebuilds, max_active):
        lat = np.array([r.latency for r in records]) if records else np.zeros(0)
        # the requests whose solve finished (status OK), apart from those that
        # ended LBM_E_UNSTABLE or failed
        ok = np.array([r.latency for r in records if r.status == 0]) if records else np.zeros(0)
        work = sum(r.nodes * r.steps for r in records if r.status in (0, LBM_E_UNSTABLE))
        arrivals = [q.arrival for q in requests]
        window = (max(arrivals) - min(arrivals)) if len(arrivals) > 1 else 0.0
        offered = sum(q.problem.nx * q.problem.ny * q.steps for q in requests)
        return {
            "requests": len(requests), "completed": len(records), "rejected": len(rejected),
            "unstable": int(sum(1 for r in records if r.status == LBM_E_UNSTABLE)),
            "failed": int(sum(1 for r in records if r.status not in (0, LBM_E_UNSTABLE))),
            "p50_s": float(np.percentile(lat, 50)) if len(lat) else None,
            "p99_s": float(np.percentile(lat, 99)) if len(lat) else None,
            "mean_s": float(lat.mean()) if len(lat) else None,
            "stable_completed": int(len(ok)),
            "stable_p50_s": float(np.percentile(ok, 50)) if len(ok) else None,
            "stable_p99_s": float(np.percentile(ok, 99)) if len(ok) else None,
            "makespan_s": makespan, "gpu_busy_s": busy,
            "served_mlups": work / makespan / 1e6 if makespan > 0 else None,
            "offered_mlups": offered / window / 1e6 if window > 0 else None,
            "arrival_window_s": window,
            "peak_hbm_bytes": peak_used, "hbm_budget_bytes": self.budget,
            "chunks": chunks, "batch_rebuilds": rebuilds, "max_active": max_active,
            "admission": "FCFS, head of line blocks while it does not fit the budget; arrivals join at "
                         "the next chunk boundary (chunks aim at target_chunk_s of GPU time)",
            "records": records,
        }


def trace_at_rate(requests, rate: float, seed: int = 11):
    """The same requests with Poisson arrivals at `rate` per second."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for r in requests:
        t += float(rng.exponential(1.0 / rate))
        out.append(dataclasses.replace(r, arrival=t))
    return out
