"""Scheduling logic of the continuous-batching server, on the host with a
simulated backend (no GPU): exact step counts, FCFS admission, the memory
budget, rejection of requests that can never fit, latency accounting."""
import dataclasses

import numpy as np

from paper_2208_13769_gb300 import serve
from paper_2208_13769_gb300 import workloads as W


@dataclasses.dataclass
class _P:
    nx: int
    ny: int


class FakeClock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t

    def sleep(self, s):
        self.t += max(0.0, s)


class FakeBackend:
    """A GPU stand-in: a step of a batch takes (sum of member nodes) / rate
    seconds of the fake clock; it records every step each body receives."""

    def __init__(self, clock, rate=1e9, per_node=100):
        self.clock, self.rate, self.per_node = clock, rate, per_node
        self.steps_of = {}
        self.admit_order = []
        self.live = 0
        self.peak_live = 0
        self.next_id = 0

    def estimate(self, prob):
        return prob.nx * prob.ny * self.per_node

    def create(self, prob):
        h = {"id": self.next_id, "nodes": prob.nx * prob.ny}
        self.next_id += 1
        self.steps_of[h["id"]] = 0
        self.admit_order.append(h["id"])
        self.live += 1
        self.peak_live = max(self.peak_live, self.live)
        return h

    def memory(self, h):
        return h["nodes"] * self.per_node

    def batch(self, bodies):
        return list(bodies)

    def step(self, batch, n):
        for h in batch:
            self.steps_of[h["id"]] += n
        self.clock.t += n * sum(h["nodes"] for h in batch) / self.rate

    def sync(self, batch):
        return [0] * len(batch)

    def result(self, h):
        return np.zeros((1, 1, 2))

    def close(self, h):
        self.live -= 1

    def close_batch(self, batch):
        pass


def _trace(n=40, seed=3):
    rng = np.random.default_rng(seed)
    t, out = 0.0, []
    for _ in range(n):
        t += float(rng.exponential(0.01))
        p = _P(int(rng.integers(50, 400)), int(rng.integers(50, 400)))
        out.append(W.Request(arrival=t, problem=p, steps=int(rng.integers(30, 3000))))
    return out


def test_every_request_gets_exactly_its_steps_in_fcfs_order():
    clock = FakeClock()
    be = FakeBackend(clock)
    reqs = _trace()
    st = serve.Server(be, hbm_budget=1e12, clock=clock, sleep=clock.sleep).run(reqs)
    assert st["completed"] == len(reqs) and st["rejected"] == 0
    order = sorted(range(len(reqs)), key=lambda i: reqs[i].arrival)
    # bodies are created in arrival order and each receives its own step count
    assert [be.steps_of[k] for k in be.admit_order] == [reqs[i].steps for i in order]
    recs = {r.index: r for r in st["records"]}
    for i, q in enumerate(reqs):
        r = recs[i]
        assert r.admitted >= q.arrival - 1e-12 and r.completed > r.admitted
        # no faster than the request alone on the simulated device
        assert r.latency >= q.steps * q.problem.nx * q.problem.ny / be.rate - 1e-9
    assert st["p50_s"] <= st["p99_s"]


def test_budget_bounds_memory_and_head_of_line_blocks():
    clock = FakeClock()
    be = FakeBackend(clock)
    reqs = _trace(30, seed=5)
    biggest = max(q.problem.nx * q.problem.ny for q in reqs) * be.per_node
    budget = 1.5 * biggest
    st = serve.Server(be, hbm_budget=budget, clock=clock, sleep=clock.sleep).run(reqs)
    assert st["completed"] == len(reqs)
    assert st["peak_hbm_bytes"] <= budget
    assert be.peak_live < len(reqs)  # the budget forced queueing
    order = sorted(range(len(reqs)), key=lambda i: reqs[i].arrival)
    assert [be.steps_of[k] for k in be.admit_order] == [reqs[i].steps for i in order]


def test_request_larger_than_the_budget_is_rejected():
    clock = FakeClock()
    be = FakeBackend(clock)
    reqs = _trace(10, seed=7)
    reqs[4] = dataclasses.replace(reqs[4], problem=_P(5000, 5000))
    st = serve.Server(be, hbm_budget=5000 * 4000 * be.per_node, clock=clock, sleep=clock.sleep).run(reqs)
    assert st["rejected"] == 1 and st["completed"] == 9


def test_idle_server_waits_for_arrivals():
    clock = FakeClock()
    be = FakeBackend(clock, rate=1e12)
    reqs = [W.Request(arrival=10.0 * k, problem=_P(64, 64), steps=100) for k in range(3)]
    st = serve.Server(be, clock=clock, sleep=clock.sleep).run(reqs)
    assert st["completed"] == 3
    for r in st["records"]:
        assert r.admitted >= r.arrival and r.latency < 1.0
    assert st["makespan_s"] >= 20.0


def test_trace_at_rate_keeps_requests_and_sets_poisson_arrivals():
    reqs = _trace(200)
    out = serve.trace_at_rate(reqs, rate=50.0)
    assert [q.steps for q in out] == [q.steps for q in reqs]
    gaps = np.diff([0.0] + [q.arrival for q in out])
    assert (gaps > 0).all() and abs(gaps.mean() - 1 / 50.0) < 0.3 / 50.0


class _Failure(RuntimeError):
    def __init__(self, status):
        super().__init__(f"injected failure {status}")
        self.status = status


class FailingBackend(FakeBackend):
    """FakeBackend whose k-th create, k-th batch step and k-th result read
    raise (host-side fault injection: nothing runs on a GPU)."""

    def __init__(self, clock, fail_create=3, fail_step=6, fail_result=2, **kw):
        super().__init__(clock, **kw)
        self.fail = {"create": fail_create, "step": fail_step, "result": fail_result}
        self.calls = {"create": 0, "step": 0, "result": 0}
        self.failed_ids = set()
        self.creates_tried = 0

    def _maybe(self, what, status):
        self.calls[what] += 1
        if self.calls[what] == self.fail[what]:
            raise _Failure(status)

    def create(self, prob):
        self._maybe("create", 2)  # as lbm_create's LBM_E_OOM
        return super().create(prob)

    def step(self, batch, n):
        try:
            self._maybe("step", 3)  # as a failed launch: LBM_E_CUDA
        except _Failure:
            self.failed_ids.update(h["id"] for h in batch)
            raise
        super().step(batch, n)

    def result(self, h):
        self._maybe("result", 3)
        return super().result(h)


def test_failed_requests_complete_with_their_status_and_the_others_go_on():
    clock = FakeClock()
    be = FailingBackend(clock)
    reqs = _trace(40, seed=9)
    st = serve.Server(be, hbm_budget=1e12, clock=clock, sleep=clock.sleep).run(reqs)
    assert st["completed"] == len(reqs) and st["rejected"] == 0  # every request got an answer
    recs = {r.index: r for r in st["records"]}
    order = sorted(range(len(reqs)), key=lambda i: reqs[i].arrival)
    failed_create = order[be.fail["create"] - 1]
    assert recs[failed_create].status == 2
    bad = [i for i, r in recs.items() if r.status != 0]
    n_step = len(be.failed_ids)
    assert n_step >= 1  # the failed batch step took its members with it
    assert len(bad) == 1 + n_step + 1 and st["failed"] == len(bad)
    # the requests that did not fail got exactly their steps
    created = [i for i in order if i != failed_create]
    for k, i in zip(be.admit_order, created):
        if recs[i].status == 0:
            assert be.steps_of[k] == reqs[i].steps
    assert st["p50_s"] is not None


class UnstableBackend(FakeBackend):
    """Every third body reports LBM_E_UNSTABLE when its batch is synced."""

    def sync(self, batch):
        return [4 if h["id"] % 3 == 2 else 0 for h in batch]


def test_stable_only_percentiles_leave_out_the_unstable_solves():
    clock = FakeClock()
    be = UnstableBackend(clock)
    reqs = _trace(60, seed=11)
    st = serve.Server(be, hbm_budget=1e12, clock=clock, sleep=clock.sleep).run(reqs)
    ok = sorted(r.latency for r in st["records"] if r.status == 0)
    assert st["unstable"] == 20 and st["stable_completed"] == len(ok) == 40
    assert abs(st["stable_p50_s"] - float(np.percentile(ok, 50))) < 1e-12
    assert abs(st["stable_p99_s"] - float(np.percentile(ok, 99))) < 1e-12
    assert st["p50_s"] is not None and st["completed"] == 60


def test_stable_materials_trace_draws_the_stable_poisson_ratios():
    lit = W.serving_trace(max_requests=200)
    st = W.serving_trace(max_requests=200, stable_materials=True)
    assert [q.arrival for q in st] == [q.arrival for q in lit]  # the same draws otherwise
    assert [q.problem.nx for q in st] == [q.problem.nx for q in lit]
    for q in st:
        nu = q.problem.lam / (2.0 * (q.problem.lam + q.problem.mu))
        if q.problem.periodic(0):
            assert 0.2 - 1e-12 <= nu <= 0.4 + 1e-12
        else:
            assert abs(nu - 0.25) < 1e-12


class PreparingBackend(FakeBackend):
    """FakeBackend with a prepare() step, as the GPU backend builds a
    request's initial fields: it records the problems it prepared and which
    problem each create received."""

    def __init__(self, clock, **kw):
        super().__init__(clock, **kw)
        self.prepared = []
        self.created_from = []

    def prepare(self, prob):
        self.prepared.append(id(prob))
        return ("prepared", prob)

    def create(self, prob):
        assert isinstance(prob, tuple) and prob[0] == "prepared"
        self.created_from.append(id(prob[1]))
        return super().create(prob[1])

    def estimate(self, prob):
        return super().estimate(prob)


def test_loader_threads_prepare_each_admitted_request_once():
    clock = FakeClock()
    be = PreparingBackend(clock)
    reqs = _trace(50, seed=13)
    st = serve.Server(be, hbm_budget=1e12, clock=clock, sleep=clock.sleep, loader_threads=4, prefetch=8).run(reqs)
    assert st["completed"] == len(reqs)
    order = sorted(range(len(reqs)), key=lambda i: reqs[i].arrival)
    # every request prepared exactly once, and created from its prepared form in FCFS order
    assert sorted(be.prepared) == sorted(id(q.problem) for q in reqs)
    assert be.created_from == [id(reqs[i].problem) for i in order]
    assert [be.steps_of[k] for k in be.admit_order] == [reqs[i].steps for i in order]
