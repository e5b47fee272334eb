"""The serving loop on the GPU: every request of a small trace completes with
exactly the result of solving it alone (same kernels, exact step counts),
under a memory budget that forces queueing."""
import numpy as np
import pytest

from paper_2208_13769_gb300 import lbm, serve
from paper_2208_13769_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _small_trace(n=10, seed=5):
    rng = np.random.default_rng(seed)
    out, t = [], 0.0
    for _ in range(n):
        t += float(rng.exponential(0.002))
        prob = W.random_body(rng, 40, 180)
        out.append(W.Request(arrival=t, problem=prob, steps=int(rng.integers(30, 300))))
    return out


@pytest.mark.parametrize("storage", ["f32", "f16"])
def test_served_results_equal_solving_alone(storage):
    reqs = _small_trace()
    be = serve.GpuBackend(storage=storage)
    budget = 3.2 * max(be.estimate(q.problem) for q in reqs)
    srv = serve.Server(be, hbm_budget=budget, target_chunk_s=0.002, keep_results=True)
    st = srv.run(reqs)
    assert st["completed"] == len(reqs) and st["rejected"] == 0
    assert st["peak_hbm_bytes"] <= budget
    assert st["max_active"] < len(reqs)  # the budget made requests queue
    for i, q in enumerate(reqs):
        with lbm.Body(q.problem, storage=storage, scheme=be.scheme) as b:
            b.step(q.steps)
            u = b.read(lbm.LBM_FIELD_U, allow_unstable=True)["u"]
        # bit for bit (a request that went unstable has NaNs in the same places)
        assert np.array_equal(srv.results[i].view(np.int64), u.view(np.int64)), i
