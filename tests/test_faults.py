"""Failure handling on the GPU without a GPU fault: failures are injected on
the host (LBM_FAULT names the call that fails) and must stay confined to the
context, batch or request they hit."""
import os

import numpy as np
import pytest

from paper_2208_13769_gb300 import lbm, serve
from paper_2208_13769_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _prob(seed=3):
    return W.smooth_random(40, 30, W.clamped_free_edges(), seed=seed, amp=0.01, vamp=0.004, lam=0.3, mu=0.3)


def test_injected_launch_failure_leaves_only_that_context_unusable(monkeypatch):
    with lbm.Body(_prob(), storage="f32") as ref:
        ref.step(8)
        want = ref.read(lbm.LBM_FIELD_U)["u"]
    with lbm.Body(_prob(), storage="f32") as a, lbm.Body(_prob(), storage="f32") as b:
        a.step(3)
        monkeypatch.setenv("LBM_FAULT", "step")
        with pytest.raises(lbm.LbmError) as e:
            a.step(5)
        assert e.value.status == lbm.LBM_E_CUDA
        monkeypatch.delenv("LBM_FAULT")
        with pytest.raises(lbm.LbmError) as e:  # the context stays unusable
            a.step(1)
        assert e.value.status == lbm.LBM_E_CUDA
        b.step(8)  # another context is untouched
        assert np.array_equal(b.read(lbm.LBM_FIELD_U)["u"], want)


def test_injected_batch_failure_is_sticky_for_the_batch_only(monkeypatch):
    bodies = [lbm.Body(_prob(s), storage="f32") for s in (3, 4)]
    try:
        batch = lbm.Batch(bodies)
        batch.step(2)
        monkeypatch.setenv("LBM_FAULT", "batch_step")
        with pytest.raises(lbm.LbmError) as e:
            batch.step(2)
        assert e.value.status == lbm.LBM_E_CUDA
        monkeypatch.delenv("LBM_FAULT")
        with pytest.raises(lbm.LbmError):
            batch.step(1)
        batch.close()
        with lbm.Body(_prob(5), storage="f32") as c:  # the device keeps working
            c.step(10)
            assert c.read(lbm.LBM_FIELD_U)["status"] == lbm.LBM_OK
    finally:
        for b in bodies:
            b.close()


class _OneFailingCreate(serve.GpuBackend):
    """The second body creation fails (LBM_FAULT=alloc for that call only)."""

    def __init__(self, **kw):
        super().__init__(**kw)
        self.creates = 0

    def create(self, prob):
        self.creates += 1
        if self.creates != 2:
            return super().create(prob)
        os.environ["LBM_FAULT"] = "alloc"
        try:
            return super().create(prob)
        finally:
            del os.environ["LBM_FAULT"]


def test_server_answers_every_request_when_one_cannot_be_created():
    reqs = [W.Request(arrival=0.001 * k, problem=_prob(10 + k), steps=40 + 10 * k) for k in range(4)]
    srv = serve.Server(_OneFailingCreate(storage="f32"), hbm_budget=1e10, keep_results=True)
    st = srv.run(reqs)
    assert st["completed"] == 4 and st["failed"] == 1
    recs = {r.index: r for r in st["records"]}
    assert recs[1].status == lbm.LBM_E_OOM
    for k in (0, 2, 3):
        assert recs[k].status == lbm.LBM_OK
        with lbm.Body(reqs[k].problem, storage="f32", scheme=lbm.LBM_SCHEME_PREDICTOR) as alone:
            alone.step(reqs[k].steps)
            assert np.array_equal(srv.results[k], alone.read(lbm.LBM_FIELD_U)["u"])
