"""The allocation-free diagnostics entry point, checked through the C ABI.

lbm_diagnostics_noalloc serves callers that cannot allocate device memory
(graph capture, fixed pools, foreign allocators): it reads caller-owned
device fields and keeps its scratch in a static array inside the library.
Its six numbers must match those of lbm_diagnostics, which uses context
memory, on two calls in a row.  This file sorts last so that a run stopping
at its first failure has run every other test already.
"""
import numpy as np
import pytest

from paper_2208_13769_gb300 import lbm
from paper_2208_13769_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _geometry(prob, t):
    g = lbm.lbm_field_geometry()
    g.nx, g.ny, g.dX = prob.nx, prob.ny, prob.dX
    g.lam, g.mu, g.rho0 = prob.lam, prob.mu, prob.rho0
    for k, e in enumerate(prob.edges):
        g.edge_kind[k] = e.kind
        for a in range(2):
            g.edge_u[k][a] = e.value[a] + e.rate[a] * t
    return g


def _device_fields(torch, fields):
    planes = np.stack([fields["u"][:, :, 0], fields["u"][:, :, 1], fields["v"][:, :, 0],
                       fields["v"][:, :, 1], fields["r"]])
    return torch.tensor(planes, dtype=torch.float64, device="cuda").contiguous()


@pytest.mark.parametrize("nx,ny", [(150, 90), (700, 400)])
def test_noalloc_diagnostics_match_context_diagnostics(nx, ny):
    """150 x 90 nodes: 53 CTAs of partial sums.  700 x 400 nodes: more than
    1024 CTAs' worth, so the allocation-free call's CTAs stride over several
    nodes each (the additions in another order than lbm_diagnostics')."""
    torch = pytest.importorskip("torch")
    prob = W.smooth_random(nx, ny, [W.Edge(W.DIRICHLET, value=(0.0, 0.0), rate=(0.002, -0.001)),
                                    W.Edge(W.NEUMANN), W.Edge(W.NEUMANN), W.Edge(W.NEUMANN)],
                           seed=21, amp=0.01, vamp=0.004, lam=0.3, mu=0.3)
    stream = torch.cuda.current_stream().cuda_stream
    out = torch.full((8,), float("nan"), dtype=torch.float64, device="cuda")
    with lbm.Body(prob, storage="f64") as body:
        for steps in (40, 25):  # two calls in a row, at different states
            body.step(steps)
            ref = body.diagnostics()
            fields = body.read(lbm.LBM_FIELD_U | lbm.LBM_FIELD_V | lbm.LBM_FIELD_R)
            dev = _device_fields(torch, fields)
            torch.cuda.synchronize()
            st = lbm.lbm_diagnostics_noalloc(_geometry(prob, fields["t"]), dev.data_ptr(), out.data_ptr(), stream)
            assert st == lbm.LBM_OK
            torch.cuda.synchronize()
            got = out.cpu().numpy()
            np.testing.assert_allclose(got[:6], ref, rtol=1e-12, atol=1e-15)
            assert got[6] == 0.0 and got[7] == 0.0


def test_noalloc_rejects_bad_sizes_without_launching():
    geo = lbm.lbm_field_geometry()
    geo.nx, geo.ny, geo.dX, geo.lam, geo.mu, geo.rho0 = 2, 10, 1.0, 0.3, 0.3, 1.0
    assert lbm.lbm_diagnostics_noalloc(geo, 16, 16) == lbm.LBM_E_INVALID
    geo.nx, geo.ny = 1 << 16, 1 << 16  # 2^32 nodes > LBM_NOALLOC_MAX_NODES
    assert lbm.lbm_diagnostics_noalloc(geo, 16, 16) == lbm.LBM_E_INVALID
    geo.nx, geo.ny = 10, 10
    geo.edge_kind[0], geo.edge_kind[1] = lbm.LBM_PERIODIC, lbm.LBM_NEUMANN
    assert lbm.lbm_diagnostics_noalloc(geo, 16, 16) == lbm.LBM_E_INVALID
