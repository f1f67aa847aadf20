"""Failure detection on the device without a fault: a kernel's bounded wait
on a barrier that nothing completes gives up after its limit, reports
DPSR_ETIMEOUT through the status word, and the context stays usable (a
solve right after it still matches the oracle)."""
import time

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2106_03452_gb300 import build
    build.build()


def test_bounded_wait_gives_up_and_context_survives(oracle):
    from gpu_util import gpu_fwd_bwd, relmax
    from paper_2106_03452_gb300 import libdpsr as L
    from paper_2106_03452_gb300 import synth
    assert L.dpsr_check_bounded_wait(0.0) == L.DPSR_EINVAL
    t0 = time.perf_counter()
    assert L.dpsr_check_bounded_wait(0.05) == L.DPSR_ETIMEOUT
    dt = time.perf_counter() - t0
    assert 0.04 <= dt < 5.0, dt  # the wait ran out near its limit, not at some other bound
    w = synth.workload_sphere_r32()
    g = gpu_fwd_bwd(w["r"], w["sigma"], w["points"], w["normals"], None)
    assert g["status"] == 0
    ref = oracle.forward(w["r"], w["sigma"], w["points"].astype(np.float64), w["normals"].astype(np.float64))
    assert relmax(g["chi"], ref) <= 1e-5


def test_timeout_surfaces_through_sync(oracle):
    """A bounded wait that gives up on a plan's stream comes back from
    dpsr_sync as DPSR_ETIMEOUT (ahead of any other status), the status is
    cleared by that sync, and the next solve on the same plan is correct."""
    import torch
    from gpu_util import relmax
    from paper_2106_03452_gb300 import libdpsr as L
    from paper_2106_03452_gb300 import synth
    from paper_2106_03452_gb300.dpsr import Plan
    w = synth.workload_sphere_r32()
    plan = Plan(w["r"], w["sigma"])
    assert L.dpsr_plan_check_bounded_wait(plan.handle, 0.0) == L.DPSR_EINVAL
    assert L.dpsr_plan_check_bounded_wait(plan.handle, 0.05) == L.DPSR_OK
    assert plan.sync() == L.DPSR_ETIMEOUT
    assert plan.sync() == L.DPSR_OK  # cleared
    P = torch.from_numpy(w["points"]).cuda()
    N = torch.from_numpy(w["normals"]).cuda()
    # zero normals make chi' vanish: a degenerate scale of Eq. 4 on its own ...
    plan.forward(P, torch.zeros_like(N))
    assert plan.sync() == L.DPSR_EDEGENERATE
    # ... and with a timed-out wait in the same sync window, the timeout wins
    plan.forward(P, torch.zeros_like(N))
    assert L.dpsr_plan_check_bounded_wait(plan.handle, 0.02) == L.DPSR_OK
    assert plan.sync() == L.DPSR_ETIMEOUT
    chi = plan.forward(P, N)
    assert plan.sync() == L.DPSR_OK
    ref = oracle.forward(w["r"], w["sigma"], w["points"].astype(np.float64), w["normals"].astype(np.float64))
    assert relmax(chi.cpu().numpy(), ref) <= 1e-5
    plan.close()
