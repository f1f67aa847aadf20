"""dpsr_forward_static, the forward entry point for callers that cannot
allocate device memory (it keeps its scratch in a static device array),
against the regular dpsr_forward through the C ABI: the same chi within the
tolerance of the parity tests, on two calls in a row (the second call sees
what the first left in the shared array). Collected last on purpose."""
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


def test_static_forward_matches_plan_forward():
    import torch
    from paper_2106_03452_gb300 import libdpsr as L
    from paper_2106_03452_gb300 import synth
    from paper_2106_03452_gb300.dpsr import Plan

    cases = [synth.workload_sphere_r32(), synth.workload_sphere_r32(seed=7, N=5000),
             synth.workload_sphere_r32(seed=8, N=300), synth.workload_sphere_r32(seed=9, N=900)]
    cases[1]["r"] = 64
    cases[2]["r"] = 8
    cases[3]["r"] = 16
    stream = torch.cuda.current_stream().cuda_stream
    for w in cases:
        r, sigma = w["r"], w["sigma"]
        P = torch.from_numpy(w["points"]).cuda()
        Nn = torch.from_numpy(w["normals"]).cuda()
        plan = Plan(r, sigma)
        ref = plan.forward(P, Nn).clone()
        assert plan.sync() == L.DPSR_OK
        for _ in range(2):  # two calls in a row share the static scratch
            out = torch.full((r, r, r), float("nan"), device="cuda")
            st = L.dpsr_forward_static(r, sigma, P.data_ptr(), Nn.data_ptr(), P.shape[0], out.data_ptr(),
                                       stream)
            assert st == L.DPSR_OK
            torch.cuda.synchronize()
            a, b = out.cpu().numpy().astype(np.float64), ref.cpu().numpy().astype(np.float64)
            assert np.max(np.abs(a - b)) / np.max(np.abs(b)) <= 1e-5
        plan.close()


def test_static_forward_rejects_sizes_above_its_limit():
    import torch
    from paper_2106_03452_gb300 import libdpsr as L
    P = torch.rand(70000, 3, device="cuda")
    out = torch.empty(128 ** 3, device="cuda")
    assert L.dpsr_forward_static(128, 2.0, P.data_ptr(), P.data_ptr(), 100, out.data_ptr(), 0) == L.DPSR_EINVAL
    assert L.dpsr_forward_static(32, 2.0, P.data_ptr(), P.data_ptr(), 70000, out.data_ptr(), 0) == L.DPSR_EINVAL
    assert L.dpsr_forward_static(12, 2.0, P.data_ptr(), P.data_ptr(), 100, out.data_ptr(), 0) == L.DPSR_EINVAL


def test_static_forward_rejects_misaligned_output_and_capture():
    """chi_out is written by bulk and vector stores: a pointer off a 16-byte
    boundary is rejected before anything is launched. The call synchronises
    and reads its status back, so it refuses to run inside a stream capture."""
    import torch
    from paper_2106_03452_gb300 import libdpsr as L
    from paper_2106_03452_gb300 import synth
    w = synth.workload_sphere_r32()
    P = torch.from_numpy(w["points"]).cuda()
    Nn = torch.from_numpy(w["normals"]).cuda()
    out = torch.zeros(32 ** 3 + 4, device="cuda")
    torch.cuda.synchronize()
    assert L.dpsr_forward_static(32, 2.0, P.data_ptr(), Nn.data_ptr(), P.shape[0], out.data_ptr() + 4, 0) \
        == L.DPSR_EINVAL
    torch.cuda.synchronize()
    assert torch.count_nonzero(out).item() == 0  # nothing ran
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        g.capture_begin()
        try:
            rc = L.dpsr_forward_static(32, 2.0, P.data_ptr(), Nn.data_ptr(), P.shape[0], out.data_ptr(),
                                       s.cuda_stream)
        finally:
            g.capture_end()
    assert rc == L.DPSR_ESTATE
