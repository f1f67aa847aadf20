"""The request server: mixed requests (r in {64, 128, 256}, forward only and
forward + backward) submitted together give the same results as the same
requests run alone, within the parity tolerances; admission by budget."""
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


def _rel(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def test_mix_equals_alone():
    import torch
    from paper_2106_03452_gb300 import libdpsr as L
    from paper_2106_03452_gb300 import serve, synth
    trace = synth.serving_trace(duration_s=0.2)[:24]
    trace[0].update(r=256, N=60000, backward=True)
    trace[1].update(r=64, N=1000, backward=False)
    pool = serve.InputPool(n_clouds=3, n_max=60000)
    for q in trace:
        q["N"] = min(q["N"], 60000)

    def run(slots, realtime=False):
        srv = serve.Server(8 << 30, slots)
        res = []
        ring = serve.OutputRing()
        for i, q in enumerate(trace):
            pts, nrm = pool.inputs(i, q["N"])
            chi, dp, dn = ring.get(q["r"], 60000, q["backward"])
            res.append((srv.submit(q["r"], pts, nrm, chi, pool.dchi[q["r"]] if q["backward"] else None,
                                   dp[:q["N"]] if q["backward"] else None,
                                   dn[:q["N"]] if q["backward"] else None), chi, dp, dn))
            if slots == 1:
                assert srv.wait(res[-1][0], 120.0) == 0     # alone: one at a time
        for t, chi, dp, dn in res:
            if slots != 1:
                assert srv.wait(t, 120.0) == 0
        st = srv.stats()
        srv.close()
        return [(chi.clone(), None if dp is None else dp.clone(), None if dn is None else dn.clone())
                for _, chi, dp, dn in res], st

    alone, _ = run(1)
    mixed, st = run(8)
    assert st["max_in_flight"] >= 2          # requests overlapped on the GPU
    for q, a, m in zip(trace, alone, mixed):
        assert _rel(m[0], a[0]) <= 1e-5
        if q["backward"]:
            N = q["N"]
            assert _rel(m[1][:N], a[1][:N]) <= 1e-4 and _rel(m[2][:N], a[2][:N]) <= 1e-4


def test_budget_admission():
    import torch
    from paper_2106_03452_gb300 import libdpsr as L
    from paper_2106_03452_gb300 import serve
    small = serve.Server(64 << 20, 4)             # 64 MiB: an r = 256 request cannot fit
    pts = torch.rand(5000, 3).pin_memory()
    nrm = torch.randn(5000, 3).pin_memory()
    chi = torch.empty(256 ** 3).pin_memory()
    t = small.submit(256, pts, nrm, chi)
    assert small.wait(t, 60.0) == L.DPSR_EBUSY
    chi64 = torch.empty(64 ** 3).pin_memory()
    t = small.submit(64, pts, nrm, chi64)
    assert small.wait(t, 60.0) == 0
    small.close()
