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

    alone, st1 = run(1)
    mixed, st = run(8)
    assert st1["groups"] == 0                # one at a time: nothing to coalesce
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


def test_coalesced_groups_equal_alone_at_each_size(oracle):
    """Eight forward + backward requests of one grid size submitted at once to
    a one-slot server with coalescing on run as a single batched launch; each
    result equals the same request run alone, and two of them match the FP64
    oracle."""
    import torch
    from paper_2106_03452_gb300 import serve, synth
    for r in (64, 128):
        rng = synth.Rng(4100 + r)
        reqs = []
        for i in range(8):
            N = 1000 + 2500 * i
            pts, nrm = synth.ellipsoid_cloud(rng, N, 1 + i % 4)
            reqs.append((torch.from_numpy(pts).pin_memory(), torch.from_numpy(nrm).pin_memory(),
                         torch.from_numpy(synth.upstream_grad(rng, r)).pin_memory()))

        def outs(N):
            return (torch.empty((r, r, r)).pin_memory(), torch.empty((N, 3)).pin_memory(),
                    torch.empty((N, 3)).pin_memory())

        res = {}
        for mode, groups in (("alone", 1), ("group", 8)):
            srv = serve.Server(8 << 30, 1, max_group=groups)
            o = [outs(p.shape[0]) for (p, _, _) in reqs]
            if mode == "alone":
                for (p, n, g), (c, d, e) in zip(reqs, o):
                    assert srv.wait(srv.submit(r, p, n, c, g, d, e), 120.0) == 0
            else:
                # hold the slot with an r = 256 request (solo, several milliseconds)
                # so that the eight queue up behind it
                hp, hn = synth.ellipsoid_cloud(synth.Rng(4099), 200000, 3)
                hp, hn = torch.from_numpy(hp).pin_memory(), torch.from_numpy(hn).pin_memory()
                hg = torch.from_numpy(synth.upstream_grad(synth.Rng(4098), 256)).pin_memory()
                h_out = (torch.empty((256,) * 3).pin_memory(), torch.empty((200000, 3)).pin_memory(),
                         torch.empty((200000, 3)).pin_memory())
                t0 = srv.submit(256, hp, hn, h_out[0], hg, h_out[1], h_out[2])
                ts = [srv.submit(r, p, n, c, g, d, e) for (p, n, g), (c, d, e) in zip(reqs, o)]
                assert srv.wait(t0, 120.0) == 0
                assert all(srv.wait(t, 120.0) == 0 for t in ts)
                st = srv.stats()
                assert st["groups"] >= 1 and st["grouped_requests"] >= 7, st
            res[mode] = o
            srv.close()
        for i in range(8):
            a, g = res["alone"][i], res["group"][i]
            assert _rel(g[0], a[0]) <= 1e-5
            assert _rel(g[1], a[1]) <= 1e-4 and _rel(g[2], a[2]) <= 1e-4
        for i in (0, 7):
            p, n, G = reqs[i]
            ref = oracle.forward(r, 2.0, p.numpy(), n.numpy())
            assert _rel(res["group"][i][0], ref) <= 1e-5
            rdp, rdn = oracle.backward(r, 2.0, p.numpy(), n.numpy(), G.numpy())
            assert _rel(res["group"][i][1], rdp) <= 1e-4 and _rel(res["group"][i][2], rdn) <= 1e-4


def test_cancel_queued_request():
    """A request still queued behind others is cancelled: its wait returns
    DPSR_ECANCELED and its output buffer keeps its contents; an admitted or
    finished request cannot be cancelled (DPSR_EBUSY) and completes normally;
    a retired ticket is unknown (DPSR_EINVAL)."""
    import torch
    from paper_2106_03452_gb300 import libdpsr as L
    from paper_2106_03452_gb300 import serve
    pool = serve.InputPool(n_clouds=2, n_max=200000, rs=(256,))
    srv = serve.Server(8 << 30, slots=1, max_group=1)
    pts, nrm = pool.inputs(0, 200000)
    outs = [torch.full((256, 256, 256), float("nan")).pin_memory() for _ in range(6)]
    tickets = [srv.submit(256, pts, nrm, outs[i]) for i in range(6)]
    # five 200 000-point r = 256 solves run one at a time ahead of the last
    assert srv.cancel(tickets[5]) == L.DPSR_OK
    assert srv.wait(tickets[5], 60.0) == L.DPSR_ECANCELED
    assert srv.cancel(tickets[0]) == L.DPSR_EBUSY       # admitted first
    for t in tickets[:5]:
        assert srv.wait(t, 120.0) == 0
    assert torch.isnan(outs[5]).all()                  # never written
    assert all(torch.isfinite(o).all() for o in outs[:5])
    with pytest.raises(L.DPSRError) as e:
        srv.cancel(tickets[0])                         # retired by its wait
    assert e.value.code == L.DPSR_EINVAL
    st = srv.stats()
    assert st["completed"] == 5
    srv.close()


def test_producer_thread_dies_mid_queue():
    """A submitting thread that raises after queueing its requests (so that
    nobody waits for them) leaves the server consistent: those requests still
    run, another producer's requests complete, and the server shuts down
    cleanly with the orphaned tickets never retired."""
    import threading
    import time

    import torch
    from paper_2106_03452_gb300 import serve
    pool = serve.InputPool(n_clouds=2, n_max=50000, rs=(64, 128))
    srv = serve.Server(8 << 30, slots=4)
    keep = []

    def dying_producer():
        for i in range(6):
            pts, nrm = pool.inputs(i, 50000)
            chi = torch.empty((128, 128, 128)).pin_memory()
            keep.append(chi)                            # the buffers outlive the thread
            srv.submit(128, pts, nrm, chi)
        raise RuntimeError("producer died with its requests in the queue")

    errors = []
    th = threading.Thread(target=lambda: errors.append(_run_catching(dying_producer)))
    th.start()
    mine = []
    for i in range(6):
        pts, nrm = pool.inputs(i + 1, 20000)
        chi = torch.empty((64, 64, 64)).pin_memory()
        mine.append((srv.submit(64, pts, nrm, chi), chi))
    th.join()
    assert errors and isinstance(errors[0], RuntimeError)
    for t, chi in mine:
        assert srv.wait(t, 120.0) == 0 and torch.isfinite(chi).all()
    deadline = time.time() + 60.0
    while srv.stats()["completed"] < 12 and time.time() < deadline:
        time.sleep(0.01)
    assert srv.stats()["completed"] == 12
    assert all(torch.isfinite(c).all() for c in keep)
    srv.close()


def _run_catching(fn):
    try:
        fn()
    except Exception as exc:  # the producer's own failure, recorded for the test
        return exc
    return None


def test_wait_any_retires_in_completion_batches():
    """dpsr_server_wait_any hands back every completed request once, with its
    status, and skips tickets that poll or wait already retired."""
    import torch
    from paper_2106_03452_gb300 import libdpsr as L
    from paper_2106_03452_gb300 import serve
    pool = serve.InputPool(n_clouds=2, n_max=30000, rs=(64, 128))
    srv = serve.Server(8 << 30, slots=4)
    keep, tickets = [], []
    for i in range(12):
        r = 64 if i % 2 else 128
        pts, nrm = pool.inputs(i, 30000)
        chi = torch.empty((r, r, r)).pin_memory()
        keep.append(chi)
        tickets.append(srv.submit(r, pts, nrm, chi))
    assert srv.wait(tickets[0], 120.0) == 0          # retired by wait: never returned below
    seen = {}
    while len(seen) < 11:
        got = srv.wait_any(5, 60.0)
        assert got, "timed out"
        assert len(got) <= 5
        for t, st in got:
            assert t not in seen and st == 0
            seen[t] = st
    assert sorted(seen) == sorted(tickets[1:])
    assert srv.wait_any(5, 0.05) == []               # nothing left
    with pytest.raises(L.DPSRError):
        L.check(L.dpsr_server_wait(srv.handle, tickets[3], 1.0), "wait")   # already retired
    assert all(torch.isfinite(c).all() for c in keep)
    srv.close()


def test_queued_same_size_requests_are_coalesced():
    """With one slot held by a long r = 256 request, six r = 64 requests queue
    behind it; when the slot frees, the head and the five behind it (same
    size, same mode) are admitted as one batched launch, and each still
    equals its solo result."""
    import torch
    from paper_2106_03452_gb300 import serve
    pool = serve.InputPool(n_clouds=2, n_max=100000, rs=(64, 256))
    srv = serve.Server(8 << 30, slots=1, max_group=8)
    serve.warm(srv, pool, rs=(64, 256), slots=1, n=100000)
    g0 = srv.stats()
    pts, nrm = pool.inputs(0, 100000)
    big = torch.empty((256,) * 3).pin_memory()
    d = [torch.empty(100000, 3).pin_memory() for _ in range(2)]
    t_big = srv.submit(256, pts, nrm, big, pool.dchi[256], d[0], d[1])
    small = []
    for i in range(6):
        p, n = pool.inputs(i + 1, 3000 + 500 * i)
        chi = torch.empty((64,) * 3).pin_memory()
        small.append((srv.submit(64, p, n, chi), p, n, chi))
    assert srv.wait(t_big, 120.0) == 0
    for t, _, _, _ in small:
        assert srv.wait(t, 120.0) == 0
    st = srv.stats()
    assert st["groups"] - g0["groups"] >= 1 and st["grouped_requests"] - g0["grouped_requests"] >= 2
    srv.close()
    solo = serve.Server(8 << 30, slots=1, max_group=1)
    for _, p, n, chi in small:
        ref = torch.empty((64,) * 3).pin_memory()
        assert solo.wait(solo.submit(64, p, n, ref), 120.0) == 0
        assert _rel(chi, ref) <= 1e-5
    solo.close()
