"""Seeded sweeps over the other entry points, each against the plain
device-buffer solve of the same inputs: the no-allocation forward
(dpsr_forward_static) over its size range, the one-call host-buffer solve
(dpsr_solve_host) over sizes that grow and shrink between calls on one plan,
and the server with a random request mix, some of the queued requests
cancelled. Tolerances: chi 1e-5 of its largest entry (plus the scale-rounding
term for near-degenerate draws), gradients 1e-4."""
import numpy as np
import pytest

from paper_2106_03452_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2106_03452_gb300 import build
    build.build()


def _draw(rng, rs, n_lo, n_hi):
    u = rng.uniform(3)
    r = rs[min(int(u[0] * len(rs)), len(rs) - 1)]
    N = int(round(np.exp(np.log(n_lo) + (np.log(n_hi) - np.log(n_lo)) * u[1])))
    sigma = round(float(4.0 * u[2]), 2)
    pts = (rng.uniform(N, 3) * 1.3 - 0.15).astype(np.float32)
    nrm = rng.normal(N, 3).astype(np.float32)
    return r, N, sigma, pts, nrm


def _tol(chi_ref):
    return 1e-5 + 4 * 2.0 ** -24 * 2.0 * float(np.max(np.abs(chi_ref)))


def test_static_forward_sweep():
    import torch
    from gpu_util import relmax
    from paper_2106_03452_gb300 import libdpsr as L
    from paper_2106_03452_gb300.dpsr import Plan
    rng = synth.Rng(71000)
    stream = torch.cuda.current_stream().cuda_stream
    for case in range(10):
        r, N, sigma, pts, nrm = _draw(rng, [8, 16, 32, 64], 1, 65536)
        P, Nn = torch.from_numpy(pts).cuda(), torch.from_numpy(nrm).cuda()
        plan = Plan(r, sigma)
        ref = plan.forward(P, Nn).clone()
        st = plan.sync()
        out = torch.full((r, r, r), float("nan"), device="cuda")
        st2 = L.dpsr_forward_static(r, sigma, P.data_ptr(), Nn.data_ptr(), N, out.data_ptr(), stream)
        torch.cuda.synchronize()
        assert st2 == st, (case, r, N, sigma, st, st2)   # same verdict on degenerate draws
        if st == 0:
            ref = ref.cpu().numpy()
            assert relmax(out.cpu().numpy(), ref) <= _tol(ref), (case, r, N, sigma)
        plan.close()


def test_solve_host_sweep():
    """One plan, sizes that grow and shrink between calls (the staging is
    reused or regrown), pageable host buffers."""
    import torch
    from gpu_util import relmax
    from paper_2106_03452_gb300 import libdpsr as L
    from paper_2106_03452_gb300.dpsr import Plan
    rng = synth.Rng(72000)
    for r in (32, 128):
        host = Plan(r, 2.0)
        for case in range(5):
            _, N, _, pts, nrm = _draw(rng, [r], 10, 60000)
            g = rng.normal(r, r, r).astype(np.float32)
            dev = Plan(r, 2.0)
            P, Nn = torch.from_numpy(pts).cuda(), torch.from_numpy(nrm).cuda()
            chi = dev.forward(P, Nn).clone()
            dp, dn = dev.backward(torch.from_numpy(g).cuda())
            assert dev.sync() == 0
            hchi = np.zeros((r, r, r), np.float32)
            hdp, hdn = np.zeros_like(pts), np.zeros_like(pts)
            L.dpsr_solve_host(host.handle, pts.ctypes.data, nrm.ctypes.data, N, g.ctypes.data,
                              hchi.ctypes.data, hdp.ctypes.data, hdn.ctypes.data)  # raises on an error
            ref = chi.cpu().numpy()
            assert relmax(hchi, ref) <= _tol(ref), (r, case, N)
            assert relmax(hdn, dn.cpu().numpy()) <= 1e-4 and relmax(hdp, dp.cpu().numpy()) <= 1e-4, (r, case, N)
            dev.close()
        host.close()


def test_server_sweep_with_cancellations():
    """A random mix of 40 requests (r 32/64/128, fwd or fwd+bwd, N up to
    40 000) submitted at once to a 3-slot coalescing server, every fifth one
    cancelled right after submission: each request completes with status 0
    (equal to its solo solve) or, if it was still queued, with
    DPSR_ECANCELED and its buffer untouched."""
    import torch
    from gpu_util import relmax
    from paper_2106_03452_gb300 import libdpsr as L
    from paper_2106_03452_gb300 import serve
    from paper_2106_03452_gb300.dpsr import Plan
    rng = synth.Rng(73000)
    srv = serve.Server(8 << 30, slots=3, max_group=8)
    reqs = []
    for i in range(40):
        r, N, sigma, pts, nrm = _draw(rng, [32, 64, 128], 100, 40000)
        bwd = rng.uniform() < 0.3
        P, Nn = torch.from_numpy(pts).pin_memory(), torch.from_numpy(nrm).pin_memory()
        chi = torch.full((r, r, r), float("nan")).pin_memory()
        G = torch.from_numpy(rng.normal(r, r, r).astype(np.float32)).pin_memory() if bwd else None
        dp = torch.zeros((N, 3)).pin_memory() if bwd else None
        dn = torch.zeros((N, 3)).pin_memory() if bwd else None
        t = srv.submit(r, P, Nn, chi, G, dp, dn)
        cancelled = False
        if i % 5 == 4:
            cancelled = srv.cancel(t) == L.DPSR_OK
        reqs.append((t, r, P, Nn, chi, G, dp, dn, cancelled))
    for (t, r, P, Nn, chi, G, dp, dn, cancelled) in reqs:
        st = srv.wait(t, 120.0)
        if cancelled:
            assert st == L.DPSR_ECANCELED and torch.isnan(chi).all()
            continue
        assert st == 0
        plan = Plan(r, 2.0)
        ref = plan.forward(P.cuda(), Nn.cuda()).cpu().numpy()
        assert relmax(chi.numpy(), ref) <= _tol(ref)
        if G is not None:
            d0, n0 = plan.backward(G.cuda())
            assert relmax(dn.numpy(), n0.cpu().numpy()) <= 1e-4 and relmax(dp.numpy(), d0.cpu().numpy()) <= 1e-4
        assert plan.sync() == 0
        plan.close()
    srv.close()
