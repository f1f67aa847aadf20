"""Serving driver for libdpsr's request server (include/dpsr.h, dpsr_server_*).

Replays a Poisson arrival trace in real time: each request is submitted at
its arrival time with page-locked host buffers, a completion thread polls the
server, and latency = completion time - arrival time. The server admits
requests by device-memory budget into CUDA-stream slots as they free up
(continuous batching); with slots = 1 it degenerates into a per-solve loop.

Request inputs come from a pool of pre-generated clouds (a cloud of at least
N points cut to N), so that a long trace needs bounded host memory; r, N, the
backward flag and the arrival times follow the trace exactly.
"""
from __future__ import annotations

import threading
import time

import numpy as np
import torch

from . import libdpsr as L
from . import synth


class Server:
    """max_group: requests of grid size <= 128 coalesced per batched launch
    (1 = every request solo; with one slot that is the per-solve loop)."""

    def __init__(self, hbm_budget_bytes: int = 8 << 30, slots: int = 8, sigma: float = 2.0,
                 max_group: int = 8):
        self.handle = L.dpsr_server_create(hbm_budget_bytes, slots, sigma)
        self.slots, self.max_group = slots, max_group
        L.dpsr_server_set_max_group(self.handle, max_group)

    def submit(self, r, points, normals, chi_out, dchi=None, dpoints=None, dnormals=None) -> int:
        p = lambda t: t.data_ptr() if t is not None else 0
        return L.dpsr_server_submit(self.handle, r, points.data_ptr(), normals.data_ptr(),
                                    points.shape[0], p(dchi), chi_out.data_ptr(), p(dpoints), p(dnormals))

    def poll(self, ticket):
        return L.dpsr_server_poll(self.handle, ticket)

    def wait(self, ticket, timeout_s=0.0) -> int:
        return L.dpsr_server_wait(self.handle, ticket, timeout_s)

    def wait_any(self, max_n=64, timeout_s=0.0):
        return L.dpsr_server_wait_any(self.handle, max_n, timeout_s)

    def cancel(self, ticket) -> int:
        return L.dpsr_server_cancel(self.handle, ticket)

    def stats(self):
        d = L.dpsr_server_stats(self.handle)
        d.update(L.dpsr_server_group_stats(self.handle))
        return d

    def close(self):
        if getattr(self, "handle", None):
            L.dpsr_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class InputPool:
    """Pinned clouds per (pool index) and one pinned dchi per r."""

    def __init__(self, n_clouds=8, n_max=200000, rs=(64, 128, 256), seed=2024):
        rng = synth.Rng(seed)
        self.clouds = []
        for k in range(n_clouds):
            pts, nrm = synth.ellipsoid_cloud(rng, n_max, 1 + k % 6)
            self.clouds.append((torch.from_numpy(pts).pin_memory(), torch.from_numpy(nrm).pin_memory()))
        self.dchi = {r: torch.from_numpy(synth.upstream_grad(rng, r)).pin_memory() for r in rs}

    def inputs(self, i, N):
        pts, nrm = self.clouds[i % len(self.clouds)]
        return pts[:N], nrm[:N]


class OutputRing:
    """Pinned output buffers reused across requests (one set per in-flight
    request; grows on demand)."""

    def __init__(self):
        self.free = {}
        self.lock = threading.Lock()

    def get(self, r, n_max, bwd):
        key = (r, bwd)
        with self.lock:
            lst = self.free.setdefault(key, [])
            if lst:
                return lst.pop()
        chi = torch.empty((r, r, r), dtype=torch.float32).pin_memory()
        if bwd:
            return (chi, torch.empty((n_max, 3)).pin_memory(), torch.empty((n_max, 3)).pin_memory())
        return (chi, None, None)

    def prefill(self, keys, count, n_max):
        for r, bwd in keys:
            bufs = [self.get(r, n_max, bwd) for _ in range(count)]
            for b in bufs:
                self.put(r, bwd, b)

    def put(self, r, bwd, bufs):
        with self.lock:
            self.free.setdefault((r, bwd), []).append(bufs)


def replay(trace, server: Server, pool: InputPool, realtime=True, n_max=200000, on_done=None,
           ring=None):
    """Submit every request of `trace` (at its arrival time if realtime, all
    at once otherwise). Returns per-request dicts with arrival, submit and
    completion times (seconds from start) and the status."""
    ring = ring or OutputRing()
    pending = {}
    results = []
    lock = threading.Lock()
    stop = threading.Event()

    def completer():
        # completed requests come back in batches from one blocking call
        # (dpsr_server_wait_any), not from a poll of every outstanding ticket
        while not stop.is_set() or pending:
            got = server.wait_any(64, 0.02)
            now = time.perf_counter() - t0
            for t, st in got:
                with lock:
                    rec = pending.pop(t, None)
                if rec is None:  # not one of this replay's requests
                    continue
                rec["done"] = now
                rec["status"] = st
                ring.put(rec["r"], rec["bwd"], rec.pop("bufs"))
                if on_done is not None:
                    on_done(rec)
                with lock:
                    results.append(rec)

    th = threading.Thread(target=completer, daemon=True)
    t0 = time.perf_counter()
    th.start()
    for i, q in enumerate(trace):
        if realtime:
            # sleep to just short of the arrival time, then spin: a plain
            # sleep overshoots by a scheduler tick, which would count as latency
            dt = q["t"] - (time.perf_counter() - t0)
            if dt > 0.0005:
                time.sleep(dt - 0.0005)
            while time.perf_counter() - t0 < q["t"]:
                time.sleep(0)  # yields the interpreter lock to the completion thread
        r, N, bwd = q["r"], q["N"], q["backward"]
        pts, nrm = pool.inputs(i, N)
        bufs = ring.get(r, n_max, bwd)
        chi, dp, dn = bufs
        rec = dict(i=i, r=r, N=N, bwd=bwd, arrival=q["t"] if realtime else 0.0, bufs=bufs)
        rec["submit"] = time.perf_counter() - t0
        with lock:
            t = server.submit(r, pts, nrm, chi, pool.dchi[r] if bwd else None,
                              dp[:N] if bwd else None, dn[:N] if bwd else None)
            pending[t] = rec
    stop.set()
    th.join()
    return results


def summarize(results, wall_s):
    lat = np.array([r["done"] - r["arrival"] for r in results]) * 1e3
    ok = sum(1 for r in results if r["status"] == 0)
    return {"requests": len(results), "ok": ok, "p50_ms": float(np.percentile(lat, 50)),
            "p99_ms": float(np.percentile(lat, 99)), "mean_ms": float(lat.mean()),
            "solves_per_s": len(results) / wall_s, "wall_s": wall_s}


def warm(server: Server, pool: InputPool, rs=(64, 128, 256), slots=1, n=20000):
    """Fill the server's plan and batch pools before a measurement: for every
    grid size, `slots` concurrent groups of fwd+bwd requests of n points
    (max_group requests per group where the server coalesces that size), so
    that the pools hold a plan or a batch per slot at full capacity (plans and
    batches are created, and grown, only when none in the pool fits; that
    allocates device memory and tunes, which would otherwise stall the GPU in
    the middle of a measurement). The first request per grid size also runs
    the plan autotuner, alone."""
    ring = OutputRing()
    for r in rs:
        pts, nrm = pool.inputs(0, n)
        chi, dp, dn = ring.get(r, n, True)
        st = server.wait(server.submit(r, pts, nrm, chi, pool.dchi[r], dp, dn), 120.0)
        if st != 0:
            raise RuntimeError(f"warm-up request r={r} failed with status {st}")
        per = getattr(server, "max_group", 1) if r <= 128 else 1
        bufs = [ring.get(r, n, True) for _ in range(slots * per)]
        tickets = [server.submit(r, pts, nrm, c, pool.dchi[r], d, e) for (c, d, e) in bufs]
        for t in tickets:
            st = server.wait(t, 120.0)
            if st != 0:
                raise RuntimeError(f"warm-up request r={r} failed with status {st}")
