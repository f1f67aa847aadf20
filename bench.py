#!/usr/bin/env python
"""Benchmark of the spectral DPSR layer (forward + backward) on GB300.

One step = one DPSR forward + backward solve of the r = 128 workload (20 000
points on a union of 4 random ellipsoids, sigma = 2, dchi ~ N(0, 1)) with
every input resident in HBM. Between timed steps a 512 MiB buffer is written
to flush L2 (the r = 128 working set would otherwise stay in the 129 MB L2);
each step is timed with CUDA events on the stream its kernels run on.

The JSON line also carries:
  e2e        the same solve through the host-buffer entry point dpsr_solve_host:
             inputs copied from pinned host memory and results copied back
             inside the timed region (copies overlapped with the kernels);
  roofline   the dominant kernel's algorithmic bytes per launch over its
             average event-timed duration, against the measured HBM copy peak;
  r256       the r = 256 solve (100 000 points, torus + 2 ellipsoids): solves/s
             and the fraction of the HBM roofline for the whole-solve byte
             model 23 r^3 * 4 B + 200 N B;
  cpu_baseline  the FP64 oracle on this host's cores on a bounded sample.

--impl reference times the FP64 oracle (the only reference there is: the
paper ships no code) on the same workload, one solve per step.
Multi-GPU (torchrun): replicas only, each rank solves its own copy of the
workload; value = solves of all ranks / max time over ranks.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "DPSR fwd+bwd solves/s at r=128/256 (% HBM roofline); served p50/p99 ms vs per-solve loop"
WORKLOAD = "r128: plain DPSR fwd+bwd, r=128, sigma=2, N=20000 on a union of 4 random ellipsoids"


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons while running."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-f", self.path], stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        if self.proc is None:
            return out
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        try:
            rows = [ln.split(",") for ln in open(self.path).read().strip().splitlines() if ln.strip()]
            os.unlink(self.path)
        except Exception:
            return out
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        sm, mx, reasons = [], [], set()
        for r in rows:
            r = [x.strip() for x in r]
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except ValueError:
                continue
            for i, n in enumerate(names):
                if r[5 + i].lower().startswith("active"):
                    reasons.add(n)
        if sm:
            out.update(sm_mhz=statistics.median(sm), sm_max_mhz=max(mx), reasons=sorted(reasons),
                       samples=len(sm))
        return out


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import datetime

        import torch.distributed as dist
        # a rank that dies ends the others' next collective with an error
        # instead of a hang: gloo sees the closed connection, and at worst the
        # group's timeout (DPSR_PG_TIMEOUT_S, default 300 s) expires
        timeout = datetime.timedelta(seconds=float(os.environ.get("DPSR_PG_TIMEOUT_S", "300")))
        dist.init_process_group("gloo", timeout=timeout)
        return dist, rank, ws, local
    return None, rank, ws, local


def _max_over_ranks(dist, x: float) -> float:
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _barrier(dist):
    if dist is not None:
        dist.barrier()


# ----------------------------------------------------------------------------
# algorithmic byte model (per launch / per solve): the bytes each plane kind
# must move at least, whichever path (cluster or pencil) runs it
# ----------------------------------------------------------------------------
def kernel_bytes(r: int, N: int):
    U = 4 * r ** 3                      # one FP32 real grid
    H = 8 * r * r * (r // 2 + 1)        # one complex half spectrum
    rec = 32                            # sorted point record
    return {
        "plane_fwd": 3 * H + 2 * rec * N,
        "xpass_fwd": 4 * H,
        "plane_inv": H + U + 2 * (rec + 16) * N,
        "plane_bfwd": 2 * U + H,
        "xpass_bwd": 4 * H,
        "plane_binv": 2 * H + 2 * (rec + 24) * N,
        "bin": 2 * 24 * N + 4 * N + (rec + 4) * N,
        "combine": (32 * 2 + 16 * 2 + 8 + 24) * N,
    }


# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) of a
# plane kind's kernel at (grid size, plane path), from one ncu capture of the
# current build on the same workload (profiles/traffic_r128_kinds.md);
# a kind, size or path not listed reports traffic as null.
MEASURED_TRAFFIC = {
    # k_zfwd<128> + k_yfwd<128, 0> (the pencil forward plane kind), r = 128 ellipsoids, N = 20000
    ("plane_fwd", 128, 0): 682240 + 37711872,
    ("plane_binv", 128, 1): 21772288,   # k_plane_binv<128, 1> (512 threads), same workload
    ("plane_binv", 128, 3): 21667072,   # k_plane_binv_ch<128> (one CTA per plane and channel)
}


def solve_bytes_model(r: int, N: int) -> float:
    """Whole fwd+bwd solve: 23 one-grid units plus ~200 B per point."""
    return 23 * 4 * r ** 3 + 200 * N


def run_gpu(args):
    import numpy as np
    import torch

    from paper_2106_03452_gb300 import libdpsr as L
    from paper_2106_03452_gb300 import synth
    from paper_2106_03452_gb300.dpsr import Plan

    dist, rank, ws, local = _dist()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    hbm_peak, peak_kind = _peaks()
    flush = torch.empty(512 * 2 ** 20 // 4, dtype=torch.float32, device=dev)

    def timed(step, K, W, flush_l2=True):
        for _ in range(W):
            step()
        torch.cuda.synchronize()
        _barrier(dist)
        torch.cuda.synchronize()
        evs = []
        t0 = time.perf_counter()
        for _ in range(K):
            if flush_l2:
                flush.fill_(1.0)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            step()
            b.record()
            evs.append((a, b))
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        ms = sum(a.elapsed_time(b) for a, b in evs)
        _barrier(dist)
        return ms, wall

    # ---------------- headline: r = 128 ----------------
    w = synth.workload_ellipsoids_r128()
    r, N = w["r"], w["points"].shape[0]
    plan = Plan(r, w["sigma"], device=dev, n_max=N)
    P = torch.from_numpy(w["points"]).to(dev)
    Nn = torch.from_numpy(w["normals"]).to(dev)
    G = torch.from_numpy(w["dchi"]).to(dev)
    chi = torch.empty((r, r, r), device=dev)
    dp, dn = torch.empty_like(P), torch.empty_like(P)

    def step():
        plan.forward(P, Nn, chi)
        plan.backward(G, dp, dn)

    plan.forward(P, Nn, chi)
    per_step = plan.last_launches()
    plan.backward(G, dp, dn)
    per_step += plan.last_launches()
    st = plan.sync()
    if st != 0:
        raise RuntimeError(f"device status {st}: {L.dpsr_strerror(st)}")
    clocks = Clocks(local)
    clocks.start()
    ms, wall = timed(step, args.steps, args.warmup)
    clk = clocks.stop()
    ms_max = _max_over_ranks(dist, ms)
    value = ws * args.steps / (ms_max / 1e3)
    launches = args.steps * per_step

    # per-kernel profile of the same step (events around every launch)
    L.dpsr_plan_profile(plan.handle, True)
    for _ in range(args.steps):
        flush.fill_(1.0)
        step()
    prof = L.dpsr_plan_profile_read(plan.handle)
    L.dpsr_plan_profile(plan.handle, False)
    kb = kernel_bytes(r, N)
    per = {k: {"ms": v[0] / max(v[1], 1), "launches": v[1], "bytes": kb.get(k)} for k, v in prof.items() if v[1]}
    dom = max((k for k in per if per[k]["bytes"]), key=lambda k: per[k]["ms"] * per[k]["launches"])
    ach = per[dom]["bytes"] / (per[dom]["ms"] / 1e3) / 1e9
    kind_index = {"plane_fwd": 0, "plane_inv": 1, "plane_bfwd": 2, "plane_binv": 3}
    paths = L.dpsr_plan_clusters(plan.handle)
    traffic = None
    if dom in kind_index:
        traffic = MEASURED_TRAFFIC.get((dom, r, paths[kind_index[dom]]))

    # ---------------- e2e through the host-buffer entry points ----------------
    hp = torch.from_numpy(w["points"]).pin_memory()
    hn = torch.from_numpy(w["normals"]).pin_memory()
    hg = torch.from_numpy(w["dchi"]).pin_memory()
    hchi = torch.empty((r, r, r)).pin_memory()
    hdp, hdn = torch.empty_like(hp).pin_memory(), torch.empty_like(hp).pin_memory()
    plan_h = Plan(r, w["sigma"], device=dev, n_max=N)
    L.dpsr_plan_set_stream(plan_h.handle, torch.cuda.current_stream(dev).cuda_stream)

    def step_e2e():
        # one call: inputs up, forward, backward, results down (the gradient's upload and
        # chi's download overlap the kernels on a second stream)
        L.dpsr_solve_host(plan_h.handle, hp.data_ptr(), hn.data_ptr(), N, hg.data_ptr(), hchi.data_ptr(),
                          hdp.data_ptr(), hdn.data_ptr())

    ms_e2e, _ = timed(step_e2e, args.steps, args.warmup)
    e2e_value = ws * args.steps / (_max_over_ranks(dist, ms_e2e) / 1e3)
    h2d = 2 * 12 * N + 4 * r ** 3
    d2h = 4 * r ** 3 + 2 * 12 * N

    # ---------------- the same workload in an anisotropic box ----------------
    # the ellipsoid cloud stretched into the periodic box (1, 0.75, 1.5): voxel
    # size L_d / 128 per axis (dpsr_plan_create_box), same kernels and bytes
    box_dims = (1.0, 0.75, 1.5)
    bx = torch.tensor(box_dims, device=dev)
    Pb = (P * bx).contiguous()
    Nb = Nn / bx
    Nb = (Nb / Nb.norm(dim=1, keepdim=True).clamp_min(1e-30)).contiguous()
    plan_b = Plan(r, w["sigma"], device=dev, n_max=N, box=box_dims)
    chib, dpb, dnb = torch.empty_like(chi), torch.empty_like(P), torch.empty_like(P)

    def step_box():
        plan_b.forward(Pb, Nb, chib)
        plan_b.backward(G, dpb, dnb)

    step_box()
    if plan_b.sync() != 0:
        raise RuntimeError("box device status")
    ms_box, _ = timed(step_box, args.steps, args.warmup)
    ms_box = _max_over_ranks(dist, ms_box)
    box_block = {"workload": "r128 workload stretched into the periodic box (1, 0.75, 1.5), fwd+bwd",
                 "box": list(box_dims), "solves_per_s": ws * args.steps / (ms_box / 1e3),
                 "ms_per_step": ms_box / args.steps, "vs_cube": ms_max / ms_box,
                 "paths": L.dpsr_plan_clusters(plan_b.handle)}
    plan_b.close()

    # ---------------- r = 256 ----------------
    r256 = None
    if not args.no_r256:
        w3 = synth.workload_torus_r256()
        r3, N3 = w3["r"], w3["points"].shape[0]
        plan3 = Plan(r3, w3["sigma"], device=dev, n_max=N3)
        P3 = torch.from_numpy(w3["points"]).to(dev)
        N3t = torch.from_numpy(w3["normals"]).to(dev)
        G3 = torch.randn((r3,) * 3, device=dev, generator=torch.Generator(device=dev).manual_seed(3))
        chi3 = torch.empty((r3,) * 3, device=dev)
        dp3, dn3 = torch.empty_like(P3), torch.empty_like(P3)

        def step3():
            plan3.forward(P3, N3t, chi3)
            plan3.backward(G3, dp3, dn3)

        step3()
        if plan3.sync() != 0:
            raise RuntimeError("r256 device status")
        k3 = max(3, args.steps // 2)
        ms3, _ = timed(step3, k3, args.warmup)
        ms3 = _max_over_ranks(dist, ms3)
        t3 = ms3 / k3 / 1e3
        bytes3 = solve_bytes_model(r3, N3)
        L.dpsr_plan_profile(plan3.handle, True)
        for _ in range(k3):
            flush.fill_(1.0)
            step3()
        prof3 = L.dpsr_plan_profile_read(plan3.handle)
        L.dpsr_plan_profile(plan3.handle, False)
        kb3 = kernel_bytes(r3, N3)
        per3 = {k: {"ms": v[0] / max(v[1], 1), "launches": v[1], "bytes": kb3.get(k),
                    "gbs": (kb3[k] / (v[0] / max(v[1], 1) / 1e3) / 1e9) if kb3.get(k) and v[0] > 0 else None}
                for k, v in prof3.items() if v[1]}
        r256 = {"workload": "r256: torus (R=0.25, tube 0.08) + 2 ellipsoids, N=100000, sigma=2, fwd+bwd",
                "solves_per_s": ws * k3 / (ms3 / 1e3), "ms_per_step": t3 * 1e3,
                "model_bytes_per_solve": bytes3,
                "roofline_frac_of_model": bytes3 / t3 / 1e9 / hbm_peak,
                "kernels": per3,
                # autotuned plane paths (0 pencil, else cluster size) of the four
                # plane kinds; DPSR_PLANE_PATHS_256 pins them for a profiler run
                "paths": L.dpsr_plan_clusters(plan3.handle)}
        # the differentiable loop of this workload: 50 Adam steps of
        # L = mean chi(q)^2 over its 200 000 clean targets through the adjoint
        if not args.no_loop:
            from paper_2106_03452_gb300.loop import optimize
            Q3 = torch.from_numpy(w3["targets"]).to(dev)
            hist, _, _, s_step = optimize(P3, N3t, Q3, r=r3, sigma=w3["sigma"], steps=50, plan=plan3)
            r256["loop"] = {"workload": "50 Adam steps of mean chi(q)^2 over 200000 targets, lr 2e-3 * 0.7^3",
                            "s_per_step": s_step, "loss_first": hist[0], "loss_last": hist[-1]}
        plan3.close()

    # ---------------- batched: 32 clouds, r in {64, 128} ----------------
    batched = None
    if not args.no_batch:
        batched = bench_batched(args, dev, dist, ws, timed)

    # ---------------- L_DPSR training step (Eq. 9) at 128^3 ----------------
    train = None
    if not args.no_train:
        train = bench_train(args, dev, dist, ws, timed)

    # ---------------- optimisation setting: the paper's full schedule ----------------
    optim = None
    if not args.no_optimize:
        optim = bench_optimize(dev)

    # ---------------- L2 read bandwidth (the ceiling of the L2-resident r = 128 solve) ----
    l2 = measure_l2_read(dev)
    # FP32 FMA throughput (the FFT butterflies' pipe), measured by the library's own kernel
    fma_tflops = L.dpsr_fp32_fma_peak(1 << 16) / 1e12
    l2_ach = per[dom]["bytes"] / (per[dom]["ms"] / 1e3) / 1e9
    solve_gbs = solve_bytes_model(r, N) / (ms_max / args.steps / 1e3) / 1e9

    # ---------------- context: the same layer in plain PyTorch ops ----------------
    torch_ctx = None
    if not args.no_torch_context and rank == 0:
        torch_ctx = torch_ops_context(dev)

    # ---------------- serving: Poisson arrivals at 200 req/s ----------------
    serving = None
    if not args.no_serve and rank == 0:
        serving = bench_serving(args)

    # ---------------- CPU baseline: the oracle ----------------
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = oracle_baseline(w, budget_s=args.cpu_budget)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "r": r, "N": N, "sigma": w["sigma"],
                       "global_batch": ws, "parallelism": f"replicas{ws}",
                       "l2": "flushed between timed steps (512 MiB write)"},
            "gpu_launches": launches,
            "e2e": {"value": e2e_value, "unit": "solves/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            "roofline": {"bound": "hbm", "achieved": ach, "peak": hbm_peak, "unit": "GB/s",
                         "frac": ach / hbm_peak, "traffic": traffic, "kernel": dom,
                         "peak_kind": peak_kind,
                         "bytes_per_launch": per[dom]["bytes"], "ms_per_launch": per[dom]["ms"],
                         # the r = 128 working set stays in L2: the same bytes against the
                         # L2 copy bandwidth measured here, and the whole solve's byte model
                         "l2": {"achieved": l2_ach, "peak": l2, "unit": "GB/s",
                                "frac": l2_ach / l2 if l2 else None,
                                "peak_kind": "measured in this run: L2 read bandwidth, 64 reads of a 24 MiB buffer in one kernel"},
                         "fp32": {"fma_tflops_measured": fma_tflops,
                                  "nominal_tflops": 152 * 128 * 2 * 2.07e9 / 1e12,
                                  "how": "8 independent FMA chains per thread, 8 x 256-thread CTAs per SM"},
                         "solve": {"model_bytes": solve_bytes_model(r, N), "achieved": solve_gbs,
                                   "frac_hbm": solve_gbs / hbm_peak,
                                   "frac_l2": solve_gbs / l2 if l2 else None}},
            "kernels": per,
            "paths": L.dpsr_plan_clusters(plan.handle),  # see r256["paths"]
            "clocks": clk,
            "r256": r256,
            "box": box_block,
            "batched": batched,
            "train": train,
            "optimize": optim,
            "torch_ops_context": torch_ctx,
            "serving": serving,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    plan.close()
    plan_h.close()
    if dist is not None:
        dist.destroy_process_group()


def bench_optimize(dev):
    """The optimisation setting (Sec. 3.2; supplementary Sec. B) with the
    paper's schedule: from a sphere of 20000 oriented points to an unoriented
    cloud of 20000 points on a torus (R = 0.25, tube 0.08: one connected
    object of genus one, as the resampling from the largest mesh component
    assumes of its input); 32^3, 64^3, 128^3
    (1000 iterations each) and 256^3 (200), sigma 2, 2, 3, 3, Adam at 2e-3
    decayed by 0.7 per level, 20000 mesh samples per Chamfer evaluation,
    resampling every 200 iterations. Wall-clock seconds for the object."""
    import torch

    from paper_2106_03452_gb300 import synth
    from paper_2106_03452_gb300.optimize import PAPER_LEVELS, reconstruct
    tgt, _ = synth.union_cloud(synth.Rng(3003), [synth.Torus()], 20000, 0.0)
    T = torch.from_numpy(tgt).to(dev)
    reconstruct(T, levels=((32, 2.0, 20),), n_points=20000, samples=20000)  # warm-up (tuners, allocations)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    _, _, hist = reconstruct(T, levels=PAPER_LEVELS, n_points=20000, samples=20000, resample=200, seed=1)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    return {"workload": "coarse-to-fine optimisation from a sphere to 20000 points on a torus: "
                        "32/64/128/256^3 for 1000/1000/1000/200 iterations, 20000 points and samples",
            "seconds_per_object": wall,
            "levels": [{"r": h[0], "sigma": h[1], "iterations": h[2], "chamfer_first": h[3],
                        "chamfer_last": h[4], "seconds": h[5]} for h in hist]}


def measure_l2_read(dev) -> float | None:
    """L2 read bandwidth: one reduction kernel reads a 24 MiB buffer 64 times
    over (a stride-0 expanded view, 1.5 GiB of reads in one launch), so every
    read after the first pass hits L2; best of 10 after warm-up."""
    import torch
    try:
        a = torch.ones(24 * 2 ** 20 // 4, device=dev)
        K = 64
        v = a.expand(K, a.numel())
        for _ in range(3):
            v.sum(1)
        best = 1e30
        for _ in range(10):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            v.sum(1)
            e1.record()
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1))
        return K * a.numel() * 4 / (best / 1e3) / 1e9
    except Exception:
        return None


def bench_train(args, dev, dist, ws, timed):
    """The L_DPSR training step of the learning setting (Sec. 3.3, Eq. 9;
    supplementary Sec. B) at 128^3: 8 instances (the paper trains with batch
    32 on two GPUs), each a predicted cloud of 3000 x 7 = 21 000 points
    against a ground-truth grid solved once from a 100 000-point sampling.
    One step = forward, fused loss and gradient, backward of every instance,
    as one CUDA graph launch; against a per-solve loop (forward, loss,
    backward per instance) of the same kernels."""
    import torch

    from paper_2106_03452_gb300 import synth
    from paper_2106_03452_gb300.dpsr import Batch, Plan
    r, sigma, count = 128, 2.0, 8
    gtb = Batch([r] * count, [sigma] * count, [100000] * count, device=dev)
    data, gts = [], []
    for i in range(count):
        rng = synth.Rng(2000 + i)
        gp, gn = synth.ellipsoid_cloud(rng, 100000, 1 + i % 4, jitter=0.0)
        pp, pn = synth.ellipsoid_cloud(rng, 21000, 1 + (i + 1) % 4, jitter=0.005)
        g = torch.empty((r, r, r), device=dev)
        gtb.bind(i, torch.from_numpy(gp).to(dev), torch.from_numpy(gn).to(dev), g)
        gts.append(g)
        data.append((torch.from_numpy(pp).to(dev), torch.from_numpy(pn).to(dev)))
    gtb.run(with_bwd=False, graph=False)
    if gtb.sync() != 0:
        raise RuntimeError("ground-truth batch device status")
    b = Batch([r] * count, [sigma] * count, [21000] * count, device=dev)
    T = []
    for i, (P, Nn) in enumerate(data):
        chi, dchi = torch.empty((r, r, r), device=dev), torch.empty((r, r, r), device=dev)
        dp, dn = torch.empty_like(P), torch.empty_like(P)
        b.bind(i, P, Nn, chi, dchi, dp, dn)
        b.bind_target(i, gts[i])
        T.append((P, Nn, chi, dchi, dp, dn))
    plans = [Plan(r, sigma, device=dev, n_max=21000) for _ in range(count)]

    def step_batch():
        b.train_step()

    def step_loop():
        for p, (P, Nn, chi, dchi, dp, dn), g in zip(plans, T, gts):
            p.forward(P, Nn, chi)
            p.mse_grad(g, dchi)
            p.backward(dchi, dp, dn)

    step_batch()
    if b.sync() != 0:
        raise RuntimeError("train batch device status")
    k = max(5, args.steps)
    ms_b, _ = timed(step_batch, k, args.warmup, flush_l2=False)
    ms_l, _ = timed(step_loop, k, args.warmup, flush_l2=False)
    ms_b, ms_l = _max_over_ranks(dist, ms_b), _max_over_ranks(dist, ms_l)
    losses = b.losses()
    out = {"workload": "L_DPSR training step, r=128, sigma=2: 8 predicted clouds of 21000 points (unions of "
                       "1-4 ellipsoids) against ground-truth grids solved from 100000-point samplings",
           "steps_per_s": ws * k / (ms_b / 1e3), "ms_per_step": ms_b / k,
           "solves_per_s": ws * count * k / (ms_b / 1e3),
           "loop_ms_per_step": ms_l / k, "speedup_vs_loop": ms_l / ms_b,
           "loss_mean": sum(losses) / len(losses), "paths": b.paths(r)}
    b.close()
    gtb.close()
    for p in plans:
        p.close()
    return out


def bench_batched(args, dev, dist, ws, timed):
    """Config 4: 32 clouds (unions of 1-6 ellipsoids, N log-uniform in
    [1000, 50000], r in {64, 128}), fwd+bwd. The batch (one CUDA graph launch
    per step) against a per-solve launch loop of the same kernels on the same
    GPU (one plan per cloud, called one after the other on one stream). The
    32 working sets (about 0.7 GB) exceed L2, so no flush is needed."""
    import torch

    from paper_2106_03452_gb300 import synth
    from paper_2106_03452_gb300.dpsr import Batch, Plan
    inst = synth.workload_batch(count=32)
    tens = []
    for w in inst:
        r = w["r"]
        P = torch.from_numpy(w["points"]).to(dev)
        Nn = torch.from_numpy(w["normals"]).to(dev)
        G = torch.from_numpy(w["dchi"]).to(dev)
        tens.append((P, Nn, G, torch.empty((r, r, r), device=dev), torch.empty_like(P), torch.empty_like(P)))
    batch = Batch([w["r"] for w in inst], [w["sigma"] for w in inst], [w["points"].shape[0] for w in inst],
                  device=dev)
    for i, t in enumerate(tens):
        batch.bind(i, *t)
    plans = [Plan(w["r"], w["sigma"], device=dev, n_max=w["points"].shape[0]) for w in inst]

    def step_batch():
        batch.run(with_bwd=True, graph=True)

    def step_loop():
        for p, (P, Nn, G, chi, dp, dn) in zip(plans, tens):
            p.forward(P, Nn, chi)
            p.backward(G, dp, dn)

    P0, Nn0, G0, chi0, dp0, dn0 = tens[0]
    plans[0].forward(P0, Nn0, chi0)
    loop_launches = plans[0].last_launches()
    plans[0].backward(G0, dp0, dn0)
    loop_launches += plans[0].last_launches()
    step_batch()
    if batch.sync() != 0:
        raise RuntimeError("batch device status")
    k = max(5, args.steps)
    ms_b, _ = timed(step_batch, k, args.warmup, flush_l2=False)
    ms_l, _ = timed(step_loop, k, args.warmup, flush_l2=False)
    ms_b, ms_l = _max_over_ranks(dist, ms_b), _max_over_ranks(dist, ms_l)
    out = {"workload": "32 clouds, unions of 1-6 ellipsoids, N log-uniform [1000, 50000], r in {64,128}, "
                       "sigma=2, fwd+bwd",
           "solves_per_s": ws * 32 * k / (ms_b / 1e3), "ms_per_batch": ms_b / k,
           "loop_solves_per_s": ws * 32 * k / (ms_l / 1e3), "loop_ms_per_batch": ms_l / k,
           "speedup_vs_loop": ms_l / ms_b, "launches_per_batch": batch.launches(True),
           "loop_launches_per_batch": 32 * loop_launches,
           "paths": {str(r): batch.paths(r) for r in sorted({w["r"] for w in inst})}}
    batch.close()
    for p in plans:
        p.close()
    return out


def bench_serving(args):
    """Config 5: Poisson arrivals at 200 req/s, each an ellipsoid-union cloud
    with N log-uniform in [1000, 200000], r in {64, 128, 256} (0.5 / 0.35 /
    0.15), 30% forward + backward, admitted by an 8 GB device budget. The
    continuous-batching server (--serve-slots stream slots) against a per-solve loop (the
    same server with one slot and no coalescing), saturated (the first 400
    requests submitted at once, best of three bursts) for throughput, then replayed in real time
    (latency = completion - arrival): the served configuration over the whole
    trace (60 s, about 12 000 requests), the loop over its first 15 s."""
    from paper_2106_03452_gb300 import serve, synth
    trace = synth.serving_trace(duration_s=args.serve_seconds)
    loop_trace = [q for q in trace if q["t"] < args.serve_loop_seconds]
    pool = serve.InputPool(n_clouds=6, n_max=200000)
    keys = [(r, b) for r in (64, 128, 256) for b in (False, True)]
    out = {"rate_per_s": 200.0, "duration_s": args.serve_seconds, "requests": len(trace),
           "budget_bytes": 8 << 30}
    out["slots"] = args.serve_slots
    ring = serve.OutputRing()  # pinned output buffers, shared by both servers
    ring.prefill(keys, args.serve_slots * 8 + 2, 200000)
    # the served configuration coalesces same-size requests (grid <= 128) into
    # batched launches of up to 8; the loop is one slot, one solve at a time
    configs = ((args.serve_slots, "served", 8), (1, "loop", 1))
    servers = {}
    for slots, label, group in configs:
        servers[label] = serve.Server(8 << 30, slots, max_group=group)
        serve.warm(servers[label], pool, slots=slots, n=200000)
    # both saturation runs before either real-time replay: the replay's
    # scattered buffer traffic measurably slows a burst that follows it in
    # the same process
    # three bursts per configuration, alternating, best of three: the
    # serving path runs on the host cores (submission, completion polling,
    # the server thread), which other jobs on a shared machine disturb
    sat = trace[:400]
    sat_runs = {label: [] for _, label, _ in configs}
    for _rep in range(3):
        for slots, label, _ in configs:
            t0 = time.perf_counter()
            serve.replay(sat, servers[label], pool, realtime=False, ring=ring)
            sat_runs[label].append(len(sat) / (time.perf_counter() - t0))
    sat_rate = {label: max(v) for label, v in sat_runs.items()}
    for slots, label, group in configs:
        srv = servers[label]
        g0 = srv.stats()
        t0 = time.perf_counter()
        res = serve.replay(trace if label == "served" else loop_trace, srv, pool, realtime=True, ring=ring)
        wall = time.perf_counter() - t0
        st = srv.stats()
        out[label] = serve.summarize(res, wall)
        out[label]["saturated_solves_per_s"] = sat_rate[label]
        out[label]["saturated_runs"] = sat_runs[label]
        out[label]["max_in_flight"] = st["max_in_flight"]
        out[label]["max_group"] = group
        out[label]["coalesced_requests"] = st["grouped_requests"] - g0["grouped_requests"]
        srv.close()
    out["saturated_speedup_vs_loop"] = out["served"]["saturated_solves_per_s"] / out["loop"]["saturated_solves_per_s"]
    return out


def torch_ops_dpsr(points, normals, r: int, sigma: float):
    """Context baseline only (never a product path): the DPSR layer written
    with plain PyTorch GPU ops from Sec. 3.1 (Eq. A1-A2 splat by index_add,
    Eq. A3 torch.fft.rfftn, the solve of Eq. 3, Eq. A8 irfftn, Eq. 4
    normalisation with a trilinear gather), differentiated by autograd. The
    readings are the library's: periodic unit cube, integer frequencies, DC
    zero, the a-th term zero at a Nyquist index with |u_a| = r/2 there, the
    shifted scale s = chi'(0) - mu."""
    import math

    import torch
    dev = points.device
    x = points * r
    fl = torch.floor(x)
    t = x - fl
    i0 = fl.long() % r
    i1 = (i0 + 1) % r
    corners = []
    for d in range(8):
        dx, dy, dz = d >> 2, (d >> 1) & 1, d & 1
        w = ((t[:, 0] if dx else 1 - t[:, 0]) * (t[:, 1] if dy else 1 - t[:, 1]) *
             (t[:, 2] if dz else 1 - t[:, 2]))
        idx = ((i1[:, 0] if dx else i0[:, 0]) * r + (i1[:, 1] if dy else i0[:, 1])) * r + \
              (i1[:, 2] if dz else i0[:, 2])
        corners.append((w, idx))
    V = torch.zeros(3, r ** 3, device=dev, dtype=points.dtype)
    for w, idx in corners:
        V = V.index_add(1, idx, (w[:, None] * normals).t())
    Vh = torch.fft.rfftn(V.view(3, r, r, r), dim=(1, 2, 3))
    k = torch.arange(r, device=dev)
    f = torch.where(k < r // 2, k, k - r).float()
    fa = torch.where(k == r // 2, torch.full_like(f, r // 2), f)     # |u| at Nyquist
    kz = torch.arange(r // 2 + 1, device=dev)
    fz = kz.float()
    U = [f.view(r, 1, 1), f.view(1, r, 1), torch.where(kz == r // 2, torch.zeros_like(fz), fz).view(1, 1, -1)]
    A = [fa.view(r, 1, 1), fa.view(1, r, 1), fz.view(1, 1, -1)]
    U[0] = torch.where((k == r // 2).view(r, 1, 1), torch.zeros_like(U[0]), U[0])
    U[1] = torch.where((k == r // 2).view(1, r, 1), torch.zeros_like(U[1]), U[1])
    u2 = A[0] ** 2 + A[1] ** 2 + A[2] ** 2
    g = torch.exp(-2.0 * sigma ** 2 * u2 / r ** 2)
    div = U[0] * Vh[0] + U[1] * Vh[1] + U[2] * Vh[2]
    H = g / (-2.0 * math.pi * torch.where(u2 > 0, u2, torch.ones_like(u2)))
    H = torch.where(u2 > 0, H, torch.zeros_like(H))
    chih = 1j * div * H
    chip = torch.fft.irfftn(chih, s=(r, r, r), dim=(0, 1, 2))
    flat = chip.reshape(-1)
    mu = sum(w * flat[idx] for w, idx in corners).mean()
    s = flat[0] - mu
    return 0.5 / s.abs() * (chip - mu)


def torch_ops_context(dev, steps=10, warmup=3):
    """Fwd+bwd solves/s of torch_ops_dpsr on this GPU at the r = 128 and
    r = 256 workloads (L2 flushed between steps, CUDA events)."""
    import torch

    from paper_2106_03452_gb300 import synth
    out = {"what": "the DPSR layer in plain PyTorch ops (cuFFT rfftn/irfftn, index_add splat, "
                   "autograd backward): context, not a product path"}
    flush = torch.empty(512 * 2 ** 20 // 4, dtype=torch.float32, device=dev)
    for name, w in (("r128", synth.workload_ellipsoids_r128()), ("r256", synth.workload_torus_r256())):
        r, sigma = w["r"], w["sigma"]
        P = torch.from_numpy(w["points"]).to(dev).requires_grad_(True)
        Nn = torch.from_numpy(w["normals"]).to(dev).requires_grad_(True)
        G = torch.randn((r,) * 3, device=dev)

        def step():
            chi = torch_ops_dpsr(P, Nn, r, sigma)
            dp, dn = torch.autograd.grad((chi * G).sum(), (P, Nn))
            return dp, dn

        def timed_ms(fn):
            for _ in range(warmup):
                fn()
            torch.cuda.synchronize()
            ms = 0.0
            for _ in range(steps):
                flush.fill_(1.0)
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record()
                fn()
                b.record()
                torch.cuda.synchronize()
                ms += a.elapsed_time(b)
            return ms / steps

        res = {}
        ms = timed_ms(step)
        res["eager"] = {"solves_per_s": 1e3 / ms, "ms_per_step": ms}
        # the same step captured as one CUDA graph (removes the per-op launch cost)
        try:
            side = torch.cuda.Stream(dev)
            side.wait_stream(torch.cuda.current_stream(dev))
            with torch.cuda.stream(side):
                for _ in range(warmup):
                    step()
            torch.cuda.current_stream(dev).wait_stream(side)
            graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(graph):
                step()
            ms = timed_ms(graph.replay)
            res["graph"] = {"solves_per_s": 1e3 / ms, "ms_per_step": ms}
        except Exception as exc:  # the context number is optional: say why it is missing
            res["graph"] = {"unavailable": f"{type(exc).__name__}: {exc}"[:200]}
        out[name] = res
    return out


def oracle_baseline(w, budget_s=12.0):
    """The FP64 oracle as it stands, forward + backward, on this host's cores:
    repeats whole solves of the workload until budget_s has passed."""
    import oracle
    oracle.build()
    r, sigma = w["r"], w["sigma"]
    n = 0
    t0 = time.perf_counter()
    while True:
        oracle.forward(r, sigma, w["points"], w["normals"])
        oracle.backward(r, sigma, w["points"], w["normals"], w["dchi"])
        n += 1
        if time.perf_counter() - t0 >= budget_s:
            break
    dt = time.perf_counter() - t0
    out = {"value": n / dt, "unit": "solves/s", "cores": oracle.threads(), "kind": "oracle",
           "sample": f"{n} whole fwd+bwd solves of the r=128 workload (FP64, OpenMP over FFT pencils)"}
    # the same on one core (a shorter sample: at least one whole solve)
    all_cores = oracle.threads()
    oracle.set_threads(1)
    n1 = 0
    t0 = time.perf_counter()
    while True:
        oracle.forward(r, sigma, w["points"], w["normals"])
        oracle.backward(r, sigma, w["points"], w["normals"], w["dchi"])
        n1 += 1
        if time.perf_counter() - t0 >= budget_s / 2:
            break
    dt1 = time.perf_counter() - t0
    oracle.set_threads(all_cores)
    out["single_thread"] = {"value": n1 / dt1, "unit": "solves/s", "cores": 1,
                            "sample": f"{n1} whole fwd+bwd solves of the r=128 workload on one thread"}
    return out


def run_reference(args):
    """Reference arm: the FP64 oracle, one whole r=128 solve per step."""
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    from paper_2106_03452_gb300 import synth
    oracle.build()
    w = synth.workload_ellipsoids_r128()
    r, sigma = w["r"], w["sigma"]

    def step():
        oracle.forward(r, sigma, w["points"], w["normals"])
        oracle.backward(r, sigma, w["points"], w["normals"], w["dchi"])

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = time.perf_counter() - t0
    v = args.steps / dt
    line = {
        "metric": METRIC, "value": v, "unit": "solves/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
        "config": {"workload": WORKLOAD, "r": r, "N": int(w["points"].shape[0]), "sigma": sigma,
                   "global_batch": 1, "parallelism": "cpu"},
        "cpu_baseline": {"value": v, "unit": "solves/s", "cores": oracle.threads(), "kind": "oracle",
                         "sample": f"{args.steps} whole fwd+bwd solves of the r=128 workload"},
        "e2e": {"value": v, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--no-r256", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--no-train", action="store_true")
    ap.add_argument("--no-optimize", action="store_true")
    ap.add_argument("--no-loop", action="store_true")
    ap.add_argument("--no-torch-context", action="store_true")
    ap.add_argument("--serve-seconds", type=float, default=60.0)
    ap.add_argument("--serve-loop-seconds", type=float, default=15.0)
    ap.add_argument("--serve-slots", type=int, default=8)
    ap.add_argument("--cpu-budget", type=float, default=12.0)
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
