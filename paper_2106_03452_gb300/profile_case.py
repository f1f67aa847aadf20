"""Run a DPSR workload a few times (for ncu captures and quick timings).

    python -m paper_2106_03452_gb300.profile_case --r 256 --reps 3 [--fwd-only]
    python -m paper_2106_03452_gb300.profile_case --batch --reps 3

Workloads: r=32 sphere (N=3000), r=128 ellipsoids (N=20000), r=256 torus +
ellipsoids (N=100000; --r 512 solves the same cloud on a 512^3 grid), all sigma = 2. Prints the event-timed ms per solve and
the per-kernel profile of the library. --batch runs the batched workload
instead (32 clouds, r in {64, 128}, fwd+bwd): one eager run (which tunes),
then --reps plain (not graph) runs, each launch visible to a profiler.
"""
import argparse
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))


def main():
    import torch

    from paper_2106_03452_gb300 import libdpsr as L
    from paper_2106_03452_gb300 import synth
    from paper_2106_03452_gb300.dpsr import Plan

    ap = argparse.ArgumentParser()
    ap.add_argument("--r", type=int, default=256, choices=[32, 128, 256, 512])
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--fwd-only", action="store_true")
    ap.add_argument("--batch", action="store_true")
    a = ap.parse_args()
    if a.batch:
        return run_batch(a.reps)
    w = {32: synth.workload_sphere_r32, 128: synth.workload_ellipsoids_r128,
         256: synth.workload_torus_r256, 512: synth.workload_torus_r256}[a.r]()
    r = a.r  # 512: the r = 256 torus workload (N = 100 000) on a 512^3 grid
    plan = Plan(r, w["sigma"], n_max=w["points"].shape[0])
    P = torch.from_numpy(w["points"]).cuda()
    Nn = torch.from_numpy(w["normals"]).cuda()
    G = torch.randn((r,) * 3, device="cuda")
    chi = torch.empty((r,) * 3, device="cuda")
    dp, dn = torch.empty_like(P), torch.empty_like(P)
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for _ in range(2):  # warm-up
        plan.forward(P, Nn, chi)
        if not a.fwd_only:
            plan.backward(G, dp, dn)
    torch.cuda.synchronize()
    L.dpsr_plan_profile(plan.handle, True)
    s.record()
    for _ in range(a.reps):
        plan.forward(P, Nn, chi)
        if not a.fwd_only:
            plan.backward(G, dp, dn)
    e.record()
    torch.cuda.synchronize()
    st = plan.sync()
    prof = L.dpsr_plan_profile_read(plan.handle)
    print(f"r={r} N={P.shape[0]} status={st} ms/solve={s.elapsed_time(e) / a.reps:.3f} "
          f"clusters={L.dpsr_plan_clusters(plan.handle)}")
    for k, (ms, n) in prof.items():
        if n:
            print(f"  {k:12s} {ms / n:8.4f} ms x {n}")
    if st != 0:
        sys.exit(1)


def run_batch(reps):
    import torch

    from paper_2106_03452_gb300 import synth
    from paper_2106_03452_gb300.dpsr import Batch

    inst = synth.workload_batch()
    dev = torch.device("cuda", torch.cuda.current_device())
    keep = []
    b = Batch([w["r"] for w in inst], [w["sigma"] for w in inst], [w["points"].shape[0] for w in inst],
              device=dev)
    for i, w in enumerate(inst):
        r = w["r"]
        P = torch.from_numpy(w["points"]).to(dev)
        t = (P, torch.from_numpy(w["normals"]).to(dev), torch.empty((r, r, r), device=dev),
             torch.from_numpy(w["dchi"]).to(dev), torch.empty_like(P), torch.empty_like(P))
        b.bind(i, *t)
        keep.append(t)
    b.run(with_bwd=True, graph=False)  # tunes the plane paths
    torch.cuda.synchronize()
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s.record(b.stream)
    for _ in range(reps):
        b.run(with_bwd=True, graph=False)
    e.record(b.stream)
    torch.cuda.synchronize()
    st = b.sync()
    print(f"batch of {len(inst)} status={st} ms/batch={s.elapsed_time(e) / reps:.3f} "
          f"launches={b.launches(True)} paths64={b.paths(64)} paths128={b.paths(128)}")
    if st != 0:
        sys.exit(1)


if __name__ == "__main__":
    main()
