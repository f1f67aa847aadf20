"""Run a DPSR workload a few times (for ncu captures and quick timings).

    python -m paper_2106_03452_gb300.profile_case --r 256 --reps 3 [--fwd-only]

Workloads: r=32 sphere (N=3000), r=128 ellipsoids (N=20000), r=256 torus +
ellipsoids (N=100000), all sigma = 2. Prints the event-timed ms per solve and
the per-kernel profile of the library.
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
    ap.add_argument("--r", type=int, default=256, choices=[32, 128, 256])
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--fwd-only", action="store_true")
    a = ap.parse_args()
    w = {32: synth.workload_sphere_r32, 128: synth.workload_ellipsoids_r128,
         256: synth.workload_torus_r256}[a.r]()
    r = w["r"]
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


if __name__ == "__main__":
    main()
