"""Small programs for profiler captures of one kernel family at a time.

    python -m paper_2406_18356_gb300.profile_cases fista   # 3 FISTA passes, 1024 px, FP32
    python -m paper_2406_18356_gb300.profile_cases grid    # one degrid + grid pair, 9.27M rows

`fista`: the FP32 plan of the first 2,000,000 rows of the SKA-Mid-like
workload at 1024 px, the ALL partition's dirty image, and a `single` minor
cycle of 3 iterations (so each FISTA kernel's first launch is in the first
pass).  `grid`: the FP32 plan of all 9,266,880 rows, then one degridding and
one gridding call of the ALL partition.  Each prints "ok" at the end.
"""
from __future__ import annotations

import sys


def fista():
    import torch
    import synth
    import paper_2406_18356_gb300 as ms
    ms.load_library()
    w = synth.ska_mid_like(device="cuda", max_rows=2_000_000)
    plan = ms.Plan(w.u[0], w.v[0], 1024, w.pixel_size, w.ell_px, w.delta_px, precision="fp32")
    vis = torch.from_numpy(w.vis[0]).cuda().to(plan.complex_dtype)
    res = plan.grid("ALL", vis)
    lam = plan.lam(res, 0.01, 1)
    _, st = plan.minor_cycle("single", res, lam, 3)
    torch.cuda.synchronize()
    print("ok", st.iterations)


def grid():
    import torch
    import synth
    import paper_2406_18356_gb300 as ms
    ms.load_library()
    w = synth.ska_mid_like(device="cuda")
    plan = ms.Plan(w.u[0], w.v[0], 1024, w.pixel_size, w.ell_px, w.delta_px, precision="fp32")
    vis = torch.from_numpy(w.vis[0]).cuda().to(plan.complex_dtype)
    img = torch.randn(1024, 1024, device="cuda", dtype=plan.real_dtype)
    out = torch.empty_like(vis)
    plan.degrid("ALL", img, vis, out=out)
    plan.grid("ALL", out)
    torch.cuda.synchronize()
    print("ok")


def main():
    cases = {"fista": fista, "grid": grid}
    if len(sys.argv) != 2 or sys.argv[1] not in cases:
        raise SystemExit("usage: python -m paper_2406_18356_gb300.profile_cases fista|grid")
    cases[sys.argv[1]]()


if __name__ == "__main__":
    main()
