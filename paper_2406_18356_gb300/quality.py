"""Reconstruction quality on synthetic skies with a known truth (Sect. 5).

The paper measures, on its simulated data: the PSNR of the two-step image
for 3 x 3 partitionings (centre ell, half width delta; Table Partitionings
and the PSNR table of Sect. 5.1), the two-step method against the
single-step one, the number of major cycles until the image stops
improving, and the FISTA iterations of the first major cycle of each step
(Sect. 5.2).  This module runs the same study through the library on a
seeded sky whose truth image is known (``synth.paper_like``):

* partitions: ell at 0.117, 0.205, 0.322 of the longest baseline's radius
  (the paper's 20, 35, 55 px at 512 px) and delta = 1, 3, 5 px at 512 px,
  scaled with the image side; 5 + 5 major cycles of 100 FISTA iterations,
  lambda_n = 0.05 ||i~_n||_2 2^n (both steps), 0.01 for the single step;
* major cycles: the PSNR after n = 1 .. n_max cycles per step;
* FISTA: step one's, step two's and the single step's first minor cycle
  with a long budget; iterations until the objective is within 1e-2, 1e-3,
  1e-4 (relative) of the best it reached.

PSNR = 10 log10(max|truth|^2 / mean((image - truth)^2)), the image being
the method's final image (last residual plus the models).

    python -m paper_2406_18356_gb300.quality --npix 1024
prints one JSON object.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

ELL_FRACS = (0.117, 0.205, 0.322)
DELTAS_512 = (1.0, 3.0, 5.0)


def psnr(image: np.ndarray, truth: np.ndarray) -> float:
    mse = float(np.mean((np.asarray(image, np.float64) - truth) ** 2))
    return 10.0 * float(np.log10(float(np.max(np.abs(truth))) ** 2 / mse))


def partitions(npix: int):
    """The 3 x 3 (ell, delta) grid in pixel units of an npix image."""
    r_max = npix / 3.0
    return [(f * r_max, d * npix / 512.0) for f in ELL_FRACS for d in DELTAS_512]


def iterations_to(trace, eps: float) -> int:
    f = np.asarray(trace)
    best = float(np.min(f))
    hit = np.nonzero(f <= best + eps * abs(best))[0]
    return int(hit[0]) if hit.size else len(f)


def study(ms, w, precision: str = "fp32", n_major: int = 5, fista_iters: int = 100,
          n_major_max: int = 7, fista_budget: int = 2000, grid=None, convergence: bool = True,
          convolution: str = "circular", interleaved: bool = True, multi_step: bool = True):
    """Run the study on workload w (synth.Workload with a truth image) with
    the minor cycle's PSF operator `convolution` ("circular" or "linear");
    interleaved adds the interleaved two-image pipeline's images (Sect. 6's
    sketch, n_major cycles per node)."""
    import torch
    truth = w.truth
    tv = None
    out = {"workload": w.name, "npix": w.npix, "nvis": int(w.nvis), "precision": precision,
           "schedule": f"{n_major} x {fista_iters}", "convolution": convolution,
           "partitions": []}
    grid = grid if grid is not None else partitions(w.npix)
    opts = ms.ReconOptions(n_major=n_major, fista_iters=fista_iters)
    single_done = False
    for ell, delta in grid:
        plan = ms.Plan(w.u[0], w.v[0], w.npix, w.pixel_size, ell, delta, precision=precision,
                       convolution=convolution)
        if tv is None:
            tv = torch.from_numpy(w.vis[0]).cuda()
        vis = tv.to(plan.complex_dtype)
        c = plan.partition_counts()
        t0 = time.perf_counter()
        low, img, st = plan.reconstruct_two_step(vis, opts)
        torch.cuda.synchronize()
        rec = {"ell_px": ell, "delta_px": delta, "V_L": c["L"], "V_H": c["H"], "V_LH": c["LH"],
               "psnr_two_step": psnr(img.double().cpu().numpy(), truth),
               "psnr_low": psnr(low.double().cpu().numpy(), truth),
               "fista_iterations": st.total_iterations,
               "seconds": time.perf_counter() - t0}
        if interleaved:
            t1 = time.perf_counter()
            il, il_l, il_h, ist = plan.reconstruct_interleaved(vis, opts)
            torch.cuda.synchronize()
            rec["psnr_interleaved"] = psnr(il.double().cpu().numpy(), truth)
            rec["psnr_interleaved_node_l"] = psnr(il_l.double().cpu().numpy(), truth)
            rec["psnr_interleaved_node_h"] = psnr(il_h.double().cpu().numpy(), truth)
            rec["interleaved_seconds"] = time.perf_counter() - t1
        out["partitions"].append(rec)
        if not single_done:
            single, _ = plan.reconstruct_single_step(vis, opts)
            out["psnr_single_step"] = psnr(single.double().cpu().numpy(), truth)
            single_done = True
        plan.close()
    if multi_step:
        # three bands at the smallest and largest ell of the grid (delta of the
        # middle partition), Sect. 6's "more than 2-steps"
        from . import multistep
        ells = sorted({round(e, 6) for e, _ in grid})
        if len(ells) >= 2:
            ells3 = [ells[0], ells[-1]]
            d = grid[len(grid) // 2][1]
            t0 = time.perf_counter()
            imgs, _ = multistep.reconstruct_multi_step(
                ms, w.u[0], w.v[0], tv, w.npix, w.pixel_size, ells3, d, opts,
                precision=precision, convolution=convolution)
            out["multi_step"] = {"ell_px": ells3, "delta_px": d,
                                 "psnr_per_step": [psnr(i.double().cpu().numpy(), truth)
                                                   for i in imgs],
                                 "seconds": time.perf_counter() - t0}
    best = max(r["psnr_two_step"] for r in out["partitions"])
    for r in out["partitions"]:
        r["psnr_normalized"] = r["psnr_two_step"] / best
    if not convergence:
        return out
    # major cycles and FISTA iterations at the middle partition
    ell, delta = grid[len(grid) // 2]
    plan = ms.Plan(w.u[0], w.v[0], w.npix, w.pixel_size, ell, delta, precision=precision,
                   convolution=convolution)
    vis = tv.to(plan.complex_dtype)
    curve_two, curve_single = [], []
    for n in range(1, n_major_max + 1):
        o = ms.ReconOptions(n_major=n, fista_iters=fista_iters)
        _, img, _ = plan.reconstruct_two_step(vis, o)
        single, _ = plan.reconstruct_single_step(vis, o)
        curve_two.append(psnr(img.double().cpu().numpy(), truth))
        curve_single.append(psnr(single.double().cpu().numpy(), truth))
    out["major_cycles"] = {"ell_px": ell, "delta_px": delta, "psnr_two_step": curve_two,
                           "psnr_single_step": curve_single}
    low, _, _ = plan.reconstruct_two_step(vis, opts)
    res_l, res_h, res_a = plan.grid("L", vis), plan.grid("H", vis), plan.grid("ALL", vis)
    s2 = plan.sigma2_hat(res_h)
    fista = {}
    for name, step, res, coef, kw in (
            ("low", "low", res_l, 0.05, {}),
            ("full", "full", res_h, 0.05, {"l_low": low, "sigma2": s2, "eta2": 1e-3 * s2}),
            ("single", "single", res_a, 0.01, {})):
        _, st = plan.minor_cycle(step, res, plan.lam(res, coef, 1), fista_budget, **kw)
        fista[name] = {f"iters_to_{e:g}": iterations_to(st.trace, e) for e in (1e-2, 1e-3, 1e-4)}
    out["fista_first_cycle"] = fista
    plan.close()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--npix", type=int, default=1024)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--precision", default="fp32")
    ap.add_argument("--convolution", default="circular", choices=("circular", "linear"))
    args = ap.parse_args()
    import synth
    import paper_2406_18356_gb300 as ms
    ms.load_library()
    w = synth.paper_like(args.npix, seed=args.seed, device="cuda")
    print(json.dumps(study(ms, w, precision=args.precision, convolution=args.convolution)))


if __name__ == "__main__":
    main()
