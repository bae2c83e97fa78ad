"""Learned warm start for step two of the two-step method (Sect. 3.3).

Training pairs come from the method itself: for a sky, the two-step
reconstruction gives the step-one image i^_L; the long-baseline dirty image
i~_H1 is the first residual of step two; the target is the solution W beta* of
step two's first minor cycle (Eq. FullRes, a long FISTA run).  The network
(``WarmStartNet``) maps [i^_L, i~_H1] to x0 ~ W beta*, and step two then
starts FISTA from beta_0 = W^H x0 / M (W W^H = M I, so W beta_0 = x0) instead
of zero and still runs to the same tolerance: the network only moves the
starting point, the plain solve decides the result.

Everything runs through the library's C ABI (plans, minor cycles, the
network's kernels); this module only arranges the calls.

    python -m paper_2406_18356_gb300.warm_start --train 512 --eval 16
prints one JSON line with the training loss and, for every evaluation sky,
FISTA iterations and wall time from zero, from the step-one image and from
the network's start (see ``evaluate``).
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np


def make_problem(ms, seed: int, npix: int, n_major: int = 5, fista_iters: int = 100,
                 precision: str = "fp32"):
    """The step-two problem of one synthetic sky: plan, network input
    [i^_L, i~_H1] (FP32 [N, N, 2] on the GPU), its normalisation, and the
    parameters of step two's first minor cycle."""
    import torch
    import synth
    w = synth.c1_style(npix, seed, device="cuda")
    plan = ms.Plan(w.u[0], w.v[0], npix, w.pixel_size, w.ell_px, w.delta_px,
                   precision=precision)
    vis = torch.from_numpy(w.vis[0]).cuda().to(plan.complex_dtype)
    low, _, _ = plan.reconstruct_two_step(vis, ms.ReconOptions(n_major=n_major,
                                                               fista_iters=fista_iters))
    res = plan.grid("H", vis)
    s2 = plan.sigma2_hat(res)
    # training pairs use the scaling ms_warm_start_coefficients applies to the
    # network's input at inference: images divided by max|i~_H1|
    scale = 1.0 / float(res.abs().max())
    x = torch.stack([low.float(), res.float()], dim=2).mul(scale).contiguous()
    return {"plan": plan, "x": x, "scale": scale, "low": low, "res": res,
            "lam": plan.lam(res, 0.05, 1), "sigma2": s2, "eta2": 1e-3 * s2}


def solve(ms, prob, max_iters: int, rel_tol: float, net=None):
    """Step two's first minor cycle, from zero or from the network's start
    (the library's ms_warm_start_coefficients), with the relative-change stop
    rel_tol (0: exactly max_iters iterations); returns (model image, stats,
    wall ms)."""
    import torch
    plan = prob["plan"]
    beta = None
    if net is not None:
        beta, _ = plan.warm_start_coefficients(net, prob["low"], prob["res"])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    model, st = plan.minor_cycle("full", prob["res"], prob["lam"], max_iters,
                                 l_low=prob["low"], sigma2=prob["sigma2"], eta2=prob["eta2"],
                                 rel_tol=rel_tol, beta=beta)
    torch.cuda.synchronize()
    return model, st, 1000.0 * (time.perf_counter() - t0)


def make_pair(ms, seed: int, npix: int, iters: int = 1500):
    """(network input, target) of one training sky, both normalised; the
    target is the minor cycle's solution after a fixed, long FISTA run."""
    prob = make_problem(ms, seed, npix)
    model, _, _ = solve(ms, prob, iters, 0.0)
    target = model.float().mul(prob["scale"]).contiguous()
    x = prob["x"]
    prob["plan"].close()
    return x, target


def train(net, pairs, epochs: int, lr: float, seed: int = 0):
    """Adam on the mean squared error, one pair per step, shuffled epochs;
    returns the mean loss of every epoch."""
    rng = np.random.default_rng(seed)
    history = []
    for _ in range(epochs):
        losses = []
        for i in rng.permutation(len(pairs)):
            x, t = pairs[i]
            losses.append(net.train_step(x, t, lr))
        history.append(float(np.mean(losses)))
    return history


def iterations_to(trace, f_best: float, eps: float) -> int:
    """First iteration whose objective is within eps (relative) of f_best."""
    hit = np.nonzero(np.asarray(trace) <= f_best + eps * abs(f_best))[0]
    return int(hit[0]) if hit.size else len(trace)


def evaluate(ms, net, seeds, npix: int, rel_tol: float = 1e-6, max_iters: int = 2000,
             eps=(1e-2, 1e-3, 1e-4)):
    """Step two's first minor cycle on each held-out sky from three starts:
    zero (the plain method), the step-one image (no learning) and the
    network's output.  Two measures: (a) FISTA with the relative-change stop
    rel_tol (iterations, wall time, objective reached); (b) a fixed budget of
    max_iters iterations, and for each relative suboptimality e in eps the
    first iteration within e of the best objective any start reached (and the
    time to it from the run's per-iteration time)."""
    out = []
    # an untrained network returns its first input channel: the step-one
    # image as the start, through the same library call
    identity = ms.WarmStartNet(levels=net.levels, width=8, max_side=net.max_side, seed=0)
    for seed in seeds:
        prob = make_problem(ms, seed, npix)
        starts = {"zero": None, "low": identity, "net": net}
        rec = {"seed": int(seed)}
        runs = {}
        x0s = {}
        for name, nt in starts.items():
            if nt is not None:
                x0s[name] = prob["plan"].warm_start_coefficients(nt, prob["low"], prob["res"])[1]
            _, st, ms_ = solve(ms, prob, max_iters, rel_tol, net=nt)
            rec[f"stop_iters_{name}"] = st.iterations
            rec[f"stop_ms_{name}"] = ms_
            rec[f"stop_objective_{name}"] = st.objective
            model, lt, lms = solve(ms, prob, max_iters, 0.0, net=nt)
            runs[name] = (model, lt.trace, lms / max(lt.iterations, 1))
        f_best = min(float(np.min(r[1])) for r in runs.values())
        for name, (_, trace, ms_per_iter) in runs.items():
            for e in eps:
                k = iterations_to(trace, f_best, e)
                rec[f"iters_{name}_{e:g}"] = k
                rec[f"ms_{name}_{e:g}"] = k * ms_per_iter
        ref = runs["zero"][0].double()
        for name in ("low", "net"):
            rec[f"solution_rel_diff_{name}"] = float((runs[name][0].double() - ref).norm()
                                                     / ref.norm())
            x0 = x0s[name].double()
            rec[f"start_rel_err_{name}"] = float((x0 - ref).norm() / ref.norm())
        out.append(rec)
        prob["plan"].close()
    identity.close()
    return out


def conv_flops(levels: int, width: int, side: int) -> int:
    """Convolution FLOPs of one forward pass (2 per multiply-add), in the
    network's execution order: per encoder level two convs, the bottom
    level, per decoder level two convs on the upsampled-and-concatenated
    input, the head."""
    shapes, lv = [], []
    cin = 2
    for l in range(levels):
        c = width << l
        shapes += [(c, cin), (c, c)]
        lv += [l, l]
        cin = c
    for l in range(levels - 2, -1, -1):
        c = width << l
        shapes += [(c, (width << (l + 1)) + c), (c, c)]
        lv += [l, l]
    shapes.append((1, width))
    lv.append(0)
    return sum(2 * 9 * ci * co * (side >> l) ** 2 for (co, ci), l in zip(shapes, lv))


def time_network(ms, levels: int, width: int, side: int, reps: int = 10, warmup: int = 3):
    """CUDA-event times of a training step (forward, backward, Adam) and of a
    forward pass on random [side, side, 2] inputs, and the rates they give."""
    import torch
    net = ms.WarmStartNet(levels=levels, width=width, max_side=side, seed=1)
    x = torch.randn(side, side, 2, device="cuda")
    t = torch.randn(side, side, device="cuda")
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn):
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize()
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    step_ms = timed(lambda: net.train_step(x, t, 1e-4))
    fwd_ms = timed(lambda: net.forward(x))
    f = conv_flops(levels, width, side)
    rec = {"levels": levels, "width": width, "params": net.param_count(), "side": side,
           "train_step_ms": step_ms, "forward_ms": fwd_ms, "forward_gflop": f / 1e9,
           "train_step_tflops": 3 * f / step_ms / 1e9, "forward_tflops": f / fwd_ms / 1e9}
    net.close()
    return rec


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--time", action="store_true",
                    help="only time a training step and a forward pass of the network "
                         "(--levels, --width) at --train-npix and --eval-npix")
    ap.add_argument("--train", type=int, default=512, help="training skies (seeds 1..n)")
    ap.add_argument("--eval", type=int, default=16, help="held-out skies")
    ap.add_argument("--train-npix", type=int, default=512)
    ap.add_argument("--eval-npix", type=int, default=1024)
    ap.add_argument("--epochs", type=int, default=20)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--levels", type=int, default=3)
    ap.add_argument("--width", type=int, default=16)
    ap.add_argument("--save", default="")
    args = ap.parse_args()
    import paper_2406_18356_gb300 as ms
    ms.load_library()
    if args.time:
        for side in sorted({args.train_npix, args.eval_npix}):
            print(json.dumps(time_network(ms, args.levels, args.width, side)))
        return
    t0 = time.perf_counter()
    pairs = [make_pair(ms, s, args.train_npix) for s in range(1, args.train + 1)]
    t1 = time.perf_counter()
    net = ms.WarmStartNet(levels=args.levels, width=args.width,
                          max_side=max(args.train_npix, args.eval_npix), seed=0)
    hist = train(net, pairs, args.epochs, args.lr)
    t2 = time.perf_counter()
    if args.save:
        np.save(args.save, net.get_params())
    ev = evaluate(ms, net, range(100001, 100001 + args.eval), args.eval_npix)
    t3 = time.perf_counter()
    summ = {k: float(np.mean([e[k] for e in ev])) for k in ev[0] if k != "seed"}
    print(json.dumps({
        "network": {"levels": args.levels, "width": args.width, "params": net.param_count()},
        "train": {"skies": args.train, "npix": args.train_npix, "epochs": args.epochs,
                  "lr": args.lr, "loss_first_epoch": hist[0], "loss_last_epoch": hist[-1],
                  "pair_generation_s": t1 - t0, "training_s": t2 - t1},
        "eval": {"skies": args.eval, "npix": args.eval_npix, "rel_tol": 1e-6,
                 "mean": summ, "eval_s": t3 - t2, "per_sky": ev}}))


if __name__ == "__main__":
    main()
