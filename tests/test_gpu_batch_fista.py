"""Batched minor cycles (several channels' FISTA problems per launch, one
CUDA graph per 8 passes) and the batched reconstruction, against the
per-job calls and the FP64 oracle (GPU)."""
import numpy as np
import pytest

import synth
from oracle import gridding as og
from oracle import solver as osv
from oracle.wavelets import Dictionary

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ms():
    import torch
    import paper_2406_18356_gb300 as pkg
    from paper_2406_18356_gb300 import _build
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    _build.build()
    pkg.load_library()
    return pkg


@pytest.fixture(scope="module")
def obs64():
    # 4 channels of one layout, uneven random flagging per channel
    return synth.multi_channel(npix=64, nchan=4, n_ant=12, n_dumps=10, span_h=4.0,
                               flag_max=0.5, with_vis=True, seed=2)


@pytest.fixture(scope="module")
def obs256():
    # wide enough that the plain minor cycle runs its coarse levels as one
    # cooperative launch, which the batched form replaces by per-level launches
    return synth.multi_channel(npix=256, nchan=2, n_ant=16, n_dumps=16, span_h=4.0,
                               flag_max=0.3, with_vis=True, seed=3)


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _plan(ms, w, precision, J=4):
    return ms.Plan(w.u, w.v, w.npix, w.pixel_size, w.ell_px, w.delta_px, flags=w.flags,
                   precision=precision, levels=J, n_bases=8)


def _jobs(plan, w, nchan):
    """low, full and single problems of every channel (12 different jobs for
    4 channels): residuals are the partitions' dirty images."""
    import torch
    jobs = []
    for c in range(nchan):
        v = torch.from_numpy(w.vis[c]).cuda().to(plan.complex_dtype)
        rl, rh, ra = plan.grid("L", v, chan=c), plan.grid("H", v, chan=c), plan.grid("ALL", v, chan=c)
        s2 = plan.sigma2_hat(rh)
        jobs.append({"step": "low", "chan": c, "residual": rl, "lam": plan.lam(rl, 0.05, 1)})
        jobs.append({"step": "full", "chan": c, "residual": rh, "lam": plan.lam(rh, 0.05, 1),
                     "l_low": 0.5 * rl, "sigma2": s2, "eta2": 1e-3 * s2})
        jobs.append({"step": "single", "chan": c, "residual": ra, "lam": plan.lam(ra, 0.01, 1)})
    return jobs


def _per_job(plan, j, iters, rel_tol=0.0):
    return plan.minor_cycle(j["step"], j["residual"], j["lam"], iters, l_low=j.get("l_low"),
                            sigma2=j.get("sigma2", 0.0), eta2=j.get("eta2", 0.0),
                            rel_tol=rel_tol, chan=j["chan"])


@pytest.mark.parametrize("npix", [64, 256])
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-11), ("fp32", 2e-5)])
def test_minor_cycle_batch_matches_per_job_calls(ms, obs64, obs256, npix, precision, tol):
    w, nchan = (obs64, 4) if npix == 64 else (obs256, 2)
    plan = _plan(ms, w, precision)
    jobs = _jobs(plan, w, nchan)
    iters = 30
    models, stats = plan.minor_cycle_batch(jobs, iters)
    for j, m, st in zip(jobs, models, stats):
        ref, rst = _per_job(plan, j, iters)
        assert st.iterations == rst.iterations == iters
        assert st.theta == pytest.approx(rst.theta, rel=1e-12)
        np.testing.assert_allclose(st.trace, rst.trace, rtol=tol)
        e = rel(m.double().cpu().numpy(), ref.double().cpu().numpy())
        assert e <= tol, (j["step"], j["chan"], e)
    plan.close()


def test_minor_cycle_batch_matches_oracle(ms, obs64):
    """Two jobs of different channels and problems against the oracle's
    Algorithm 1 on the same inputs (FP64)."""
    w = obs64
    plan = _plan(ms, w, "fp64")
    jobs = _jobs(plan, w, 4)
    pick = [jobs[1 * 3 + 0], jobs[2 * 3 + 1]]   # channel 1 low, channel 2 full
    iters = 25
    models, stats = plan.minor_cycle_batch(pick, iters)
    for j, m, st in zip(pick, models, stats):
        c = j["chan"]
        keep = w.flags[c] == 0
        in_l, in_h = og.partition(w.u[c][keep], w.v[c][keep], w.npix, w.pixel_size, w.ell_px,
                                  w.delta_px)
        mask = in_l if j["step"] == "low" else in_h
        A = og.GriddedOperator(w.u[c][keep][mask], w.v[c][keep][mask], w.npix, w.pixel_size)
        Hhat = osv.psf_spectrum(A.psf())
        res = j["residual"].cpu().numpy()
        W = Dictionary(w.npix, 8, 4)
        if j["step"] == "low":
            prob = osv.Problem("low", W, Hhat, res, j["lam"])
        else:
            gl, gh = osv.filter_responses(w.npix, w.ell_px, w.delta_px, j["sigma2"], j["eta2"])
            prob = osv.Problem("full", W, Hhat, res, j["lam"], gl=gl, gh=gh,
                               l_low=j["l_low"].cpu().numpy())
        ref = osv.fista(prob, iters)
        np.testing.assert_allclose(st.trace, ref.objective, rtol=1e-9)
        assert rel(m.cpu().numpy(), W.synth(ref.beta)) <= 1e-8
    plan.close()


def test_minor_cycle_batch_stops_each_job_on_its_own(ms, obs64):
    """With a relative-change stop every job ends at the iteration its own
    per-job call ends at (the done flags are per job, on the device)."""
    plan = _plan(ms, obs64, "fp64")
    jobs = _jobs(plan, obs64, 4)[:6]
    models, stats = plan.minor_cycle_batch(jobs, 400, rel_tol=1e-4)
    its = [st.iterations for st in stats]
    assert len(set(its)) > 1, its
    for j, m, st in zip(jobs, models, stats):
        ref, rst = _per_job(plan, j, 400, rel_tol=1e-4)
        assert st.iterations == rst.iterations
        assert st.converged == rst.converged
        assert rel(m.cpu().numpy(), ref.cpu().numpy()) <= 1e-11
    plan.close()


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("fp32", 1e-4)])
def test_reconstruct_batch_matches_per_channel(ms, obs64, precision, tol):
    """The batched two-step and single-step reconstructions of 4 channels
    (batched residual images, batched minor cycles) against the per-channel
    calls."""
    import torch
    w = obs64
    plan = _plan(ms, w, precision, J=3)
    vis = [torch.from_numpy(w.vis[c]).cuda().to(plan.complex_dtype) for c in range(4)]
    opts = ms.ReconOptions(n_major=3, fista_iters=20)
    lows, imgs, stats = plan.reconstruct_two_step_batch(vis, opts)
    for c in range(4):
        low, img, st = plan.reconstruct_two_step(vis[c], opts, chan=c)
        e_low = rel(lows[c].double().cpu().numpy(), low.double().cpu().numpy())
        e_img = rel(imgs[c].double().cpu().numpy(), img.double().cpu().numpy())
        print(f"channel {c} {precision}: low {e_low:.2e} image {e_img:.2e}")
        assert e_low <= tol and e_img <= tol
        assert stats[c].total_iterations == st.total_iterations == 2 * 3 * 20
        assert stats[c].gridded_vis == st.gridded_vis
        assert stats[c].sigma2 == pytest.approx(st.sigma2, rel=1e-9 if precision == "fp64" else 1e-4)
    singles, _ = plan.reconstruct_single_step_batch(vis[1:3], opts, chans=[1, 2])
    for s, c in zip(singles, (1, 2)):
        ref, _ = plan.reconstruct_single_step(vis[c], opts, chan=c)
        assert rel(s.double().cpu().numpy(), ref.double().cpu().numpy()) <= tol
    plan.close()


def test_batch_needs_the_fused_spectral_step(ms):
    import torch
    w = synth.tiny(npix=48)
    plan = ms.Plan(w.u[0], w.v[0], 48, w.pixel_size, w.ell_px, w.delta_px, precision="fp64",
                   levels=3, n_bases=2)
    res = plan.grid("L", torch.from_numpy(w.vis[0]).cuda())
    with pytest.raises(ms.MsError):
        plan.minor_cycle_batch([{"step": "low", "residual": res, "lam": 1.0}], 5)
    plan.close()
