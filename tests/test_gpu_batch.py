"""The batched form: several (channel, partition) jobs through one gridding /
degridding launch, against the per-job calls and the FP64 oracle (GPU)."""
import numpy as np
import pytest

import synth
from oracle import gridding as og

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
def obs():
    # 4 channels of one layout, uneven random flagging per channel
    return synth.multi_channel(npix=64, nchan=4, n_ant=12, n_dumps=10, span_h=4.0,
                               flag_max=0.5, with_vis=True, seed=2)


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _plan(ms, w, precision):
    return ms.Plan(w.u, w.v, w.npix, w.pixel_size, w.ell_px, w.delta_px, flags=w.flags,
                   precision=precision)


JOBS = [(c, p) for c in range(4) for p in ("L", "H")]


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 2e-6),
                                           ("fp32_kahan", 2e-6)])
def test_grid_batch_matches_per_job_grid(ms, obs, precision, tol):
    import torch
    plan = _plan(ms, obs, precision)
    vis = [torch.from_numpy(obs.vis[c]).cuda().to(plan.complex_dtype) for c, _ in JOBS]
    outs = plan.grid_batch(JOBS, vis)
    for (c, p), v, o in zip(JOBS, vis, outs):
        ref = plan.grid(p, v, chan=c).cpu().numpy()
        assert np.abs(ref).max() > 0
        assert rel(o.cpu().numpy(), ref) <= tol
    plan.close()


def test_grid_batch_matches_oracle_with_flags(ms, obs):
    import torch
    plan = _plan(ms, obs, "fp64")
    vis = [torch.from_numpy(obs.vis[c]).cuda() for c, _ in JOBS]
    outs = plan.grid_batch(JOBS, vis)
    for (c, p), o in zip(JOBS, outs):
        keep = obs.flags[c] == 0
        u, v = obs.u[c][keep], obs.v[c][keep]
        in_l, in_h = og.partition(u, v, obs.npix, obs.pixel_size, obs.ell_px, obs.delta_px)
        m = in_l if p == "L" else in_h
        A = og.GriddedOperator(u[m], v[m], obs.npix, obs.pixel_size)
        ref = A.dirty(obs.vis[c][keep][m])
        assert rel(o.cpu().numpy(), ref) <= 1e-10
    plan.close()


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 2e-6)])
@pytest.mark.parametrize("with_obs", [False, True])
def test_degrid_batch_matches_per_job_degrid(ms, obs, precision, tol, with_obs):
    import torch
    plan = _plan(ms, obs, precision)
    rng = np.random.default_rng(5)
    images = [torch.from_numpy(rng.standard_normal((64, 64))).cuda().to(plan.real_dtype)
              for _ in JOBS]
    vobs = [torch.from_numpy(obs.vis[c]).cuda().to(plan.complex_dtype) for c, _ in JOBS]
    outs = plan.degrid_batch(JOBS, images, vis_obs=vobs if with_obs else None)
    for (c, p), x, vo, o in zip(JOBS, images, vobs, outs):
        ref = torch.zeros(plan.nvis, dtype=plan.complex_dtype, device="cuda")
        plan.degrid(p, x, vo if with_obs else None, out=ref, chan=c)
        r, g = ref.cpu().numpy(), o.cpu().numpy()
        rows = plan.partition_rows(p, c)
        assert len(rows) > 0
        others = np.ones(plan.nvis, bool)
        others[rows] = False
        assert np.all(g[others] == 0)          # only the job's rows are written
        assert rel(g[rows], r[rows]) <= tol
    plan.close()


def test_batch_workspace_grows_and_shrinks(ms, obs):
    import torch
    plan = _plan(ms, obs, "fp32")
    vis = {c: torch.from_numpy(obs.vis[c]).cuda().to(plan.complex_dtype) for c in range(4)}
    for jobs in (JOBS[:2], JOBS, JOBS[3:5]):
        outs = plan.grid_batch(jobs, [vis[c] for c, _ in jobs])
        for (c, p), o in zip(jobs, outs):
            ref = plan.grid(p, vis[c], chan=c).cpu().numpy()
            assert rel(o.cpu().numpy(), ref) <= 2e-6
    plan.close()


def test_batch_rejects_bad_jobs(ms, obs):
    import torch
    plan = _plan(ms, obs, "fp32")
    v = torch.from_numpy(obs.vis[0]).cuda().to(plan.complex_dtype)
    with pytest.raises(ms.MsError) as e:
        plan.grid_batch([(7, "L")], [v])
    assert e.value.status == ms.MS_ERR_ARG
    plan.close()


def test_autotune_picks_a_candidate(ms, obs):
    t, c, ms_ = ms.ms_plan_autotune(obs.u, obs.v, obs.npix, obs.pixel_size, obs.ell_px,
                                    obs.delta_px, flags=obs.flags, precision="fp32", reps=2)
    assert t in (16, 32) and c in (512, 1024, 2048, 4096, 8192)
    assert ms_ > 0
