"""The precision form at the 4096^2, 125.6M-row SKA-Low-like scale (GPU, slow):
FP32 and Kahan-compensated FP32 gridding / degridding of all (channel,
partition) jobs against the FP64 form on the same GPU, and the FP64 form
against the oracle on every 16th row of one channel."""
import numpy as np
import pytest

import synth
from oracle import gridding as og

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


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
def low():
    return synth.ska_low_like(seed=0)


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_precision_forms_against_fp64_at_full_scale(ms, low):
    import torch
    w = low
    assert w.u.size == 125_583_360
    jobs = [(c, p) for c in range(w.u.shape[0]) for p in ("L", "H")]
    image = torch.from_numpy(np.random.default_rng(1).standard_normal((w.npix, w.npix))).cuda()
    ref = None
    for prec in ("fp64", "fp32", "fp32_kahan"):
        plan = ms.Plan(w.u, w.v, w.npix, w.pixel_size, w.ell_px, w.delta_px, precision=prec)
        vis = {c: torch.from_numpy(w.vis[c]).cuda().to(plan.complex_dtype)
               for c in range(w.u.shape[0])}
        dirty = [o.double() for o in plan.grid_batch(jobs, [vis[c] for c, _ in jobs])]
        rows = [torch.from_numpy(plan.partition_rows(p, c)).cuda().long() for c, p in jobs]
        model = [v[r].to(torch.complex128) for v, r in
                 zip(plan.degrid_batch(jobs, [image.to(plan.real_dtype)] * len(jobs)), rows)]
        plan.close()
        del vis
        if ref is None:
            ref = (dirty, model)
            continue
        e_grid = max(float((d - d64).norm() / d64.norm()) for d, d64 in zip(dirty, ref[0]))
        e_degrid = max(float((m - m64).norm() / m64.norm()) for m, m64 in zip(model, ref[1]))
        print(f"{prec}: dirty images max rel L2 vs FP64 {e_grid:.3e}, "
              f"degridded values max rel L2 vs FP64 {e_degrid:.3e}")
        assert e_grid <= 1e-5 and e_degrid <= 1e-5
        del dirty, model
        torch.cuda.empty_cache()


def test_fp64_form_matches_oracle_on_every_16th_row(ms, low):
    import torch
    w = low
    u, v, vis = w.u[0][::16], w.v[0][::16], w.vis[0][::16]
    plan = ms.Plan(u, v, w.npix, w.pixel_size, w.ell_px, w.delta_px, precision="fp64")
    got = plan.grid("ALL", torch.from_numpy(vis).cuda()).cpu().numpy()
    plan.close()
    A = og.GriddedOperator(u, v, w.npix, w.pixel_size)
    ref = A.dirty(vis)
    e = rel(got, ref)
    print(f"fp64 GPU vs oracle on {len(u)} rows at {w.npix}^2: rel L2 {e:.3e}")
    assert e <= 1e-10
