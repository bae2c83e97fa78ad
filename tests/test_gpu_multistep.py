"""The method with more than two steps through ms_reconstruct_step, against
the oracle (GPU)."""
import numpy as np
import pytest

import synth
from oracle import imaging as oi
from oracle import multistep as oms

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


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-8), ("fp32", 1e-4)])
def test_three_bands_match_oracle(ms, precision, tol):
    import torch
    from paper_2406_18356_gb300 import multistep
    w = synth.tiny(npix=32, n_ant=12, n_dumps=10, seed=9)
    u, v, vis = w.u[0], w.v[0], w.vis[0]
    ells, delta = [3.0, 6.0], 1.0
    opts = ms.ReconOptions(n_major=2, fista_iters=20)
    ro = oi.ReconOptions(n_major=2, fista_iters=20, levels=3)
    imgs, stats = multistep.reconstruct_multi_step(ms, u, v, torch.from_numpy(vis).cuda(), 32,
                                                   w.pixel_size, ells, delta, opts,
                                                   precision=precision, levels=3)
    ref = oms.reconstruct_multi_step(vis, u, v, 32, w.pixel_size, ells, delta, ro)
    errs = [rel(i.double().cpu().numpy(), r.image) for i, r in zip(imgs, ref)]
    print(f"three bands {precision}: " + ", ".join(f"{e:.2e}" for e in errs))
    assert len(imgs) == 3 and max(errs) <= tol
    masks = oms.band_masks(u, v, 32, w.pixel_size, ells, delta)
    assert [s.gridded_vis for s in stats] == [3 * int(m.sum()) for m in masks]


def test_two_bands_are_the_two_step_call(ms):
    import torch
    from paper_2406_18356_gb300 import multistep
    w = synth.tiny(npix=32, n_ant=12, n_dumps=10, seed=4)
    tv = torch.from_numpy(w.vis[0]).cuda()
    opts = ms.ReconOptions(n_major=2, fista_iters=20)
    imgs, _ = multistep.reconstruct_multi_step(ms, w.u[0], w.v[0], tv, 32, w.pixel_size,
                                               [w.ell_px], w.delta_px, opts, precision="fp64",
                                               levels=3)
    plan = ms.Plan(w.u[0], w.v[0], 32, w.pixel_size, w.ell_px, w.delta_px, precision="fp64",
                   levels=3)
    low, img, _ = plan.reconstruct_two_step(tv, opts)
    assert rel(imgs[0].cpu().numpy(), low.cpu().numpy()) <= 1e-13
    assert rel(imgs[1].cpu().numpy(), img.cpu().numpy()) <= 1e-13
    plan.close()
