"""The quality study (Sect. 5) through the library against the FP64 oracle
at 128 pixels: the PSNRs of the two-step image over partitions and of the
single-step image match the oracle's reconstructions of the same sky (GPU,
slow)."""
import numpy as np
import pytest

import synth
from oracle import imaging as oi

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


def test_study_psnrs_match_the_oracle(ms):
    from paper_2406_18356_gb300 import quality as q
    w = synth.paper_like(128, seed=2)
    grid = [q.partitions(128)[1], q.partitions(128)[7]]   # ell 0.117 / 0.322, delta 3 @ 512
    got = q.study(ms, w, precision="fp64", n_major=3, fista_iters=50, grid=grid,
                  convergence=False)
    ro = oi.ReconOptions(n_major=3, fista_iters=50)
    u, v, vis = w.u[0], w.v[0], w.vis[0]
    for rec, (ell, delta) in zip(got["partitions"], grid):
        _, full = oi.reconstruct_two_step(vis, u, v, 128, w.pixel_size, ell, delta, ro)
        want = oi.psnr(full.image, w.truth)
        print(f"ell {ell:.1f} delta {delta:.2f}: library {rec['psnr_two_step']:.4f} dB, "
              f"oracle {want:.4f} dB")
        assert abs(rec["psnr_two_step"] - want) <= 1e-3
    single = oi.reconstruct_single_step(vis, u, v, 128, w.pixel_size, ro)
    want = oi.psnr(single.image, w.truth)
    print(f"single step: library {got['psnr_single_step']:.4f} dB, oracle {want:.4f} dB")
    assert abs(got["psnr_single_step"] - want) <= 1e-3
    # the interleaved pipeline's combined image, first partition
    from oracle import interleaved as oil
    (ell, delta), rec = grid[0], got["partitions"][0]
    il = oil.reconstruct_interleaved(vis, u, v, 128, w.pixel_size, ell, delta, ro)
    want = oi.psnr(il.image, w.truth)
    print(f"interleaved: library {rec['psnr_interleaved']:.4f} dB, oracle {want:.4f} dB")
    assert abs(rec["psnr_interleaved"] - want) <= 1e-3


def test_study_reports_every_measure(ms):
    """The full study's structure on a small sky: 9 partitions, the
    major-cycle curves and the first-cycle FISTA counts."""
    from paper_2406_18356_gb300 import quality as q
    w = synth.paper_like(128, seed=3)
    out = q.study(ms, w, precision="fp32", n_major=2, fista_iters=30, n_major_max=3,
                  fista_budget=300)
    assert len(out["partitions"]) == 9
    for r in out["partitions"]:
        assert np.isfinite(r["psnr_two_step"]) and r["V_L"] + r["V_H"] - r["V_LH"] == w.nvis
    assert len(out["major_cycles"]["psnr_two_step"]) == 3
    for name in ("low", "full", "single"):
        f = out["fista_first_cycle"][name]
        assert f["iters_to_0.01"] <= f["iters_to_0.001"] <= f["iters_to_0.0001"] <= 301


def test_linear_study_psnrs_match_the_oracle(ms):
    """The same study with the linear PSF operator against the oracle's
    linear reading; with it the major cycles keep improving the image."""
    from paper_2406_18356_gb300 import quality as q
    w = synth.paper_like(128, seed=2)
    grid = [q.partitions(128)[4]]   # ell 0.205, delta 3 @ 512
    got = q.study(ms, w, precision="fp64", n_major=3, fista_iters=50, grid=grid,
                  convergence=False, convolution="linear")
    ro = oi.ReconOptions(n_major=3, fista_iters=50, convolution="linear")
    u, v, vis = w.u[0], w.v[0], w.vis[0]
    (ell, delta), rec = grid[0], got["partitions"][0]
    _, full = oi.reconstruct_two_step(vis, u, v, 128, w.pixel_size, ell, delta, ro)
    want = oi.psnr(full.image, w.truth)
    print(f"linear: library {rec['psnr_two_step']:.4f} dB, oracle {want:.4f} dB")
    assert abs(rec["psnr_two_step"] - want) <= 1e-3
    single = oi.reconstruct_single_step(vis, u, v, 128, w.pixel_size, ro)
    want = oi.psnr(single.image, w.truth)
    print(f"linear single step: library {got['psnr_single_step']:.4f} dB, oracle {want:.4f} dB")
    assert abs(got["psnr_single_step"] - want) <= 1e-3
