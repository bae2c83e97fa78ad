"""Checks of the oracle's major-cycle orchestration (CPU only).

The end-to-end images have no printed worked example in the paper: these are
structural checks and special-case reductions, the reconstructions themselves
stay "parity unpinned" beyond the pins of their parts."""
import numpy as np

import synth
from oracle import imaging as oi
from oracle.gridding import GriddedOperator, partition


def _opts(**kw):
    base = dict(n_major=2, fista_iters=15, levels=3)
    base.update(kw)
    return oi.ReconOptions(**base)


def test_step_one_with_all_baselines_is_single_step():
    """ell + delta >= r_max puts every row in V_L, and step one is then the
    single-step method (Sect. 5) when the lambda coefficients agree."""
    w = synth.tiny(npix=32, n_ant=8, n_dumps=6, seed=5)
    u, v, vis = w.u[0], w.v[0], w.vis[0]
    in_l, _ = partition(u, v, 32, w.pixel_size, 40.0, 2.0)
    assert in_l.all()
    opts = _opts(lambda_low=0.02, lambda_single=0.02)
    low = oi.run_low_step(vis[in_l], u[in_l], v[in_l], 32, w.pixel_size, opts, opts.lambda_low)
    single = oi.reconstruct_single_step(vis, u, v, 32, w.pixel_size, opts)
    np.testing.assert_array_equal(low.image, single.image)


def test_final_image_is_residual_plus_model_and_residual_is_consistent():
    w = synth.tiny(npix=32, n_ant=8, n_dumps=6, seed=6)
    u, v, vis = w.u[0], w.v[0], w.vis[0]
    opts = _opts()
    low, full = oi.reconstruct_two_step(vis, u, v, 32, w.pixel_size, w.ell_px, w.delta_px, opts)
    for st in (low, full):
        assert len(st.residuals) == opts.n_major + 1
        np.testing.assert_allclose(st.image, st.residuals[-1] + st.model, atol=1e-15)
    # the last residual of step two is the dirty image of V_H minus its model
    _, in_h = partition(u, v, 32, w.pixel_size, w.ell_px, w.delta_px)
    A = GriddedOperator(u[in_h], v[in_h], 32, w.pixel_size)
    np.testing.assert_allclose(full.residuals[-1], A.dirty(vis[in_h] - A.forward(full.model)),
                               atol=1e-12)
    assert full.sigma2 > 0 and abs(full.eta2 - 1e-3 * full.sigma2) < 1e-18


def test_lambda_rules():
    r = np.full((4, 4), 0.5)
    assert oi._lambda("norm2_2n", 0.05, r, r, 3) == 0.05 * 2.0 * 8
    first = np.zeros((4, 4)); first[1, 1] = -3.0
    assert oi._lambda("max_fixed", 1e-3, r, first, 4) == 3e-3


def test_minor_cycles_lower_their_objective():
    """Soft sanity (not a pin): every minor cycle ends below where it started,
    and the single-step image beats the dirty image's PSNR."""
    w = synth.tiny(npix=32, n_ant=12, n_dumps=10, seed=7, n_points=3, n_blobs=1)
    u, v, vis = w.u[0], w.v[0], w.vis[0]
    opts = _opts(n_major=3, fista_iters=40)
    low, full = oi.reconstruct_two_step(vis, u, v, 32, w.pixel_size, w.ell_px, w.delta_px, opts)
    single = oi.reconstruct_single_step(vis, u, v, 32, w.pixel_size, opts)
    for st in (low, full, single):
        for trace in st.objectives:
            assert trace[-1] <= trace[0]
    dirty = GriddedOperator(u, v, 32, w.pixel_size).dirty(vis)
    assert oi.psnr(single.image, w.truth) > oi.psnr(dirty, w.truth)
