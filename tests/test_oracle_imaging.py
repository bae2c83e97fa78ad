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


def _complete_coverage(npix, dl, rng):
    """One visibility at every frequency of the npix x npix image DFT (on the
    oversampled grid's cells) for a random real sky, exact under the gridded
    model (no noise)."""
    k = np.arange(-npix // 2, npix // 2)
    kx, ky = np.meshgrid(k, k)
    u = kx.ravel() / (npix * dl)
    v = ky.ravel() / (npix * dl)
    sky = rng.standard_normal((npix, npix))
    return u, v, sky, GriddedOperator(u, v, npix, dl).forward(sky)


def test_single_step_recovers_the_sky_with_complete_coverage():
    # With every image frequency sampled on the grid, A^H A is exactly the
    # PSF's circular convolution, so with lambda = 0 the minor cycle's model
    # is exact and the major cycles reach the sky itself (the fixed point
    # A^H (v - A x) = 0 of a full-rank A): a check of the residual and PSF
    # normalization, the model update and image = residual + model.
    rng = np.random.default_rng(3)
    u, v, sky, vis = _complete_coverage(16, 1e-4, rng)
    opts = oi.ReconOptions(n_major=3, fista_iters=100, lambda_single=0.0, levels=2, n_bases=2)
    out = oi.reconstruct_single_step(vis, u, v, 16, 1e-4, opts)
    assert np.linalg.norm(out.image - sky) <= 1e-12 * np.linalg.norm(sky)
    assert np.linalg.norm(out.residuals[-1]) <= 1e-12 * np.linalg.norm(out.residuals[0])


def test_two_step_recovers_the_sky_with_complete_coverage():
    # Step one (V_L) fixes the frequencies inside its disk, step two (V_H and
    # the low-passed step-one image) the rest; with lambda = 0 the final
    # image converges to the sky as the major cycles proceed.
    rng = np.random.default_rng(4)
    u, v, sky, vis = _complete_coverage(16, 1e-4, rng)
    errs = []
    for n_major in (1, 3, 6):
        opts = oi.ReconOptions(n_major=n_major, fista_iters=300, lambda_low=0.0, lambda_full=0.0,
                               levels=2, n_bases=2, sigma2=1.0, eta2=1e-3)
        low, full = oi.reconstruct_two_step(vis, u, v, 16, 1e-4, 4.0, 1.5, opts)
        errs.append(np.linalg.norm(full.image - sky) / np.linalg.norm(sky))
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] <= 1e-5
    # step one alone only knows the frequencies its baselines sample
    assert np.linalg.norm(low.image - sky) > 0.1 * np.linalg.norm(sky)


def test_psnr_closed_form():
    truth = np.zeros((8, 8))
    truth[2, 3] = -4.0                    # peak magnitude 4
    image = truth + 0.5                   # mse 0.25
    assert abs(oi.psnr(image, truth) - 10.0 * np.log10(16.0 / 0.25)) < 1e-12
