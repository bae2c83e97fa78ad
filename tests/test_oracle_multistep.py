"""Pins of the oracle's method with more than two steps (CPU)."""
import numpy as np

import synth
from oracle import imaging as oi
from oracle import multistep as oms
from oracle.gridding import GriddedOperator, partition


def test_bands_cover_every_row_and_overlap_only_near_their_edges():
    w = synth.tiny(npix=32, n_ant=12, n_dumps=10, seed=3)
    u, v = w.u[0], w.v[0]
    ells, delta = (3.0, 6.0, 9.0), 1.0
    masks = oms.band_masks(u, v, 32, w.pixel_size, ells, delta)
    r = np.hypot(u, v) * 32 * w.pixel_size
    assert len(masks) == 4
    assert np.all(np.any(masks, axis=0))
    for k in range(3):
        both = masks[k] & masks[k + 1]
        assert np.all(np.abs(r[both] - ells[k]) <= delta + 1e-9)
    # rows of a band lie inside its closed interval
    assert np.all(r[masks[1]] >= ells[0] - delta - 1e-9) and np.all(r[masks[1]] <= ells[1] + delta + 1e-9)


def test_two_bands_are_the_two_step_method():
    w = synth.tiny(npix=32, n_ant=12, n_dumps=10, seed=9)
    u, v, vis = w.u[0], w.v[0], w.vis[0]
    opts = oi.ReconOptions(n_major=2, fista_iters=15, levels=3, n_bases=2)
    steps = oms.reconstruct_multi_step(vis, u, v, 32, w.pixel_size, [w.ell_px], w.delta_px, opts)
    low, full = oi.reconstruct_two_step(vis, u, v, 32, w.pixel_size, w.ell_px, w.delta_px, opts)
    np.testing.assert_array_equal(steps[0].image, low.image)
    np.testing.assert_array_equal(steps[1].image, full.image)


def test_three_steps_recover_the_sky_with_complete_coverage():
    """Every frequency sampled, lambda = 0: the last step's image approaches
    the sky as the major cycles proceed; the first step alone does not."""
    rng = np.random.default_rng(7)
    N, dl = 16, 1e-4
    k = np.arange(-N // 2, N // 2)
    kx, ky = np.meshgrid(k, k)
    u, v = kx.ravel() / (N * dl), ky.ravel() / (N * dl)
    sky = rng.standard_normal((N, N))
    vis = GriddedOperator(u, v, N, dl).forward(sky)
    errs = []
    for n_major in (1, 3, 6):
        opts = oi.ReconOptions(n_major=n_major, fista_iters=300, lambda_low=0.0,
                               lambda_full=0.0, levels=2, n_bases=2, sigma2=1.0, eta2=1e-3)
        steps = oms.reconstruct_multi_step(vis, u, v, N, dl, [3.0, 6.0], 1.0, opts)
        errs.append(np.linalg.norm(steps[-1].image - sky) / np.linalg.norm(sky))
    assert errs[0] > errs[1] > errs[2], errs
    assert errs[2] <= 1e-4, errs
    assert np.linalg.norm(steps[0].image - sky) > 0.1 * np.linalg.norm(sky)
