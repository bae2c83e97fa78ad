"""Pins of the oracle's interleaved two-image pipeline (Sect. 6's sketch, in
the reading the module states): filter identities, its first cycle against
the already-pinned steps, and recovery of the sky under complete coverage
(CPU)."""
import numpy as np

from oracle import imaging as oi
from oracle import interleaved as oil
from oracle import solver as osv
from oracle.gridding import GriddedOperator, partition


def _complete_coverage(npix, dl, rng):
    """One visibility at every frequency of the npix x npix DFT for a random
    real sky, exact under the gridded model (no noise)."""
    k = np.arange(-npix // 2, npix // 2)
    kx, ky = np.meshgrid(k, k)
    u = kx.ravel() / (npix * dl)
    v = ky.ravel() / (npix * dl)
    sky = rng.standard_normal((npix, npix))
    return u, v, sky, GriddedOperator(u, v, npix, dl).forward(sky)


def test_mirrored_filters_and_combination_weights_partition_unity():
    """Node L's filters are Sect. 3.3's with the sides exchanged:
    sigma^2 data^2 + eta^2 prior^2 = 1, data = 1/sigma below ell - delta and
    0 above ell + delta; the combination weights sum to one."""
    N, ell, delta, s2, e2 = 32, 6.0, 2.0, 0.3, 4e-4
    data, prior = oil.mirrored_filters(N, ell, delta, s2, e2)
    np.testing.assert_allclose(s2 * data ** 2 + e2 * prior ** 2, 1.0, atol=1e-12)
    r = osv.radial_frequency(N)
    np.testing.assert_allclose(data[r < ell - delta], 1.0 / np.sqrt(s2))
    assert np.all(data[r > ell + delta] == 0.0) and np.all(prior[r < ell - delta] == 0.0)
    gl, gh = osv.filter_responses(N, ell, delta, s2, e2)
    np.testing.assert_allclose(e2 * gl ** 2 + s2 * gh ** 2, 1.0, atol=1e-12)


def test_first_cycle_is_each_partitions_low_resolution_problem():
    """Cycle 1 of node L is step one's first minor cycle on V_L; cycle 1 of
    node H is the same problem on V_H (the single-step problem of V_H)."""
    rng = np.random.default_rng(5)
    N, dl = 16, 1e-4
    u, v, sky, vis = _complete_coverage(N, dl, rng)
    opts = oi.ReconOptions(n_major=1, fista_iters=20, levels=2, n_bases=2,
                           lambda_low=0.02, lambda_full=0.03, lambda_single=0.03)
    res = oil.reconstruct_interleaved(vis, u, v, N, dl, 4.0, 1.5, opts)
    low, _ = oi.reconstruct_two_step(vis, u, v, N, dl, 4.0, 1.5, opts)
    np.testing.assert_allclose(res.node_l.objectives[0], low.objectives[0], rtol=1e-12)
    np.testing.assert_allclose(res.node_l.image, low.image, rtol=1e-12, atol=1e-14)
    in_l, in_h = partition(u, v, N, dl, 4.0, 1.5)
    single_h = oi.reconstruct_single_step(vis[in_h], u[in_h], v[in_h], N, dl, opts)
    np.testing.assert_allclose(res.node_h.objectives[0], single_h.objectives[0], rtol=1e-12)


def test_second_cycle_exchanges_the_models():
    """From cycle 2 each node's prior image is the other node's model minus
    its own: node H's cycle-2 problem equals step two's form with
    l = model_L - model_H (recomputed here from the cycle-1 models)."""
    rng = np.random.default_rng(6)
    N, dl = 16, 1e-4
    u, v, sky, vis = _complete_coverage(N, dl, rng)
    o1 = oi.ReconOptions(n_major=1, fista_iters=15, levels=2, n_bases=2)
    o2 = oi.ReconOptions(n_major=2, fista_iters=15, levels=2, n_bases=2)
    r1 = oil.reconstruct_interleaved(vis, u, v, N, dl, 4.0, 1.5, o1)
    r2 = oil.reconstruct_interleaved(vis, u, v, N, dl, 4.0, 1.5, o2)
    in_l, in_h = partition(u, v, N, dl, 4.0, 1.5)
    A = GriddedOperator(u[in_h], v[in_h], N, dl)
    res = A.residual_image(vis[in_h], r1.node_h.model)
    np.testing.assert_allclose(res, r2.node_h.residuals[1], rtol=1e-12, atol=1e-14)
    gl, gh = osv.filter_responses(N, 4.0, 1.5, r2.node_h.sigma2, r2.node_h.eta2)
    from oracle.wavelets import Dictionary
    W = Dictionary(N, 2, 2)
    lam = 0.05 * np.linalg.norm(res) * 4
    prob = osv.Problem("full", W, osv.psf_spectrum(A.psf()), res, lam, gl=gl, gh=gh,
                       l_low=r1.node_l.model - r1.node_h.model)
    assert abs(prob.objective(np.zeros((2, N, N))) - r2.node_h.objectives[1][0]) <= \
        1e-12 * abs(r2.node_h.objectives[1][0])


def test_interleaved_pipeline_recovers_the_sky_with_complete_coverage():
    """With every frequency sampled and lambda = 0, the combined image
    approaches the sky as the major cycles proceed, while each node's own
    image stays off on the other side of the band."""
    rng = np.random.default_rng(4)
    N, dl = 16, 1e-4
    u, v, sky, vis = _complete_coverage(N, dl, rng)
    errs = []
    for n_major in (1, 3, 6):
        opts = oi.ReconOptions(n_major=n_major, fista_iters=300, lambda_low=0.0,
                               lambda_full=0.0, levels=2, n_bases=2)
        out = oil.reconstruct_interleaved(vis, u, v, N, dl, 4.0, 1.5, opts)
        errs.append(np.linalg.norm(out.image - sky) / np.linalg.norm(sky))
    np.testing.assert_allclose(out.c_low + out.c_high, 1.0, atol=1e-12)
    assert errs[0] > errs[1] > errs[2], errs
    assert errs[2] <= 1e-4, errs
