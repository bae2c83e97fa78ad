"""Pins of the oracle's linear reading of the PSF operator (the minor
cycle's H as the linear convolution that A^H A / sum(w) is on the N x N
field) and of why it is needed: the circular N x N reading makes the major
cycle diverge on a wide PSF (CPU)."""
import numpy as np
import pytest

import synth
from oracle import gridding as og
from oracle import imaging as oi
from oracle import solver as osv


def _coverage(N=32, n=400, seed=0):
    rng = np.random.default_rng(seed)
    u, v = synth.random_uv(n, N, 1e-3, rng, frac_of_grid=0.3)
    return u, v, 1e-3


def test_linear_convolution_by_brute_force():
    """apply_linear equals the explicit double sum over the 2N x 2N PSF."""
    N = 8
    rng = np.random.default_rng(1)
    psf2 = rng.standard_normal((2 * N, 2 * N))
    psf2 = 0.5 * (psf2 + np.roll(psf2[::-1, ::-1], 1, axis=(0, 1)))   # point-symmetric about N
    x = rng.standard_normal((N, N))
    H2 = np.fft.rfft2(np.fft.ifftshift(psf2)).real
    want = np.zeros((N, N))
    for p in range(N):
        for q in range(N):
            for a in range(N):
                for b in range(N):
                    want[p, q] += psf2[N + p - a, N + q - b] * x[a, b]
    np.testing.assert_allclose(osv.apply_linear(x, H2), want, atol=1e-12)


def test_linear_reading_is_the_normal_operator():
    """H (linear, from the 2N-field PSF) equals A^H A / sum(w) on images of
    the N x N field to the gridding accuracy; the circular reading does not."""
    N = 32
    u, v, dl = _coverage(N)
    A = og.GriddedOperator(u, v, N, dl)
    H2 = osv.psf_spectrum(og.GriddedOperator(u, v, 2 * N, dl).psf())
    H1 = osv.psf_spectrum(A.psf())
    x = np.random.default_rng(2).standard_normal((N, N))
    truth = A.dirty(A.forward(x))
    lin = osv.apply_linear(x, H2)
    circ = osv.apply_spectral(x, H1)
    e_lin = np.linalg.norm(lin - truth) / np.linalg.norm(truth)
    e_circ = np.linalg.norm(circ - truth) / np.linalg.norm(truth)
    assert e_lin <= 1e-5, e_lin
    assert e_circ > 1e-2, e_circ


def test_linear_closed_form_bounds_the_power_iteration():
    N = 16
    u, v, dl = _coverage(N, 300, 3)
    A = og.GriddedOperator(u, v, N, dl)
    H2 = osv.psf_spectrum(og.GriddedOperator(u, v, 2 * N, dl).psf())
    from oracle.wavelets import Dictionary
    W = Dictionary(N, 2, 2)
    res = np.zeros((N, N))
    prob = osv.Problem("low", W, osv.psf_spectrum(A.psf()), res, 0.0, Hhat2=H2)
    bound = prob.lipschitz_closed_form()
    power = prob.lipschitz_power_iteration(iters=300)
    assert power <= bound * (1 + 1e-12)   # a valid step size for FISTA
    assert power >= 0.2 * bound           # and not a vacuous one (0.34 here, N = 16)


@pytest.mark.parametrize("conv,converges", [("linear", True), ("circular", False)])
def test_major_cycle_convergence_on_a_wide_psf(conv, converges):
    """Single-step major cycles on a paper-like sky at 128 px: with the
    linear reading the residual falls with every cycle after the first; the
    circular reading lets it grow (the minor cycle under-estimates the
    low-frequency gain of A^H A and over-corrects)."""
    w = synth.paper_like(128, seed=0)
    ro = oi.ReconOptions(n_major=5, fista_iters=60, lambda_single=0.01, convolution=conv)
    r = oi.reconstruct_single_step(w.vis[0], w.u[0], w.v[0], 128, w.pixel_size, ro)
    norms = [float(np.linalg.norm(x)) for x in r.residuals]
    if converges:
        assert all(b < a for a, b in zip(norms[1:], norms[2:])), norms
        assert norms[-1] < 0.1 * norms[0]
    else:
        assert norms[-1] > norms[1], norms


def test_splitmix64_published_outputs():
    """The generator of the power iteration's start vector: the first outputs
    of SplitMix64 from state 0, and the first from state 1234567, as the
    generator's reference implementation prints them."""
    np.testing.assert_array_equal(
        osv.splitmix64(3, 0),
        np.array([0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F], dtype=np.uint64))
    assert int(osv.splitmix64(1, 1234567)[0]) == 6457827717110365317
    s = osv.power_start((2, 4, 4))
    assert s.shape == (2, 4, 4) and np.all(s >= -1.0) and np.all(s < 1.0)


def test_linear_step_size_is_the_power_estimate_below_the_bound():
    """The linear reading's step size: 100 power iterations from the fixed
    start, within 1 % of 2 M lambda_max (dense eigenvalue of the N x N
    operator, M lambda_max(K) since W W^H = M I) and below the bound."""
    N, M = 12, 2
    u, v, dl = _coverage(N, 200, 5)
    A = og.GriddedOperator(u, v, N, dl)
    H2 = osv.psf_spectrum(og.GriddedOperator(u, v, 2 * N, dl).psf())
    from oracle.wavelets import Dictionary
    W = Dictionary(N, M, 2)
    prob = osv.Problem("low", W, osv.psf_spectrum(A.psf()), np.zeros((N, N)), 0.0, Hhat2=H2)
    K = np.stack([prob.H(prob.H(e.reshape(N, N))).ravel() for e in np.eye(N * N)], axis=1)
    exact = 2.0 * M * float(np.linalg.eigvalsh(0.5 * (K + K.T))[-1])
    theta = oi._step_size(prob, None)
    assert theta <= exact * (1 + 1e-9)
    assert theta >= 0.99 * exact
    assert exact <= prob.lipschitz_closed_form()
    assert oi._step_size(prob, 3.5) == 3.5   # computed once per step
