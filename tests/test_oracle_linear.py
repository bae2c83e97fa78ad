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
