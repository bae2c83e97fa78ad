"""Pins of the oracle's measurement operator and partition (CPU only)."""
import math
import os

import numpy as np
import pytest
from scipy import integrate

from oracle import gridding as og
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_es_kernel_values():
    W, beta = 7, og.es_beta(7)
    assert og.es_kernel(0.0, W, beta) == 1.0
    # edge of support: exp(beta (0 - 1)); outside: 0
    assert math.isclose(float(og.es_kernel(3.5, W, beta)), math.exp(-beta), rel_tol=1e-15)
    assert og.es_kernel(3.5000001, W, beta) == 0.0
    t = np.linspace(-3.4, 3.4, 41)
    np.testing.assert_array_equal(og.es_kernel(t, W, beta), og.es_kernel(-t, W, beta))


def test_deapodization_against_adaptive_quadrature():
    # psi(a) = int phi(t) cos(2 pi t a / Ng) dt, checked by scipy's adaptive quad
    W, beta, N = 7, og.es_beta(7), 32
    psi = og.deapodization(N, 2 * N, W, beta)
    for a in (-16, -7, 0, 5, 15):
        ref, _ = integrate.quad(
            lambda t: math.exp(beta * (math.sqrt(max(0.0, 1 - (2 * t / W) ** 2)) - 1))
            * math.cos(2 * math.pi * t * a / (2 * N)), -W / 2, W / 2,
            epsabs=0.0, epsrel=1e-13, limit=400)
        assert abs(psi[a + N // 2] - ref) <= 1e-12 * abs(ref)


def test_nudft_closed_forms():
    rng = np.random.default_rng(3)
    N, dl = 16, 1e-3
    u, v = rng.uniform(-300, 300, 50), rng.uniform(-300, 300, 50)
    # unit impulse at the phase centre: V = 1 everywhere
    img = np.zeros((N, N)); img[N // 2, N // 2] = 1.0
    np.testing.assert_allclose(og.nudft_forward(img, u, v, dl), np.ones(50), atol=1e-14)
    # point source at (p, q): V = f exp(-2 pi i (u l + v m))
    img = np.zeros((N, N)); img[3, 11] = 2.5
    l, m = (11 - N // 2) * dl, (3 - N // 2) * dl
    ref = 2.5 * np.exp(-2j * np.pi * (u * l + v * m))
    np.testing.assert_allclose(og.nudft_forward(img, u, v, dl), ref, rtol=1e-13)


def _tiny_uv(n, N, dl, rng, frac=0.49):
    # grid coordinate |g| = |u| Ng dl up to frac * Ng: reaches past the wrap
    return synth.random_uv(n, N, dl, rng, frac_of_grid=frac)


@pytest.mark.parametrize("N", [16, 32])
def test_gridded_forward_matches_nudft(N):
    """The gridded operator approximates the exact model within the ES bound
    (W = 7, 2x oversampling: ~1e-6 relative); visibilities reach the grid edge."""
    rng = np.random.default_rng(N)
    dl = 1e-3
    u, v = _tiny_uv(400, N, dl, rng)
    x = rng.standard_normal((N, N))
    A = og.GriddedOperator(u, v, N, dl)
    exact = og.nudft_forward(x, u, v, dl)
    err = np.linalg.norm(A.forward(x) - exact) / np.linalg.norm(exact)
    assert err < 3e-6, err
    # adjoint too
    y = rng.standard_normal(400) + 1j * rng.standard_normal(400)
    exact_h = og.nudft_adjoint(y, u, v, N, dl)
    err_h = np.linalg.norm(A.adjoint(y) - exact_h) / np.linalg.norm(exact_h)
    assert err_h < 3e-6, err_h


def test_gridded_error_falls_with_kernel_width():
    """Sanity of the kernel: a wider support gives a smaller error (a dropped
    term or wrong deapodization would not show this)."""
    rng = np.random.default_rng(5)
    N, dl = 16, 1e-3
    u, v = _tiny_uv(200, N, dl, rng, 0.4)
    x = rng.standard_normal((N, N))
    exact = og.nudft_forward(x, u, v, dl)
    errs = []
    for W in (3, 5, 7, 9):
        A = og.GriddedOperator(u, v, N, dl, width=W)
        errs.append(np.linalg.norm(A.forward(x) - exact) / np.linalg.norm(exact))
    assert errs[0] > errs[1] > errs[2] > errs[3]
    assert errs[3] < 1e-7


def test_adjointness():
    """<A x, y> = <x, A^H y> with <a, b> = Re sum conj(a) b, to 1e-12."""
    rng = np.random.default_rng(11)
    N, dl = 32, 1e-3
    u, v = _tiny_uv(500, N, dl, rng)
    A = og.GriddedOperator(u, v, N, dl)
    x = rng.standard_normal((N, N))
    y = rng.standard_normal(500) + 1j * rng.standard_normal(500)
    lhs = np.real(np.vdot(A.forward(x), y))
    rhs = float(np.sum(x * A.adjoint(y)))
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), 1.0)


def test_psf_properties():
    w = synth.tiny(npix=32, n_ant=6, n_dumps=4, seed=2)
    A = og.GriddedOperator(w.u[0], w.v[0], 32, w.pixel_size)
    psf = A.psf()
    assert abs(psf[16, 16] - 1.0) < 1e-5          # peak one (normalized by sum of weights)
    # point symmetry about the centre
    np.testing.assert_allclose(psf[1:, 1:], psf[1:, 1:][::-1, ::-1], atol=1e-12)
    # equals the exact A^H A delta within the gridding bound
    delta = np.zeros((32, 32)); delta[16, 16] = 1
    exact = og.nudft_adjoint(og.nudft_forward(delta, w.u[0], w.v[0], w.pixel_size),
                             w.u[0], w.v[0], 32, w.pixel_size) / w.nvis
    assert np.max(np.abs(psf - exact)) < 5e-6


def test_partition_invariant_and_band():
    w = synth.small_fp64()
    u, v = w.u[0], w.v[0]
    in_l, in_h = og.partition(u, v, w.npix, w.pixel_size, w.ell_px, w.delta_px)
    assert in_l.sum() + in_h.sum() - (in_l & in_h).sum() == w.nvis
    assert np.all(in_l | in_h)
    r = og.baseline_radius_px(u, v, w.npix, w.pixel_size)
    both = in_l & in_h
    assert np.all(np.abs(r[both] - w.ell_px) <= w.delta_px)
    assert abs(r.max() - w.npix / 3.0) < 1e-9       # pixel size = 1/(3 max|uv|)


def test_partition_table_invariant_from_paper():
    """Every row of the paper's partition table satisfies
    |V_L| + |V_H| - |V_L n V_H| = |V| = 249600 (Sects. 4.1, 4.2), which pins
    the reading that overlap rows belong to both partitions."""
    rows = np.loadtxt(os.path.join(GOLDEN, "partition_table.txt"))
    assert rows.shape == (9, 5)
    np.testing.assert_array_equal(rows[:, 2] + rows[:, 3] - rows[:, 4], 249600)


def test_workload_row_counts():
    # 32 antennas, 64 dumps, no autocorrelations: 496 * 64 rows
    w = synth.small_fp64()
    assert w.nvis == 31744 and w.npix == 128
