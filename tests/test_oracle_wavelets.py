"""Pins of the oracle's Daubechies filters, DWT and dictionary (CPU only)."""
import math

import numpy as np
import pytest

from oracle import wavelets as ow

S2 = math.sqrt(2.0)


def test_db1_db2_db3_closed_forms():
    np.testing.assert_array_equal(ow.daubechies_lowpass(1), (1 / S2, 1 / S2))
    r3 = math.sqrt(3.0)
    db2 = np.array([1 + r3, 3 + r3, 3 - r3, 1 - r3]) / (4 * S2)
    np.testing.assert_allclose(ow.daubechies_lowpass(2), db2, atol=1e-15)
    # Daubechies' closed form for 3 vanishing moments
    a = math.sqrt(10.0)
    b = math.sqrt(5 + 2 * a)
    db3 = np.array([1 + a + b, 5 + a + 3 * b, 10 - 2 * a + 2 * b,
                    10 - 2 * a - 2 * b, 5 + a - 3 * b, 1 + a - b]) / (16 * S2)
    np.testing.assert_allclose(ow.daubechies_lowpass(3), db3, atol=1e-15)


@pytest.mark.parametrize("p", range(1, 9))
def test_filter_identities(p):
    h = np.array(ow.daubechies_lowpass(p))
    g = ow.highpass(h)
    L = h.size
    assert L == 2 * p
    assert abs(h.sum() - S2) < 1e-14
    for m in range(p):
        s = sum(h[k] * h[k + 2 * m] for k in range(L - 2 * m))
        assert abs(s - (1.0 if m == 0 else 0.0)) < 1e-14
    # p vanishing moments of the wavelet: sum g_k (k/L)^j = 0, j < p
    for j in range(p):
        assert abs(sum(g[k] * (k / L) ** j for k in range(L))) < 1e-13
    # the next moment does not vanish
    assert abs(sum(g[k] * (k / L) ** p for k in range(L))) > 1e-6


@pytest.mark.parametrize("p", [1, 4, 8])
@pytest.mark.parametrize("n", [2, 4, 8, 16, 32])
def test_periodized_matrix_orthogonal(p, n):
    """Periodization keeps the transform orthogonal even when n < 2p."""
    T = ow.analysis_matrix(p, n)
    np.testing.assert_allclose(T @ T.T, np.eye(n), atol=1e-13)


def test_haar_2x2_hand_values():
    # rows then columns with h = (1, 1)/sqrt2, g = (1, -1)/sqrt2:
    # LL = 10/2, low-y/high-x = -1, high-y/low-x = -2, high/high = 0
    y = ow.dwt2(np.array([[1.0, 2.0], [3.0, 4.0]]), 1, 1)
    np.testing.assert_allclose(y, [[5.0, -1.0], [-2.0, 0.0]], atol=1e-15)


def test_shift_equivariance_one_level():
    """Shifting the input by 2 pixels shifts each subband by 1 (periodic)."""
    rng = np.random.default_rng(0)
    x = rng.standard_normal((16, 16))
    y0 = ow.dwt2(x, 5, 1)
    y1 = ow.dwt2(np.roll(x, (2, 2), axis=(0, 1)), 5, 1)
    for sl in [(slice(0, 8), slice(0, 8)), (slice(0, 8), slice(8, 16)),
               (slice(8, 16), slice(0, 8)), (slice(8, 16), slice(8, 16))]:
        np.testing.assert_allclose(y1[sl], np.roll(y0[sl], (1, 1), axis=(0, 1)), atol=1e-13)


@pytest.mark.parametrize("N,J", [(16, 4), (32, 4), (64, 3)])
def test_perfect_reconstruction_and_dictionary(N, J):
    rng = np.random.default_rng(N)
    x = rng.standard_normal((N, N))
    for p in range(1, 9):
        np.testing.assert_allclose(ow.idwt2(ow.dwt2(x, p, J), p, J), x, atol=1e-12)
        # Parseval: orthonormal
        assert abs(np.sum(ow.dwt2(x, p, J) ** 2) - np.sum(x ** 2)) < 1e-10 * np.sum(x ** 2)
    W = ow.Dictionary(N, 8, J)
    np.testing.assert_allclose(W.synth(W.analysis(x)), 8 * x, atol=1e-11)   # W W^H = M I
    a = rng.standard_normal((8, N, N))
    # adjoint pair: <W a, x> = <a, W^H x>
    assert abs(np.sum(W.synth(a) * x) - np.sum(a * W.analysis(x))) < 1e-10 * N * N


def test_constant_image_only_in_approximation():
    """A constant image has zero detail coefficients and its level-J
    approximation is the constant times 2^J (orthonormal scaling)."""
    N, J = 32, 4
    x = np.full((N, N), 3.0)
    for p in range(1, 9):
        y = ow.dwt2(x, p, J)
        n = N >> J
        np.testing.assert_allclose(y[:n, :n], 3.0 * 2 ** J, atol=1e-12)
        y[:n, :n] = 0
        assert np.max(np.abs(y)) < 1e-12
