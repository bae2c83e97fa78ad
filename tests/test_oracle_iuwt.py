"""Pins of the oracle's IUWT dictionary (App. A.1's alternative dictionary;
Sect. 3.4's power-iteration step size) against closed forms, brute force and
invariants (CPU)."""
import numpy as np
import pytest

from oracle import iuwt as oi
from oracle import solver as osv


def test_b3_filter():
    assert np.isclose(oi.B3.sum(), 1.0)
    np.testing.assert_array_equal(oi.B3, oi.B3[::-1])
    np.testing.assert_allclose(oi.B3 * 16, [1, 4, 6, 4, 1])


@pytest.mark.parametrize("j", [1, 2, 3])
def test_smoothing_equals_direct_convolution(j):
    """h_j * c by explicit loops over the 25 taps (periodic), tiny N."""
    N = 16
    c = np.random.default_rng(j).standard_normal((N, N))
    d = 1 << (j - 1)
    want = np.zeros((N, N))
    for p in range(N):
        for q in range(N):
            for a in range(5):
                for b in range(5):
                    want[p, q] += oi.B3[a] * oi.B3[b] * c[(p + (a - 2) * d) % N, (q + (b - 2) * d) % N]
    np.testing.assert_allclose(oi.smooth(c, j), want, rtol=0, atol=1e-13)


@pytest.mark.parametrize("J", [1, 3, 4])
def test_planes_sum_to_the_image(J):
    """The IUWT's defining property: w_1 + ... + w_J + c_J = x."""
    x = np.random.default_rng(J).standard_normal((32, 32))
    np.testing.assert_allclose(oi.iuwt(x, J).sum(axis=0), x, rtol=0, atol=1e-13)


@pytest.mark.parametrize("J", [1, 2, 4])
def test_adjoint(J):
    rng = np.random.default_rng(10 + J)
    x = rng.standard_normal((32, 32))
    a = rng.standard_normal((J + 1, 32, 32))
    lhs = float(np.sum(oi.iuwt(x, J) * a))
    rhs = float(np.sum(x * oi.iuwt_adjoint(a, J)))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_frame_symbol_matches_the_operator():
    """T^H T is circulant: its response to a unit impulse has the DFT given by
    frame_symbol (independent of both routines' internals)."""
    N, J = 32, 3
    delta = np.zeros((N, N))
    delta[0, 0] = 1.0
    resp = oi.iuwt_adjoint(oi.iuwt(delta, J), J)
    np.testing.assert_allclose(np.fft.rfft2(resp).real, oi.frame_symbol(N, J), atol=1e-13)
    assert np.max(np.abs(np.fft.rfft2(resp).imag)) < 1e-13


def test_not_a_tight_frame():
    """W W^H = T^H T is not a multiple of the identity (why the closed form of
    Sect. 3.4 does not apply)."""
    S = oi.frame_symbol(32, 4)
    assert S.max() - S.min() > 0.1


@pytest.mark.parametrize("kind", ["low", "full"])
def test_power_iteration_reaches_the_fourier_value(kind):
    """Sect. 3.4's power iteration through W = T^H equals the Fourier-space
    value max_k K(k) S(k) (all operators circulant) on a separated spectrum."""
    N, J = 16, 2
    W = oi.IUWTDictionary(N, J)
    r = osv.radial_frequency(N)
    Hhat = np.exp(-0.5 * r ** 2)
    res = np.zeros((N, N))
    if kind == "low":
        prob = osv.Problem("low", W, Hhat, res, 0.0)
    else:
        gl, gh = osv.filter_responses(N, 1.0, 0.5, 1.0, 1.2)
        prob = osv.Problem("full", W, Hhat, res, 0.0, gl=gl, gh=gh, l_low=res)
    want = oi.lipschitz_fourier(prob.normal_spectrum(), N, J)
    got = prob.lipschitz_power_iteration(iters=400)
    assert abs(got - want) <= 1e-10 * want, (got, want)
    # the Daubechies closed form would be wrong here
    assert abs(prob.lipschitz_closed_form() - want) > 1e-3 * want


def test_ista_with_iuwt_is_monotone_and_fista_converges():
    N, J = 32, 3
    rng = np.random.default_rng(5)
    W = oi.IUWTDictionary(N, J)
    r = osv.radial_frequency(N)
    Hhat = np.exp(-0.5 * (r / 6.0) ** 2)
    res = rng.standard_normal((N, N))
    prob = osv.Problem("low", W, Hhat, res, 0.05)
    theta = oi.lipschitz_fourier(prob.normal_spectrum(), N, J)
    ista = osv.fista(prob, 60, theta=theta, momentum=False)
    assert np.all(np.diff(ista.objective) <= 1e-12 * abs(ista.objective[0]))
    fast = osv.fista(prob, 300, theta=theta)
    assert fast.objective[-1] <= ista.objective[-1]
