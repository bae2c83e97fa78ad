"""Pins of the oracle's filters, gradients, Lipschitz constants, FISTA and
noise estimators (CPU only)."""
import math

import numpy as np
import pytest

from oracle import solver as osv
from oracle.wavelets import Dictionary


def test_soft_threshold_closed_form():
    x = np.array([-3.0, -1.0, -0.5, 0.0, 0.5, 1.0, 2.5])
    np.testing.assert_array_equal(osv.soft_threshold(x, 1.0),
                                  [-2.0, 0.0, 0.0, 0.0, 0.0, 0.0, 1.5])


@pytest.mark.parametrize("sigma2,eta2", [(1.0, 1.2), (2.5e-4, 2.5e-7)])
def test_filter_constraints(sigma2, eta2):
    """Sect. 3.3: eta^2 g_L^2 + sigma^2 g_H^2 = 1 everywhere, the outer values,
    and continuity at r = ell +- delta (Fig. FilterResponse uses sigma^2 = 1,
    eta^2 = 1.2)."""
    N, ell, delta = 64, 12.0, 3.0
    gl, gh = osv.filter_responses(N, ell, delta, sigma2, eta2)
    np.testing.assert_allclose(eta2 * gl ** 2 + sigma2 * gh ** 2, 1.0, rtol=1e-13)
    r = osv.radial_frequency(N)
    np.testing.assert_array_equal(gh[r < ell - delta], 0.0)
    np.testing.assert_array_equal(gl[r > ell + delta], 0.0)
    np.testing.assert_allclose(gh[r > ell + delta], 1 / math.sqrt(sigma2), rtol=1e-15)
    np.testing.assert_allclose(gl[r < ell - delta], 1 / math.sqrt(eta2), rtol=1e-15)
    # band formula at the edges reaches the outer values (continuity)
    for edge, want_l, want_h in [(ell - delta, 1 / math.sqrt(eta2), 0.0),
                                 (ell + delta, 0.0, 1 / math.sqrt(sigma2))]:
        s = math.sin(math.pi * (edge - ell) / (2 * delta))
        a = 1 / math.sqrt(eta2 * (1 - s) ** 2 + sigma2 * (1 + s) ** 2)
        assert abs(a * (1 - s) - want_l) < 1e-12 * max(1, want_l)
        assert abs(a * (1 + s) - want_h) < 1e-12 * max(1, want_h)
    # g_H rises and g_L falls across the band
    band = (r >= ell - delta) & (r <= ell + delta)
    order = np.argsort(r[band])
    assert np.all(np.diff(gh[band][order]) >= -1e-12)
    assert np.all(np.diff(gl[band][order]) <= 1e-12)


def _symmetric_psf(N, rng):
    h = rng.standard_normal((N, N))
    h = h + h[(-np.arange(N)) % N][:, (-np.arange(N)) % N]     # h[-a] = h[a]
    return np.fft.fftshift(h)


def test_spectral_filter_equals_direct_circular_convolution():
    rng = np.random.default_rng(1)
    N = 12
    psf = _symmetric_psf(N, rng)
    x = rng.standard_normal((N, N))
    Hhat = osv.psf_spectrum(psf)
    y = osv.apply_spectral(x, Hhat)
    h = np.fft.ifftshift(psf)
    direct = np.zeros((N, N))
    for p in range(N):
        for q in range(N):
            for a in range(N):
                for b in range(N):
                    direct[p, q] += h[(p - a) % N, (q - b) % N] * x[a, b]
    np.testing.assert_allclose(y, direct, atol=1e-12)


def _small_problem(kind, N=16, M=3, J=2, seed=0, lam=0.05):
    rng = np.random.default_rng(seed)
    W = Dictionary(N, M, J)
    psf = _symmetric_psf(N, rng) * 0.1
    psf[N // 2, N // 2] += 1.0
    Hhat = osv.psf_spectrum(psf)
    res = rng.standard_normal((N, N))
    if kind == "low":
        return osv.Problem("low", W, Hhat, res, lam)
    gl, gh = osv.filter_responses(N, 3.0, 1.5, 0.7, 0.2)
    return osv.Problem("full", W, Hhat, res, lam, gl=gl, gh=gh,
                       l_low=rng.standard_normal((N, N)))


@pytest.mark.parametrize("kind", ["low", "full"])
def test_gradient_finite_differences(kind):
    prob = _small_problem(kind)
    rng = np.random.default_rng(7)
    a = rng.standard_normal((prob.W.M, 16, 16))
    g = prob.grad(a)
    for _ in range(6):
        d = rng.standard_normal(a.shape)
        eps = 1e-5
        fd = (prob.smooth(a + eps * d) - prob.smooth(a - eps * d)) / (2 * eps)
        an = float(np.sum(g * d))
        assert abs(fd - an) <= 1e-7 * max(abs(an), 1.0), (fd, an)


@pytest.mark.parametrize("kind", ["low", "full"])
def test_quadratic_expansion(kind):
    """f(alpha) = <x, K x> - 2 <b, x> + c0 with x = W alpha, K^ the normal
    spectrum, b = H G_H^2 i~ + G_L^2 l (the identity the CUDA minor cycle
    evaluates in the Fourier domain)."""
    prob = _small_problem(kind)
    rng = np.random.default_rng(2)
    a = rng.standard_normal((prob.W.M, 16, 16))
    x = prob.W.synth(a)
    Kx = osv.apply_spectral(x, prob.normal_spectrum())
    if kind == "low":
        b = prob.H(prob.residual)
        c0 = np.sum(prob.residual ** 2)
    else:
        b = prob.H(prob.GH(prob.GH(prob.residual))) + prob.GL(prob.GL(prob.l_low))
        c0 = np.sum(prob.GH(prob.residual) ** 2) + np.sum(prob.GL(prob.l_low) ** 2)
    val = np.sum(x * Kx) - 2 * np.sum(b * x) + c0
    assert abs(val - prob.smooth(a)) <= 1e-10 * abs(prob.smooth(a))


@pytest.mark.parametrize("kind", ["low", "full"])
def test_lipschitz_power_iteration_matches_closed_form(kind):
    """Sect. 3.4: theta = 2 M max|K^| for M orthogonal bases and circular
    convolutions; the power iteration through W must agree.  The PSF spectrum
    here is radial and decreasing so the top eigenvalue is well separated."""
    N, M, J = 16, 3, 2
    W = Dictionary(N, M, J)
    r = osv.radial_frequency(N)
    Hhat = np.exp(-0.5 * r ** 2)
    res = np.zeros((N, N))
    if kind == "low":
        prob = osv.Problem("low", W, Hhat, res, 0.0)
    else:
        # band [0.5, 1.5]: only the DC term gets the full 1/eta^2
        gl, gh = osv.filter_responses(N, 1.0, 0.5, 1.0, 1.2)
        prob = osv.Problem("full", W, Hhat, res, 0.0, gl=gl, gh=gh, l_low=res)
    closed = prob.lipschitz_closed_form()
    power = prob.lipschitz_power_iteration(iters=300)
    assert abs(power - closed) <= 1e-10 * closed, (power, closed)


@pytest.mark.parametrize("p", [1, 2, 5, 8])
def test_fista_one_step_exact_for_orthonormal_identity(p):
    """With one orthonormal basis (M = 1) and H = I, the minimiser of
    ||i - Psi a||^2 + lam ||a||_1 is soft(Psi^H i, lam/2), and FISTA from zero
    with mu = 1/theta = 1/2 lands on it in one step and stays."""
    from oracle.wavelets import dwt2
    N, J, lam = 16, 3, 0.3
    rng = np.random.default_rng(p)
    res = rng.standard_normal((N, N))

    class OneBasis(Dictionary):
        def synth(self, alpha):
            from oracle.wavelets import idwt2
            return idwt2(alpha[0], p, self.levels)

        def analysis(self, x):
            return dwt2(x, p, self.levels)[None]

    W = OneBasis(N, 1, J)
    prob = osv.Problem("low", W, np.ones((N, N // 2 + 1)), res, lam)
    assert prob.lipschitz_closed_form() == 2.0
    star = osv.soft_threshold(dwt2(res, p, J), lam / 2)
    r1 = osv.fista(prob, 1)
    np.testing.assert_allclose(r1.beta[0], star, atol=1e-12)
    r5 = osv.fista(prob, 5)
    np.testing.assert_allclose(r5.beta[0], star, atol=1e-12)


def _c1_like_problem(kind="low", N=32):
    from oracle.gridding import GriddedOperator
    import synth
    w = synth.tiny(npix=N, n_ant=10, n_dumps=8, seed=4)
    A = GriddedOperator(w.u[0], w.v[0], N, w.pixel_size)
    res = A.dirty(w.vis[0])
    Hhat = osv.psf_spectrum(A.psf())
    W = Dictionary(N, 8, 3)
    lam = 0.05 * np.linalg.norm(res) * 2
    if kind == "low":
        return osv.Problem("low", W, Hhat, res, lam)
    gl, gh = osv.filter_responses(N, 3.0, 1.5, osv.sigma2_hat(res), 1e-3 * osv.sigma2_hat(res))
    return osv.Problem("full", W, Hhat, res, lam, gl=gl, gh=gh, l_low=0.5 * res)


@pytest.mark.parametrize("kind", ["low", "full"])
def test_ista_objective_monotone(kind):
    """Without momentum the proximal gradient objective never increases."""
    prob = _c1_like_problem(kind)
    r = osv.fista(prob, 40, momentum=False)
    F = np.array(r.objective)
    assert np.all(np.diff(F) <= 1e-12 * np.abs(F[1:]))
    assert F[-1] < F[0]


def test_fista_rate_bound_and_kkt():
    """Beck-Teboulle: F(beta_k) - F* <= 2 theta ||beta_0 - a*||^2 / (k+1)^2;
    at the (long-run) solution the KKT conditions hold."""
    N = 16
    prob = _small_problem("low", N=N, M=2, J=2, seed=3, lam=0.3)
    theta = prob.lipschitz_closed_form()
    long = osv.fista(prob, 4000, theta=theta)
    a_star = long.beta
    F_star = min(long.objective)
    short = osv.fista(prob, 150, theta=theta)
    d0 = float(np.sum(a_star ** 2))        # beta_0 = 0
    for k in range(1, 151):
        assert short.objective[k] - F_star <= 2 * theta * d0 / (k + 1) ** 2 + 1e-9
    # KKT: grad_i = -lam sign(beta_i) on the support, |grad_i| <= lam off it
    g = prob.grad(a_star)
    on = a_star != 0
    # (first-order accuracy of a 4000-iteration run: 1e-3 relative)
    assert np.max(np.abs(g[on] + prob.lam * np.sign(a_star[on]))) < 1e-3 * prob.lam
    assert np.max(np.abs(g[~on])) <= prob.lam * (1 + 1e-3)
    # and the objective has settled
    assert abs(long.objective[-1] - long.objective[-2]) < 1e-10 * abs(long.objective[-1])


def test_full_step_reduces_to_scaled_low_step():
    """With g_L = 0 and g_H = 1/sigma everywhere, the full-resolution problem
    is the low-resolution one divided by sigma^2: same FISTA iterates when
    lambda is scaled likewise."""
    N, M, J = 16, 3, 2
    prob_low = _small_problem("low", N=N, M=M, J=J, seed=8, lam=0.2)
    s2 = 0.37
    shape = prob_low.Hhat.shape
    prob_full = osv.Problem("full", prob_low.W, prob_low.Hhat, prob_low.residual,
                            0.2 / s2, gl=np.zeros(shape),
                            gh=np.full(shape, 1 / math.sqrt(s2)),
                            l_low=np.random.default_rng(0).standard_normal((N, N)))
    a = osv.fista(prob_low, 25)
    b = osv.fista(prob_full, 25)
    np.testing.assert_allclose(a.beta, b.beta, atol=1e-10)
    np.testing.assert_allclose(np.array(a.objective) / s2, b.objective, rtol=1e-10)


def test_sigma2_hat_exact_cases():
    N = 20
    assert osv.sigma2_hat(np.full((N, N), 4.0)) == 0.0
    # ramp along x: each window holds 5 consecutive integers 5 times: var 2
    ramp = np.tile(np.arange(N, dtype=float), (N, 1))
    assert abs(osv.sigma2_hat(ramp) - 2.0) < 1e-12
    # checkerboard +-1: every window is 13 of one sign, 12 of the other
    cb = (-1.0) ** np.add.outer(np.arange(N), np.arange(N))
    assert abs(osv.sigma2_hat(cb) - (1 - 1 / 625)) < 1e-12
    assert osv.eta2_hat(2.0) == 2e-3
