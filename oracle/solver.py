"""Oracle: the minor-cycle problems and FISTA.

Test infrastructure only (see ``oracle/__init__``).

Operators on N x N real images (all circulant, Sect. 3.4 allows circular
convolutions):
  H x   = PSF convolution:  irfft2( H^ . rfft2(x) ),  H^ = rfft2(ifftshift(psf))
          (psf is real and point-symmetric, so H^ is real and H^H = H),
  G_L x = irfft2( g_L(r) . rfft2(x) ),  G_H x likewise, with r the radial
          frequency in pixel units of the N x N DFT grid (Sect. 3.3).

Step one (Sect. 3.2, Eq. LowRes):
  f_L(alpha) = || i~_L - H_L W alpha ||^2,
  grad f_L   = 2 W^H H_L^H (H_L W alpha - i~_L)                    (Eq. GradL)
Step two (Sect. 3.3, Eq. FullRes):
  f_H(alpha) = || G_H (i~_H - H_H W alpha) ||^2 + || G_L (l_L - W alpha) ||^2,
  grad f_H   = 2 W^H ( H_H^H G_H^H G_H (H_H W alpha - i~_H)
                      + G_L^H G_L (W alpha - l_L) )                 (Eq. GradH)
Both are minimised with an added lambda ||alpha||_1 by FISTA (Algorithm 1),
step mu = 1/theta with theta the Lipschitz constant of the gradient (Sect. 3.4).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Callable, List, Optional

import numpy as np
from numpy.lib.stride_tricks import sliding_window_view

from .wavelets import Dictionary


# ---------------------------------------------------------------------------
# circulant operators
# ---------------------------------------------------------------------------
def radial_frequency(npix: int) -> np.ndarray:
    """r = sqrt(kx^2 + ky^2) on the rfft2 half-plane, k in pixel units."""
    ky = np.fft.fftfreq(npix) * npix
    kx = np.fft.rfftfreq(npix) * npix
    return np.sqrt(ky[:, None] ** 2 + kx[None, :] ** 2)


def apply_spectral(x: np.ndarray, response: np.ndarray) -> np.ndarray:
    """Circular filter with a real spectral response on the rfft2 half-plane."""
    return np.fft.irfft2(response * np.fft.rfft2(x), s=x.shape)


def apply_linear(x: np.ndarray, response2: np.ndarray) -> np.ndarray:
    """Linear convolution of an N x N image with the PSF whose 2N x 2N
    half-plane spectrum is response2, restricted to the image: zero-pad x to
    2N x 2N, filter circularly there (offsets within +-N never wrap), keep
    the first N x N."""
    n = x.shape[0]
    xp = np.zeros((2 * n, 2 * n))
    xp[:n, :n] = x
    return np.fft.irfft2(response2 * np.fft.rfft2(xp), s=xp.shape)[:n, :n]


def psf_spectrum(psf: np.ndarray) -> np.ndarray:
    """H^ = DFT of the PSF centred at pixel (N/2, N/2); real by symmetry, so
    the (rounding-level) imaginary part is dropped."""
    return np.fft.rfft2(np.fft.ifftshift(psf)).real


def filter_responses(npix: int, ell: float, delta: float, sigma2: float, eta2: float):
    """g_L(r), g_H(r) of Sect. 3.3:
      r > ell + delta:  |g_H|^2 = 1/sigma^2, g_L = 0
      r < ell - delta:  g_H = 0, |g_L|^2 = 1/eta^2
      inside the band:  g_L = a(r)(1 - s), g_H = a(r)(1 + s),
                        s = sin(pi (r - ell) / (2 delta)),
                        a(r) such that eta^2 g_L^2 + sigma^2 g_H^2 = 1.
    The responses are taken non-negative (the paper fixes only |g|^2 outside
    the band); the printed g_L(u) in the first condition is read as g_L(r)."""
    if not (sigma2 > 0 and eta2 > 0):
        raise ValueError("filters need sigma^2 > 0 and eta^2 > 0")
    r = radial_frequency(npix)
    gl = np.zeros_like(r)
    gh = np.zeros_like(r)
    hi = r > ell + delta
    lo = r < ell - delta
    band = ~(hi | lo)
    gh[hi] = 1.0 / math.sqrt(sigma2)
    gl[lo] = 1.0 / math.sqrt(eta2)
    s = np.sin(np.pi * (r[band] - ell) / (2.0 * delta))
    a = 1.0 / np.sqrt(eta2 * (1.0 - s) ** 2 + sigma2 * (1.0 + s) ** 2)
    gl[band] = a * (1.0 - s)
    gh[band] = a * (1.0 + s)
    return gl, gh


# ---------------------------------------------------------------------------
# the smooth parts, their gradients and Lipschitz constants
# ---------------------------------------------------------------------------
@dataclass
class Problem:
    """One minor-cycle problem: f(alpha) + lam ||alpha||_1.

    ``kind`` is "low" (Eq. LowRes; also the single-step problem) or "full"
    (Eq. FullRes).  Spectra live on the rfft2 half-plane."""

    kind: str
    W: Dictionary
    Hhat: np.ndarray
    residual: np.ndarray                 # i~_n
    lam: float
    gl: Optional[np.ndarray] = None      # full step only
    gh: Optional[np.ndarray] = None
    l_low: Optional[np.ndarray] = None   # l_{L_n}, full step only
    Hhat2: Optional[np.ndarray] = None   # 2N PSF spectrum: H is a linear convolution

    def H(self, x):
        """The PSF operator: circular convolution on N x N (Sect. 3.4's
        reading), or, given the 2N x 2N PSF's spectrum, the linear
        convolution that A^H A / sum(w) is on images of the N x N field."""
        if self.Hhat2 is not None:
            return apply_linear(x, self.Hhat2)
        return apply_spectral(x, self.Hhat)

    def GL(self, x):
        return apply_spectral(x, self.gl)

    def GH(self, x):
        return apply_spectral(x, self.gh)

    def smooth(self, alpha) -> float:
        x = self.W.synth(alpha)
        if self.kind == "low":
            r = self.residual - self.H(x)
            return float(np.sum(r * r))
        a = self.GH(self.residual - self.H(x))
        b = self.GL(self.l_low - x)
        return float(np.sum(a * a) + np.sum(b * b))

    def objective(self, alpha) -> float:
        return self.smooth(alpha) + self.lam * float(np.sum(np.abs(alpha)))

    def grad(self, alpha) -> np.ndarray:
        x = self.W.synth(alpha)
        if self.kind == "low":                                   # Eq. GradL
            return 2.0 * self.W.analysis(self.H(self.H(x) - self.residual))
        inner = self.H(self.GH(self.GH(self.H(x) - self.residual)))  # Eq. GradH
        inner = inner + self.GL(self.GL(x - self.l_low))
        return 2.0 * self.W.analysis(inner)

    # Sect. 3.4: theta = 2 lambda_max(W^H (...) W); closed form for M
    # concatenated orthogonal bases and circular convolutions
    def normal_spectrum(self) -> np.ndarray:
        if self.kind == "low":
            return self.Hhat ** 2
        return (self.gh * self.Hhat) ** 2 + self.gl ** 2

    def lipschitz_closed_form(self) -> float:
        """2 M max K^ (exact for circulant operators); with the linear
        convolution an upper bound: ||P H P^T|| <= max|H2^|, so
        2 M (max g_H^2 max H2^2 + max g_L^2) (full) or 2 M max H2^2."""
        if self.Hhat2 is not None:
            h2 = float(np.max(self.Hhat2 ** 2))
            if self.kind == "low":
                return 2.0 * self.W.M * h2
            return 2.0 * self.W.M * (float(np.max(self.gh ** 2)) * h2 + float(np.max(self.gl ** 2)))
        return 2.0 * self.W.M * float(np.max(self.normal_spectrum()))

    def normal_op(self, alpha) -> np.ndarray:
        """W^H (H^H G_H^H G_H H + G_L^H G_L) W alpha (or W^H H^H H W alpha)."""
        x = self.W.synth(alpha)
        if self.kind == "low":
            return self.W.analysis(self.H(self.H(x)))
        return self.W.analysis(self.H(self.GH(self.GH(self.H(x)))) + self.GL(self.GL(x)))

    def lipschitz_power_iteration(self, iters: int = 200, seed: int = 0,
                                  tol: float = 0.0,
                                  start: Optional[np.ndarray] = None) -> float:
        """theta = 2 lambda_max by power iteration (Sect. 3.4, the method the
        paper names for dictionaries without the closed form), from `start`
        (else a normal random vector drawn with `seed`)."""
        shape = (self.W.M, self.W.npix, self.W.npix)
        if start is None:
            v = np.random.default_rng(seed).standard_normal(shape)
        else:
            v = np.array(start, dtype=np.float64).reshape(shape)
        v /= np.linalg.norm(v)
        lam = 0.0
        for _ in range(iters):
            w = self.normal_op(v)
            new = float(np.vdot(v, w))        # Rayleigh quotient
            v = w / np.linalg.norm(w)
            if tol and abs(new - lam) <= tol * abs(new):
                lam = new
                break
            lam = new
        return 2.0 * lam


def splitmix64(n: int, seed: int) -> np.ndarray:
    """Outputs 1..n of the SplitMix64 generator (Steele, Lea and Flood, 2014)
    from state `seed`: the state advances by the odd constant 0x9E3779B97F4A7C15
    and each output is the state through the two xor-shift-multiply rounds
    (30, 0xBF58476D1CE4E5B9; 27, 0x94D049BB133111EB) and a final xor-shift by
    31, all modulo 2^64."""
    k = np.arange(1, n + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed) + np.uint64(0x9E3779B97F4A7C15) * k
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
    return z ^ (z >> np.uint64(31))


# The start vector of the power iterations that set the step size where the
# closed form does not hold: SplitMix64 outputs from this seed, their top 53
# bits as a fraction of 2^53 mapped to [-1, 1), in the coefficients' flat
# order; 100 iterations (the counter-based start lets the CUDA path, which
# implements the same generator, reach the same estimate).
POWER_SEED = 12345
POWER_ITERS = 100


def power_start(shape) -> np.ndarray:
    n = int(np.prod(shape))
    z = splitmix64(n, POWER_SEED)
    return ((z >> np.uint64(11)).astype(np.float64) * (2.0 / 2.0 ** 53) - 1.0).reshape(shape)


def soft_threshold(x: np.ndarray, t: float) -> np.ndarray:
    """Proximal operator of t ||.||_1: sign(x) max(|x| - t, 0) (Sect. 3.4)."""
    return np.sign(x) * np.maximum(np.abs(x) - t, 0.0)


@dataclass
class FistaResult:
    beta: np.ndarray                   # last prox output
    alpha: np.ndarray                  # last extrapolated point (Algorithm 1's literal return)
    objective: List[float] = field(default_factory=list)  # F(beta_0), F(beta_1), ...
    iterations: int = 0


def fista(problem: Problem, iters: int, theta: Optional[float] = None,
          beta0: Optional[np.ndarray] = None, rel_tol: float = 0.0,
          momentum: bool = True) -> FistaResult:
    """Algorithm 1:  beta <- tau_gamma(alpha - mu grad f(alpha));
    alpha <- beta + (k-1)/(k+2) (beta - beta_p);  beta_p <- beta,
    for k = 1..iters, from beta_p = alpha = beta0 (zero by default), with
    mu = 1/theta and the threshold gamma = mu * lambda (the lambda of
    Eqs. LowRes / FullRes).  ``momentum=False`` gives ISTA (t = 0).

    Stops early when |F_k - F_{k-1}| <= rel_tol |F_k| for successive prox
    outputs; returns the last prox output beta (and alpha for reference)."""
    W = problem.W
    shape = (W.M, W.npix, W.npix)
    beta_p = np.zeros(shape) if beta0 is None else np.array(beta0, dtype=np.float64)
    alpha = beta_p.copy()
    theta = problem.lipschitz_closed_form() if theta is None else theta
    mu = 1.0 / theta
    res = FistaResult(beta=beta_p.copy(), alpha=alpha.copy())
    res.objective.append(problem.objective(beta_p))
    beta = beta_p
    for k in range(1, iters + 1):
        beta = soft_threshold(alpha - mu * problem.grad(alpha), mu * problem.lam)
        t = (k - 1.0) / (k + 2.0) if momentum else 0.0
        alpha = beta + t * (beta - beta_p)
        beta_p = beta
        res.objective.append(problem.objective(beta))
        res.iterations = k
        if rel_tol > 0 and abs(res.objective[-1] - res.objective[-2]) <= rel_tol * abs(res.objective[-1]):
            break
    res.beta = beta
    res.alpha = alpha
    return res


# ---------------------------------------------------------------------------
# noise-level estimates (Sect. 4.3)
# ---------------------------------------------------------------------------
def sigma2_hat(image: np.ndarray, window: int = 5) -> float:
    """Mean over all fully-inside window x window positions of the population
    variance of the pixels in the window (Sect. 4.3)."""
    win = sliding_window_view(np.asarray(image, dtype=np.float64), (window, window))
    return float(win.var(axis=(-2, -1)).mean())


def eta2_hat(sigma2: float) -> float:
    """eta^2 = 1e-3 sigma^2 (Sect. 4.3)."""
    return 1e-3 * sigma2
