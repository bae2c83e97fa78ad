"""Oracle: major cycles, the two-step method and the single-step baseline.

Test infrastructure only (see ``oracle/__init__``).

Readings of the paper taken here (each also listed in the design notes):
* The model starts at zero in both steps; step two's residual is taken
  against its own model sum_{j<n} i_j (Sect. 3.3, Eq. FullRes).
* A step's final image is its last residual plus the sum of its deconvolved
  residuals, i^ = i~_{N+1} + sum_n i_n (Sects. 3.2, 3.3); the model-only sum is
  returned as well.
* lambda rules: "norm2_2n" is lambda_n = c ||i~_n||_2 2^n with n counted from 1
  (Sect. 5, App. A.2; c = 0.05 for both steps, 0.01 single-step); "max_fixed"
  is lambda = c max|i~_1| held for all cycles of a step.
* sigma^2 is estimated on i~_{H_1} by the 5 x 5 window rule and eta^2 =
  1e-3 sigma^2 (Sect. 4.3) unless given.
* FISTA starts from zero each major cycle and returns its last prox output.
* The PSF operator of the minor cycle is a circular N x N convolution
  (Sect. 3.4 allows circulant operators) or, with convolution="linear",
  the linear convolution by the 2N x 2N PSF that A^H A / sum(w) is on the
  N x N field (the circular one makes the major cycle diverge when the PSF
  is wide; see the pins).  Its step size is a power iteration from a fixed
  counter-based start (the closed form is then only a bound).
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

from .gridding import GriddedOperator, partition
from .solver import (POWER_ITERS, Problem, eta2_hat, filter_responses, fista, power_start,
                     psf_spectrum, sigma2_hat)
from .wavelets import Dictionary


@dataclass
class ReconOptions:
    n_major: int = 5
    fista_iters: int = 100
    rel_tol: float = 0.0
    lambda_rule: str = "norm2_2n"        # or "max_fixed"
    lambda_low: float = 0.05
    lambda_full: float = 0.05
    lambda_single: float = 0.01
    sigma2: Optional[float] = None
    eta2: Optional[float] = None
    width: int = 7
    oversample: int = 2
    beta: Optional[float] = None
    levels: int = 4
    n_bases: int = 8
    convolution: str = "circular"        # or "linear": the PSF operator on the N x N field


@dataclass
class StepResult:
    image: np.ndarray                 # i~_{N+1} + sum i_n
    model: np.ndarray                 # sum i_n
    residuals: List[np.ndarray] = field(default_factory=list)   # i~_1 .. i~_{N+1}
    lambdas: List[float] = field(default_factory=list)
    objectives: List[List[float]] = field(default_factory=list)
    thetas: List[float] = field(default_factory=list)
    sigma2: Optional[float] = None
    eta2: Optional[float] = None


def _lambda(rule: str, coef: float, residual: np.ndarray, first: np.ndarray, n: int) -> float:
    if rule == "norm2_2n":
        return coef * float(np.linalg.norm(residual)) * (2.0 ** n)
    if rule == "max_fixed":
        return coef * float(np.max(np.abs(first)))
    raise ValueError(rule)


def _operator(u, v, npix, pixel_size, opts: ReconOptions) -> GriddedOperator:
    return GriddedOperator(u, v, npix, pixel_size, width=opts.width,
                           oversample=opts.oversample, beta=opts.beta)


def _psf2_spectrum(u, v, npix, pixel_size, opts: ReconOptions):
    """Spectrum of the PSF on a 2N x 2N field (offsets up to +-N), for the
    linear reading of the PSF operator; None for the circular one."""
    if opts.convolution != "linear":
        return None
    return psf_spectrum(_operator(u, v, 2 * npix, pixel_size, opts).psf())


def _step_size(prob: Problem, previous: Optional[float]) -> float:
    """theta of Sect. 3.4: the closed form 2 M max K^ for the circular
    operator; for the linear one (not circulant, where the closed form is only
    a bound, 2-5x above the constant on small cases) a power iteration from the
    fixed start, once per step (the operator is the same in every cycle)."""
    if prob.Hhat2 is None:
        return prob.lipschitz_closed_form()
    if previous is not None:
        return previous
    return prob.lipschitz_power_iteration(
        iters=POWER_ITERS, start=power_start((prob.W.M, prob.W.npix, prob.W.npix)))


def run_low_step(vis, u, v, npix, pixel_size, opts: ReconOptions, coef: float) -> StepResult:
    """Step one (Sect. 3.2, Eq. LowRes); also the single-step method on all
    visibilities (Sect. 5)."""
    A = _operator(u, v, npix, pixel_size, opts)
    W = Dictionary(npix, opts.n_bases, opts.levels)
    Hhat = psf_spectrum(A.psf())
    Hhat2 = _psf2_spectrum(u, v, npix, pixel_size, opts)
    model = np.zeros((npix, npix))
    out = StepResult(image=model, model=model)
    first = None
    for n in range(1, opts.n_major + 1):
        res = A.residual_image(vis, model)
        first = res if first is None else first
        lam = _lambda(opts.lambda_rule, coef, res, first, n)
        prob = Problem("low", W, Hhat, res, lam, Hhat2=Hhat2)
        theta = _step_size(prob, theta if n > 1 else None)
        fr = fista(prob, opts.fista_iters, theta=theta, rel_tol=opts.rel_tol)
        model = model + W.synth(fr.beta)
        out.residuals.append(res)
        out.lambdas.append(lam)
        out.objectives.append(fr.objective)
        out.thetas.append(theta)
    last = A.residual_image(vis, model)
    out.residuals.append(last)
    out.model = model
    out.image = last + model
    return out


def run_full_step(vis, u, v, npix, pixel_size, low_image, ell, delta,
                  opts: ReconOptions, beta0_first: Optional[np.ndarray] = None) -> StepResult:
    """Step two (Sect. 3.3, Eq. FullRes) with l_{L_n} = i^_L - sum_{j<n} i_j.
    beta0_first: start of the first minor cycle (a warm start) instead of
    zero; the later cycles start from zero."""
    A = _operator(u, v, npix, pixel_size, opts)
    W = Dictionary(npix, opts.n_bases, opts.levels)
    Hhat = psf_spectrum(A.psf())
    Hhat2 = _psf2_spectrum(u, v, npix, pixel_size, opts)
    model = np.zeros((npix, npix))
    out = StepResult(image=model, model=model)
    first = None
    gl = gh = None
    for n in range(1, opts.n_major + 1):
        res = A.residual_image(vis, model)
        if first is None:
            first = res
            s2 = opts.sigma2 if opts.sigma2 is not None else sigma2_hat(res)
            e2 = opts.eta2 if opts.eta2 is not None else eta2_hat(s2)
            out.sigma2, out.eta2 = s2, e2
            gl, gh = filter_responses(npix, ell, delta, s2, e2)
        lam = _lambda(opts.lambda_rule, opts.lambda_full, res, first, n)
        l_low = low_image - model
        prob = Problem("full", W, Hhat, res, lam, gl=gl, gh=gh, l_low=l_low, Hhat2=Hhat2)
        theta = _step_size(prob, theta if n > 1 else None)
        fr = fista(prob, opts.fista_iters, theta=theta, rel_tol=opts.rel_tol,
                   beta0=beta0_first if n == 1 else None)
        model = model + W.synth(fr.beta)
        out.residuals.append(res)
        out.lambdas.append(lam)
        out.objectives.append(fr.objective)
        out.thetas.append(theta)
    last = A.residual_image(vis, model)
    out.residuals.append(last)
    out.model = model
    out.image = last + model
    return out


def reconstruct_two_step(vis, u, v, npix, pixel_size, ell, delta,
                         opts: Optional[ReconOptions] = None,
                         beta0_full: Optional[np.ndarray] = None):
    """Partition (Sect. 3.1), step one on V_L, step two on V_H and i^_L;
    beta0_full optionally starts step two's first minor cycle."""
    opts = opts or ReconOptions()
    in_l, in_h = partition(u, v, npix, pixel_size, ell, delta)
    low = run_low_step(vis[in_l], u[in_l], v[in_l], npix, pixel_size, opts, opts.lambda_low)
    full = run_full_step(vis[in_h], u[in_h], v[in_h], npix, pixel_size, low.image,
                         ell, delta, opts, beta0_first=beta0_full)
    return low, full


def reconstruct_single_step(vis, u, v, npix, pixel_size,
                            opts: Optional[ReconOptions] = None) -> StepResult:
    """All baselines at once with step one's problem (Sect. 5)."""
    opts = opts or ReconOptions()
    return run_low_step(vis, u, v, npix, pixel_size, opts, opts.lambda_single)


def psnr(image: np.ndarray, truth: np.ndarray) -> float:
    """Peak signal-to-noise ratio in dB against the truth's peak."""
    mse = float(np.mean((image - truth) ** 2))
    return 10.0 * np.log10(float(np.max(np.abs(truth))) ** 2 / mse)
