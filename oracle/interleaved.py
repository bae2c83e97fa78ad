"""Oracle: the interleaved two-image pipeline (Sect. 6, future work; Fig.
InterleavedMultiStepPipeline).

Test infrastructure only (see ``oracle/__init__``).

The paper sketches two nodes, one per baseline partition, that reconstruct
full-resolution images side by side and exchange their deconvolved
residuals after every major cycle, the two final images being combined at
the end.  It fixes no problem for the nodes beyond that, so this module
writes out one reading (listed with the others in the design notes):

* node L holds V_L, node H holds V_H; each keeps its own model, the sum of
  its deconvolved residuals, starting from zero;
* major cycle 1: each node solves Eq. LowRes on its own residual with its
  own PSF (node L gives the low-resolution image i_L1, node H the
  high-resolution image i_H1 of the figure);
* major cycle n >= 2: node H solves Eq. FullRes on its residual with
  l = (node L's model) - (node H's model), the low frequencies it still
  lacks; node L solves the same problem with the roles of the two sides of
  the band exchanged: data term ||G'_L (i~_L - H_L x)||^2 with weight
  1 / sigma_L^2 below ell - delta, prior ||G'_H (h - x)||^2 with weight
  1 / eta_L^2 above ell + delta and h = (node H's model) - (node L's
  model); G'_L, G'_H are Sect. 3.3's filters with sigma^2 and eta^2
  exchanged (so eta_L^2 G'_H^2 + sigma_L^2 G'_L^2 = 1 as there);
* sigma^2 of each node is Sect. 4.3's estimate on its first residual,
  eta^2 = 1e-3 sigma^2; lambda_n = c ||i~_n||_2 2^n with each node's own
  residual (c: lambda_low for node L, lambda_full for node H);
* each node's final image is its last residual plus its model (as a step's
  final image); the combined image takes the low frequencies from node L's
  and the high ones from node H's with the weights eta_H^2 g_L^2 and
  sigma_H^2 g_H^2 of node H's filters, which sum to one at every frequency.

Both nodes' minor cycles of a major cycle are independent (they read only
the models of the previous cycle), which is the pipeline's parallelism.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import Optional

import numpy as np

from .gridding import partition
from .imaging import (ReconOptions, StepResult, _lambda, _operator, _psf2_spectrum,
                      _step_size)
from .solver import (Problem, eta2_hat, filter_responses, fista, psf_spectrum,
                     sigma2_hat)
from .wavelets import Dictionary


@dataclass
class InterleavedResult:
    image: np.ndarray        # combined final image
    node_l: StepResult       # node L: image = last residual + model, per-cycle records
    node_h: StepResult
    c_low: np.ndarray        # weight of node L's image on the rfft half-plane
    c_high: np.ndarray       # weight of node H's image (c_low + c_high = 1)


def mirrored_filters(npix: int, ell: float, delta: float, sigma2: float, eta2: float):
    """(data, prior) responses of node L's problem: data weight 1/sigma^2
    below ell - delta, prior weight 1/eta^2 above ell + delta, Sect. 3.3's
    band rule with the two sides exchanged."""
    low, high = filter_responses(npix, ell, delta, sigma2=eta2, eta2=sigma2)
    return low, high


def combine(image_l: np.ndarray, image_h: np.ndarray, c_low: np.ndarray,
            c_high: np.ndarray) -> np.ndarray:
    """The combined image: c_low F(image_l) + c_high F(image_h), back to the
    image domain."""
    spec = c_low * np.fft.rfft2(image_l) + c_high * np.fft.rfft2(image_h)
    return np.fft.irfft2(spec, s=image_l.shape)


def reconstruct_interleaved(vis, u, v, npix, pixel_size, ell, delta,
                            opts: Optional[ReconOptions] = None) -> InterleavedResult:
    opts = opts or ReconOptions()
    in_l, in_h = partition(u, v, npix, pixel_size, ell, delta)
    A = {"L": _operator(u[in_l], v[in_l], npix, pixel_size, opts),
         "H": _operator(u[in_h], v[in_h], npix, pixel_size, opts)}
    V = {"L": vis[in_l], "H": vis[in_h]}
    W = Dictionary(npix, opts.n_bases, opts.levels)
    Hhat = {k: psf_spectrum(A[k].psf()) for k in A}
    Hhat2 = {"L": _psf2_spectrum(u[in_l], v[in_l], npix, pixel_size, opts),
             "H": _psf2_spectrum(u[in_h], v[in_h], npix, pixel_size, opts)}
    coef = {"L": opts.lambda_low, "H": opts.lambda_full}
    model = {k: np.zeros((npix, npix)) for k in A}
    out = {k: StepResult(image=model[k], model=model[k]) for k in A}
    first, filt, theta = {}, {}, {}
    for n in range(1, opts.n_major + 1):
        res = {k: A[k].residual_image(V[k], model[k]) for k in A}
        if n == 1:
            for k in A:
                first[k] = res[k]
                s2 = sigma2_hat(res[k])
                out[k].sigma2, out[k].eta2 = s2, eta2_hat(s2)
            gl, gh = filter_responses(npix, ell, delta, out["H"].sigma2, out["H"].eta2)
            dl, ph = mirrored_filters(npix, ell, delta, out["L"].sigma2, out["L"].eta2)
            filt = {"H": (gl, gh), "L": (ph, dl)}   # (prior, data) of each node
        prob = {}
        for k in A:
            lam = _lambda(opts.lambda_rule, coef[k], res[k], first[k], n)
            if n == 1:
                prob[k] = Problem("low", W, Hhat[k], res[k], lam, Hhat2=Hhat2[k])
            else:
                other = "H" if k == "L" else "L"
                prior, data = filt[k]
                prob[k] = Problem("full", W, Hhat[k], res[k], lam, gl=prior, gh=data,
                                  l_low=model[other] - model[k], Hhat2=Hhat2[k])
            # the operator changes from cycle 1 to cycle 2, then stays
            theta[k] = _step_size(prob[k], theta.get(k) if n > 2 else None)
        for k in A:
            fr = fista(prob[k], opts.fista_iters, theta=theta[k], rel_tol=opts.rel_tol)
            out[k].residuals.append(res[k])
            out[k].lambdas.append(prob[k].lam)
            out[k].objectives.append(fr.objective)
            out[k].thetas.append(theta[k])
            model[k] = model[k] + W.synth(fr.beta)
    for k in A:
        last = A[k].residual_image(V[k], model[k])
        out[k].residuals.append(last)
        out[k].model = model[k]
        out[k].image = last + model[k]
    gl, gh = filt["H"][0], filt["H"][1]
    c_low = out["H"].eta2 * gl ** 2
    c_high = out["H"].sigma2 * gh ** 2
    return InterleavedResult(combine(out["L"].image, out["H"].image, c_low, c_high),
                             out["L"], out["H"], c_low, c_high)
