"""Oracle: measurement operator, gridding and the baseline partition.

Test infrastructure only (see ``oracle/__init__``).

Model (Sect. 2, Eq. RIME, reduced form with D = 1, C = 1, w = 0): an image x
of N x N real pixels, pixel (p, q) at l = (q - N/2) dl, m = (p - N/2) dl,
measured at baseline (u_k, v_k) as

    V_k = sum_{p,q} x[p,q] exp(-2 pi i (u_k l_q + v_k m_p)).

Only one visibility of each conjugate pair is stored, so the adjoint under
<a, b> = Re sum conj(a) b is  (A^H y)[p,q] = Re sum_k y_k exp(+2 pi i (...)).

The method evaluates this operator as the residual of the major cycle
(Sect. 2):  i~ = F^H G^H (v - G F x),  with F the FFT and G the (de)gridding
operator.  The paper names no kernel; it cites the exponential-of-semicircle
(ES) kernel of Barnett et al. as prior art for gridding, which is used here:

    phi(t) = exp(beta (sqrt(1 - (2t/W)^2) - 1)),  |t| <= W/2  (t in grid cells)

with W = 7 cells, 2x oversampling (grid of Ng = 2N cells) and beta = 2.30 W.
The gridded forward operator is A = G F Z D:
  D  divide pixel a by psi(a), psi the Fourier transform of phi at a/Ng,
  Z  zero-pad N -> Ng (pixel a at FFT index a mod Ng),
  F  forward FFT (exp(-2 pi i ...)),
  G  visibility k = sum over the W x W cells c nearest to g_k = (u_k, v_k) Ng dl
     of phi(g_u - c_u) phi(g_v - c_v) Fx[c mod Ng].
The footprint of a visibility is the W cells starting at floor(g - W/2) + 1
(the nearest cell and (W-1)/2 on either side).  The grid is periodic.
"""
from __future__ import annotations

import numpy as np

ES_BETA_PER_WIDTH = 2.30   # Barnett et al. (cited in Sect. 2) for 2x upsampling


def es_beta(width: int) -> float:
    return ES_BETA_PER_WIDTH * width


def es_kernel(t, width: int, beta: float) -> np.ndarray:
    """phi(t) on |t| <= W/2, zero outside."""
    z = 2.0 * np.asarray(t, dtype=np.float64) / width
    out = np.zeros(z.shape, dtype=np.float64)
    inside = np.abs(z) <= 1.0
    out[inside] = np.exp(beta * (np.sqrt(1.0 - z[inside] ** 2) - 1.0))
    return out


def deapodization(npix: int, ngrid: int, width: int, beta: float,
                  n_quad: int = 400) -> np.ndarray:
    """psi(a) = integral_{-W/2}^{W/2} phi(t) cos(2 pi t a / Ng) dt for the
    image offsets a = -N/2 .. N/2-1, by Gauss-Legendre quadrature in t."""
    x, w = np.polynomial.legendre.leggauss(n_quad)
    t = x * (width / 2.0)
    wt = w * (width / 2.0)
    a = np.arange(npix) - npix // 2
    phi = es_kernel(t, width, beta)
    return (np.cos(2.0 * np.pi * np.outer(a, t) / ngrid) * (wt * phi)[None, :]).sum(axis=1)


# ---------------------------------------------------------------------------
# exact model (the pin for the gridded operator)
# ---------------------------------------------------------------------------
def pixel_lm(npix: int, pixel_size: float) -> np.ndarray:
    return (np.arange(npix) - npix // 2) * pixel_size


def nudft_forward(image: np.ndarray, u: np.ndarray, v: np.ndarray, pixel_size: float) -> np.ndarray:
    """Exact V_k = sum x[p,q] exp(-2 pi i (u_k l_q + v_k m_p)) (Sect. 2, Eq. RIME)."""
    npix = image.shape[0]
    lm = pixel_lm(npix, pixel_size)
    eu = np.exp(-2j * np.pi * np.outer(u, lm))   # [k, q]
    ev = np.exp(-2j * np.pi * np.outer(v, lm))   # [k, p]
    return np.einsum("kp,pq,kq->k", ev, image, eu)


def nudft_adjoint(vis: np.ndarray, u: np.ndarray, v: np.ndarray, npix: int,
                  pixel_size: float) -> np.ndarray:
    """Exact adjoint Re sum_k y_k exp(+2 pi i (u_k l_q + v_k m_p))."""
    lm = pixel_lm(npix, pixel_size)
    eu = np.exp(2j * np.pi * np.outer(u, lm))
    ev = np.exp(2j * np.pi * np.outer(v, lm))
    return np.einsum("k,kp,kq->pq", vis, ev, eu).real


# ---------------------------------------------------------------------------
# gridded operator A = G F Z D and its adjoint
# ---------------------------------------------------------------------------
class GriddedOperator:
    """A = G F Z D for one set of baselines (Sect. 2, residual equation)."""

    def __init__(self, u, v, npix, pixel_size, width=7, oversample=2, beta=None):
        self.u = np.asarray(u, dtype=np.float64)
        self.v = np.asarray(v, dtype=np.float64)
        self.npix = int(npix)
        self.ngrid = int(oversample * npix)
        self.width = int(width)
        self.beta = es_beta(width) if beta is None else float(beta)
        self.pixel_size = float(pixel_size)
        self.psi = deapodization(self.npix, self.ngrid, self.width, self.beta)
        # continuous grid coordinates (cells, uv origin at cell 0)
        self.gu = self.u * self.ngrid * self.pixel_size
        self.gv = self.v * self.ngrid * self.pixel_size
        self.c0u = np.floor(self.gu - self.width / 2.0).astype(np.int64) + 1
        self.c0v = np.floor(self.gv - self.width / 2.0).astype(np.int64) + 1
        self.pad_index = (np.arange(self.npix) - self.npix // 2) % self.ngrid

    @property
    def nvis(self) -> int:
        return self.u.shape[0]

    def _taps(self):
        """Yield (cell_v, cell_u, weight) for the W x W footprint taps."""
        for j in range(self.width):
            cv = self.c0v + j
            wv = es_kernel(self.gv - cv, self.width, self.beta)
            for i in range(self.width):
                cu = self.c0u + i
                wu = es_kernel(self.gu - cu, self.width, self.beta)
                yield cv % self.ngrid, cu % self.ngrid, wu * wv

    def forward(self, image: np.ndarray) -> np.ndarray:
        """V = A x (degridding)."""
        xd = np.asarray(image, dtype=np.float64) / np.outer(self.psi, self.psi)      # D
        padded = np.zeros((self.ngrid, self.ngrid), dtype=np.complex128)           # Z
        padded[np.ix_(self.pad_index, self.pad_index)] = xd
        grid = np.fft.fft2(padded)                                                 # F
        out = np.zeros(self.nvis, dtype=np.complex128)
        for cv, cu, w in self._taps():                                             # G
            out += w * grid[cv, cu]
        return out

    def adjoint(self, vis: np.ndarray) -> np.ndarray:
        """A^H y (gridding, inverse FFT, crop, deapodize, real part)."""
        vis = np.asarray(vis, dtype=np.complex128)
        n2 = self.ngrid * self.ngrid
        acc_re = np.zeros(n2)
        acc_im = np.zeros(n2)
        for cv, cu, w in self._taps():                                             # G^H
            flat = cv * self.ngrid + cu
            acc_re += np.bincount(flat, weights=w * vis.real, minlength=n2)
            acc_im += np.bincount(flat, weights=w * vis.imag, minlength=n2)
        grid = (acc_re + 1j * acc_im).reshape(self.ngrid, self.ngrid)
        img = np.fft.ifft2(grid) * n2                                              # F^H (unnormalized)
        img = img[np.ix_(self.pad_index, self.pad_index)].real                     # Z^H, real part
        return img / np.outer(self.psi, self.psi)                                  # D^H

    # -- the images the major cycle works with (natural weights) ---------------
    def dirty(self, vis: np.ndarray) -> np.ndarray:
        """Residual/dirty image normalized by the sum of (unit) weights."""
        return self.adjoint(vis) / max(self.nvis, 1)

    def residual_image(self, vis: np.ndarray, model: np.ndarray) -> np.ndarray:
        """i~_n = F^H G^H (v - G F i^_n) (Sect. 2), normalized by sum of weights."""
        return self.dirty(vis - self.forward(model))

    def psf(self) -> np.ndarray:
        """A^H A applied to a unit impulse at pixel (N/2, N/2), normalized."""
        delta = np.zeros((self.npix, self.npix))
        delta[self.npix // 2, self.npix // 2] = 1.0
        return self.dirty(self.forward(delta))


# ---------------------------------------------------------------------------
# baseline partition (Sect. 3.1)
# ---------------------------------------------------------------------------
def baseline_radius_px(u, v, npix, pixel_size) -> np.ndarray:
    """|uv| in pixel units of the N x N image DFT grid (the paper measures
    ell and delta in pixel distances, Sect. 3.1)."""
    return np.hypot(u, v) * npix * pixel_size


def partition(u, v, npix, pixel_size, ell, delta):
    """Masks of V_L (r <= ell + delta) and V_H (r >= ell - delta); the overlap
    band [ell - delta, ell + delta] belongs to both (Sect. 3.1, Fig. Partitioning)."""
    r = baseline_radius_px(u, v, npix, pixel_size)
    return r <= ell + delta, r >= ell - delta
