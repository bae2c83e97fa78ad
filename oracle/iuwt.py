"""Oracle: the isotropic undecimated wavelet transform (IUWT) as a dictionary.

Test infrastructure only (see ``oracle/__init__``).

The paper compares its Daubechies dictionary with IUWT wavelets (App. A.1,
citing Starck et al. 2007) and notes (Sect. 3.4) that for dictionaries
without the closed-form step size the Lipschitz constant comes from power
iteration.  This module writes the transform out plainly:

* B3-spline scaling filter h = (1, 4, 6, 4, 1) / 16, applied separably along
  rows and columns with holes ("a trous"): at scale j the taps sit at
  offsets -2d, -d, 0, d, 2d with d = 2^(j-1), on a periodic N x N grid;
* analysis T: c_0 = x, c_j = h_j * c_{j-1}, w_j = c_{j-1} - c_j for
  j = 1..J; coefficients [w_1, ..., w_J, c_J] ([J + 1, N, N]); the planes sum
  back to x;
* the dictionary is W = T^H (so the FISTA gradient 2 W^H (K W alpha - b)
  applies T to an image); W W^H = T^H T is not a multiple of the identity,
  hence no closed-form step size from Sect. 3.4.

T^H follows from <T x, a> = <c_0, a_1> + sum_{j=1}^{J-1} <c_j, a_{j+1} - a_j>
+ <c_J, a_{J+1} - a_J> and c_j = h_j * c_{j-1} (h symmetric, so each
smoothing is its own adjoint): with y_J = a_{J+1} - a_J and
y_{j-1} = (a_j - a_{j-1}) + h_j * y_j for j = J..2, T^H a = a_1 + h_1 * y_1.
"""
from __future__ import annotations

import numpy as np

B3 = np.array([1.0, 4.0, 6.0, 4.0, 1.0]) / 16.0


def smooth(c: np.ndarray, j: int) -> np.ndarray:
    """h_j * c: the B3 filter with holes of 2^(j-1) along rows, then columns,
    periodic boundaries."""
    d = 1 << (j - 1)
    rows = sum(B3[t] * np.roll(c, -(t - 2) * d, axis=0) for t in range(5))
    return sum(B3[t] * np.roll(rows, -(t - 2) * d, axis=1) for t in range(5))


def iuwt(x: np.ndarray, levels: int) -> np.ndarray:
    """T x = [w_1, ..., w_J, c_J]."""
    c = np.asarray(x, dtype=np.float64)
    planes = []
    for j in range(1, levels + 1):
        cj = smooth(c, j)
        planes.append(c - cj)
        c = cj
    planes.append(c)
    return np.stack(planes)


def iuwt_adjoint(a: np.ndarray, levels: int) -> np.ndarray:
    """T^H a for coefficients a = [a_1, ..., a_{J+1}] (a[0] .. a[J])."""
    J = levels
    y = a[J] - a[J - 1]
    for j in range(J, 1, -1):
        y = (a[j - 1] - a[j - 2]) + smooth(y, j)
    return a[0] + smooth(y, 1)


def scaling_symbol(npix: int, j: int) -> np.ndarray:
    """DFT of the level-j smoothing on the rfft2 half-plane (real: h is
    symmetric): prod over the two axes of sum_t h_t cos(2 pi (t - 2) d k / N)."""
    d = 1 << (j - 1)
    ky = np.fft.fftfreq(npix) * npix
    kx = np.fft.rfftfreq(npix) * npix
    off = np.arange(-2, 3)
    sy = (B3[None, :] * np.cos(2 * np.pi * off[None, :] * d * ky[:, None] / npix)).sum(1)
    sx = (B3[None, :] * np.cos(2 * np.pi * off[None, :] * d * kx[:, None] / npix)).sum(1)
    return sy[:, None] * sx[None, :]


def frame_symbol(npix: int, levels: int) -> np.ndarray:
    """DFT of T^H T (a circulant operator): sum_j (C_{j-1} - C_j)^2 + C_J^2
    with C_0 = 1 and C_j = prod_{i <= j} (the level-i symbol)."""
    C = np.ones((npix, npix // 2 + 1))
    S = np.zeros_like(C)
    for j in range(1, levels + 1):
        Cj = C * scaling_symbol(npix, j)
        S += (C - Cj) ** 2
        C = Cj
    return S + C ** 2


class IUWTDictionary:
    """W = T^H on [J + 1, N, N] coefficients (the same interface as
    ``wavelets.Dictionary``: M planes, synth = W, analysis = W^H)."""

    def __init__(self, npix: int, levels: int = 4):
        self.npix = npix
        self.levels = levels
        self.M = levels + 1

    def synth(self, alpha: np.ndarray) -> np.ndarray:
        return iuwt_adjoint(alpha, self.levels)

    def analysis(self, x: np.ndarray) -> np.ndarray:
        return iuwt(x, self.levels)


def lipschitz_fourier(normal_spectrum: np.ndarray, npix: int, levels: int) -> float:
    """2 lambda_max(T K T^H) for a circulant K with real half-plane spectrum
    normal_spectrum: the nonzero spectrum of T K T^H is that of
    K^(1/2) T^H T K^(1/2), diagonal in Fourier space, so
    lambda_max = max_k K(k) S(k) with S the symbol of T^H T."""
    return 2.0 * float(np.max(normal_spectrum * frame_symbol(npix, levels)))
