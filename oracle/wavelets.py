"""Oracle: Daubechies wavelets and the concatenated dictionary W.

Test infrastructure only (see ``oracle/__init__``).

The paper's dictionary is the concatenation of the first eight Daubechies
wavelets (Sect. 4.3, Sect. 5, App. A.1), M = 8 orthonormal bases, and the
closed-form Lipschitz constant it uses (Sect. 3.4) assumes each basis is an
orthogonal decomposition with circular boundaries; so each basis here is the
periodized, orthonormal, separable 2-D DWT with J levels, and W alpha is the
plain sum of the M syntheses (W W^H = M I).

Filters: db_p has p vanishing moments and 2p taps.  With z = exp(-i w) and
y = sin^2(w/2) = (2 - z - 1/z)/4, Daubechies' construction writes
|m0|^2 = cos^{2p}(w/2) P(y), P(y) = sum_{k<p} C(p-1+k, k) y^k, and factors
P into Q(z) Q(1/z) choosing one root of each reciprocal pair; the roots with
|z| > 1 give the filter with h_0 > 0 in Daubechies' table ordering
(db2: h = ((1+sqrt3), (3+sqrt3), (3-sqrt3), (1-sqrt3)) / (4 sqrt2)).
High-pass: g_k = (-1)^k h_{L-1-k}.

Periodized analysis of a length-n signal (n even):
  a_i = sum_k h_k x[(2i + k) mod n],  d_i = sum_k g_k x[(2i + k) mod n].
One 2-D level on an n x n block X is Y = T X T^T with T the n x n analysis
matrix (rows 0..n/2-1 low-pass, n/2..n-1 high-pass).  Layout (Mallat): after a
level, Y[:n/2, :n/2] is the approximation (low in y and x), Y[:n/2, n/2:] low
in y / high in x, Y[n/2:, :n/2] high in y / low in x, Y[n/2:, n/2:] high/high;
the next level works on Y[:n/2, :n/2].
"""
from __future__ import annotations

from functools import lru_cache
from math import comb, sqrt

import numpy as np


@lru_cache(maxsize=None)
def daubechies_lowpass(p: int) -> tuple:
    """Low-pass filter of db_p (2p taps, sum = sqrt 2).

    Roots y_i of P(y) (degree p-1, positive coefficients) are mapped to z by
    z + 1/z = 2 - 4 y_i, keeping the root with |z| > 1; then
    h ~ (1 + z)^p prod_i (z - z_i) in ascending powers of z, scaled to
    sum h = sqrt 2."""
    if p == 1:
        return (1.0 / sqrt(2.0), 1.0 / sqrt(2.0))
    pc = np.array([comb(p - 1 + k, k) for k in range(p)], dtype=np.float64)
    ys = np.roots(pc[::-1])
    # Newton polish on P(y)
    for _ in range(4):
        ys = ys - np.polyval(pc[::-1], ys) / np.polyval(np.polyder(pc[::-1]), ys)
    q = np.array([1.0 + 0j])                        # ascending powers of z
    for y in ys:
        s = 1.0 - 2.0 * y                           # z^2 - 2 s z + 1 = 0
        disc = np.sqrt(s * s - 1.0 + 0j)
        z = s + disc
        if abs(z) < 1.0:
            z = s - disc
        q = np.convolve(q, np.array([-z, 1.0]))
    binom = np.array([comb(p, k) for k in range(p + 1)], dtype=np.float64)
    h = np.convolve(binom, q).real
    h = h * (sqrt(2.0) / h.sum())
    return tuple(float(x) for x in h)


def highpass(h) -> np.ndarray:
    h = np.asarray(h, dtype=np.float64)
    L = h.size
    return np.array([(-1) ** k * h[L - 1 - k] for k in range(L)])


@lru_cache(maxsize=None)
def _analysis_matrix_cached(p: int, n: int) -> np.ndarray:
    h = np.asarray(daubechies_lowpass(p))
    g = highpass(h)
    T = np.zeros((n, n))
    half = n // 2
    for i in range(half):
        for k in range(h.size):
            T[i, (2 * i + k) % n] += h[k]
            T[half + i, (2 * i + k) % n] += g[k]
    return T


def analysis_matrix(p: int, n: int) -> np.ndarray:
    """n x n periodized one-level analysis matrix of db_p."""
    if n % 2:
        raise ValueError("periodized DWT needs an even length")
    return _analysis_matrix_cached(p, n)


def dwt2(x: np.ndarray, p: int, levels: int) -> np.ndarray:
    """Psi_p^H x: J-level 2-D analysis, Mallat layout (same shape as x)."""
    y = np.array(x, dtype=np.float64, copy=True)
    n = y.shape[0]
    for _ in range(levels):
        T = analysis_matrix(p, n)
        y[:n, :n] = T @ y[:n, :n] @ T.T
        n //= 2
    return y


def idwt2(y: np.ndarray, p: int, levels: int) -> np.ndarray:
    """Psi_p c: J-level 2-D synthesis (the transpose, and inverse, of dwt2)."""
    x = np.array(y, dtype=np.float64, copy=True)
    n = x.shape[0] >> (levels - 1)
    for _ in range(levels):
        T = analysis_matrix(p, n)
        x[:n, :n] = T.T @ x[:n, :n] @ T
        n *= 2
    return x


class Dictionary:
    """W = [Psi_1 ... Psi_M], Psi_m the db_m basis (Sect. 4.3 / App. A.1).

    Coefficients alpha have shape [M, N, N]; W alpha = sum_m Psi_m alpha_m and
    W^H x = [Psi_1^H x, ..., Psi_M^H x]."""

    def __init__(self, npix: int, n_bases: int = 8, levels: int = 4):
        if npix % (1 << levels):
            raise ValueError("image side must be divisible by 2^levels")
        self.npix = npix
        self.M = n_bases
        self.levels = levels

    def synth(self, alpha: np.ndarray) -> np.ndarray:
        return sum(idwt2(alpha[m], m + 1, self.levels) for m in range(self.M))

    def analysis(self, x: np.ndarray) -> np.ndarray:
        return np.stack([dwt2(x, m + 1, self.levels) for m in range(self.M)])
