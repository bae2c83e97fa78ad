"""Oracle: the method with more than two steps (Sect. 6 names it as a
direction: "more than 2-steps", to find the limit of partitioning by
baseline).

Test infrastructure only (see ``oracle/__init__``).

Reading (listed with the others in the design notes): K - 1 partition radii
ell_1 < ... < ell_{K-1} with one half width delta cut the baselines into K
bands with Sect. 3.1's closed intervals,

    V_1 = {r <= ell_1 + delta},
    V_k = {ell_{k-1} - delta <= r <= ell_k + delta}   (1 < k < K),
    V_K = {r >= ell_{K-1} - delta};

step 1 is Eq. LowRes on V_1 (step one), and step k > 1 is Eq. FullRes on V_k
with the filters of Sect. 3.3 at ell_{k-1} and l = the image of step k - 1
(step two's problem, one band up).  With K = 2 this is the two-step method.
"""
from __future__ import annotations

from typing import List, Optional, Sequence

import numpy as np

from .gridding import partition
from .imaging import ReconOptions, StepResult, run_full_step, run_low_step


def band_masks(u, v, npix, pixel_size, ells: Sequence[float], delta: float) -> List[np.ndarray]:
    """The K row masks of the bands for radii ells (increasing)."""
    ells = list(ells)
    if any(b <= a for a, b in zip(ells, ells[1:])):
        raise ValueError("partition radii must increase")
    low = [partition(u, v, npix, pixel_size, e, delta)[0] for e in ells]    # r <= ell + delta
    high = [partition(u, v, npix, pixel_size, e, delta)[1] for e in ells]   # r >= ell - delta
    masks = [low[0]]
    for k in range(1, len(ells)):
        masks.append(high[k - 1] & low[k])
    masks.append(high[-1])
    return masks


def reconstruct_multi_step(vis, u, v, npix, pixel_size, ells: Sequence[float], delta: float,
                           opts: Optional[ReconOptions] = None) -> List[StepResult]:
    """Steps 1..K in order; the last one's image is the method's image."""
    opts = opts or ReconOptions()
    masks = band_masks(u, v, npix, pixel_size, ells, delta)
    m = masks[0]
    out = [run_low_step(vis[m], u[m], v[m], npix, pixel_size, opts, opts.lambda_low)]
    for k in range(1, len(masks)):
        m = masks[k]
        out.append(run_full_step(vis[m], u[m], v[m], npix, pixel_size, out[-1].image,
                                 ells[k - 1], delta, opts))
    return out
