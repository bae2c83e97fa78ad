"""The method with more than two steps (Sect. 6's "more than 2-steps"),
through ms_reconstruct_step: K - 1 partition radii ell_1 < ... < ell_K-1 and
one half width delta cut the baselines into K bands (V_1 = {r <= ell_1 +
delta}, V_k = {ell_k-1 - delta <= r <= ell_k + delta}, V_K = {r >= ell_K-1 -
delta}); step 1 is Eq. LowRes on V_1 and step k > 1 Eq. FullRes on V_k with
the filters at ell_k-1 and the previous step's image.  Step k > 1 runs on a
plan whose partition radius is ell_k-1 and whose flags drop the rows above
ell_k + delta (read back from a plan at ell_k, so that band membership is the
library's own classification).  With K = 2 this is ms_reconstruct_two_step.
"""
from __future__ import annotations

from typing import Optional, Sequence

import numpy as np


def reconstruct_multi_step(ms, u, v, vis, npix: int, pixel_size: float, ells: Sequence[float],
                           delta: float, opts=None, precision: str = "fp32", flags=None,
                           **plan_kw):
    """Images of steps 1..K (device tensors) and their Stats; vis is a device
    complex [nvis] tensor of the rows u, v (one channel)."""
    ells = list(ells)
    if not ells or any(b <= a for a, b in zip(ells, ells[1:])):
        raise ValueError("partition radii must be given and increase")
    u = np.asarray(u, dtype=np.float64)
    v = np.asarray(v, dtype=np.float64)
    base = np.zeros(u.shape, np.uint8) if flags is None else np.asarray(flags, np.uint8).copy()
    images, stats = [], []
    prev = None
    for k in range(len(ells) + 1):
        ell = ells[max(k - 1, 0)]
        fl = base.copy()
        if 0 < k < len(ells):
            # drop the rows above ell_k + delta: the L partition of a plan at ell_k
            probe = ms.Plan(u, v, npix, pixel_size, ells[k], delta, flags=base,
                            precision=precision, **plan_kw)
            keep = np.zeros(u.shape, bool)
            keep[probe.partition_rows("L")] = True
            probe.close()
            fl[~keep] = 1
        plan = ms.Plan(u, v, npix, pixel_size, ell, delta, flags=fl, precision=precision,
                       **plan_kw)
        img, st = plan.reconstruct_step("low" if k == 0 else "full", vis.to(plan.complex_dtype),
                                        opts, low_image=prev)
        plan.close()
        images.append(img)
        stats.append(st)
        prev = img
    return images, stats
