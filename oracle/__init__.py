"""Plain, slow, FP64 CPU oracle of the multi-step reconstruction hot path.

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it.
The CUDA library never calls it, and nothing in it is shared with the CUDA
path: no kernels, tables, constants or helpers.

Every function cites the passage of the paper (Wang, Prunet, Mignot, Ferrari,
"Multi-Step Reconstruction of Radio-Interferometric Images") it follows.  The
code is written for being checked by eye: the paper's equations in its order
and notation, numpy primitives (FFT, matmul, scatter-add) as single steps, no
blocking or fusion.

Modules
-------
``gridding``   reduced measurement equation (Sect. 2, Eq. RIME), exact NUDFT,
               the gridded operator A = G F Z D with an exponential-of-semicircle
               kernel, dirty images, PSFs, the baseline partition (Sect. 3.1).
``wavelets``   Daubechies filters db1..db8, periodized orthonormal 2-D DWT,
               the concatenated dictionary W (Sect. 4.3, App. A.1).
``solver``     filters G_L, G_H (Sect. 3.3), objectives, gradients (Eqs. GradL,
               GradH), Lipschitz constants and power iteration (Sect. 3.4),
               soft threshold and FISTA (Algorithm 1), sigma/eta estimators
               (Sect. 4.3).
``imaging``    major cycles, the two-step method (Eqs. LowRes, FullRes) and the
               single-step baseline (Sect. 5).
``unet``       the learned warm start's network (a small U-Net: convolutions,
               pooling, upsampling, bfloat16 rounding points), its gradients
               and the Adam update.

Parity status
-------------
Every function is pinned by a ``-m "not gpu"`` test against something other
than itself (closed forms, brute force, invariants, special cases).  The
end-to-end reconstructions of ``imaging`` have no printed worked example in
the paper; they are pinned by exact recovery: with one noise-free visibility
at every image frequency and lambda = 0, the single-step image is the sky and
the two-step image converges to it.
"""
