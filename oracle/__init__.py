"""FP64 CPU oracle for preconditioned-BFGS elastic FWI (Liu et al. 2020).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports this package:
only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may use it.  It shares no code with
the CUDA library; the two meet only in the seeded input generators of
``synth``.

Modules
-------
sem      spectral-element forward / adjoint / gradient / preconditioners (C, FP64)
bfgs     dense BFGS (Eq. 3), two-loop recursions (Algorithms 1 and 2),
         single-pass randomized SVD (Algorithm 3), posterior std (Eq. 14)
philox   Philox4x32-10 counter-based generator (Salmon et al. 2011)
unet     learned diagonal preconditioner: U-Net forward / backward, MSE, Adam,
         bilinear node-grid <-> image resampling, input features (optional
         bfloat16 rounding at the CUDA path's storage points)
"""
