"""Plain FP64 CPU oracle of InfiniteDiffusion sampling (test infrastructure).

This package is test infrastructure, not part of the product.  Only the test
suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py``
may import it.  It shares no code with the CUDA library and imports nothing
from it; the only inputs both sides share come from the seeded generators in
``synth``.

Everything is written to be read against the paper:

* ``noise``     -- the seed function G(s, p) of App. B ("Seeds and initial
                   noise"): Philox4x32-10 and Box-Muller in binary32.
* ``kappa``     -- Alg. 3 (windows intersecting a region) and the window
                   layout of Sec. 3.2.
* ``schedule``  -- sigma schedule, EDM preconditioning, the separable linear
                   weight window of Sec. 6.
* ``unet``      -- the window denoiser Phi (Sec. 5.3; the synthetic UNet
                   reading) in FP64 via im2col + matmul.
* ``sampler``   -- Eq. 1 (bounded MultiDiffusion, eager), Eq. 2 / Alg. 1
                   (lazy InfiniteDiffusion with A_t, B_t, P_t and an LRU of
                   per-window contributions, Sec. 3.3), the DAG chaining of
                   App. C.3.
* ``laplacian`` -- signed square root (Sec. 5.1, App. H) and the Laplacian
                   encoding / denoising decode (Sec. 5.2).

Parity status of each function is stated in its module header.
"""
