"""FP64 CPU oracle of the widefield measurement operator (test infrastructure).

This package is the correctness reference for the CUDA library and nothing
else: only the tests, the smoke check and the benchmark's CPU-baseline leg may
import it.  It shares no code with the CUDA path.  Every function follows the
paper's definitions step by step in plain NumPy/SciPy at double precision:

* ``direct``   - the direct measurement equation (Eq. 1 and Eq. 2), brute force.
* ``kb``       - the Kaiser-Bessel NUFFT interpolation kernel, its Fourier
                 transform and the grid correction (Section 2, NUFFT of Fessler).
* ``wterm``    - w-term chirp, w-layers and residual w-kernels (Section 3.1, Fig. 1).
* ``plan``     - k-means w-bins, support table, cost/memory models and the
                 planning decision tree (Section 3.1, Section 3.4, Eq. 5, Eq. 9,
                 Eq. 10, Fig. 2).
* ``operator`` - Phi = [G_p F Z_p]_p, its adjoint, Phi^dagger Phi, the PSF and the
                 holographic matrices H_p = G_p^dagger G_p (Eq. 6, Eq. 7, Eq. 8,
                 Section 3.3).
* ``mlp``      - FP64 forward/backward of the kernel-surrogate MLP.
"""
