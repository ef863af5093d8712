"""CPU oracle for the rectangular-cavity solver (Chen, Jiang, Lai, Li: fast
algorithm for electromagnetic scattering from a large rectangular cavity in 3D).

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, complex128 restatement
of the paper's discretised problem.  Only the test-suite, the smoke check and the
CPU-baseline leg of the benchmark may import it; the product path (the CUDA
library and its Python binding) never does, and shares no code with it.

Modules
  geometry    index sets N1, N2, N3 (Sec. 3), Appendix A ordering, layer levels
  zsystem     per-mode finite-difference systems in x3 (Sec. 3, Sec. 4),
              solved directly with banded LU (partial pivoting, Algorithm I/II
              Step 2)
  khat        Fourier transform of the truncated Green's function (Sec. 5.2)
  tbc         the singular integrals I1, I2, I3 by the FFT route of Sec. 5.2
              (closed-form transform of the truncated basis, kernel table,
              inverse DFT to the aperture nodes, trapezoid outer rule)
  excitation  incident plane wave (Sec. 2, Sec. 7) and the vectors g1, g2
  aperture    the reduced aperture system (EJ1) / (uT1): dense or matrix-free
  field       interior back-substitution (EInter) and cos/sin synthesis (E123F)
  rcs         backscatter radar cross section from the aperture field (EGa2)
  brute       the full unreduced system on tiny grids (for pinning the
              elimination)
  solver      end-to-end driver

Every function cites the equation or section of the paper it follows.
"""

from .geometry import Cavity, Layer  # noqa: F401
