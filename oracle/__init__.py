"""FP64 CPU oracle for the SENSE / unrolled-reconstruction hot path.

TEST INFRASTRUCTURE ONLY.  Nothing in the product package imports, links or
runs this code; only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may use it.  It shares no code with the CUDA path.

Every function is a plain, slow, obviously-correct NumPy (complex128/float64)
implementation of what the paper defines, each citing the passage it follows
(Blumenthal et al., "Deep, Deep Learning with BART"):

* ``fft``      centred unitary 2-D DFT F (the Fourier factor of A = PFC, Eq. 4
               "inverse_problem", Sec. 2.3)
* ``sense``    A = P F C, its adjoint A^H and the normal operator A^H A + lambda I
               (Eq. 4 and the MoDL update, Eq. 6 "update_modl")
* ``cg``       conjugate gradient applying S_lambda^{-1}, and its derivative
               (the inversion nlop S^{-1} and its derivatives, Sec. 2.3.2, MoDL)
* ``nn``       direct-sum convolutions, ReLU, Gaussian-RBF activation
               (MoDL residual CNN D_W; VarNet regulariser K, Phi')
* ``unrolled`` MoDL (Eq. 6) and VarNet (Eq. 5 "update_vn") blocks, forward and
               reverse mode, with the paper's complex-gradient convention
* ``ipalm``    the iPALM update of the VarNet parameters with the filter constraints
               (Sec. 2.3.1, training)
* ``noncart``  non-Cartesian SENSE: direct non-uniform DFT pair, the PSF and the
               Toeplitz-embedded normal operator (Sec. 2.3.3)
               (Sec. 2.2.2 "Complex numbers": the real part of the gradient is
               the derivative with respect to the real part, the imaginary
               part with respect to the imaginary part).

Every function here is pinned by a ``-m "not gpu"`` test against something
other than itself (naive O(N^2) DFT, adjoint identity, closed forms, dense
direct solves, brute-force loops, finite differences); see ``tests/``.
"""
from . import fft, sense, cg, nn, unrolled, noncart, ipalm  # noqa: F401
