"""FP64 CPU oracle for the multicoil non-Cartesian MRI hot path of
"Robust Plug-and-Play Methods for Highly Accelerated Non-Cartesian MRI
Reconstruction" (Comby, Lapostolle, Terris, Ciuciu; arXiv 2411.01955).

THIS PACKAGE IS TEST INFRASTRUCTURE.  Only the test suite, the smoke check of
the package entry file and the CPU-baseline leg of the benchmark may import it.
The CUDA library never calls it, and it shares no code with the CUDA path:
every formula here is written out again from the paper (and, where the paper
is silent, from the readings listed in the design notes), in plain NumPy,
float64, with no blocking, fusion or reordering beyond what the definitions
state.

Modules
-------
kb        Kaiser-Bessel kernel, its own I0 power series and closed-form transform.
nudft     exact non-uniform DFT forward/adjoint (the definition of A in Eq. (1)).
nufft     gridding NUFFT with the same kernel parameters as the GPU path.
toeplitz  Toeplitz embedding of A^H A and the Strang circulant preconditioner.
nufft3d   volumetric operator: exact 3D NUDFT, 3D gridding, 2N^3 Toeplitz embedding.
solvers   PCG, flexible CG, CG energy, power iteration.
smaps     S-map estimation from the windowed k-space centre (Sec. 4.1).
hqs       PnP-HQS / PnP-PGD loops (Sec. 3.3), Gaussian-smoothing denoiser,
          P-metric prox coefficients (Sec. 3.4).
convnet   small 2-channel conv net: forward, backward, Adam.

Parity status: every function has an independent pin in tests/test_oracle_pins.py
(tests/test_oracle_pins_3d.py for nufft3d)
except the annealed HQS run with a non-proximal denoiser, which has no closed
form: there only iterate-level agreement is checked ("parity unpinned" beyond that).
"""
