"""FP64 CPU oracle for band-limited Jacobi PDE-EPDiff LDDMM (Hernandez, arXiv:1807.11560).

TEST INFRASTRUCTURE ONLY.  This package is the plain, slow, obviously correct
restatement of what the GPU library computes.  Only the test-suite, the smoke
check and the timed CPU baseline of the benchmark may import it; the product
path (the C-ABI library and its Python binding) never does.

It shares no code with the CUDA path: band-limited maps go through
``numpy.fft`` instead of the truncated DFT matrices the kernels use, the
semi-Lagrangian interpolation is written out corner by corner on whole arrays,
and every quantity is float64.

Modules
-------
bl         band-limited algebra of Section 3.1: iota, pi, L~, K~, spectral
           derivatives, the truncated convolution, ad~ (Eq. 49) and
           ad~^dagger (Eq. 48), V-inner product (Eq. 47).
sweeps     the time sweeps: Heun shoot of BL EPDiff (Eq. 51), its tangent
           (Eq. 30 in BL form), the backward reduced adjoint Jacobi sweep
           (Eqs. 53-54) as the exact discrete transpose of the Jacobi-field
           tangent, semi-Lagrangian state transport (Eq. 52) and incremental
           state transport (Eq. 31).
objective  energy (Eq. 50), V-gradient (Eqs. 53-55), Gauss-Newton
           Hessian-vector product (Eqs. 30-31, 56-58 under the GN reading),
           the J-form diagnostic, PCG in the V inner product and the
           Gauss-Newton-Krylov outer loop with Armijo backtracking (Eqs. 44-45).
deformation  the deformation-state form of Section 3.3: the band-limited
           inverse-map displacement swept jointly with the shoot, its tangent,
           the terminal image I0(x + u(1)), U~(1) = K~(D~phi~(1)^T * rho~(1)) and
           the energy, gradient and GN product built on them.

Every function is pinned by ``tests/test_oracle_*.py`` against closed forms,
identities, brute-force sums and convergence orders.  Parity status: pinned
for every function listed above (no function here is "parity unpinned").
"""

from . import bl, sweeps, objective  # noqa: F401
