"""CPU oracle for the circulant-preconditioned voxel VIE (Groth, Polimeridis,
Tambova, White, "Circulant preconditioning in the volume integral equation
method for silicon photonics").

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The product path
(the CUDA library and its Python binding) never imports, calls or links it, and
this package imports nothing from the CUDA path: the only module both sides
share is the input generator ``paper_1903_07884_gb300.inputs``.

Everything here is plain FP64 NumPy/SciPy, written from the paper's equations
and in their order; library primitives (FFT, LU, triangular solve) serve as
single steps.  Each function cites the passage it follows.

Parity status per function (see the pin tests in tests/test_oracle_*.py):
  greens.entries / self_term      pinned (finite differences, quadrature,
                                   static limit, trace identity, parity)
  operator.dense_matrix           pinned (symmetry, single voxel closed form)
  operator.material / rhs         pinned (Table 1 contrasts; the single voxel's
                                   static limit is the Clausius-Mossotti factor)
  operator.background_k           pinned (the cladding wavelength lambda0 /
                                   sqrt(eps_b) puts whole periods of phase
                                   between the radiating traces)
  operator.fft_matvec             pinned (equals dense on brute-force grids)
  circulant.*                     pinned (Eq. Chan hand example, Frobenius
                                   optimality, eigen-decomposition)
  precond.*                       pinned (dense definition vs per-frequency,
                                   P^-1 P x = x, S1 symmetry, tau = 0)
  precond2.* (2-level)            pinned (2-level Frobenius projection of the
                                   dense box matrix, level-by-level Chan-Olkin
                                   identity, dense solve, x/y parity, ny = 1
                                   reduces to 1-level)
  homogenize.*                    pinned (hand examples)
  gmres.gmres                     pinned (dense LU solve, 1-step exactness)
"""
