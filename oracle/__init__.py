"""FP64 CPU oracle for the bilateral-filter graph operator and its Krylov filters.

TEST INFRASTRUCTURE, NOT PART OF THE PRODUCT.  Only the test suite, the smoke check and
the CPU-baseline leg of the benchmark may import anything from this package.  The CUDA
library never calls it and it never calls the CUDA library: the two share no code.

Plain numpy / scipy.sparse in float64, written step by step from the paper
(Knyazev & Malyshev, "Accelerated graph-based spectral polynomial filters", 2015):

* ``graph``    -- the weights of Eq. 2 over a window, the adjacency W, degree D,
                  Laplacian L = D - W (Eq. 4), the BF step D^-1 W (Eq. 3) and the two
                  normalised Laplacians (Section 4), as explicit CSR matrices.
* ``solvers``  -- simple iteration (Section 4), preconditioned CG (Algorithm 2, with the
                  flexible beta of Section 5) and block LOBPCG (Algorithm 3, Section 6).
* ``spectral`` -- dense eigendecompositions (Eq. 8) used as pins: the CG polynomial
                  filter evaluated spectrally, and exact low-pass projections.
* ``convnet``  -- the small conv net used as a learned preconditioner (forward, backward).
* ``precond_spd`` -- a learned symmetric positive definite preconditioner
                  T = D^-1/2 (I + K^T K) D^-1/2 (K a small convolution), its A-norm
                  training loss and gradient.
* ``guided``   -- Section 3's guided filter: Algorithm 1 with truncated mean filters and
                  the matrix of Eq. 6 it applies (degree, Laplacian) as explicit CSR.

Every function is pinned by ``tests/test_oracle_*.py`` against facts the paper or the
mathematics fixes (symmetry, row sums, null vector, closed-form spectra, Krylov
optimality, hand-computed values), never against the CUDA path.
"""
