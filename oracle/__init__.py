"""FP64 CPU oracle for the HOTRG coarse-graining step and its backward.

TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check of the
package entry module and the CPU-baseline leg of the benchmark may import
anything from here.  The product (the CUDA library and its Python binding)
never imports, links or calls this package, and this package never imports
the product: the two share no code, no headers, no constants and no helpers.
The only common module is ``synth`` (seeded input generators, no HOTRG
arithmetic).

Contents
--------
ising      site tensor T0(beta, J, h) of the square-lattice Ising model and
           its beta derivative (SM Sec. A).
hotrg      plain NumPy/LAPACK HOTRG forward (SM Sec. B, HOTRG step equation;
           isometry from the local higher-order SVD, i.e. the eigenvectors
           of the environment Gram matrix) and its reverse-mode backward
           (SM Sec. B second-renormalization recursion, SM Sec. E Jacobian
           and chain rule, plus the adjoint of the truncated eigensolve).
dtrg       differentiable-TRG sweeps: environments of the isometries and
           the MERA update (main text Eq. (1) and the MERA paragraph).
xy         quantum XY chain: exact partition functions (SM Sec. G, with
           exact diagonalisation as their pin) and the second-order
           Trotter MPO of rho(tau) (SM Sec. F).
xtrg       scheme (b) of main text Fig. 1b: vertical-only coarse-graining
           of the MPO (exponential cooling), the exact final product, its
           backward and the differentiable-TRG cooling with depth n_d.
exact      closed forms and exact small-lattice references used as pins:
           Onsager's free energy (two independent integral forms), brute-force
           enumeration of periodic tori (C), and exact transfer-matrix
           contraction of a torus of T0 tensors.

Parity status: every function here is pinned by tests under ``tests/``
(test_oracle_*.py) against brute force, closed forms, invariants or finite
differences; none is "parity unpinned".
"""
