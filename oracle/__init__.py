"""CPU oracle for ChASE on pseudo-hermitian (BSE) Hamiltonians (arXiv 2601.10557).

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, complex128 NumPy/SciPy
restatement of the paper's method, used to check the CUDA library.  Only the
test-suite, the smoke check and the benchmark's CPU-baseline leg may import it;
the library itself never does, and this package imports nothing from the
library.  Inputs come from the seeded generator module ``bse_inputs``.

Modules
-------
dense          brute-force eigensolves of H (two independent routes + Jacobi)
chebyshev      the Chebyshev filter on H^2 (Section 4.2, eq. three-term_recurrence_pseudo-hermitian);
               also the explicit-H^2 variant (H^2 from its blocks, not the paper's method)
lanczos        pseudo-hermitian Lanczos spectral bounds (Section 4.1)
qr             CholeskyQR2 with a Householder fallback (Section 4.3)
rayleigh_ritz  oblique Rayleigh-Ritz with hermitian spectral equivalence (Algorithm 2);
               also the non-hermitian fallback dual basis (Section 4.4, last paragraph)
solver         the outer subspace iteration (Algorithm 3)
gradient       eigenvalue gradient with respect to A and B (Theorem SH_HPD: u = S v)

Parity status: every function is pinned by tests in ``tests/test_oracle_*.py``:
the DOS estimate of mu_nevex and the per-vector degree rule by hand-worked cases
(``tests/test_oracle_pins.py``), mu_N as an upper bound of the spectral radius.
Only the iteration trajectory of the solver as a whole (how many iterations, which
degrees in which iteration) is "parity unpinned": it changes speed, not the
converged result, and is reported, not compared.
"""
