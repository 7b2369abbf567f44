"""Pins of the oracle for the two variants beyond the paper's default path:

* the explicit-H^2 filter (H^2 = [[P, Q], [conj Q, conj P]] formed once, one product
  per H^2 step) against the dense square of H and against the implicit filter;
* the non-hermitian fallback Rayleigh-Ritz (Section 4.4, last paragraph: a dual basis
  that needs only a nonzero diagonal of Q^* S Q) against its bi-orthogonality and the
  exact eigenpairs of invariant subspaces.
"""
import numpy as np
import pytest

import bse_inputs as bi
from oracle import chebyshev, dense, rayleigh_ritz


@pytest.mark.parametrize("real,b_zero", [(False, False), (True, False), (False, True)])
def test_h2_blocks_equal_the_dense_square(real, b_zero):
    P = bi.make_problem(36, seed=5, real=real, b_zero=b_zero)
    H = dense.hamiltonian(P.A, P.B)
    Pb, Qb = chebyshev.h2_blocks(P.A, P.B)
    H2 = np.block([[Pb, Qb], [Qb.conj(), Pb.conj()]])
    ref = H @ H
    assert np.linalg.norm(H2 - ref) <= 1e-14 * np.linalg.norm(ref)
    if b_zero:  # H^2 = diag(A^2, conj(A)^2)
        assert np.array_equal(Qb, np.zeros_like(Qb))


def test_explicit_filter_matches_the_implicit_filter():
    P = bi.make_problem(48, seed=2)
    W0 = bi.start_block(48, 10, 4)
    degs = np.random.default_rng(0).integers(1, 9, size=10)
    lam, _ = dense.eig_cholesky(P.A, P.B)
    pos = lam[P.n:]
    mus = (0.9 * pos[0], pos[len(pos) // 5], 1.05 * pos[-1])
    Pb, Qb = chebyshev.h2_blocks(P.A, P.B)
    Y1 = chebyshev.chebyshev_filter(P.A, P.B, W0.T, degs, *mus)
    Y2 = chebyshev.chebyshev_filter_explicit(Pb, Qb, W0.T, degs, *mus)
    for i in range(10):
        assert np.linalg.norm(Y2[:, i] - Y1[:, i]) <= 1e-12 * np.linalg.norm(Y1[:, i]), i


def test_explicit_filter_keeps_the_k_conjugate_symmetry():
    """Theorem relation_polynomial: p(H^2) K conj(W) = K conj(p(H^2) W)."""
    n = 30
    P = bi.make_problem(n, seed=8)
    W = bi.start_block(n, 4, 1).T
    Kc = lambda V: np.vstack([V[n:].conj(), V[:n].conj()])
    Pb, Qb = chebyshev.h2_blocks(P.A, P.B)
    mus = (0.8, 2.0, 30.0)
    Yp = chebyshev.chebyshev_filter_explicit(Pb, Qb, W, [5] * 4, *mus)
    Ym = chebyshev.chebyshev_filter_explicit(Pb, Qb, Kc(W), [5] * 4, *mus)
    assert np.linalg.norm(Ym - Kc(Yp)) <= 1e-12 * np.linalg.norm(Yp)


def _singular_qsq_pair(n: int) -> np.ndarray:
    """Two orthonormal columns with Q^* S Q = [[1/2, 1/2], [1/2, 1/2]] (singular, nonzero
    diagonal): q1 = (sqrt(3/4) e1; 1/2 f1), q2 = (a e1 + b e2; -1/2 f1)."""
    Q = np.zeros((2 * n, 2), dtype=complex)
    a = 0.25 / np.sqrt(0.75)
    Q[0, 0], Q[n, 0] = np.sqrt(0.75), 0.5
    Q[0, 1], Q[1, 1], Q[n, 1] = a, np.sqrt(0.75 - a * a), -0.5
    return Q


def test_fallback_dual_basis_is_biorthogonal():
    n = 20
    rng = np.random.default_rng(3)
    Z = rng.standard_normal((2 * n, 8)) + 1j * rng.standard_normal((2 * n, 8))
    Q, _ = np.linalg.qr(Z)
    QL = rayleigh_ritz.fallback_dual_basis(Q)
    assert np.abs(QL.conj().T @ Q - np.eye(8)).max() <= 1e-13
    Qs = _singular_qsq_pair(n)
    S = np.diag(np.r_[np.ones(n), -np.ones(n)])
    M = Qs.conj().T @ S @ Qs
    assert abs(np.linalg.det(M)) <= 1e-15 and np.allclose(np.diag(M), 0.5)
    QLs = rayleigh_ritz.fallback_dual_basis(Qs)
    assert np.abs(QLs.conj().T @ Qs - np.eye(2)).max() <= 1e-14


@pytest.mark.parametrize("m", [1, 4])
def test_fallback_rr_is_exact_on_invariant_subspaces(m):
    """Q spanning the eigenvectors of +-lambda_1..lambda_m: both Rayleigh-Ritz variants
    return lambda_1..lambda_m and eigenvectors (brute force: the dense eigensolve)."""
    n = 32
    P = bi.make_problem(n, seed=4)
    lam, V, _ = dense.eig_general(P.A, P.B)
    order = np.argsort(lam)
    pos = order[lam[order] > 0][:m]
    neg = order[lam[order] < 0][::-1][:m]
    Q, _ = np.linalg.qr(np.hstack([V[:, pos], V[:, neg]]))
    ritz, W = rayleigh_ritz.rayleigh_ritz_fallback(P.A, P.B, Q)
    np.testing.assert_allclose(ritz, lam[pos], rtol=1e-11)
    H = dense.hamiltonian(P.A, P.B)
    assert np.linalg.norm(H @ W - W * ritz[None, :], axis=0).max() <= 1e-10 * np.linalg.norm(H, 2)
    ritz2, _ = rayleigh_ritz.rayleigh_ritz(P.A, P.B, Q)
    np.testing.assert_allclose(ritz, ritz2, rtol=1e-11)


def test_oracle_solve_with_the_fallback_rr_reaches_the_dense_eigenpairs():
    """Algorithm 3 with the fallback Rayleigh-Ritz in place of Algorithm 2 still returns
    the nev smallest positive eigenpairs of the dense brute force."""
    from oracle import solver
    n, nev, nex = 64, 6, 6
    P = bi.make_problem(n, seed=0)
    W0, V0 = bi.start_block(n, nev + nex, 0), bi.lanczos_starts(n, 4, 0)
    ref, _ = dense.smallest_positive(P.A, P.B, nev)
    out = solver.solve(P.A, P.B, nev, nex, 12, 1e-10, W0, V0, deg_min=4, deg_max=24, maxiter=40, rr="fallback")
    assert out["converged"] == nev
    np.testing.assert_allclose(out["lam"], ref, rtol=1e-10)
    H = dense.hamiltonian(P.A, P.B)
    R = H @ out["V"] - out["V"] * out["lam"][None, :]
    assert np.linalg.norm(R, axis=0).max() <= 1e-9 * np.linalg.norm(H, 2)
