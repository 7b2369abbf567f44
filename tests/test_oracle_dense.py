"""Pins of the brute-force eigensolves against facts the paper and mathematics fix."""
import numpy as np
import pytest
import scipy.linalg as sla

import bse_inputs as bi
from oracle import dense


@pytest.mark.parametrize("seed", [0, 1])
def test_two_routes_agree_and_pm_pairs(seed):
    P = bi.make_problem(40, seed=seed)
    lam_g, V_g, im = dense.eig_general(P.A, P.B)
    lam_c, V_c = dense.eig_cholesky(P.A, P.B)
    H = dense.hamiltonian(P.A, P.B)
    # Theorem SH_HPD: real spectrum
    assert im < 1e-10
    np.testing.assert_allclose(lam_g, lam_c, rtol=0, atol=1e-11 * np.abs(lam_c).max())
    # +- pairs (Theorem pseudo-hermitian_hamiltonian_eigenvalues_relation)
    np.testing.assert_allclose(lam_c, -lam_c[::-1], atol=1e-11 * np.abs(lam_c).max())
    for lam, V in ((lam_g, V_g), (lam_c, V_c)):
        R = H @ V - V * lam[None, :]
        assert np.linalg.norm(R, axis=0).max() < 1e-11 * np.abs(lam).max()


def test_closed_form_n1():
    # H = [[a, b], [-conj(b), -a]]: det(H - x) = x^2 - a^2 + |b|^2
    for a, b in [(2.0, 0.5 + 0.3j), (1.0, 0.9j), (5.0, -1.2)]:
        A = np.array([[a]], dtype=complex)
        B = np.array([[b]], dtype=complex)
        lam, _ = dense.eig_cholesky(A, B)
        ref = np.sqrt(a * a - abs(b) ** 2)
        np.testing.assert_allclose(lam, [-ref, ref], rtol=1e-14)


def test_closed_form_block_diagonal():
    rng = np.random.default_rng(5)
    n = 12
    a = rng.uniform(1, 4, n)
    b = rng.uniform(0, 0.9, n) * a * np.exp(2j * np.pi * rng.uniform(size=n))
    lam, V = dense.eig_cholesky(np.diag(a).astype(complex), np.diag(b))
    ref = np.sort(np.sqrt(a * a - np.abs(b) ** 2))
    np.testing.assert_allclose(lam[n:], ref, rtol=1e-13)
    lam_g, _, _ = dense.eig_general(np.diag(a).astype(complex), np.diag(b))
    np.testing.assert_allclose(lam_g[n:], ref, rtol=1e-13)


def test_b_zero_planted_spectrum():
    P = bi.make_problem(48, seed=3, b_zero=True)
    lam, _ = dense.eig_cholesky(P.A, P.B)
    np.testing.assert_allclose(lam[48:], np.sort(P.d), rtol=1e-12)
    np.testing.assert_allclose(lam[:48], -np.sort(P.d)[::-1], rtol=1e-12)


def test_real_case_squared_spectrum():
    # A, B real symmetric: H^2 restricted gives lambda^2 = eig((A - B)(A + B))
    P = bi.make_problem(40, seed=2, real=True)
    A, B = P.A.real, P.B.real
    lam, _ = dense.eig_cholesky(P.A, P.B)
    ref = np.sort(np.linalg.eigvals((A - B) @ (A + B)).real)
    np.testing.assert_allclose(np.sort(lam[40:] ** 2), ref, rtol=1e-11)


def test_left_eigenvectors_and_k_conjugacy():
    P = bi.make_problem(32, seed=4)
    n = 32
    H = dense.hamiltonian(P.A, P.B)
    S = dense.s_matrix(n)
    K = dense.k_matrix(n)
    lam, V = dense.eig_cholesky(P.A, P.B)
    for i in [n, n + 3, 2 * n - 1]:
        v = V[:, i]
        u = S @ v  # Theorem SH_HPD
        assert np.linalg.norm(u.conj() @ H - lam[i] * u.conj()) < 1e-11 * abs(lam).max()
        w = K @ v.conj()  # H K conj(v) = -lambda K conj(v)
        assert np.linalg.norm(H @ w + lam[i] * w) < 1e-11 * abs(lam).max()
    # D = V^* S V diagonal with D_- = -D_+ (eq. bi-orthogonality, symmetry_diagonals)
    D = V.conj().T @ S @ V
    off = D - np.diag(np.diag(D))
    assert np.abs(off).max() < 1e-10
    dpos = np.diag(D)[n:].real
    dneg = np.diag(D)[:n].real[::-1]
    assert np.all(dpos > 0)
    np.testing.assert_allclose(dneg, -dpos, rtol=1e-9)


def test_bounds_tda_and_spectral_radius():
    for seed in range(3):
        P = bi.make_problem(60, seed=seed)
        lam, _ = dense.eig_cholesky(P.A, P.B)
        pos = lam[60:]
        # Lemma interval_of_real_eigenvalues
        assert np.abs(lam).max() <= np.abs(np.linalg.eigvalsh(P.A)).max() * (1 + 1e-12)
        # eigenvalues of A bound the positive eigenvalues index-wise (Section 3)
        assert np.all(pos <= np.sort(P.d) * (1 + 1e-12))


def test_condition_numbers_equal():
    P = bi.make_problem(24, seed=6)
    H = dense.hamiltonian(P.A, P.B)
    SH = dense.s_matrix(24) @ H
    np.testing.assert_allclose(np.linalg.cond(H), np.linalg.cond(SH), rtol=1e-9)


@pytest.mark.parametrize("m", [1, 2, 9, 24])
def test_jacobi_matches_planted_and_library(m):
    rng = np.random.default_rng(m)
    Qm = bi.haar_unitary(m, rng)
    d = np.sort(rng.uniform(-3, 3, m))
    M = (Qm * d) @ Qm.conj().T
    M = 0.5 * (M + M.conj().T)
    lam, V = dense.jacobi_eigh(M)
    np.testing.assert_allclose(lam, d, atol=1e-13)
    assert np.linalg.norm(M @ V - V * lam) < 1e-12
    assert np.linalg.norm(V.conj().T @ V - np.eye(m)) < 1e-12


def test_jacobi_pins_structure_route():
    P = bi.make_problem(16, seed=7)
    n = 16
    SH = np.block([[P.A, P.B], [P.B.conj(), P.A.conj()]])
    L = sla.cholesky(SH, lower=True)
    M = L.conj().T @ dense.s_matrix(n) @ L
    lam_j, _ = dense.jacobi_eigh(0.5 * (M + M.conj().T))
    lam_c, _ = dense.eig_cholesky(P.A, P.B)
    np.testing.assert_allclose(lam_j, lam_c, atol=1e-12 * np.abs(lam_c).max())
