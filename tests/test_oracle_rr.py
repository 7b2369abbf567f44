"""Pins of the oblique Rayleigh-Ritz oracle (Section 4.4, Algorithm 2, Section 5)."""
import numpy as np
import pytest
import scipy.linalg as sla

import bse_inputs as bi
from oracle import dense, qr, rayleigh_ritz as rr
from oracle.solver import k_conj, s_flip


def _problem(n=30, seed=0):
    P = bi.make_problem(n, seed=seed)
    lam, V = dense.eig_cholesky(P.A, P.B)
    return P, lam[n:], V[:, n:]


def _basis(Wp):
    Q, _ = qr.cholesky_qr2(np.concatenate([Wp, k_conj(Wp)], axis=1))
    return Q


def test_qsq_identity_and_pm_symmetry():
    n = 30
    P, _, _ = _problem(n)
    Wp = bi.start_block(n, 6, 0).T
    Wp[n:] *= 1e-3
    Q = _basis(Wp)
    ritz, W, theta, M2 = rr.rayleigh_ritz(P.A, P.B, Q, return_all=True)
    # Algorithm 2: I - 2 Q_2^* Q_2 = Q^* S Q
    np.testing.assert_allclose(M2, Q.conj().T @ s_flip(Q), atol=1e-13)
    # Theorem positive-negative-symmetry_oblique_RR: spectrum of G is +- symmetric
    np.testing.assert_allclose(np.sort(theta), -np.sort(theta)[::-1], atol=1e-12 * np.abs(theta).max())
    assert len(ritz) == 6 and np.all(ritz > 0) and np.all(np.diff(ritz) >= 0)


def test_exact_on_invariant_subspace():
    n = 30
    P, lam, V = _problem(n, seed=1)
    Q = _basis(V[:, :5])
    ritz, W = rr.rayleigh_ritz(P.A, P.B, Q)
    np.testing.assert_allclose(ritz, lam[:5], rtol=1e-12)
    res = rr.residuals(P.A, P.B, W, ritz)
    assert res.max() < 1e-11 * lam.max()


def test_printed_back_transform_reading():
    # The right Ritz vector is z = L^{-*} y (Theorem spectral_equivalent: y = L^* z);
    # the L^{-1} y printed in Algorithm 2 does not give eigenvectors.
    n = 30
    P, lam, V = _problem(n, seed=2)
    Q = _basis(V[:, :4])
    H = dense.hamiltonian(P.A, P.B)
    T = s_flip(H @ Q)
    L = np.linalg.cholesky(0.5 * (Q.conj().T @ T + (Q.conj().T @ T).conj().T))
    M2 = Q.conj().T @ s_flip(Q)
    G = sla.solve_triangular(L, M2, lower=True)
    G = sla.solve_triangular(L, G.conj().T, lower=True).conj().T
    th, Y = np.linalg.eigh(0.5 * (G + G.conj().T))
    i = np.argmax(th)
    for back, ok in ((sla.solve_triangular(L.conj().T, Y[:, i], lower=False), True),
                     (sla.solve_triangular(L, Y[:, i], lower=True), False)):
        w = Q @ back
        w /= np.linalg.norm(w)
        r = np.linalg.norm(H @ w - w / th[i])
        assert (r < 1e-10) == ok


def test_ritz_interval():
    # Theorem field_of_values_ritz_hermitian_variant
    n = 30
    P, _, _ = _problem(n, seed=3)
    SH = np.block([[P.A, P.B], [P.B.conj(), P.A.conj()]])
    rho = np.linalg.eigvalsh(SH).max()
    for s in range(3):
        Wp = bi.start_block(n, 5, s).T
        Wp[n:] *= 0.3
        Q = _basis(Wp)
        _, _, theta, M2 = rr.rayleigh_ritz(P.A, P.B, Q, return_all=True)
        bound = rho / np.abs(np.linalg.eigvalsh(M2)).min()
        assert np.all(np.abs(1.0 / theta) <= bound * (1 + 1e-12))


def test_quadratic_convergence():
    # Lemma hermitian_equivalent_rayleigh-ritz_quadratic: |lambda - ritz| = O(sigma^2)
    n = 30
    P, lam, V = _problem(n, seed=4)
    E = bi.start_block(n, 3, 4).T
    errs = []
    sig = np.array([1e-2, 1e-3, 1e-4, 1e-5])
    for s in sig:
        Q = _basis(V[:, :3] + s * E)
        ritz, _ = rr.rayleigh_ritz(P.A, P.B, Q)
        errs.append(np.abs(ritz - lam[:3]).max())
    slope = np.polyfit(np.log(sig), np.log(errs), 1)[0]
    assert 1.8 < slope < 2.3, (slope, errs)


def test_not_definite_raises():
    n = 8
    A = np.eye(n, dtype=complex)
    B = 2.0 * np.eye(n, dtype=complex)   # ||B|| > min eig(A): S H indefinite
    Q, _ = np.linalg.qr(bi.start_block(n, 4, 0).T)
    with pytest.raises(rr.NotDefinite):
        rr.rayleigh_ritz(A, B, Q)
