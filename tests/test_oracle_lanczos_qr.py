"""Pins of the Lanczos bounds (Section 4.1) and the QR step (Section 4.3)."""
import numpy as np
import pytest

import bse_inputs as bi
from oracle import dense, lanczos, qr


def test_lanczos_basis_is_sh_orthonormal_and_tridiagonal():
    n = 20
    P = bi.make_problem(n, seed=0)
    H = dense.hamiltonian(P.A, P.B)
    M = dense.s_matrix(n) @ H
    v0 = bi.lanczos_starts(n, 1, 0)[0]
    al, be, Vb = lanczos.lanczos_tridiagonal(P.A, P.B, v0, 8, return_basis=True)
    G = Vb.conj().T @ M @ Vb
    assert np.abs(G - np.eye(8)).max() < 1e-10
    T = Vb.conj().T @ M @ H @ Vb
    Tref = np.diag(al) + np.diag(be[:7], 1) + np.diag(be[:7], -1)
    assert np.abs(T - Tref).max() < 1e-9


def test_full_lanczos_recovers_spectrum():
    n = 6
    P = bi.make_problem(n, seed=1)
    lam, _ = dense.eig_cholesky(P.A, P.B)
    v0 = bi.lanczos_starts(n, 1, 1)[0]
    al, be = lanczos.lanczos_tridiagonal(P.A, P.B, v0, 2 * n)
    th, tau = lanczos.ritz_and_weights(al, be)
    np.testing.assert_allclose(np.sort(th), lam, atol=1e-8 * np.abs(lam).max())
    assert abs(tau.sum() - 1.0) < 1e-12


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_mu_n_bounds_spectral_radius(seed):
    n = 64
    P = bi.make_problem(n, seed=seed)
    lam, _ = dense.eig_cholesky(P.A, P.B)
    mu1, mune, muN = lanczos.spectral_bounds(P.A, P.B, bi.lanczos_starts(n, 4, seed), 26, 12)
    assert muN >= np.abs(lam).max()
    assert 0 < mu1 <= mune <= muN


def test_cholesky_qr2_orthonormal_and_triangular():
    rng = np.random.default_rng(0)
    X = rng.standard_normal((50, 9)) + 1j * rng.standard_normal((50, 9))
    Q, hh = qr.cholesky_qr2(X)
    assert not hh
    assert np.abs(Q.conj().T @ Q - np.eye(9)).max() < 1e-13
    R = Q.conj().T @ X
    assert np.abs(np.tril(R, -1)).max() < 1e-12   # X = Q R with R upper triangular
    assert np.linalg.norm(Q @ R - X) < 1e-12 * np.linalg.norm(X)


def test_householder_fallback_on_ill_conditioned():
    rng = np.random.default_rng(1)
    U, _ = np.linalg.qr(rng.standard_normal((60, 8)) + 1j * rng.standard_normal((60, 8)))
    X = U * np.logspace(0, -9, 8)[None, :]          # cond 1e9 -> cond(X^*X) = 1e18
    Q, hh = qr.cholesky_qr2(X)
    assert hh
    assert np.abs(Q.conj().T @ Q - np.eye(8)).max() < 1e-13
    R = Q.conj().T @ X
    assert np.abs(np.tril(R, -1)).max() < 1e-12 * np.abs(R).max()
