"""Pins of the oracle Chebyshev filter on H^2 (Section 4.2)."""
import numpy as np
import pytest

import bse_inputs as bi
from oracle import chebyshev, dense
from oracle.solver import k_conj


def _mus(lam_pos):
    return 0.9 * lam_pos[0], lam_pos[len(lam_pos) // 5], 1.05 * lam_pos[-1]


@pytest.mark.parametrize("seed", [0, 1])
def test_filter_equals_spectral_closed_form(seed):
    n, k = 20, 7
    P = bi.make_problem(n, seed=seed)
    lam, V = dense.eig_cholesky(P.A, P.B)
    mu1, mune, muN = _mus(lam[n:])
    W0 = bi.start_block(n, k, seed).T
    degs = np.array([1, 2, 3, 5, 8, 8, 4])
    Y = chebyshev.chebyshev_filter(P.A, P.B, W0, degs, mu1, mune, muN)
    C = np.linalg.solve(V, W0)  # W0 = V C
    for i, d in enumerate(degs):
        p = chebyshev.filter_polynomial(lam ** 2, d, mu1, mune, muN)
        ref = V @ (p * C[:, i])
        assert np.linalg.norm(Y[:, i] - ref) <= 1e-11 * np.linalg.norm(ref)


def test_filter_planted_eigenvectors_b_zero():
    # Theorem polynomial_effect_eigenvectors: on an eigenvector the filter is the scalar p(lambda^2)
    n = 24
    P = bi.make_problem(n, seed=3, b_zero=True)
    w, Qm = np.linalg.eigh(P.A)
    V = np.concatenate([Qm, np.zeros_like(Qm)], axis=0)  # v_i = [q_i; 0]
    mu1, mune, muN = 0.95 * w[0], w[6], 1.02 * w[-1]
    Y = chebyshev.chebyshev_filter(P.A, P.B, V, np.full(n, 6), mu1, mune, muN)
    p = chebyshev.filter_polynomial(w ** 2, 6, mu1, mune, muN)
    np.testing.assert_allclose(Y, V * p[None, :], atol=1e-11 * np.abs(p).max())
    # normalisation: p(mu_1^2) = 1 and |p| <= 1/|T_deg(t_1)| on the damped interval
    assert abs(chebyshev.filter_polynomial(np.array([mu1 ** 2]), 6, mu1, mune, muN)[0] - 1) < 1e-13


def test_filter_commutes_with_k_conjugation():
    # Theorem relation_polynomial: p(H^2) K conj(W) = K conj(p(H^2) W)
    n, k = 16, 5
    P = bi.make_problem(n, seed=2)
    lam, _ = dense.eig_cholesky(P.A, P.B)
    mu1, mune, muN = _mus(lam[n:])
    W = bi.start_block(n, k, 2).T
    degs = np.array([3, 3, 7, 1, 4])
    Y1 = chebyshev.chebyshev_filter(P.A, P.B, k_conj(W), degs, mu1, mune, muN)
    Y2 = k_conj(chebyshev.chebyshev_filter(P.A, P.B, W, degs, mu1, mune, muN))
    assert np.linalg.norm(Y1 - Y2) <= 1e-12 * np.linalg.norm(Y2)


def test_degree_one_is_shifted_square():
    n = 10
    P = bi.make_problem(n, seed=1)
    H = dense.hamiltonian(P.A, P.B)
    W = bi.start_block(n, 3, 1).T
    mu1, mune, muN = 0.8, 2.0, 15.0
    c, e, s1 = chebyshev.coefficients(mu1, mune, muN)
    Y = chebyshev.chebyshev_filter(P.A, P.B, W, [1, 1, 1], mu1, mune, muN)
    np.testing.assert_allclose(Y, (s1 / e) * (H @ H @ W - c * W), rtol=1e-13, atol=1e-13)


def test_chebyshev_closed_form_matches_recurrence():
    t = np.array([-3.0, -1.0, -0.3, 0.0, 0.7, 1.0, 2.5])
    T0, T1 = np.ones_like(t), t.copy()
    for m in range(2, 12):
        T0, T1 = T1, 2 * t * T1 - T0
        np.testing.assert_allclose(chebyshev.chebyshev_t(m, t), T1, rtol=1e-12, atol=1e-12)


def test_empty_block():
    P = bi.make_problem(4, seed=0)
    Y = chebyshev.chebyshev_filter(P.A, P.B, np.zeros((8, 0), complex), [], 1.0, 2.0, 10.0)
    assert Y.shape == (8, 0)
