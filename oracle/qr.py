"""Orthonormalisation of the search space (oracle; test infrastructure).

Section 4.3 and Section 2: the search space is orthonormalised with a Cholesky QR
or, when it is ill-conditioned, a Householder QR.  Reading used here (the switch
rule is in a reference not available): CholeskyQR2 -- R = chol(X^* X)^*,
X <- X R^{-1}, done twice -- and Householder QR (LAPACK zgeqrf via numpy) when
the first Cholesky factorisation breaks down or its estimated condition
(max r_ii / min r_ii)^2 exceeds 1e12.  Q is unique up to a unitary
diagonal; the Rayleigh-Ritz step is invariant to it.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

COND_LIMIT = 1e12


def cholesky_qr2(X: np.ndarray):
    """Returns (Q, used_householder)."""
    G = X.conj().T @ X
    G = 0.5 * (G + G.conj().T)
    try:
        L = np.linalg.cholesky(G)
    except np.linalg.LinAlgError:
        return householder_qr(X), True
    r = np.abs(np.diag(L))
    if r.min() == 0.0 or (r.max() / r.min()) ** 2 > COND_LIMIT:
        return householder_qr(X), True
    Q1 = sla.solve_triangular(L, X.conj().T, lower=True).conj().T  # X L^{-*}
    G2 = Q1.conj().T @ Q1
    G2 = 0.5 * (G2 + G2.conj().T)
    L2 = np.linalg.cholesky(G2)
    Q = sla.solve_triangular(L2, Q1.conj().T, lower=True).conj().T
    return Q, False


def householder_qr(X: np.ndarray) -> np.ndarray:
    Q, _ = np.linalg.qr(X, mode="reduced")
    return Q
