"""Oblique Rayleigh-Ritz with hermitian spectral equivalence (oracle; test infrastructure).

Section 4.4, Algorithm 2 and Theorem spectral_equivalent_hermitian_eigenvalue_problem:
with the dual basis Q_L = S Q (Q^* S Q)^{-1} the Rayleigh quotient is
G = (Q^* S Q)^{-1} Q^* S H Q; with Q^* S H Q = L L^* it is spectrally equivalent
to the hermitian L^* (Q^* S Q)^{-1} L, whose inverse L^{-1} (Q^* S Q) L^{-*} is
formed without any inversion.  Steps (Algorithm 2):

    T = H Q;  T <- S T;  M = Q^* T;  L = chol(M);
    M2 = I - 2 Q_2^* Q_2   (= Q^* S Q, Q_2 the lower half of Q);
    G = L^{-1} M2 L^{-*};  G y = theta y;  lambda = 1 / theta;
    z = L^{-*} y.

The printed back-transform uses L^{-1}; from y = L^* z (Theorem
spectral_equivalent) the right Ritz vector is z = L^{-*} y, which is what is
used here.  By Theorem positive-negative-symmetry_oblique_RR the spectrum of G is
+-symmetric, so only the k/2 positive theta are kept (Section 4.5), and only
W_+ = Q Z_+ is back-transformed (Algorithm 3).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

from .dense import hamiltonian


class NotDefinite(RuntimeError):
    """Cholesky of Q^* S H Q failed (S H not positive definite on range(Q))."""


def rayleigh_ritz(A, B, Q, return_all: bool = False):
    """Returns (ritz ascending positive values, W_plus normalised columns).

    With ``return_all`` also returns the full theta spectrum of G and M2.
    """
    n = A.shape[0]
    H = hamiltonian(A, B)
    k = Q.shape[1]
    T = H @ Q
    T[n:, :] *= -1.0                       # T <- S T
    M = Q.conj().T @ T                     # Q^* S H Q
    M = 0.5 * (M + M.conj().T)
    try:
        L = np.linalg.cholesky(M)
    except np.linalg.LinAlgError as exc:
        raise NotDefinite(str(exc)) from exc
    Q2 = Q[n:, :]
    M2 = np.eye(k) - 2.0 * (Q2.conj().T @ Q2)   # Q^* S Q
    G = sla.solve_triangular(L, M2, lower=True)                       # L^{-1} M2
    G = sla.solve_triangular(L, G.conj().T, lower=True).conj().T      # (.) L^{-*}
    G = 0.5 * (G + G.conj().T)
    theta, Y = np.linalg.eigh(G)
    pos = np.where(theta > 0)[0]
    pos = pos[np.argsort(-theta[pos])]     # largest theta = smallest lambda first
    ritz = 1.0 / theta[pos]
    Z = sla.solve_triangular(L.conj().T, Y[:, pos], lower=False)      # L^{-*} Y_+
    W = Q @ Z
    W = W / np.linalg.norm(W, axis=0, keepdims=True)
    if return_all:
        return ritz, W, theta, M2
    return ritz, W


def residuals(A, B, W, ritz):
    """||H w_i - lambda_i w_i||_2 for unit columns w_i (Section 4.5)."""
    H = hamiltonian(A, B)
    R = H @ W - W * ritz[None, :]
    return np.linalg.norm(R, axis=0)


def fallback_dual_basis(Q: np.ndarray) -> np.ndarray:
    """The dual basis of the non-hermitian fallback (Section 4.4, last paragraph):
    Q_L = [S Q - Q (M - diag M)] diag(M)^{-1} with M = Q^* S Q, defined whenever the
    diagonal of M has no zero (M itself may be singular).  For orthonormal Q,
    Q_L^* Q = I."""
    n = Q.shape[0] // 2
    SQ = Q.copy()
    SQ[n:, :] *= -1.0
    M = Q.conj().T @ SQ
    d = np.real(np.diag(M))
    if np.any(d == 0.0):
        raise ZeroDivisionError("Q^* S Q has a zero diagonal entry")
    return (SQ - Q @ (M - np.diag(np.diag(M)))) / d[None, :]


def rayleigh_ritz_fallback(A, B, Q):
    """Non-hermitian fallback Rayleigh-Ritz: G = Q_L^* H Q with the dual basis of
    ``fallback_dual_basis``, a general (non-hermitian) eigensolve of G, and the
    Ritz pairs with positive real part, ascending: returns (ritz, W_plus) with unit
    columns W_plus = Q Z_plus.  No spectral equivalence to a hermitian matrix is used."""
    H = hamiltonian(A, B)
    QL = fallback_dual_basis(Q)
    G = QL.conj().T @ (H @ Q)
    lam, Z = np.linalg.eig(G)
    pos = np.where(lam.real > 0)[0]
    pos = pos[np.argsort(lam.real[pos])]
    W = Q @ Z[:, pos]
    W = W / np.linalg.norm(W, axis=0, keepdims=True)
    return lam[pos].real, W
