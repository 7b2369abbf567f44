"""Brute-force dense eigensolves of the BSE Hamiltonian (oracle; test infrastructure).

The wanted result of the method is the nev smallest positive eigenvalues of
H = [[A, B], [-conj(B), -conj(A)]] (Section 1, eq. introduction::hamiltonian_definition)
with their right eigenvectors, for S H hermitian positive definite
(eq. introduction::quasi_hermitian_condition).  Two independent routes compute it:

* ``eig_general``   -- the general non-hermitian eigensolver (LAPACK zgeev) on H;
* ``eig_cholesky``  -- the structure route from the proof of Theorem SH_HPD:
                       S H = L L^*, the hermitian problem L^* S L y = lambda y,
                       and v = L^{-*} y;

plus ``jacobi_eigh``, a hand-written cyclic Jacobi method for hermitian matrices
(Golub & Van Loan, Matrix Computations, Sec. 8.5) that pins the library routine
at small sizes.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla


def hamiltonian(A: np.ndarray, B: np.ndarray) -> np.ndarray:
    """H = [[A, B], [-conj(B), -conj(A)]] (Section 1)."""
    return np.block([[A, B], [-B.conj(), -A.conj()]])


def s_matrix(n: int) -> np.ndarray:
    """S = diag(I_n, -I_n) (eq. introduction::pseudo_hermitian_condition)."""
    return np.diag(np.concatenate([np.ones(n), -np.ones(n)])).astype(np.complex128)


def k_matrix(n: int) -> np.ndarray:
    """K = [[0, I], [I, 0]] (Theorem pseudo-hermitian_hamiltonian_eigenvalues_relation)."""
    Z = np.zeros((n, n))
    I = np.eye(n)
    return np.block([[Z, I], [I, Z]]).astype(np.complex128)


def _normalise(V: np.ndarray) -> np.ndarray:
    V = V / np.linalg.norm(V, axis=0, keepdims=True)
    return V


def fix_phase(V: np.ndarray) -> np.ndarray:
    """Unit-phase convention: the largest-magnitude entry of the upper block of
    each column is made real and positive."""
    n = V.shape[0] // 2
    idx = np.argmax(np.abs(V[:n]), axis=0)
    ph = V[idx, np.arange(V.shape[1])]
    return V * (np.abs(ph) / ph)[None, :]


def eig_general(A: np.ndarray, B: np.ndarray):
    """All eigenpairs of H by zgeev.  Returns (lam ascending, V normalised).

    Eigenvalues of a definite H are real (Theorem SH_HPD); the tiny imaginary
    parts left by the non-hermitian solver are returned separately so tests can
    check them.
    """
    H = hamiltonian(A, B)
    w, V = sla.eig(H)
    order = np.argsort(w.real)
    w = w[order]
    V = _normalise(V[:, order])
    return w.real.copy(), V, np.abs(w.imag).max()


def eig_cholesky(A: np.ndarray, B: np.ndarray):
    """All eigenpairs of H through S H = L L^* and L^* S L y = lambda y (proof of
    Theorem SH_HPD).  Returns (lam ascending, V normalised right eigenvectors)."""
    n = A.shape[0]
    SH = np.block([[A, B], [B.conj(), A.conj()]])
    L = sla.cholesky(SH, lower=True)
    s = np.concatenate([np.ones(n), -np.ones(n)])
    M = L.conj().T @ (s[:, None] * L)
    M = 0.5 * (M + M.conj().T)
    lam, Y = sla.eigh(M)
    V = sla.solve_triangular(L.conj().T, Y, lower=False)
    return lam, _normalise(V)


def smallest_positive(A: np.ndarray, B: np.ndarray, nev: int, route: str = "cholesky"):
    """The nev smallest positive eigenvalues and their right eigenvectors
    (phase-fixed), by the chosen brute-force route."""
    if route == "cholesky":
        lam, V = eig_cholesky(A, B)
    else:
        lam, V, _ = eig_general(A, B)
    pos = np.where(lam > 0)[0]
    sel = pos[:nev]
    return lam[sel].copy(), fix_phase(V[:, sel])


def jacobi_eigh(M: np.ndarray, tol: float = 1e-15, max_sweeps: int = 60):
    """Cyclic-by-row Jacobi method for a hermitian matrix M.

    Each (p, q) rotation is the unitary J = diag(1, e^{-i phi}) R(c, s), where
    phi = arg(M_pq) makes the 2x2 block real and the real rotation R zeroes it
    (Golub & Van Loan, Algorithm 8.5.1 "sym.schur2").  Returns (eigenvalues
    ascending, eigenvectors).
    """
    M = np.array(M, dtype=np.complex128, copy=True)
    m = M.shape[0]
    V = np.eye(m, dtype=np.complex128)
    fro = np.linalg.norm(M)
    for _ in range(max_sweeps):
        off = np.linalg.norm(M - np.diag(np.diag(M)))
        if off <= tol * fro:
            break
        for p in range(m - 1):
            for q in range(p + 1, m):
                apq = M[p, q]
                r = abs(apq)
                if r == 0.0:
                    continue
                e_phi = apq / r
                app = M[p, p].real
                aqq = M[q, q].real
                tau = (aqq - app) / (2.0 * r)
                t = (1.0 if tau >= 0 else -1.0) / (abs(tau) + np.sqrt(1.0 + tau * tau))
                c = 1.0 / np.sqrt(1.0 + t * t)
                s = t * c
                J = np.array([[c, s], [-s * np.conj(e_phi), c * np.conj(e_phi)]])
                idx = [p, q]
                M[:, idx] = M[:, idx] @ J
                M[idx, :] = J.conj().T @ M[idx, :]
                V[:, idx] = V[:, idx] @ J
    lam = np.diag(M).real.copy()
    order = np.argsort(lam)
    return lam[order], V[:, order]
