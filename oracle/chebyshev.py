"""Chebyshev filter on H^2 (oracle; test infrastructure).

Section 4.2 (eq. three-term_recurrence_pseudo-hermitian) filters with a
Chebyshev polynomial of H^2 so that the spectrum is folded at zero and the
smallest |lambda| are amplified.  The paper leaves the recurrence coefficients
unstated (its "W_1 := A W_0" is carried over from the hermitian case); this
oracle uses the scaled three-term recurrence of Zhou, Saad, Tiago & Chelikowsky
(J. Comput. Phys. 219, 2006) on the operator H^2:

    a = mu_nevex^2,  b = mu_N^2,  c = (a + b) / 2,  e = (b - a) / 2,
    sigma_1 = e / (mu_1^2 - c),  tau = 2 / sigma_1,
    Y_1     = (sigma_1 / e) (H^2 Y_0 - c Y_0),
    sigma_{j+1} = 1 / (tau - sigma_j),
    Y_{j+1} = (2 sigma_{j+1} / e) (H^2 Y_j - c Y_j) - sigma_j sigma_{j+1} Y_{j-1},

so that Y_deg = T_deg((H^2 - c)/e) Y_0 / T_deg((mu_1^2 - c)/e).  "deg" counts
H^2 steps; H^2 is applied as H (H Y).  Column i stops after deg_i steps
(per-vector degrees, Section 6 convergence experiments).
"""
from __future__ import annotations

import numpy as np

from .dense import hamiltonian


def coefficients(mu1: float, mu_nevex: float, muN: float):
    """(c, e, sigma_1) of the scaled recurrence on H^2."""
    a = mu_nevex * mu_nevex
    b = muN * muN
    c = 0.5 * (a + b)
    e = 0.5 * (b - a)
    sigma1 = e / (mu1 * mu1 - c)
    return c, e, sigma1


def apply_h(A: np.ndarray, B: np.ndarray, W: np.ndarray) -> np.ndarray:
    """H W with H formed explicitly (Section 1)."""
    return hamiltonian(A, B) @ W


def chebyshev_filter(A, B, W0, degs, mu1, mu_nevex, muN):
    """Filter each column of W0 (2n x k) with its own degree deg_i >= 1.

    Returns Y with Y[:, i] = p_{deg_i}(H^2) W0[:, i].
    """
    H = hamiltonian(A, B)
    degs = np.asarray(degs, dtype=int)
    W0 = np.array(W0, dtype=np.complex128)
    if W0.shape[1] == 0:
        return W0.copy()
    c, e, sigma1 = coefficients(mu1, mu_nevex, muN)
    tau = 2.0 / sigma1
    out = np.empty_like(W0)
    Yprev = W0
    Y = (sigma1 / e) * (H @ (H @ W0) - c * W0)
    for i in np.where(degs == 1)[0]:
        out[:, i] = Y[:, i]
    sigma = sigma1
    for j in range(1, int(degs.max())):
        sigma_new = 1.0 / (tau - sigma)
        Ynew = (2.0 * sigma_new / e) * (H @ (H @ Y) - c * Y) - (sigma * sigma_new) * Yprev
        Yprev, Y = Y, Ynew
        sigma = sigma_new
        for i in np.where(degs == j + 1)[0]:
            out[:, i] = Y[:, i]
    return out


def chebyshev_t(m: int, t):
    """Chebyshev polynomial of the first kind T_m(t) by its closed form
    (cos(m arccos t) on [-1, 1], cosh(m arccosh |t|) * sign^m outside)."""
    t = np.asarray(t, dtype=float)
    out = np.empty_like(t)
    inside = np.abs(t) <= 1.0
    out[inside] = np.cos(m * np.arccos(t[inside]))
    ti = t[~inside]
    out[~inside] = np.sign(ti) ** m * np.cosh(m * np.arccosh(np.abs(ti)))
    return out


def filter_polynomial(x, deg: int, mu1: float, mu_nevex: float, muN: float):
    """p_deg(x) = T_deg((x - c)/e) / T_deg((mu_1^2 - c)/e) for x an eigenvalue of H^2."""
    c, e, _ = coefficients(mu1, mu_nevex, muN)
    num = chebyshev_t(deg, (np.asarray(x, dtype=float) - c) / e)
    den = chebyshev_t(deg, np.array([(mu1 * mu1 - c) / e]))[0]
    return num / den


def h2_blocks(A: np.ndarray, B: np.ndarray):
    """(P, Q) with H^2 = [[P, Q], [conj(Q), conj(P)]] for H = [[A, B], [-conj(B), -conj(A)]]:
    P = A A - B conj(B), Q = A B - B conj(A) (block product of H with itself; the
    lower blocks are the conjugates because H^2 commutes with K conj).  Not the
    paper's method, which applies H twice; this is the explicit-H^2 variant."""
    P = A @ A - B @ B.conj()
    Q = A @ B - B @ A.conj()
    return P, Q


def apply_h2_blocks(P: np.ndarray, Q: np.ndarray, W: np.ndarray) -> np.ndarray:
    """H^2 W from the blocks of H^2: top P x + Q y, bottom conj(Q) x + conj(P) y."""
    n = P.shape[0]
    X, Y = W[:n], W[n:]
    return np.vstack([P @ X + Q @ Y, Q.conj() @ X + P.conj() @ Y])


def chebyshev_filter_explicit(P, Q, W0, degs, mu1, mu_nevex, muN):
    """The filter of ``chebyshev_filter`` (same recurrence and per-column degrees) with
    H^2 applied from its blocks (P, Q) of ``h2_blocks``: one product per H^2 step."""
    degs = np.asarray(degs, dtype=int)
    W0 = np.array(W0, dtype=np.complex128)
    if W0.shape[1] == 0:
        return W0.copy()
    c, e, sigma1 = coefficients(mu1, mu_nevex, muN)
    tau = 2.0 / sigma1
    out = np.empty_like(W0)
    Yprev = W0
    Y = (sigma1 / e) * (apply_h2_blocks(P, Q, W0) - c * W0)
    for i in np.where(degs == 1)[0]:
        out[:, i] = Y[:, i]
    sigma = sigma1
    for j in range(1, int(degs.max())):
        sigma_new = 1.0 / (tau - sigma)
        Ynew = (2.0 * sigma_new / e) * (apply_h2_blocks(P, Q, Y) - c * Y) - (sigma * sigma_new) * Yprev
        Yprev, Y = Y, Ynew
        sigma = sigma_new
        for i in np.where(degs == j + 1)[0]:
            out[:, i] = Y[:, i]
    return out
