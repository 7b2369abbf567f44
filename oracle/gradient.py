"""Gradient of L = sum_i w_i lambda_i with respect to A and B (oracle; test infrastructure).

Not in the paper; it follows from Theorem SH_HPD: the left eigenvector of a
definite H is u = S v, so first-order perturbation theory gives
d lambda = (S v)^* dH v / (v^* S v).  With v = [x; y], s = |x|^2 - |y|^2 and
dH = [[dA, dB], [-conj(dB), -conj(dA)]]:

    d lambda = (x^* dA x + y^* conj(dA) y + x^* dB y + y^* conj(dB) x) / s.

For a real loss and the convention dL = Re sum conj(G) * dZ (the one PyTorch
uses for complex tensors) this gives, with c_i = w_i / s_i,

    grad_A = sum_i c_i (x_i x_i^* + conj(y_i) y_i^T)   (hermitian)
    grad_B = sum_i c_i (x_i y_i^* + conj(y_i) x_i^T)   (symmetric).
"""
from __future__ import annotations

import numpy as np

from .dense import smallest_positive


def gradient_from_vectors(V: np.ndarray, w: np.ndarray):
    n = V.shape[0] // 2
    X, Y = V[:n], V[n:]
    s = np.sum(np.abs(X) ** 2, axis=0) - np.sum(np.abs(Y) ** 2, axis=0)
    c = np.asarray(w, dtype=float) / s
    gA = (X * c) @ X.conj().T + (Y.conj() * c) @ Y.T
    gB = (X * c) @ Y.conj().T + (Y.conj() * c) @ X.T
    return gA, gB


def eigenvalue_gradient(A, B, nev, w):
    """Gradient from the dense eigendecomposition (brute force)."""
    lam, V = smallest_positive(A, B, nev)
    gA, gB = gradient_from_vectors(V, w)
    return lam, gA, gB


def loss(A, B, nev, w):
    lam, _ = smallest_positive(A, B, nev)
    return float(np.dot(w, lam))
