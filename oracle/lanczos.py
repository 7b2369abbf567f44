"""Pseudo-hermitian Lanczos spectral bounds (oracle; test infrastructure).

Section 4.1: a few Lanczos steps estimate mu_1 (smallest |lambda|), mu_N (an
upper bound of the spectral radius) and mu_nevex (the value below which the
positive axis holds nevex/n of the spectral weight); the filter uses their
squares.  The paper follows a Lanczos defined with S-inner products and an even
number of steps so that the +-symmetry of the spectral density is kept.

Reading used here (the paper does not spell out the recurrence): Lanczos for
the operator H in the inner product <x, y>_M = y^* M x with M = S H, which is
hermitian positive definite for a definite problem.  H is self-adjoint in it
because (S H) H = H^* (S H).  Each start vector v gives a real symmetric
tridiagonal T (alpha_j on the diagonal, beta_j beside it) whose eigenvalues
theta_j are Ritz values of H and whose squared first eigenvector components
tau_j are the weights of the spectral density of v (Lin, Saad & Yang, SIAM Rev.
58, 2016).

* mu_1     = min |theta| over all start vectors
* mu_N     = max |theta| + |beta_last| (upper bound after Zhou, Linear Algebra
             Appl. 435, 2011)
* mu_nevex = positive-axis quantile of the density of eigenvalues.  In the
             S H inner product the weight an eigenvalue lambda receives from a
             random start vector is proportional to lambda times its share of
             the start vector, so the counting density is recovered with the
             weights tau_j / theta_j.  These are pooled over the start vectors
             for theta > 0 and renormalised; the cumulative weight is linearly
             interpolated between (mu_1, 0) and the successive (theta_j, C_j),
             and mu_nevex is where it reaches nevex / n.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

from .dense import hamiltonian


def lanczos_tridiagonal(A, B, v0, steps: int, return_basis: bool = False):
    """Run ``steps`` Lanczos steps in the S H inner product from v0.
    Returns (alpha[steps], beta[steps]) with beta[j] coupling step j and j+1
    (and the basis vectors as columns when ``return_basis``)."""
    n = A.shape[0]
    H = hamiltonian(A, B)
    s = np.concatenate([np.ones(n), -np.ones(n)])
    M = s[:, None] * H  # S H

    def ip(x, y):
        return np.vdot(y, M @ x)

    v = v0 / np.sqrt(ip(v0, v0).real)
    v_prev = np.zeros_like(v)
    beta_prev = 0.0
    alpha = np.zeros(steps)
    beta = np.zeros(steps)
    basis = []
    for j in range(steps):
        basis.append(v)
        w = H @ v
        alpha[j] = ip(w, v).real
        w = w - alpha[j] * v - beta_prev * v_prev
        beta[j] = np.sqrt(max(ip(w, w).real, 0.0))
        if beta[j] == 0.0:
            alpha, beta = alpha[: j + 1], beta[: j + 1]
            break
        v_prev, v = v, w / beta[j]
        beta_prev = beta[j]
    if return_basis:
        return alpha, beta, np.stack(basis, axis=1)
    return alpha, beta


def ritz_and_weights(alpha, beta):
    """Eigenvalues theta and weights tau = |z[0]|^2 of the tridiagonal T."""
    theta, Z = sla.eigh_tridiagonal(alpha, beta[: len(alpha) - 1])
    return theta, np.abs(Z[0, :]) ** 2


def spectral_bounds(A, B, starts, steps: int, nevex: int):
    """(mu_1, mu_nevex, mu_N) from Lanczos runs on each start vector (rows of
    ``starts``, shape (nvec, 2n))."""
    n = A.shape[0]
    thetas, taus, betas = [], [], []
    for v0 in starts:
        al, be = lanczos_tridiagonal(A, B, np.asarray(v0, dtype=np.complex128), steps)
        th, ta = ritz_and_weights(al, be)
        thetas.append(th)
        taus.append(ta)
        betas.append(abs(be[len(al) - 1]))
    allth = np.concatenate(thetas)
    mu1 = np.abs(allth).min()
    muN = max(np.abs(th).max() + b for th, b in zip(thetas, betas))
    # positive-axis density, averaged over start vectors
    th_pos = np.concatenate([th[th > 0] for th in thetas])
    w_pos = np.concatenate([ta[th > 0] / th[th > 0] for th, ta in zip(thetas, taus)])
    order = np.argsort(th_pos)
    th_pos = th_pos[order]
    w_pos = w_pos[order] / w_pos.sum()
    cum = np.cumsum(w_pos)
    target = nevex / n
    xs = np.concatenate([[mu1], th_pos])
    ys = np.concatenate([[0.0], cum])
    j = int(np.searchsorted(ys, target))
    if j >= len(ys):
        mu_nevex = xs[-1]
    elif j == 0:
        mu_nevex = xs[0]
    else:
        t = (target - ys[j - 1]) / (ys[j] - ys[j - 1])
        mu_nevex = xs[j - 1] + t * (xs[j] - xs[j - 1])
    return float(mu1), float(mu_nevex), float(muN)
