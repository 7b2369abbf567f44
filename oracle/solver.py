"""The outer subspace iteration of ChASE for pseudo-hermitian H (oracle; test infrastructure).

Algorithm 3 (Section 4), step by step:

 1. W_+ <- randn(2n, nevex); its lower half is scaled by gamma = 1e-3 so the
    search space starts on the S-positive side (Section 4.6).
 2. mu_1, mu_nevex, mu_N from pseudo-hermitian Lanczos (Section 4.1).
 3. while locked < nev:
    a. W_+ <- p(H^2) W_+                      (Section 4.2)
    b. W_- <- K conj(W_+)                     (Theorem relation_polynomial)
    c. Q <- [S Y_+, S Y_-, W_+, W_-] R^{-1}    (Section 4.3), keep Q[:, 2 locked:]
    d. Ritz values and W_+ = Q Z_+             (Algorithm 2)
    e. residuals of the positive half          (Section 4.5)
    f. lock converged positive pairs, Y_- = K conj(Y_+)

Readings where the paper is silent (the same ones the CUDA driver follows):

* residual r_i = ||H w_i - lambda_i w_i||_2 / rho_hat with ||w_i|| = 1 and
  rho_hat = max |theta| of the Lanczos Ritz values (no beta padding);
* lock every i among the first (nev - locked) active pairs (ascending lambda)
  with r_i <= tol;
* after locking, mu_nevex <- largest non-locked positive Ritz value
  (Section 4.1) among those below mu_N: a Ritz value above the Lanczos upper
  bound of the spectrum is spurious (Theorem field_of_values_ritz_hermitian_variant
  and the remark after it) and is ignored; spurious values below mu_N also
  occur in the first iterations, so mu_nevex grows by at most a factor 2 per
  iteration; mu_1 <- min(mu_1, lambda_1);
* mu_1 is only the normalisation point of the filter (p(mu_1^2) = 1) and must
  stay below mu_nevex, otherwise it falls inside the damped interval where the
  scaled recurrence divides by values of T_j near zero; mu_1 <- min(mu_1,
  mu_nevex / 2) is applied after every update (a lower mu_1 only rescales);
* per-vector degree from the convergence rate (Section 6 cites a formula not
  available here): the predicted rate per H^2 step is
  rho_i = 1/(|t_i| + sqrt(t_i^2 - 1)) with t_i = (lambda_i^2 - c)/e (1 when
  |t_i| <= 1); once a column has a residual history, the observed rate
  (r_i / r_i_prev)^(1/deg_i_prev) is used instead when it is slower; then
  deg_i = clamp(ceil(ln(tol/r_i)/ln(rho_i)) + 1, deg_min, deg_max).  The first
  iteration uses ``deg`` for every column.
"""
from __future__ import annotations

import math
import numpy as np

from .chebyshev import chebyshev_filter, coefficients
from .dense import fix_phase
from .lanczos import spectral_bounds, lanczos_tridiagonal, ritz_and_weights
from .qr import cholesky_qr2
from .rayleigh_ritz import rayleigh_ritz, rayleigh_ritz_fallback, residuals

GAMMA = 1e-3


def k_conj(W: np.ndarray) -> np.ndarray:
    """K conj(W) with K = [[0, I], [I, 0]]."""
    n = W.shape[0] // 2
    return np.concatenate([W[n:].conj(), W[:n].conj()], axis=0)


def s_flip(W: np.ndarray) -> np.ndarray:
    """S W with S = diag(I, -I)."""
    n = W.shape[0] // 2
    return np.concatenate([W[:n], -W[n:]], axis=0)


def rho_hat(A, B, starts, steps):
    """max |theta| over the Lanczos runs (no beta padding)."""
    m = 0.0
    for v0 in starts:
        al, be = lanczos_tridiagonal(A, B, np.asarray(v0, dtype=np.complex128), steps)
        th, _ = ritz_and_weights(al, be)
        m = max(m, float(np.abs(th).max()))
    return m


def degrees(ritz, res, tol, mu1, mu_nevex, muN, deg_min, deg_max, prev_res=None, prev_deg=None):
    c, e, _ = coefficients(mu1, mu_nevex, muN)
    out = np.empty(len(ritz), dtype=int)
    for i, (lam, r) in enumerate(zip(ritz, res)):
        t = (lam * lam - c) / e
        rho = 1.0 if abs(t) <= 1.0 else 1.0 / (abs(t) + math.sqrt(t * t - 1.0))
        if prev_res is not None and np.isfinite(prev_res[i]) and 0.0 < r < prev_res[i]:
            rho = max(rho, (r / prev_res[i]) ** (1.0 / prev_deg[i]))
        if r <= tol:
            d = deg_min
        elif rho >= 1.0:
            d = deg_max
        else:
            d = math.ceil(math.log(tol / r) / math.log(rho)) + 1
        out[i] = min(max(d, deg_min), deg_max)
    return out


def solve(A, B, nev, nex, deg, tol, W0raw, starts, lanczos_steps=26, deg_min=None,
          deg_max=None, maxiter=25, rr="oblique"):
    """Returns dict(lam[nev], V[2n, nev], iterations, history, mu).

    rr: "oblique" (Algorithm 2) or "fallback" (the non-hermitian dual basis of the last
    paragraph of Section 4.4, for a singular Q^* S Q)."""
    if rr not in ("oblique", "fallback"):
        raise ValueError("rr must be 'oblique' or 'fallback'")
    rr_step = rayleigh_ritz if rr == "oblique" else rayleigh_ritz_fallback
    n = A.shape[0]
    nevex = nev + nex
    deg_min = deg if deg_min is None else deg_min
    deg_max = deg if deg_max is None else deg_max
    W = np.array(W0raw, dtype=np.complex128).T.copy()   # (2n, nevex)
    W[n:, :] *= GAMMA
    mu1, mu_nevex, muN = spectral_bounds(A, B, starts, lanczos_steps, nevex)
    mu1 = min(mu1, 0.5 * mu_nevex)
    rhat = rho_hat(A, B, starts, lanczos_steps)
    Yp = np.zeros((2 * n, 0), dtype=np.complex128)
    lam_locked = np.zeros(0)
    degs = np.full(nevex, deg, dtype=int)
    prev_res = np.full(nevex, np.inf)
    history = []
    it = 0
    while Yp.shape[1] < nev and it < maxiter:
        it += 1
        locked = Yp.shape[1]
        Wf = chebyshev_filter(A, B, W, degs, mu1, mu_nevex, muN)
        X = np.concatenate([s_flip(Yp), s_flip(k_conj(Yp)), Wf, k_conj(Wf)], axis=1)
        Q, used_hh = cholesky_qr2(X)
        Q = Q[:, 2 * locked:]
        ritz, Wpos = rr_step(A, B, Q)
        res = residuals(A, B, Wpos, ritz) / rhat
        history.append(dict(ritz=ritz.copy(), res=res.copy(), degs=degs.copy(),
                            locked=locked, householder=used_hh,
                            mu=(mu1, mu_nevex, muN)))
        want = min(nev - locked, len(ritz))
        conv = [i for i in range(want) if res[i] <= tol]
        keep = [i for i in range(len(ritz)) if i not in set(conv)]
        if conv:
            Yp = np.concatenate([Yp, Wpos[:, conv]], axis=1)
            lam_locked = np.concatenate([lam_locked, ritz[conv]])
        W = Wpos[:, keep]
        if Yp.shape[1] >= nev or not keep:
            break
        # mu_nevex: the largest kept Ritz value below mu_N (larger ones are spurious); after
        # the first Rayleigh-Ritz (which replaces the Lanczos estimate, growing by at most 2x)
        # it never increases: the top Ritz values of the unconverged guard vectors approach
        # the spectrum from above, so a growing value means drift, not information
        cand = ritz[keep][ritz[keep] < muN]
        if len(cand):
            if it == 1:
                mu_nevex = min(float(cand.max()), 2.0 * mu_nevex)
            else:
                mu_nevex = min(float(cand.max()), mu_nevex)
        if ritz[0] > 0:
            mu1 = min(mu1, float(ritz[0]))
        mu1 = min(mu1, 0.5 * mu_nevex)
        degs = degrees(ritz[keep], res[keep], tol, mu1, mu_nevex, muN, deg_min, deg_max,
                       prev_res=prev_res[keep], prev_deg=degs[keep])
        prev_res = res[keep]
    order = np.argsort(lam_locked)[:nev]
    V = fix_phase(Yp[:, order]) if len(order) else Yp
    return dict(lam=lam_locked[order], V=V, iterations=it, history=history,
                mu=(mu1, mu_nevex, muN), converged=len(order))
