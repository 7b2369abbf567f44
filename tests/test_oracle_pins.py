"""Pins of the two oracle functions that shape the iteration but not its result:
the DOS estimate of mu_nevex (Section 4.1) and the per-vector degree rule (the
convergence-rate degree the Section 6 experiments use), each against values
worked out by hand; then the library's own degree rule (chase_bse_degrees, host
code, no GPU) against the oracle's on random inputs, integer for integer.
"""
import math
import os

import numpy as np
import pytest

from oracle import lanczos, solver as osolver


# ---------------------------------------------------------------- DOS mu_nevex
def _diagonal_problem(d):
    """A = diag(d), B = 0: H = diag(d, -d), eigenvectors e_i, S H = diag(d, d)."""
    n = len(d)
    A = np.diag(np.asarray(d, dtype=np.complex128))
    B = np.zeros((n, n), dtype=np.complex128)
    return A, B


def test_dos_quantile_of_a_planted_spectrum():
    """Full-length Lanczos (2n steps) on H = diag(d, -d) returns every eigenvalue.  In the
    S H inner product the start vector v0 = sum x_i e_i + sum y_i e_{n+i} gives the
    eigenvalue d_i the weight tau_i = d_i x_i^2 / <v0, v0>_SH, so tau_i / theta_i is
    proportional to x_i^2.  With x_i^2 = 1, 2, ..., 6 on d = 1, 2, 3.5, 4, 6, 7.5 the
    cumulative positive-axis weights are 1, 3, 6, 10, 15, 21 (/21); the target
    nevex / n = 3/6 = 10.5/21 lies between (4, 10/21) and (6, 15/21), a tenth of the way:
    mu_nevex = 4 + 0.1 * 2 = 4.2.  mu_1 = 1 and mu_N = 7.5 (the last beta vanishes)."""
    d = [1.0, 2.0, 3.5, 4.0, 6.0, 7.5]
    A, B = _diagonal_problem(d)
    x = np.sqrt(np.arange(1, 7, dtype=float))
    y = np.array([0.7, -1.1, 0.4, 0.9, -0.3, 1.3])  # the negative half does not enter
    v0 = np.concatenate([x, y]).astype(np.complex128)
    mu1, mune, muN = lanczos.spectral_bounds(A, B, [v0], steps=12, nevex=3)
    assert abs(mu1 - 1.0) < 1e-9
    assert abs(mune - 4.2) < 1e-8
    assert abs(muN - 7.5) < 1e-8


def test_dos_quantile_on_a_grid_point_and_pooled_vectors():
    """Equal weights put the cumulative weight j/n exactly on the j-th eigenvalue, so
    mu_nevex = d_(nevex); two start vectors with the same weights pool to the same
    density.  nevex = 2 of n = 5 on d = 1.5, 2.5, 3, 5, 8 gives 2.5."""
    d = [3.0, 1.5, 8.0, 2.5, 5.0]
    A, B = _diagonal_problem(d)
    v1 = np.concatenate([np.ones(5), 0.5 * np.ones(5)]).astype(np.complex128)
    v2 = np.concatenate([-np.ones(5), np.ones(5)]).astype(np.complex128)
    mu1, mune, muN = lanczos.spectral_bounds(A, B, [v1, v2], steps=10, nevex=2)
    assert abs(mune - 2.5) < 1e-8
    assert abs(mu1 - 1.5) < 1e-9 and abs(muN - 8.0) < 1e-8


def test_dos_quantile_below_the_first_eigenvalue_interpolates_from_mu1():
    """A target below the first cumulative weight interpolates from (mu_1, 0): weights
    x_i^2 = 9, 1, 1, 1 on d = 1, 2, 3, 4 (cumulative 9/12 at d = 1) and nevex/n = 1/4
    lie on the segment from (1, 0) to (1, 0.75), so mu_nevex = mu_1 = 1; with
    weights 1, 1, 1, 9 the cumulative weights are 1, 2, 3, 12 (/12) and the target 3/12
    falls on d = 3 exactly."""
    d = [1.0, 2.0, 3.0, 4.0]
    A, B = _diagonal_problem(d)
    v = np.concatenate([np.sqrt([9.0, 1.0, 1.0, 1.0]), np.ones(4)]).astype(np.complex128)
    _, mune, _ = lanczos.spectral_bounds(A, B, [v], steps=8, nevex=1)
    assert abs(mune - 1.0) < 1e-8
    v = np.concatenate([np.sqrt([1.0, 1.0, 1.0, 9.0]), np.ones(4)]).astype(np.complex128)
    _, mune, _ = lanczos.spectral_bounds(A, B, [v], steps=8, nevex=1)
    assert abs(mune - 3.0) < 1e-8


# ------------------------------------------------------------------- degrees
def _ce(mune, muN):
    a, b = mune * mune, muN * muN
    return 0.5 * (a + b), 0.5 * (b - a)


def test_degree_rule_closed_forms():
    """mu_nevex = 3, mu_N = 5: c = 17, e = 8.
    * lambda = 1: t = -2, rho = 1/(2 + sqrt 3) = 0.2679492; r = 1e-2, tol = 1e-10:
      ln(1e-8)/ln(rho) = 13.98729 -> 14 + 1 = 15
    * lambda = 4: t = -1/8 inside the damped interval: rho = 1 -> deg_max
    * r <= tol -> deg_min
    * observed rate: prev r = 1e-1 after 10 steps, r = 1e-2: (0.1)^(1/10) = 0.7943 is
      slower than 0.268, so ln(3e-10/1e-2)/ln(0.1^0.1) = 75.23 -> 76 + 1 = 77
    * a faster observed rate keeps the predicted one: prev r = 1, r = 1e-12 after 10 steps
      (rate 0.063 < 0.268) with tol 1e-13: ln(0.1)/ln(rho) = 1.75 -> 2 + 1 = 3
    * a residual that grew uses the predicted rate: 15 as in the first case."""
    c, e = _ce(3.0, 5.0)
    assert (c, e) == (17.0, 8.0)
    rho = 1.0 / (2.0 + math.sqrt(3.0))
    assert abs(math.log(1e-8) / math.log(rho) - 13.98729) < 1e-5
    inf = float("inf")
    cases = [
        # (lambda, r, prev_r, prev_deg, tol, expected)
        (1.0, 1e-2, inf, 20, 1e-10, 15),
        (4.0, 1e-2, inf, 20, 1e-10, 100),
        (1.0, 1e-11, inf, 20, 1e-10, 1),
        (1.0, 1e-2, 1e-1, 10, 3e-10, 77),
        (1.0, 1e-12, 1.0, 10, 1e-13, 3),
        (1.0, 1e-2, 5e-3, 10, 1e-10, 15),
    ]
    for lam, r, pr, pd, tol, want in cases:
        got = osolver.degrees([lam], [r], tol, 0.5, 3.0, 5.0, 1, 100, prev_res=np.array([pr]),
                              prev_deg=np.array([pd]))
        assert int(got[0]) == want, (lam, r, pr, pd, tol, int(got[0]))


def test_degree_rule_clamps():
    """The same first case clamped to [16, 40] and to [4, 12]."""
    for lo, hi, want in [(16, 40, 16), (4, 12, 12)]:
        got = osolver.degrees([1.0], [1e-2], 1e-10, 0.5, 3.0, 5.0, lo, hi)
        assert int(got[0]) == want


# ----------------------------------------------- the library's rule = the oracle's
@pytest.fixture(scope="module")
def libdeg():
    from paper_2601_10557_gb300 import _lib
    if not os.path.exists(_lib.LIB_PATH):
        import __graft_entry__
        __graft_entry__.build()
    return _lib.degrees


def test_library_degree_rule_matches_oracle(libdeg):
    rng = np.random.default_rng(3)
    k = 400
    mune, muN = 2.5, 40.0
    ritz = rng.uniform(0.5, 3.5, size=k)
    res = 10.0 ** rng.uniform(-12, 0, size=k)
    prev = res * 10.0 ** rng.uniform(-1, 3, size=k)
    prev[rng.random(k) < 0.2] = np.inf
    pdeg = rng.integers(8, 37, size=k)
    for tol, lo, hi in [(1e-10, 8, 36), (1e-8, 1, 100), (1e-12, 20, 20)]:
        want = osolver.degrees(ritz, res, tol, 0.5, mune, muN, lo, hi, prev_res=prev, prev_deg=pdeg)
        got = libdeg(ritz, res, prev, pdeg, tol, mune, muN, lo, hi)
        assert list(map(int, want)) == got
