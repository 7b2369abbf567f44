"""Pins of the oracle solver (Algorithm 3) and the eigenvalue gradient."""
import numpy as np
import pytest

import bse_inputs as bi
from oracle import dense, gradient, solver


def _solve(P, nev, nex, deg=12, tol=1e-10, seed=0):
    n = P.n
    return solver.solve(P.A, P.B, nev, nex, deg, tol, bi.start_block(n, nev + nex, seed),
                        bi.lanczos_starts(n, 4, seed), deg_min=4, deg_max=24)


@pytest.mark.parametrize("kind", ["complex", "real", "bzero"])
def test_solver_matches_brute_force(kind):
    n, nev, nex = 64, 8, 6
    P = bi.make_problem(n, seed=11, real=(kind == "real"), b_zero=(kind == "bzero"))
    r = _solve(P, nev, nex)
    assert r["converged"] == nev
    ref, Vref = dense.smallest_positive(P.A, P.B, nev)
    np.testing.assert_allclose(r["lam"], ref, rtol=1e-10)
    H = dense.hamiltonian(P.A, P.B)
    normH = np.linalg.norm(H, 2)
    R = H @ r["V"] - r["V"] * r["lam"][None, :]
    assert np.linalg.norm(R, axis=0).max() / normH <= 1e-10
    if kind == "bzero":
        np.testing.assert_allclose(r["lam"], np.sort(P.d)[:nev], rtol=1e-10)
    if kind == "real":
        A, B = P.A.real, P.B.real
        ref2 = np.sort(np.linalg.eigvals((A - B) @ (A + B)).real)[:nev]
        np.testing.assert_allclose(r["lam"] ** 2, ref2, rtol=1e-9)


def test_pm_residuals_equal():
    # Section 4.5: residuals of the +- Ritz pairs are equal
    n = 40
    P = bi.make_problem(n, seed=5)
    r = _solve(P, 6, 4)
    H = dense.hamiltonian(P.A, P.B)
    Vm = solver.k_conj(r["V"])
    rp = np.linalg.norm(H @ r["V"] - r["V"] * r["lam"], axis=0)
    rm = np.linalg.norm(H @ Vm + Vm * r["lam"], axis=0)
    np.testing.assert_allclose(rp, rm, rtol=1e-6, atol=1e-14)


def test_maxiter_partial():
    n = 64
    P = bi.make_problem(n, seed=1)
    r = solver.solve(P.A, P.B, 8, 4, 4, 1e-12, bi.start_block(n, 12, 1),
                     bi.lanczos_starts(n, 4, 1), maxiter=1)
    assert r["iterations"] == 1 and r["converged"] < 8


def _herm(rng, n):
    E = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    return E + E.conj().T


def _sym(rng, n):
    E = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    return E + E.T


def test_gradient_matches_central_fd():
    n, nev = 14, 4
    P = bi.make_problem(n, seed=9)
    w = bi.loss_weights(nev, 9)
    _, gA, gB = gradient.eigenvalue_gradient(P.A, P.B, nev, w)
    assert np.abs(gA - gA.conj().T).max() < 1e-13
    assert np.abs(gB - gB.T).max() < 1e-13
    rng = np.random.default_rng(0)
    h = 1e-6
    for _ in range(6):
        dA, dB = _herm(rng, n), _sym(rng, n)
        fd = (gradient.loss(P.A + h * dA, P.B + h * dB, nev, w)
              - gradient.loss(P.A - h * dA, P.B - h * dB, nev, w)) / (2 * h)
        an = np.real(np.sum(gA.conj() * dA) + np.sum(gB.conj() * dB))
        assert abs(fd - an) <= 1e-6 * abs(an)


def test_gradient_b_zero_textbook():
    n, nev = 16, 5
    P = bi.make_problem(n, seed=2, b_zero=True)
    w = bi.loss_weights(nev, 2)
    _, gA, gB = gradient.eigenvalue_gradient(P.A, P.B, nev, w)
    d, Qm = np.linalg.eigh(P.A)
    ref = (Qm[:, :nev] * w) @ Qm[:, :nev].conj().T
    np.testing.assert_allclose(gA, ref, atol=1e-12)
    assert np.abs(gB).max() < 1e-12
