"""The non-hermitian fallback Rayleigh-Ritz (Section 4.4, last paragraph) and its general
dense eigensolver, through the C ABI, against the oracle (oracle/rayleigh_ritz.py
fallback_dual_basis, rayleigh_ritz_fallback) and numpy's general eigensolver."""
import numpy as np
import pytest
import torch

import bse_inputs as bi
from oracle import dense, rayleigh_ritz as orr
from tests.gpu_util import dev, problem_on_device

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    import paper_2601_10557_gb300 as p
    p.lib()
    return p


def _match(got, ref):
    """Largest distance from an eigenvalue in `got` to the nearest one in `ref` and back."""
    d1 = max(np.min(np.abs(ref - g)) for g in got)
    d2 = max(np.min(np.abs(got - r)) for r in ref)
    return max(d1, d2)


@pytest.mark.parametrize("k", [1, 2, 3, 16, 100, 300])
def test_eig_general_random(pkg, k):
    rng = np.random.default_rng(k)
    G = rng.standard_normal((k, k)) + 1j * rng.standard_normal((k, k))
    lam, V = pkg.eig_general(torch.from_numpy(G).to(dev()))
    lam, V = lam.cpu().numpy(), V.cpu().numpy()
    g = np.linalg.norm(G)
    assert np.linalg.norm(G @ V - V * lam[None, :]) <= 1e-13 * k * g
    np.testing.assert_allclose(np.linalg.norm(V, axis=0), 1.0, rtol=1e-12)
    assert _match(lam, np.linalg.eigvals(G)) <= 1e-11 * g


def test_eig_general_real_spectrum_non_normal(pkg):
    """Q T Q^* with T upper triangular (diagonal -3 .. 5): the eigenvalues are T's diagonal."""
    k = 64
    rng = np.random.default_rng(5)
    Q, _ = np.linalg.qr(rng.standard_normal((k, k)) + 1j * rng.standard_normal((k, k)))
    d = np.linspace(-3.0, 5.0, k)
    T = np.triu(0.3 * rng.standard_normal((k, k)), 1) + np.diag(d)
    lam, V = pkg.eig_general(torch.from_numpy(Q @ T @ Q.conj().T).to(dev()))
    lam = lam.cpu().numpy()
    np.testing.assert_allclose(np.sort(lam.real), d, atol=1e-12)
    assert np.abs(lam.imag).max() <= 1e-12


def _rr(pkg, P, Q):
    A, B = problem_on_device(P)
    return pkg.rayleigh_ritz_fallback(A, B, torch.from_numpy(np.ascontiguousarray(Q.T)).to(dev()))


def _same_vectors(W, Wref):
    """Columns equal up to a unit phase: |w^* w_ref| = 1 for unit columns."""
    ov = np.abs(np.sum(W.conj() * Wref, axis=0))
    return np.abs(ov - 1.0).max()


def test_fallback_rr_matches_oracle_on_a_random_basis(pkg):
    n, k = 40, 16
    P = bi.make_problem(n, seed=2)
    rng = np.random.default_rng(2)
    Q, _ = np.linalg.qr(rng.standard_normal((2 * n, k)) + 1j * rng.standard_normal((2 * n, k)))
    ritz, W = _rr(pkg, P, Q)
    ref, Wref = orr.rayleigh_ritz_fallback(P.A, P.B, Q)
    assert len(ritz) == len(ref)
    np.testing.assert_allclose(ritz, ref, rtol=1e-10)
    assert _same_vectors(W.cpu().numpy().T, Wref) <= 1e-9


@pytest.mark.parametrize("m", [1, 4])
def test_fallback_rr_is_exact_on_invariant_subspaces(pkg, m):
    n = 32
    P = bi.make_problem(n, seed=4)
    lam, V, _ = dense.eig_general(P.A, P.B)
    order = np.argsort(lam)
    pos = order[lam[order] > 0][:m]
    neg = order[lam[order] < 0][::-1][:m]
    Q, _ = np.linalg.qr(np.hstack([V[:, pos], V[:, neg]]))
    ritz, W = _rr(pkg, P, Q)
    np.testing.assert_allclose(ritz, lam[pos], rtol=1e-11)
    H = dense.hamiltonian(P.A, P.B)
    Wg = W.cpu().numpy().T
    assert np.linalg.norm(H @ Wg - Wg * ritz[None, :], axis=0).max() <= 1e-10 * np.linalg.norm(H, 2)


def test_fallback_rr_singular_qsq(pkg):
    """Q^* S Q = [[1/2, 1/2], [1/2, 1/2]] (singular, nonzero diagonal) extended by random
    orthonormal columns: the dual basis still exists; the GPU matches the oracle."""
    n = 20
    a = 0.25 / np.sqrt(0.75)
    Qs = np.zeros((2 * n, 2), dtype=complex)
    Qs[0, 0], Qs[n, 0] = np.sqrt(0.75), 0.5
    Qs[0, 1], Qs[1, 1], Qs[n, 1] = a, np.sqrt(0.75 - a * a), -0.5
    rng = np.random.default_rng(7)
    Z = rng.standard_normal((2 * n, 6)) + 1j * rng.standard_normal((2 * n, 6))
    Z -= Qs @ (Qs.conj().T @ Z)
    Qz, _ = np.linalg.qr(Z)
    Q = np.hstack([Qs, Qz])
    S = np.diag(np.r_[np.ones(n), -np.ones(n)])
    M2 = Qs.conj().T @ S @ Qs
    assert abs(np.linalg.det(M2)) <= 1e-15
    P = bi.make_problem(n, seed=7)
    ritz, W = _rr(pkg, P, Q)
    ref, Wref = orr.rayleigh_ritz_fallback(P.A, P.B, Q)
    assert len(ritz) == len(ref)
    np.testing.assert_allclose(ritz, ref, rtol=1e-9)
    assert _same_vectors(W.cpu().numpy().T, Wref) <= 1e-8


def test_fallback_rr_zero_diagonal_is_rejected(pkg):
    """A column with q^* S q = 0 has no dual vector: QR_FAILED."""
    n = 16
    P = bi.make_problem(n, seed=1)
    Q = np.zeros((2 * n, 2), dtype=complex)
    Q[0, 0] = Q[n, 0] = 1.0 / np.sqrt(2.0)
    Q[1, 1] = 1.0
    with pytest.raises(pkg.ChaseBSEError) as e:
        _rr(pkg, P, Q)
    assert e.value.status == -5


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_solve_with_the_fallback_rr_matches_brute_force(pkg, precision):
    """Algorithm 3 with the fallback Rayleigh-Ritz in every iteration (as the oracle's
    solver with rr="fallback") still returns the nev smallest positive eigenpairs."""
    from tests.gpu_util import starts, to_dev
    n, nev, nex = 64, 6, 6
    P = bi.make_problem(n, seed=0)
    A, B = problem_on_device(P)
    W0, V0 = starts(n, nev + nex, 0)
    lam, V, st = pkg.solve(A, B, nev, nex, 12, 1e-10, W0=to_dev(W0), V0=to_dev(V0), deg_min=4, deg_max=24,
                           maxiter=40, rr="fallback", precision=precision)
    ref, _ = dense.smallest_positive(P.A, P.B, nev)
    np.testing.assert_allclose(lam.cpu().numpy(), ref, rtol=1e-10)
    H = dense.hamiltonian(P.A, P.B)
    Vg = V.cpu().numpy().T
    R = H @ Vg - Vg * lam.cpu().numpy()[None, :]
    assert np.linalg.norm(R, axis=0).max() <= 1e-9 * np.linalg.norm(H, 2)
    assert st["fallback_rr"] == st["iterations"]
