"""Parity of the CUDA path (called through the C ABI) with the CPU oracle."""
import numpy as np
import pytest
import torch

import bse_inputs as bi
from oracle import chebyshev, dense, gradient, lanczos, qr as oqr, rayleigh_ritz as orr, solver as osolver
from tests.gpu_util import dev, problem_on_device, rel_fro, starts, to_dev

pytestmark = pytest.mark.gpu

TOL_FP64_FILTER = 1e-12   # relative Frobenius, FP64 filter vs oracle filter
TOL_EIG = 1e-10           # relative eigenvalue error


@pytest.fixture(scope="module")
def pkg():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    import paper_2601_10557_gb300 as p
    p.lib()
    return p


def _mus(P):
    lam, _ = dense.eig_cholesky(P.A, P.B)
    pos = lam[P.n:]
    return 0.9 * pos[0], pos[len(pos) // 6], 1.05 * pos[-1]


@pytest.mark.parametrize("n,k", [(1, 1), (37, 5), (100, 37), (130, 70)])
def test_filter_fp64_matches_oracle(pkg, n, k):
    P = bi.make_problem(n, seed=n)
    A, B = problem_on_device(P)
    W0 = bi.start_block(n, k, 1)
    rng = np.random.default_rng(k)
    degs = rng.integers(1, 9, size=k)
    mu1, mune, muN = (0.5, 1.0, 30.0) if n == 1 else _mus(P)
    W = to_dev(W0)
    pkg.filter(A, B, W, degs, mu1, mune, muN)
    Y = chebyshev.chebyshev_filter(P.A, P.B, W0.T, degs, mu1, mune, muN)
    assert rel_fro(W.cpu().numpy().T, Y) < TOL_FP64_FILTER


def test_filter_empty_and_k_conjugation(pkg):
    n, k = 70, 9
    P = bi.make_problem(n, seed=3)
    A, B = problem_on_device(P)
    mu1, mune, muN = _mus(P)
    empty = torch.zeros((0, 2 * n), dtype=torch.complex128, device=dev())
    pkg.filter(A, B, empty, [], mu1, mune, muN)
    W0 = bi.start_block(n, k, 2).T
    degs = [6] * k
    W1 = to_dev(W0.T)
    W2 = to_dev(osolver.k_conj(W0).T)
    pkg.filter(A, B, W1, degs, mu1, mune, muN)
    pkg.filter(A, B, W2, degs, mu1, mune, muN)
    # Theorem relation_polynomial: p(H^2) K conj(W) = K conj(p(H^2) W)
    lhs = W2.cpu().numpy().T
    rhs = osolver.k_conj(W1.cpu().numpy().T)
    assert rel_fro(lhs, rhs) < 1e-13


def test_residuals_match_oracle(pkg):
    n, k = 90, 11
    P = bi.make_problem(n, seed=4)
    A, B = problem_on_device(P)
    W = bi.start_block(n, k, 4).T
    W /= np.linalg.norm(W, axis=0)
    lam = np.linspace(1.0, 3.0, k)
    res = pkg.residuals(A, B, to_dev(W.T), torch.from_numpy(lam)).cpu().numpy()
    ref = orr.residuals(P.A, P.B, W, lam)
    np.testing.assert_allclose(res, ref, rtol=1e-12)


@pytest.mark.parametrize("n,h", [(50, 4), (120, 33)])
def test_rayleigh_ritz_matches_oracle(pkg, n, h):
    P = bi.make_problem(n, seed=5)
    A, B = problem_on_device(P)
    Wp = bi.start_block(n, h, 5).T
    Wp[n:] *= 1e-3
    Wp = chebyshev.chebyshev_filter(P.A, P.B, Wp, [3] * h, *_mus(P))
    Q, _ = oqr.cholesky_qr2(np.concatenate([Wp, osolver.k_conj(Wp)], axis=1))
    ritz_ref, W_ref = orr.rayleigh_ritz(P.A, P.B, Q)
    ritz, Wpos = pkg.rayleigh_ritz(A, B, to_dev(Q.T))
    np.testing.assert_allclose(ritz, ritz_ref, rtol=1e-11)
    Wg = Wpos.cpu().numpy().T
    # unit vectors, equal up to a phase for well separated Ritz values
    gap = np.minimum(np.r_[np.inf, np.diff(ritz_ref)], np.r_[np.diff(ritz_ref), np.inf]) / ritz_ref
    ov = np.abs(np.sum(Wg.conj() * W_ref, axis=0))
    assert np.all(ov[gap > 1e-6] > 1 - 1e-9)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_lanczos_bounds_match_oracle(pkg, precision):
    """mu_1, mu_nevex (the DOS quantile), mu_N and rho_hat of the library's Lanczos run
    (FP64 pipe, or the FP64-accurate tensor-core products in mixed mode) against the
    oracle's on the same start vectors."""
    if precision == "mixed" and not pkg.has_mixed():
        pytest.fail("tensor-core path not available on this device")
    n, nev, nex = 128, 10, 6
    P = bi.make_problem(n, seed=6)
    A, B = problem_on_device(P)
    W0, V0 = starts(n, nev + nex, 6)
    _, _, st = pkg.solve(A, B, nev, nex, 10, 1e-10, W0=to_dev(W0), V0=to_dev(V0), deg_min=4, deg_max=24,
                         maxiter=1, allow_partial=True, precision=precision)
    mu_ref = lanczos.spectral_bounds(P.A, P.B, V0, 26, nev + nex)
    rhat = osolver.rho_hat(P.A, P.B, V0, 26)
    np.testing.assert_allclose(st["lanczos_mu1"], mu_ref[0], rtol=1e-8)
    np.testing.assert_allclose(st["lanczos_mu_nevex"], mu_ref[1], rtol=1e-8)
    np.testing.assert_allclose(st["lanczos_muN"], mu_ref[2], rtol=1e-8)
    # after one iteration mu_nevex/mu1 are updated from Ritz values; mu_N and rho_hat are the Lanczos ones
    np.testing.assert_allclose(st["muN"], mu_ref[2], rtol=1e-8)
    np.testing.assert_allclose(st["rho_hat"], rhat, rtol=1e-8)


@pytest.mark.parametrize("kind", ["complex", "real", "bzero"])
def test_solve_small_matches_brute_force(pkg, kind):
    n, nev, nex = 64, 8, 6
    P = bi.make_problem(n, seed=11, real=(kind == "real"), b_zero=(kind == "bzero"))
    A, B = problem_on_device(P)
    W0, V0 = starts(n, nev + nex, 0)
    lam, V, st = pkg.solve(A, B, nev, nex, 12, 1e-10, W0=to_dev(W0), V0=to_dev(V0), deg_min=4, deg_max=24)
    ref, Vref = dense.smallest_positive(P.A, P.B, nev)
    lam = lam.cpu().numpy()
    np.testing.assert_allclose(lam, ref, rtol=TOL_EIG)
    Vg = V.cpu().numpy().T
    H = dense.hamiltonian(P.A, P.B)
    R = H @ Vg - Vg * lam
    assert np.linalg.norm(R, axis=0).max() / np.linalg.norm(H, 2) <= 1e-10
    # phase convention: largest upper-half entry real positive
    idx = np.argmax(np.abs(Vg[:n]), axis=0)
    top = Vg[idx, np.arange(nev)]
    assert np.all(top.real > 0) and np.abs(top.imag).max() < 1e-12
    np.testing.assert_allclose(np.linalg.norm(Vg, axis=0), 1.0, rtol=1e-12)


def test_solve_n512_workload_matches_oracle(pkg):
    cfg = bi.WORKLOADS["n512"]
    n, nev, nex = cfg["n"], cfg["nev"], cfg["nex"]
    P = bi.make_problem(n, seed=0, spec=cfg["spec"], beta=cfg["beta"])
    A, B = problem_on_device(P)
    W0, V0 = starts(n, nev + nex, 0)
    lam, V, st = pkg.solve(A, B, nev, nex, cfg["deg"], cfg["tol"], W0=to_dev(W0), V0=to_dev(V0),
                           deg_min=cfg["deg_min"], deg_max=cfg["deg_max"])
    ref, _ = dense.smallest_positive(P.A, P.B, nev)
    np.testing.assert_allclose(lam.cpu().numpy(), ref, rtol=TOL_EIG)
    assert st["max_residual"] <= cfg["tol"]
    # the oracle's own solve takes the same number of iterations (same readings, same inputs)
    o = osolver.solve(P.A, P.B, nev, nex, cfg["deg"], cfg["tol"], W0, V0, deg_min=cfg["deg_min"],
                      deg_max=cfg["deg_max"])
    assert abs(o["iterations"] - st["iterations"]) <= 1


def test_gradient_matches_oracle_and_fd(pkg):
    n, nev, nex = 48, 5, 5
    P = bi.make_problem(n, seed=8)
    A, B = problem_on_device(P)
    W0, V0 = starts(n, nev + nex, 8)
    w = bi.loss_weights(nev, 8)
    kw = dict(W0=to_dev(W0), V0=to_dev(V0), deg_min=4, deg_max=24)
    At = A.clone().requires_grad_(True)
    Bt = B.clone().requires_grad_(True)
    lam = pkg.eigvals(At, Bt, nev, nex, 12, 1e-12, **kw)
    L = (lam * torch.from_numpy(w).to(dev())).sum()
    L.backward()
    _, rA, rB = gradient.eigenvalue_gradient(P.A, P.B, nev, w)
    assert rel_fro(At.grad.cpu().numpy(), rA) < 1e-6
    assert rel_fro(Bt.grad.cpu().numpy(), rB) < 1e-6
    # central FD of the GPU solve along random hermitian / symmetric directions
    rng = np.random.default_rng(1)
    h = 1e-6
    for _ in range(3):
        E = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
        F = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
        dA, dB = E + E.conj().T, F + F.T
        lp, _, _ = pkg.solve(to_dev(P.A + h * dA), to_dev(P.B + h * dB), nev, nex, 12, 1e-12, **kw)
        lm, _, _ = pkg.solve(to_dev(P.A - h * dA), to_dev(P.B - h * dB), nev, nex, 12, 1e-12, **kw)
        fd = float(np.dot(w, (lp - lm).cpu().numpy()) / (2 * h))
        an = float(np.real(np.sum(At.grad.cpu().numpy().conj() * dA) + np.sum(Bt.grad.cpu().numpy().conj() * dB)))
        assert abs(fd - an) <= 1e-6 * abs(an)


def test_householder_fallback_rank_deficient_start(pkg):
    n, nev, nex = 64, 6, 6
    P = bi.make_problem(n, seed=2)
    A, B = problem_on_device(P)
    W0, V0 = starts(n, nev + nex, 2)
    W0[1] = W0[0] * (1 + 1e-8) + 1e-8 * W0[2]   # nearly parallel: cond(X^* X) > 1e12
    lam, V, st = pkg.solve(A, B, nev, nex, 12, 1e-10, W0=to_dev(W0), V0=to_dev(V0), deg_min=4, deg_max=24)
    assert st["householder"] >= 1
    ref, _ = dense.smallest_positive(P.A, P.B, nev)
    np.testing.assert_allclose(lam.cpu().numpy(), ref, rtol=TOL_EIG)


def test_error_statuses(pkg):
    n = 32
    A = to_dev(np.eye(n, dtype=complex))
    B = to_dev(2.0 * np.eye(n, dtype=complex))   # S H indefinite
    with pytest.raises(pkg.ChaseBSEError) as e:
        pkg.solve(A, B, 4, 4, 8, 1e-10)
    assert e.value.status == -4
    P = bi.make_problem(n, seed=1)
    A, B = problem_on_device(P)
    with pytest.raises(pkg.ChaseBSEError) as e:
        pkg.solve(A, B, 30, 10, 8, 1e-10)      # nev + nex > n
    assert e.value.status == -1
    lam, V, st = pkg.solve(A, B, 4, 4, 2, 1e-14, maxiter=1, allow_partial=True)
    assert st["status"] == 1 and st["converged"] < 4


# ------------------------------------------------ FP64 on the tensor cores (FP64_TC)
@pytest.mark.parametrize("n,k", [(37, 5), (130, 70), (300, 24)])
def test_filter_fp64_tc_matches_oracle(pkg, n, k):
    """The FP64 recurrence with both H applications of every step as sliced tensor-core
    GEMMs: the oracle filter's result to 1e-12, ragged degrees; 2 max(deg) recorded
    sliced H applications."""
    P = bi.make_problem(n, seed=n + 1)
    A, B = problem_on_device(P)
    W0 = bi.start_block(n, k, 4)
    degs = np.random.default_rng(k + 1).integers(1, 9, size=k)
    mu1, mune, muN = _mus(P)
    W = to_dev(W0)
    pkg.gemm_timer(True)
    try:
        pkg.filter(A, B, W, degs, mu1, mune, muN, precision="fp64_tc")
        torch.cuda.synchronize()
        _, flops, launches = pkg.gemm_time("sliced")
    finally:
        pkg.gemm_timer(False)
    Y = chebyshev.chebyshev_filter(P.A, P.B, W0.T, degs, mu1, mune, muN)
    assert rel_fro(W.cpu().numpy().T, Y) < TOL_FP64_FILTER
    assert launches == 2 * int(degs.max())
    assert flops == 64.0 * n * n * float(degs.sum())


def test_filter_cols_fp64_tc_group_with_mixed(pkg):
    """Precision groups of one call: FP64_TC columns (1e-12) beside FP16x3 columns (1e-5);
    FP64 and FP64_TC in one call are rejected."""
    n, k = 200, 18
    P = bi.make_problem(n, seed=12)
    A, B = problem_on_device(P)
    W0 = bi.start_block(n, k, 12)
    degs = np.random.default_rng(12).integers(1, 7, size=k)
    precs = ["fp64_tc" if i % 2 == 0 else "fp16x3" for i in range(k)]
    mu1, mune, muN = _mus(P)
    W = to_dev(W0)
    pkg.filter_cols(A, B, W, degs, precs, mu1, mune, muN)
    Y = chebyshev.chebyshev_filter(P.A, P.B, W0.T, degs, mu1, mune, muN)
    got = W.cpu().numpy().T
    for j in range(k):
        err = rel_fro(got[:, j], Y[:, j])
        assert err < (TOL_FP64_FILTER if precs[j] == "fp64_tc" else 1e-5), (j, precs[j], err)
    with pytest.raises(pkg.ChaseBSEError):
        pkg.filter_cols(A, B, to_dev(W0), degs, ["fp64", "fp64_tc"] * (k // 2), mu1, mune, muN)


@pytest.mark.parametrize("kind", ["complex", "real"])
def test_solve_fp64_tc_matches_brute_force(pkg, kind):
    """An FP64_TC solve (every large product FP64-accurate on the tensor cores) reaches the
    dense eigenpairs like the FP64 solve, with the same residual bound."""
    n, nev, nex = 64, 8, 6
    P = bi.make_problem(n, seed=11, real=(kind == "real"))
    A, B = problem_on_device(P)
    W0, V0 = starts(n, nev + nex, 0)
    lam, V, st = pkg.solve(A, B, nev, nex, 12, 1e-10, W0=to_dev(W0), V0=to_dev(V0), deg_min=4, deg_max=24,
                           precision="fp64_tc")
    ref, _ = dense.smallest_positive(P.A, P.B, nev)
    lam = lam.cpu().numpy()
    np.testing.assert_allclose(lam, ref, rtol=TOL_EIG)
    Vg = V.cpu().numpy().T
    H = dense.hamiltonian(P.A, P.B)
    R = H @ Vg - Vg * lam
    assert np.linalg.norm(R, axis=0).max() / np.linalg.norm(H, 2) <= 1e-10
    assert st["filter_flops_fp64"] == st["filter_flops"]


def test_solve_fp64_tc_n512_workload(pkg):
    cfg = bi.WORKLOADS["n512"]
    n, nev, nex = cfg["n"], cfg["nev"], cfg["nex"]
    P = bi.make_problem(n, seed=0, spec=cfg["spec"], beta=cfg["beta"])
    A, B = problem_on_device(P)
    W0, V0 = starts(n, nev + nex, 0)
    lam, V, st = pkg.solve(A, B, nev, nex, cfg["deg"], cfg["tol"], W0=to_dev(W0), V0=to_dev(V0),
                           deg_min=cfg["deg_min"], deg_max=cfg["deg_max"], precision="fp64_tc")
    ref, _ = dense.smallest_positive(P.A, P.B, nev)
    np.testing.assert_allclose(lam.cpu().numpy(), ref, rtol=TOL_EIG)
    assert st["max_residual"] <= cfg["tol"]
