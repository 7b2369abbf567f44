"""Parity at full size: the n = 4096 workload in the configuration the benchmark
times (mixed precision, nev = 200, nex = 60, degrees 20-36, tol 1e-10), and the
n = 8192 gradient workload.

The dense oracle cannot solve these sizes in test time, so the checks are the
properties that fix the answer at any size, each computed on the host from the
GPU output with the plain FP64 formulas:

* residuals ||H v - lambda v|| <= tol ||H||_2 (bound ||A||_2 + ||B||_2, exact for
  the planted inputs) for every returned pair;
* lambda equals the S-Rayleigh quotient v^* S H v / v^* S v of its own vector
  (quadratically accurate in the residual);
* completeness by Sylvester's law of inertia: for the definite pencil
  (S H, S), the number of negative eigenvalues of S H - sigma S is the number of
  eigenvalues of H in (0, sigma); just above lambda_nev it is nev, just below
  lambda_1 it is 0;
* the whole filter block against the oracle filter (element by element);
* the eigenvalue gradient against the oracle's formula on the same vectors and
  against central finite differences of the solve on 32 random directions;
* at n = 16384 the same properties, the inertia from the Schur complement of the
  pencil on the device; at n = 4096 with real A and B, lambda^2 against the
  eigenvalues of (A - B)(A + B).
"""
import numpy as np
import pytest
import torch

import bse_inputs as bi
from oracle import chebyshev, gradient
from tests.gpu_util import rel_fro, to_dev

pytestmark = pytest.mark.gpu

# FP64 filter: 1e-12; tensor-core filter (FP16x3, the default mixed scheme): the 1e-5
# gate of an FP32 filter, relative Frobenius over the whole block
TOL_FILTER = {"fp64": 1e-12, "mixed": 1e-5}


@pytest.fixture(scope="module")
def pkg():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    import paper_2601_10557_gb300 as p
    return p


@pytest.fixture(scope="module")
def c2():
    wl = bi.WORKLOADS["n4096"]
    P = bi.make_problem(wl["n"], seed=0, spec=wl["spec"], beta=wl["beta"])
    nevex = wl["nev"] + wl["nex"]
    return wl, P, bi.start_block(wl["n"], nevex, 0), bi.lanczos_starts(wl["n"], 4, 0)


def _hv(A, B, V):
    """H V for V (2n x m), H = [[A, B], [-conj(B), -conj(A)]], without forming H."""
    n = A.shape[0]
    X, Y = V[:n], V[n:]
    return np.vstack([A @ X + B @ Y, -(B.conj() @ X) - A.conj() @ Y])


def _negative_count(M):
    """Number of negative eigenvalues of the hermitian M (LDL^* with 1x1 / 2x2 blocks)."""
    import scipy.linalg as sl
    _, D, _ = sl.ldl(M, lower=True, hermitian=True)
    count, i, m = 0, 0, D.shape[0]
    while i < m:
        if i + 1 < m and D[i + 1, i] != 0:
            count += int((np.linalg.eigvalsh(D[i:i + 2, i:i + 2]) < 0).sum())
            i += 2
        else:
            count += int(D[i, i].real < 0)
            i += 1
    return count


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_c2_filter_full_block(pkg, c2, precision):
    """The whole n = 4096, k = 260, degree-20 filter block against the oracle filter,
    element by element (relative Frobenius over the block)."""
    if precision == "mixed" and not pkg.has_mixed():
        pytest.fail("tensor-core filter not available on this device")
    wl, P, W0, _ = c2
    k, deg = W0.shape[0], 20
    mus = (1.0, 2.0, 45.0)
    W = to_dev(W0)
    pkg.filter(to_dev(P.A), to_dev(P.B), W, [deg] * k, *mus, precision=precision)
    got = W.cpu().numpy().T
    ref = chebyshev.chebyshev_filter(P.A, P.B, W0.T, [deg] * k, *mus)
    assert rel_fro(got, ref) < TOL_FILTER[precision]
    # and column by column (no column may hide behind the large ones)
    colerr = np.linalg.norm(got - ref, axis=0) / np.linalg.norm(ref, axis=0)
    assert colerr.max() < 10 * TOL_FILTER[precision], colerr.max()


def test_c3_filter_sampled_columns(pkg):
    """At n = 16384 (the n16384 workload's inputs, H 32768 x 32768) the tensor-core
    filter on 6 columns, degree 20, against the oracle filter (H formed on the host);
    the columns are filtered independently, so a few stand for the block."""
    if not pkg.has_mixed():
        pytest.fail("tensor-core filter not available on this device")
    wl = bi.WORKLOADS["n16384"]
    A, B, _ = bi.make_problem_device(wl["n"], 0, wl["spec"], wl["beta"], device=torch.device("cuda:0"))
    W0 = bi.start_block(wl["n"], 6, 0)
    mus = (1.0, 2.7, 75.0)
    W = to_dev(W0)
    pkg.filter(A, B, W, [20] * 6, *mus, precision="mixed")
    got = W.cpu().numpy().T
    ref = chebyshev.chebyshev_filter(A.cpu().numpy(), B.cpu().numpy(), W0.T, [20] * 6, *mus)
    colerr = np.linalg.norm(got - ref, axis=0) / np.linalg.norm(ref, axis=0)
    assert colerr.max() < TOL_FILTER["mixed"], colerr


def test_c2_mixed_solve_properties(pkg, c2):
    if not pkg.has_mixed():
        pytest.fail("tensor-core filter not available on this device")
    wl, P, W0, V0 = c2
    n, nev, nex, tol = wl["n"], wl["nev"], wl["nex"], wl["tol"]
    lam, V, st = pkg.solve(to_dev(P.A), to_dev(P.B), nev, nex, wl["deg"], tol, precision="mixed",
                           W0=to_dev(W0), V0=to_dev(V0), deg_min=wl["deg_min"], deg_max=wl["deg_max"],
                           maxiter=40)
    lam = lam.cpu().numpy()
    V = V.cpu().numpy().T  # 2n x nev
    assert st["converged"] == nev
    assert np.all(np.diff(lam) > 0) and lam[0] > 0
    np.testing.assert_allclose(np.linalg.norm(V, axis=0), 1.0, atol=1e-12)
    # phase convention: largest-magnitude entry of the upper half real and positive
    top = V[:n]
    piv = top[np.argmax(np.abs(top), axis=0), np.arange(nev)]
    assert np.all(np.abs(piv.imag) <= 1e-12 * np.abs(piv)) and np.all(piv.real > 0)
    # residuals against the exact norm bound of the planted inputs
    hnorm = P.d.max() + P.beta * P.d.min()
    HV = _hv(P.A, P.B, V)
    res = np.linalg.norm(HV - V * lam, axis=0)
    assert res.max() <= tol * hnorm, res.max() / hnorm
    # lambda is the S-Rayleigh quotient of its vector
    SV = np.vstack([V[:n], -V[n:]])
    rq = np.real(np.sum(SV.conj() * HV, axis=0) / np.sum(SV.conj() * V, axis=0))
    assert np.max(np.abs(rq - lam) / lam) < 1e-12
    # completeness: exactly nev eigenvalues of H in (0, lambda_nev (1 + 1e-9)], none below lambda_1
    SH = np.block([[P.A, P.B], [P.B.conj(), P.A.conj()]])
    S = np.concatenate([np.ones(n), -np.ones(n)])
    for sigma, want in ((lam[-1] * (1 + 1e-9), nev), (lam[0] * (1 - 1e-9), 0)):
        assert _negative_count(SH - sigma * np.diag(S)) == want


def test_c4_gradient_fullsize(pkg):
    """n = 8192, nev = 100, nex = 40: the adjoint kernel against the oracle's formula
    on the same eigenvectors, and against central differences (h = 1e-6) of the solve
    along dA = I and 32 random hermitian / complex-symmetric directions."""
    if not pkg.has_mixed():
        pytest.fail("tensor-core filter not available on this device")
    wl = bi.WORKLOADS["n8192grad"]
    n, nev, nex = wl["n"], wl["nev"], wl["nex"]
    P = bi.make_problem(n, seed=0, spec=wl["spec"], beta=wl["beta"])
    W0, V0 = bi.start_block(n, nev + nex, 0), bi.lanczos_starts(n, 4, 0)
    w = bi.loss_weights(nev, 0)
    # the dense planted spectrum (spacing ~1e-3 around lambda_nev) converges slowly:
    # adaptive degrees up to 36 and up to 100 iterations
    kw = dict(W0=to_dev(W0), V0=to_dev(V0), deg_min=wl["deg_min"], deg_max=36, maxiter=100,
              precision="mixed")
    lam, Vt, st = pkg.solve(to_dev(P.A), to_dev(P.B), nev, nex, wl["deg"], wl["tol"], **kw)
    gA, gB = pkg.grad(Vt, torch.from_numpy(w))
    gA, gB = gA.cpu().numpy(), gB.cpu().numpy()
    rA, rB = gradient.gradient_from_vectors(Vt.cpu().numpy().T, w)
    assert rel_fro(gA, rA) < 1e-12
    assert rel_fro(gB, rB) < 1e-12
    np.testing.assert_allclose(gA, gA.conj().T, atol=1e-12 * np.abs(gA).max())
    np.testing.assert_allclose(gB, gB.T, atol=1e-12 * np.abs(gB).max())
    # central differences (h = 1e-6) of the solve on 32 random directions (the
    # configuration's count): dA hermitian and dB complex symmetric, Wigner-scaled
    # (entries ~ 1/sqrt(n), ||dA||_2 ~ 2) so that h ||dA|| stays far below the eigenvalue
    # gaps of the planted spectrum, plus dA = I (which perturbs H by S); each perturbed
    # solve starts from the converged eigenvectors (a warm restart)
    rng = np.random.default_rng(5)
    h = 1e-6
    # the solver scales the start block's lower half by gamma = 1e-3 (Section 4.6): the
    # converged vectors' lower halves are divided by it beforehand
    Vc = Vt.cpu().numpy().copy()
    Vc[:, n:] /= 1e-3
    W0w = np.concatenate([Vc, W0[nev:]], axis=0)
    kw_w = dict(kw, W0=to_dev(W0w), deg_min=8)
    dirs = [(np.eye(n, dtype=complex), np.zeros((n, n), dtype=complex))]
    for _ in range(32):
        E = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
        F = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
        dirs.append(((E + E.conj().T) / (2 * np.sqrt(n)), (F + F.T) / (2 * np.sqrt(n))))
    fds, ans = [], []
    for dA, dB in dirs:
        lp, _, _ = pkg.solve(to_dev(P.A + h * dA), to_dev(P.B + h * dB), nev, nex, wl["deg"], wl["tol"], **kw_w)
        lm, _, _ = pkg.solve(to_dev(P.A - h * dA), to_dev(P.B - h * dB), nev, nex, wl["deg"], wl["tol"], **kw_w)
        fds.append(float(np.dot(w, (lp - lm).cpu().numpy()) / (2 * h)))
        ans.append(float(np.real(np.sum(gA.conj() * dA) + np.sum(gB.conj() * dB))))
    fds, ans = np.array(fds), np.array(ans)
    # dA = I on its own; the random directions as one vector of directional derivatives (a
    # random direction's derivative sum_i w_i dlambda_i can be near zero: its own relative
    # error would measure the cancellation, not the gradient)
    assert abs(fds[0] - ans[0]) <= 1e-6 * abs(ans[0]), (fds[0], ans[0])
    rel = np.linalg.norm(fds[1:] - ans[1:]) / np.linalg.norm(ans[1:])
    assert rel <= 1e-6, (rel, np.abs(fds[1:] - ans[1:]).max(), np.abs(ans[1:]).min())


def _hv_torch(A, B, V):
    """H V on the device in FP64 (torch products): V (2n x m)."""
    n = A.shape[0]
    X, Y = V[:n], V[n:]
    return torch.cat([A @ X + B @ Y, -(B.conj() @ X) - A.conj() @ Y], dim=0)


def _negative_count_schur(A, B, sigma):
    """Eigenvalues of H in (0, sigma) for the definite pencil (S H, S): the negative
    eigenvalues of S H - sigma S = [[A - sigma, B], [conj(B), conj(A) + sigma]].  Its
    lower-right block conj(A) + sigma I is positive definite (A is), so by Sylvester's law
    of inertia the count is that of the Schur complement
    M = A - sigma I - B (conj(A) + sigma I)^-1 conj(B) (torch FP64 on the device)."""
    n = A.shape[0]
    I = torch.eye(n, dtype=A.dtype, device=A.device)
    L = torch.linalg.cholesky(A.conj() + sigma * I)
    Z = torch.cholesky_solve(B.conj(), L)
    M = A - sigma * I - B @ Z
    M = 0.5 * (M + M.conj().T)
    ev = torch.linalg.eigvalsh(M)
    return int((ev < 0).sum().item())


def test_c3_mixed_solve_properties(pkg):
    """n = 16384 (H 32768), nev 1000, nex 300, degrees 8-36, tol 1e-10, the gapband
    spectrum (the benchmark's configuration): residuals against the norm bound,
    lambda = the S-Rayleigh quotient of its vector, completeness by the inertia of the
    Schur complement just above lambda_nev (nev distinct eigenpairs and exactly nev
    eigenvalues in (0, lambda_nev] leave none out, below lambda_1 included)."""
    if not pkg.has_mixed():
        pytest.fail("tensor-core filter not available on this device")
    wl = bi.WORKLOADS["n16384"]
    n, nev, nex, tol = wl["n"], wl["nev"], wl["nex"], wl["tol"]
    dev = torch.device("cuda:0")
    A, B, d = bi.make_problem_device(n, 0, wl["spec"], wl["beta"], device=dev)
    W0, V0 = bi.start_block(n, nev + nex, 0), bi.lanczos_starts(n, 4, 0)
    lam, V, st = pkg.solve(A, B, nev, nex, wl["deg"], tol, precision="mixed", W0=to_dev(W0), V0=to_dev(V0),
                           deg_min=wl["deg_min"], deg_max=wl["deg_max"], maxiter=40)
    assert st["converged"] == nev
    lam_h = lam.cpu().numpy()
    assert np.all(np.diff(lam_h) > 0) and lam_h[0] > 0
    Vt = V.T  # 2n x nev
    # ||H||_2 <= ||A||_2 + ||B||_2 = max(d) + beta min(d) (A's eigenvalues are d up to
    # the assembly's FP32 rounding, ~1e-6 ||A||: a 1e-5 margin)
    hnorm = (d.max() + wl["beta"] * d.min()) * (1 + 1e-5)
    worst_res, worst_rq = 0.0, 0.0
    for c0 in range(0, nev, 250):
        Vb = Vt[:, c0:c0 + 250]
        lb = lam[c0:c0 + 250]
        HV = _hv_torch(A, B, Vb)
        res = torch.linalg.vector_norm(HV - Vb * lb[None, :], dim=0)
        worst_res = max(worst_res, float(res.max()))
        SV = torch.cat([Vb[:n], -Vb[n:]], dim=0)
        rq = torch.real(torch.sum(SV.conj() * HV, dim=0) / torch.sum(SV.conj() * Vb, dim=0))
        worst_rq = max(worst_rq, float(((rq - lb).abs() / lb).max()))
    assert worst_res <= tol * hnorm, worst_res / hnorm
    assert worst_rq < 1e-12, worst_rq
    assert _negative_count_schur(A, B, float(lam_h[-1]) * (1 + 1e-9)) == nev


def test_c2_real_variant_squared_spectrum(pkg):
    """n = 4096 with real symmetric A and B, mixed precision: lambda^2 are the
    eigenvalues of (A - B)(A + B); with A + B = L L^T (positive definite for a definite
    problem) they are those of the symmetric L^T (A - B) L (host LAPACK)."""
    if not pkg.has_mixed():
        pytest.fail("tensor-core filter not available on this device")
    import scipy.linalg as sl
    wl = bi.WORKLOADS["n4096"]
    n, nev, nex, tol = wl["n"], wl["nev"], wl["nex"], wl["tol"]
    P = bi.make_problem(n, seed=2, spec=wl["spec"], beta=wl["beta"], real=True)
    W0, V0 = bi.start_block(n, nev + nex, 2), bi.lanczos_starts(n, 4, 2)
    lam, V, st = pkg.solve(to_dev(P.A), to_dev(P.B), nev, nex, wl["deg"], tol, precision="mixed", W0=to_dev(W0),
                           V0=to_dev(V0), deg_min=wl["deg_min"], deg_max=wl["deg_max"], maxiter=40)
    assert st["converged"] == nev
    Ar, Br = P.A.real, P.B.real
    L = sl.cholesky(Ar + Br, lower=True)
    mu = sl.eigh(L.T @ (Ar - Br) @ L, eigvals_only=True, subset_by_index=[0, nev - 1])
    np.testing.assert_allclose(lam.cpu().numpy() ** 2, mu, rtol=2e-10)
