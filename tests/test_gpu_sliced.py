"""FP64-accurate sliced GEMM on the tensor cores (chase_bse_dgemm_sliced) and the
mixed solve that uses it for its QR and Rayleigh-Ritz products.

Exactness: with entries k_i * 2^(e_r) where |k_i| < 2^20 and K <= 4096, every
product and partial sum of A B^T is an integer multiple of 2^(e_r + e_c) below
2^53, so numpy's FP64 result is exact; the 7 signed 8-bit digits of the sliced
GEMM hold 21-bit integers exactly, so its result must be bit-identical.
"""
import numpy as np
import pytest
import torch

from bse_inputs import make_problem, start_block, lanczos_starts

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cbx():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    import paper_2601_10557_gb300 as p
    if not p.has_mixed():
        pytest.fail("tensor cores (sm_103a) not available on this device")
    return p


def _int_scaled(rng, rows, K, lo_exp=-30, hi_exp=30, bits=20):
    k = rng.integers(-(2 ** bits) + 1, 2 ** bits, size=(rows, K)).astype(np.float64)
    e = rng.integers(lo_exp, hi_exp + 1, size=rows)
    return np.ldexp(k, e[:, None])


@pytest.mark.parametrize("M,N,K", [(1, 1, 2), (130, 33, 258), (300, 70, 2050), (129, 257, 4096)])
def test_sliced_gemm_exact_on_integer_data(cbx, M, N, K):
    rng = np.random.default_rng(M * 1000 + N + K)
    A = _int_scaled(rng, M, K)
    B = _int_scaled(rng, N, K)
    ref = A @ B.T
    C = cbx.dgemm_sliced(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()).cpu().numpy()
    assert np.array_equal(C, ref), f"max |diff| {np.abs(C - ref).max()}"


def test_sliced_gemm_alpha_zero_rows_and_wide_range(cbx):
    rng = np.random.default_rng(7)
    A = _int_scaled(rng, 140, 512, -200, 200)
    B = _int_scaled(rng, 40, 512, -200, 200)
    A[3] = 0.0
    B[5] = 0.0
    ref = -2.0 * (A @ B.T)
    C = cbx.dgemm_sliced(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), alpha=-2.0).cpu().numpy()
    assert np.array_equal(C, ref)


@pytest.mark.parametrize("M,N,K", [(200, 100, 1000), (520, 520, 8192)])
def test_sliced_gemm_fp64_class_on_random_data(cbx, M, N, K):
    """Random FP64 entries: the error stays within 2^-51 K max|a_r| max|b_c| (the digit
    truncation bound, 2^-56 of the row scales per term) plus FP64 rounding of the
    numpy reference."""
    rng = np.random.default_rng(M + N + K)
    A = rng.standard_normal((M, K)) * np.logspace(-8, 8, M)[:, None]
    B = rng.standard_normal((N, K))
    ref = A @ B.T
    C = cbx.dgemm_sliced(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()).cpu().numpy()
    scale = np.abs(A).max(1)[:, None] * np.abs(B).max(1)[None, :]
    bound = 2.0 ** -51 * K * scale + 2.0 ** -50 * np.sqrt(K) * np.sqrt((A * A).sum(1))[:, None] * \
        np.sqrt((B * B).sum(1))[None, :]
    err = np.abs(C - ref)
    assert (err <= bound).all(), f"worst ratio {(err / bound).max()}"
    # and far inside it in practice (an FP64-class result, not an FP32-class one)
    assert (err / (scale * np.sqrt(K))).max() < 1e-14


def test_sliced_gemm_bad_args(cbx):
    L = cbx.lib()
    st = L.chase_bse_dgemm_sliced(None, 2, None, 2, 1, 1, 2, 1.0, None, 1, None)
    assert st == -1
    A = torch.zeros((4, 3), dtype=torch.float64, device="cuda")
    with pytest.raises(cbx.ChaseBSEError):  # odd K
        cbx.dgemm_sliced(A, A)


def test_mixed_solve_sliced_matches_fp64_products(cbx):
    """The n = 512 workload in mixed precision with the QR / Rayleigh-Ritz products on
    the tensor cores (default) and on the FP64 pipe: same eigenvalues to 1e-12."""
    p = make_problem(512, seed=0, spec="uniform:1:10", beta=0.3)
    A = torch.from_numpy(p.A).cuda()
    B = torch.from_numpy(p.B).cuda()
    nev, nex = 20, 10
    W0 = torch.from_numpy(start_block(512, nev + nex, 0)).cuda()
    V0 = torch.from_numpy(lanczos_starts(512, 4, 0)).cuda()
    out = {}
    for mode in ("tensor", "fp64"):
        ev, V, st = cbx.solve(A, B, nev, nex, 20, 1e-10, precision="mixed", W0=W0, V0=V0,
                              fp64_products=mode, maxiter=40)
        out[mode] = (ev.cpu().numpy(), V, st)
        assert st["max_residual"] <= 1e-10
    e_t, e_f = out["tensor"][0], out["fp64"][0]
    assert np.max(np.abs(e_t - e_f) / np.abs(e_f)) < 1e-12
    # mu_N and rho_hat come from the Lanczos bounds alone, whose H products run on the
    # tensor cores (J-even / J-odd split) in one mode and on the FP64 pipe in the other
    for key in ("muN", "rho_hat"):
        assert abs(out["tensor"][2][key] - out["fp64"][2][key]) <= 1e-9 * out["fp64"][2][key], key
    # and both match the dense eigenvalues of H
    H = np.block([[p.A, p.B], [-p.B.conj(), -p.A.conj()]])
    lam = np.sort(np.linalg.eigvals(H).real)
    pos = lam[lam > 0][:nev]
    assert np.max(np.abs(e_t - pos) / pos) < 1e-10
