"""Parity of the tensor-core (tcgen05) filter and the mixed-precision solve with the oracle."""
import numpy as np
import pytest
import torch

import bse_inputs as bi
from oracle import chebyshev, dense
from tests.gpu_util import problem_on_device, rel_fro, starts, to_dev

pytestmark = pytest.mark.gpu

# Relative Frobenius tolerances of the tensor-core filter against the FP64 oracle.
# FP16x3 (the default mixed scheme) keeps 22 significant bits of each operand and
# BF16x6 24 (FP32 class): the 1e-5 gate of an FP32 filter applies.  BF16x3 keeps
# 16 bits of each operand: the representation error is 2 * 2^-17 = 1.5e-5 per
# product, and the recurrence adds a small factor; it is kept as a labelled
# low-accuracy option.
TOL = {"fp16x3": 1e-5, "bf16x6": 1e-5, "bf16x3": 6e-5}


@pytest.fixture(scope="module")
def pkg():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    import paper_2601_10557_gb300 as p
    if not p.has_mixed():
        pytest.fail("tensor-core filter not available on this device")
    return p


def _mus(P):
    lam, _ = dense.eig_cholesky(P.A, P.B)
    pos = lam[P.n:]
    return 0.9 * pos[0], pos[len(pos) // 6], 1.05 * pos[-1]


@pytest.mark.parametrize("scheme", ["fp16x3", "bf16x3", "bf16x6"])
# (300, 70): an odd number of row blocks, a narrow last column tile and a 2-way K split;
# (640, 24): 5 row blocks and a 4-way K split of 6 CTAs per split
@pytest.mark.parametrize("n,k,maxdeg", [(128, 8, 1), (128, 8, 4), (300, 70, 8), (129, 33, 6), (640, 24, 4)])
def test_filter_tensor_core_matches_oracle(pkg, scheme, n, k, maxdeg):
    P = bi.make_problem(n, seed=n + k)
    A, B = problem_on_device(P)
    W0 = bi.start_block(n, k, 3)
    degs = np.random.default_rng(k).integers(1, maxdeg + 1, size=k)
    mu1, mune, muN = _mus(P)
    W = to_dev(W0)
    pkg.filter(A, B, W, degs, mu1, mune, muN, precision=scheme)
    Y = chebyshev.chebyshev_filter(P.A, P.B, W0.T, degs, mu1, mune, muN)
    err = rel_fro(W.cpu().numpy().T, Y)
    assert err < TOL[scheme], err


@pytest.mark.parametrize("scheme", ["fp16x3", "bf16x3", "bf16x6"])
def test_solve_mixed_matches_brute_force(pkg, scheme):
    n, nev, nex = 64, 8, 6
    P = bi.make_problem(n, seed=11)
    A, B = problem_on_device(P)
    W0, V0 = starts(n, nev + nex, 0)
    lam, V, st = pkg.solve(A, B, nev, nex, 12, 1e-10, W0=to_dev(W0), V0=to_dev(V0), deg_min=4, deg_max=24,
                           precision=scheme)
    ref, _ = dense.smallest_positive(P.A, P.B, nev)
    np.testing.assert_allclose(lam.cpu().numpy(), ref, rtol=1e-10)
    Vg = V.cpu().numpy().T
    H = dense.hamiltonian(P.A, P.B)
    R = H @ Vg - Vg * lam.cpu().numpy()
    assert np.linalg.norm(R, axis=0).max() / np.linalg.norm(H, 2) <= 1e-10
    assert st["filter_flops_fp64"] < 0.5 * st["filter_flops"]


def test_solve_mixed_n512_workload(pkg):
    cfg = bi.WORKLOADS["n512"]
    n, nev, nex = cfg["n"], cfg["nev"], cfg["nex"]
    P = bi.make_problem(n, seed=0, spec=cfg["spec"], beta=cfg["beta"])
    A, B = problem_on_device(P)
    W0, V0 = starts(n, nev + nex, 0)
    lam, V, st = pkg.solve(A, B, nev, nex, cfg["deg"], cfg["tol"], W0=to_dev(W0), V0=to_dev(V0),
                           deg_min=cfg["deg_min"], deg_max=cfg["deg_max"], precision="mixed")
    ref, _ = dense.smallest_positive(P.A, P.B, nev)
    np.testing.assert_allclose(lam.cpu().numpy(), ref, rtol=1e-10)
    assert st["max_residual"] <= cfg["tol"]


@pytest.mark.parametrize("scheme", ["fp16x3", "bf16x6"])
def test_filter_tensor_core_column_scales(pkg, scheme):
    """Columns whose magnitudes span 1e-20 .. 1e20 (far outside FP16's range): every
    operand row is scaled by a power of two, so each column keeps the 1e-5 accuracy
    relative to its own norm."""
    n, k = 200, 12
    P = bi.make_problem(n, seed=7)
    A, B = problem_on_device(P)
    W0 = bi.start_block(n, k, 5)
    W0 *= (10.0 ** np.linspace(-20, 20, k))[:, None]
    degs = np.full(k, 5)
    mu1, mune, muN = _mus(P)
    W = to_dev(W0)
    pkg.filter(A, B, W, degs, mu1, mune, muN, precision=scheme)
    Y = chebyshev.chebyshev_filter(P.A, P.B, W0.T, degs, mu1, mune, muN)
    got = W.cpu().numpy().T
    for j in range(k):
        assert rel_fro(got[:, j], Y[:, j]) < TOL[scheme], j


def test_filter_precision_groups(pkg):
    """The precision groups of a mixed solve in one filter call (chase_bse_filter_cols):
    FP64 columns on the FP64 filter (1e-12 against the oracle), the others on the
    tensor-core filter (1e-5), with ragged degrees in both groups."""
    n, k = 300, 24
    P = bi.make_problem(n, seed=9)
    A, B = problem_on_device(P)
    W0 = bi.start_block(n, k, 9)
    rng = np.random.default_rng(9)
    degs = rng.integers(1, 7, size=k)
    precs = ["fp64" if i % 3 == 0 else "fp16x3" for i in range(k)]
    mu1, mune, muN = _mus(P)
    W = to_dev(W0)
    pkg.filter_cols(A, B, W, degs, precs, mu1, mune, muN)
    Y = chebyshev.chebyshev_filter(P.A, P.B, W0.T, degs, mu1, mune, muN)
    got = W.cpu().numpy().T
    for j in range(k):
        err = rel_fro(got[:, j], Y[:, j])
        assert err < (1e-12 if precs[j] == "fp64" else TOL["fp16x3"]), (j, precs[j], err)


def test_solve_mixed_moves_stalled_columns_to_fp64(pkg):
    """With switch_tol = 1 every column whose residual stops decreasing moves to the FP64
    filter (the precision groups inside the solve's filter calls); the result still
    matches the dense oracle."""
    n, nev, nex = 64, 8, 6
    P = bi.make_problem(n, seed=13)
    A, B = problem_on_device(P)
    W0, V0 = starts(n, nev + nex, 13)
    lam, V, st = pkg.solve(A, B, nev, nex, 4, 1e-10, W0=to_dev(W0), V0=to_dev(V0), deg_min=2, deg_max=6,
                           precision="mixed", switch_tol=1.0, maxiter=60)
    ref, _ = dense.smallest_positive(P.A, P.B, nev)
    np.testing.assert_allclose(lam.cpu().numpy(), ref, rtol=1e-10)
    assert st["filter_flops_fp64"] > 0.0
    assert st["filter_flops_fp64"] < st["filter_flops"]


@pytest.mark.parametrize("precision,kind", [("fp16x3", "tensor"), ("fp64", "fp64")])
def test_gemm_timer_counts_the_filter_launches(pkg, precision, kind):
    """The event record of the filter's H applications (the bench's roofline source):
    a filter over columns with degrees d_i applies H 2 d_i times to column i, so the
    record holds 2 max(d) launches of 32 n^2 k_j flops each, 64 n^2 sum(d) flops in
    all, with a positive device time; reading clears it, and nothing is recorded while
    the record is off."""
    n, k = 256, 40
    P = bi.make_problem(n, seed=21)
    A, B = problem_on_device(P)
    degs = np.sort(np.random.default_rng(21).integers(1, 6, size=k))[::-1].copy()
    mu1, mune, muN = _mus(P)
    pkg.gemm_timer(True)
    try:
        W = to_dev(bi.start_block(n, k, 21))
        pkg.filter(A, B, W, degs, mu1, mune, muN, precision=precision)
        torch.cuda.synchronize()
        ms, flops, launches = pkg.gemm_time(kind)
        other = pkg.gemm_time("fp64" if kind == "tensor" else "tensor")
        again = pkg.gemm_time(kind)
    finally:
        pkg.gemm_timer(False)
    assert launches == 2 * int(degs.max())
    assert flops == 64.0 * n * n * float(degs.sum())
    assert ms > 0.0
    assert other == (0.0, 0.0, 0)
    assert again == (0.0, 0.0, 0)
    W = to_dev(bi.start_block(n, k, 21))
    pkg.filter(A, B, W, degs, mu1, mune, muN, precision=precision)
    assert pkg.gemm_time(kind) == (0.0, 0.0, 0)
