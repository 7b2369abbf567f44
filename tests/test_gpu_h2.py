"""The explicit-H^2 variant (not the paper's method, which applies H twice per filter
step): the blocks of H^2 against the oracle (oracle/chebyshev.py h2_blocks), the
tensor-core filter that applies them against the oracle's explicit filter, and a mixed
solve with it against brute force."""
import numpy as np
import pytest
import torch

import bse_inputs as bi
from oracle import chebyshev, dense
from tests.gpu_util import problem_on_device, rel_fro, starts, to_dev

pytestmark = pytest.mark.gpu

# Relative Frobenius tolerance of the explicit-H^2 tensor-core filter (FP16x3) against
# the oracle: the squared operator's entries reach ||H||^2, so the 2^-22 operand error of
# a product is relative to L2 max|z| with L2 the largest row sum of [P | Q]; a CPU
# emulation of the operand rounding measured 2-5x the implicit filter's error, whose
# gate is 1e-5.
TOL_EXPLICIT = 5e-5


@pytest.fixture(scope="module")
def pkg():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    import paper_2601_10557_gb300 as p
    if not p.has_mixed():
        pytest.fail("tensor cores not available on this device")
    return p


def _mus(P):
    lam, _ = dense.eig_cholesky(P.A, P.B)
    pos = lam[P.n:]
    return 0.9 * pos[0], pos[len(pos) // 6], 1.05 * pos[-1]


@pytest.mark.parametrize("n,kind", [(1, "complex"), (64, "complex"), (200, "complex"), (130, "real"),
                                    (64, "bzero")])
def test_h2_blocks_match_oracle(pkg, n, kind):
    """FP64-accurate products: the error of every block is at the rounding level of the
    products it sums, u ||[A | B]||_F^2 (Q = A B - B conj(A) cancels: its own norm can be
    far smaller than the terms', so it is not the scale)."""
    P = bi.make_problem(n, seed=n + 3, real=(kind == "real"), b_zero=(kind == "bzero"))
    A, B = problem_on_device(P)
    Pg, Qg = pkg.h2_blocks(A, B)
    Pr, Qr = chebyshev.h2_blocks(P.A, P.B)
    scale = np.linalg.norm(P.A) ** 2 + np.linalg.norm(P.B) ** 2
    assert np.linalg.norm(Pg.cpu().numpy() - Pr) <= 1e-13 * scale
    assert np.linalg.norm(Qg.cpu().numpy() - Qr) <= 1e-13 * scale
    assert rel_fro(Pg.cpu().numpy(), Pr) <= 1e-12
    if kind == "bzero" or n == 1:
        # Q = 0: B = 0, or n = 1 where Q = b (a - conj a) with a real
        assert np.abs(Qg.cpu().numpy()).max() <= 1e-14 * scale


@pytest.mark.parametrize("n,k,maxdeg", [(128, 8, 4), (300, 70, 8), (129, 33, 6), (640, 24, 4)])
def test_filter_h2_matches_oracle(pkg, n, k, maxdeg):
    P = bi.make_problem(n, seed=n + k + 1)
    A, B = problem_on_device(P)
    W0 = bi.start_block(n, k, 5)
    degs = np.random.default_rng(k + 2).integers(1, maxdeg + 1, size=k)
    mu1, mune, muN = _mus(P)
    W = to_dev(W0)
    pkg.filter_h2(A, B, W, degs, mu1, mune, muN)
    Pr, Qr = chebyshev.h2_blocks(P.A, P.B)
    Y = chebyshev.chebyshev_filter_explicit(Pr, Qr, W0.T, degs, mu1, mune, muN)
    assert rel_fro(W.cpu().numpy().T, Y) < TOL_EXPLICIT


@pytest.mark.parametrize("n,nev,nex,deg,spec", [(64, 8, 6, 12, "uniform:1:10"), (512, 20, 10, 20, "uniform:1:10")])
def test_solve_explicit_h2_matches_brute_force(pkg, n, nev, nex, deg, spec):
    """The correction form keeps the explicit variant's solve FP64-accurate: the
    eigenvalues of brute force to 1e-10 and every residual below the tolerance."""
    P = bi.make_problem(n, seed=0, spec=spec)
    A, B = problem_on_device(P)
    W0, V0 = starts(n, nev + nex, 0)
    lam, V, st = pkg.solve(A, B, nev, nex, deg, 1e-10, W0=to_dev(W0), V0=to_dev(V0), deg_min=4, deg_max=36,
                           maxiter=40, precision="mixed", h2="explicit")
    ref, _ = dense.smallest_positive(P.A, P.B, nev)
    np.testing.assert_allclose(lam.cpu().numpy(), ref, rtol=1e-10)
    assert st["max_residual"] <= 1e-10
    assert st["ms_h2"] > 0.0
