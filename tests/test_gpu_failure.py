"""Failure paths that are tested without faulting the GPU: a device-side wait that runs
out (the grid barrier of the cooperative kernels, with its bound shortened through
chase_bse_set_wait_limit) returns DEVICE_TIMEOUT and leaves the device usable; inputs
with a NaN return NONFINITE before any work."""
import numpy as np
import pytest
import torch

import bse_inputs as bi
from oracle import dense
from tests.gpu_util import problem_on_device, starts, to_dev

pytestmark = pytest.mark.gpu

DEVICE_TIMEOUT, NONFINITE = -6, -8


@pytest.fixture(scope="module")
def pkg():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    import paper_2601_10557_gb300 as p
    return p


def _small_solve_ok(pkg):
    n, nev, nex = 64, 6, 6
    P = bi.make_problem(n, seed=3)
    A, B = problem_on_device(P)
    W0, V0 = starts(n, nev + nex, 3)
    lam, _, _ = pkg.solve(A, B, nev, nex, 12, 1e-10, W0=to_dev(W0), V0=to_dev(V0), deg_min=4, deg_max=24)
    ref, _ = dense.smallest_positive(P.A, P.B, nev)
    np.testing.assert_allclose(lam.cpu().numpy(), ref, rtol=1e-10)


def test_grid_barrier_wait_runs_out_then_device_recovers(pkg):
    """A 1 ns bound on the grid-barrier waits: the FP64 block Jacobi's first barrier (CTAs
    without a block pair wait for those with one) gives up, every CTA leaves at its next
    barrier, the call returns DEVICE_TIMEOUT; with the default bound restored, the same
    process solves a problem correctly."""
    rng = np.random.default_rng(0)
    k = 520
    Z = rng.standard_normal((k, k)) + 1j * rng.standard_normal((k, k))
    G = torch.from_numpy(0.5 * (Z + Z.conj().T)).cuda()
    try:
        pkg.set_wait_limit(1)
        with pytest.raises(pkg.ChaseBSEError) as ei:
            pkg.eigh(G, method="block")
        assert ei.value.status == DEVICE_TIMEOUT
    finally:
        pkg.set_wait_limit(0)
    theta, V = pkg.eigh(G, method="block")
    ref = np.linalg.eigvalsh(G.cpu().numpy())
    assert np.abs(np.sort(theta.cpu().numpy()) - ref).max() <= 1e-11 * np.abs(ref).max()
    _small_solve_ok(pkg)


@pytest.mark.parametrize("where", ["W0", "A"])
def test_nonfinite_input_is_rejected_then_device_recovers(pkg, where):
    """A NaN injected on the host into one column of the start block (or one entry of A)
    makes the solve return NONFINITE before any work."""
    n, nev, nex = 64, 6, 6
    P = bi.make_problem(n, seed=4)
    A, B = problem_on_device(P)
    W0, V0 = starts(n, nev + nex, 4)
    W0 = W0.copy()
    if where == "W0":
        W0[2, 5] = np.nan
    else:
        A = A.clone()
        A[3, 7] = complex(np.inf, 0.0)
    with pytest.raises(pkg.ChaseBSEError) as ei:
        pkg.solve(A, B, nev, nex, 12, 1e-10, W0=to_dev(W0), V0=to_dev(V0), deg_min=4, deg_max=24)
    assert ei.value.status == NONFINITE
    _small_solve_ok(pkg)
