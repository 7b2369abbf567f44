"""The allocation-free residual entry point (chase_bse_residuals_noalloc) against
the allocating one (chase_bse_residuals), through the C ABI.

It exists for callers that cannot let a library allocate device memory (an
application pool that owns the whole device, a fixed memory budget, loops where
an allocation may synchronise the device).  This file is collected last, so a
run that stops at the first failure has already run every other test."""
import ctypes

import numpy as np
import pytest
import torch

import bse_inputs as bi

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2601_10557_gb300 import _lib
    return _lib


def _case(n, k, seed):
    P = bi.make_problem(n, seed=seed)
    dev = torch.device("cuda:0")
    A = torch.from_numpy(P.A).to(dev)
    B = torch.from_numpy(P.B).to(dev)
    W = bi.start_block(n, k, seed)
    W /= np.linalg.norm(W, axis=1, keepdims=True)
    Wt = torch.from_numpy(W).to(dev)
    lam = torch.from_numpy(np.linspace(0.5, 4.0, k)).to(dev)
    return A, B, Wt, lam


def _call(L, fn, A, B, W, lam, out, n, k, stream):
    vp = ctypes.c_void_p
    return getattr(L, fn)(vp(A.data_ptr()), vp(B.data_ptr()), n, vp(W.data_ptr()), vp(lam.data_ptr()), k,
                          vp(out.data_ptr()), vp(stream))


# (4096, 64) and (1024, 256): 2n * k = 2^19 (the scratch limit) with an output grid small
# enough that chase_bse_residuals splits K into partial sums (workspace it allocates);
# (200, 37) and (96, 5): small cases, the second running over stale contents of the first
CASES = [(4096, 64, 1), (1024, 256, 2), (200, 37, 3), (96, 5, 4)]


def test_noalloc_matches_allocating_entry_point_on_two_calls(lib):
    """Two calls in a row per case, each against chase_bse_residuals, with no device
    allocation by the library across the no-alloc calls."""
    L = lib.lib()
    stream = torch.cuda.current_stream().cuda_stream
    for n, k, seed in CASES:
        A, B, W, lam = _case(n, k, seed)
        ref = torch.zeros(k, dtype=torch.float64, device=A.device)
        assert _call(L, "chase_bse_residuals", A, B, W, lam, ref, n, k, stream) == 0
        torch.cuda.synchronize()
        for _ in range(2):
            out = torch.full((k,), float("nan"), dtype=torch.float64, device=A.device)
            before = L.chase_bse_alloc_count()
            assert _call(L, "chase_bse_residuals_noalloc", A, B, W, lam, out, n, k, stream) == 0
            torch.cuda.synchronize()
            assert L.chase_bse_alloc_count() == before, (n, k)
            np.testing.assert_allclose(out.cpu().numpy(), ref.cpu().numpy(), rtol=1e-12, atol=0)


def test_allocating_entry_point_does_allocate_on_a_split_case(lib):
    """The counter sees the split-K workspace of chase_bse_residuals at (4096, 64), so a
    zero count for the no-alloc call above is a real observation."""
    L = lib.lib()
    stream = torch.cuda.current_stream().cuda_stream
    n, k = 4096, 64
    A, B, W, lam = _case(n, k, 1)
    out = torch.zeros(k, dtype=torch.float64, device=A.device)
    before = L.chase_bse_alloc_count()
    assert _call(L, "chase_bse_residuals", A, B, W, lam, out, n, k, stream) == 0
    torch.cuda.synchronize()
    assert L.chase_bse_alloc_count() > before


def test_noalloc_rejects_sizes_beyond_its_scratch(lib):
    L = lib.lib()
    n = 4096
    k = lib.NOALLOC_MAX_ENTRIES // (2 * n) + 1
    # rejected on the host before anything is launched (pointers are never touched)
    dummy = ctypes.c_void_p(16)
    assert L.chase_bse_residuals_noalloc(dummy, dummy, n, dummy, dummy, k, dummy, None) == -1
