"""Host logic of the benchmark (no GPU): the per-eigenvalue error bounds it reports and
the roofline traffic lookup."""
import numpy as np
import pytest
import torch

import bench
import bse_inputs as bi
from oracle import dense


def _exact_pairs(n=24, nev=5, seed=2):
    P = bi.make_problem(n, seed=seed)
    lam, V = dense.smallest_positive(P.A, P.B, nev)
    V = V / np.linalg.norm(V, axis=0, keepdims=True)
    return P, lam, V


def test_error_bounds_vanish_on_exact_pairs():
    """Exact eigenpairs (brute force): residual-based bounds and the S-Rayleigh quotient
    difference are at the rounding level."""
    P, lam, V = _exact_pairs()
    e = bench.eig_error_bounds(torch.from_numpy(P.A), torch.from_numpy(P.B), torch.from_numpy(lam),
                               torch.from_numpy(np.ascontiguousarray(V.T)), nsample=5)
    assert e["sampled_pairs"] == 5
    assert e["max_rel_bound"] <= 1e-13
    assert e["max_rel_rayleigh_diff"] <= 1e-13


def test_error_bounds_see_a_shifted_eigenvalue():
    """An eigenvalue reported 1e-6 too large (vector exact): the S-Rayleigh quotient of the
    vector is the true eigenvalue, so the quotient difference is 1e-6 relative, and the
    first-order bound ||Hv - lambda v|| / (|v^* S v| lambda) is at least that."""
    P, lam, V = _exact_pairs()
    lam2 = lam.copy()
    lam2[2] *= 1.0 + 1e-6
    e = bench.eig_error_bounds(torch.from_numpy(P.A), torch.from_numpy(P.B), torch.from_numpy(lam2),
                               torch.from_numpy(np.ascontiguousarray(V.T)), nsample=5)
    row = [r for r in e["per_eigenvalue"] if r["i"] == 2][0]
    assert abs(row["rel_rq_diff"] - 1e-6 / (1.0 + 1e-6)) <= 1e-12
    assert row["rel_bound"] >= 0.99e-6


def test_traffic_lookup_follows_the_kernel_hash(tmp_path, monkeypatch):
    """A capture counts only while the filter source hashes to the recorded value."""
    h = bench.filter_source_hash()
    doc = tmp_path / "traffic.md"
    doc.write_text(f"kernel source sha256[:16]: {h}\ntraffic_bytes_per_launch[n4096]: 5.5e8\n")
    monkeypatch.setattr(bench, "TRAFFIC_PROFILE", str(doc))
    v, _ = bench.traffic_for("n4096")
    assert v == 5.5e8
    assert bench.traffic_for("n16384")[0] is None
    doc.write_text("kernel source sha256[:16]: 0000000000000000\ntraffic_bytes_per_launch[n4096]: 5.5e8\n")
    assert bench.traffic_for("n4096")[0] is None
