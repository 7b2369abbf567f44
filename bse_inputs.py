"""Seeded synthetic inputs for the pseudo-hermitian (BSE) eigenproblem.

This module only draws random numbers and assembles the test matrices; it holds
none of the eigensolver's arithmetic.  Both the CPU oracle (``oracle/``) and the
CUDA path's tests and benchmark take their inputs from here, so that the two
sides see bit-identical data.

The Hamiltonian of the paper (Section 1, eq. ``introduction::hamiltonian_definition``)
is H = [[A, B], [-conj(B), -conj(A)]] with A hermitian and B complex symmetric;
the problem is "definite" when S H = [[A, B], [conj(B), conj(A)]] is hermitian
positive definite (eq. ``introduction::quasi_hermitian_condition``).  The
generator plants A = Q diag(d) Q^* with a Haar-unitary Q and draws
B = G + G^T scaled to ||B||_2 = beta * min(d); with beta < 1 this makes S H
positive definite, because x^* A x >= min(d) |x|^2 > ||B||_2 |x|^2.

Storage convention (shared with the C ABI): A and B are returned as C-ordered
(row-major) numpy complex128 arrays; the start vectors are returned as arrays of
shape (k, 2n), i.e. one 2n-vector per row, which is the column-major 2n x k
block the C ABI expects.
"""
from __future__ import annotations

import dataclasses
import numpy as np

__all__ = [
    "BSEProblem",
    "haar_unitary",
    "spectrum",
    "make_problem",
    "make_problem_device",
    "start_block",
    "lanczos_starts",
    "loss_weights",
    "WORKLOADS",
]


@dataclasses.dataclass
class BSEProblem:
    """A, B (row-major complex128 n x n), the planted spectrum d of A, beta."""

    A: np.ndarray
    B: np.ndarray
    d: np.ndarray
    beta: float
    seed: int
    real: bool

    @property
    def n(self) -> int:
        return self.A.shape[0]


def haar_unitary(n: int, rng: np.random.Generator, real: bool = False) -> np.ndarray:
    """Haar-distributed unitary (or orthogonal if real) matrix.

    QR of a Gaussian matrix with the phases of diag(R) moved into Q
    (Mezzadri, Notices AMS 54, 2007).
    """
    if real:
        Z = rng.standard_normal((n, n))
    else:
        Z = (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) / np.sqrt(2.0)
    Qm, R = np.linalg.qr(Z)
    ph = np.diag(R) / np.abs(np.diag(R))
    return Qm * ph[None, :]


def spectrum(kind: str, n: int, rng: np.random.Generator) -> np.ndarray:
    """Planted eigenvalues d of A for the named distribution.

    - "uniform:lo:hi"  d ~ U[lo, hi]
    - "groups8"        8 bands of n/8 values, band j ~ U[c_j, c_j + 4.375] with
                       c_j = 1 + 4.875 j: a spectrum clustered in 8 groups on
                       [1, 39.5], separated by gaps of 0.5
    - "gapband"        d ~ U[1, 50] with 5 % of the values replaced by U[1, 1.49]
                       (a dense band at the bottom of the positive spectrum)
    """
    if kind.startswith("uniform:"):
        _, lo, hi = kind.split(":")
        return rng.uniform(float(lo), float(hi), size=n)
    if kind == "groups8":
        d = np.empty(n)
        bounds = np.linspace(0, n, 9).astype(int)
        for j in range(8):
            c = 1.0 + 4.875 * j
            d[bounds[j]:bounds[j + 1]] = rng.uniform(c, c + 4.375, size=bounds[j + 1] - bounds[j])
        return d
    if kind == "gapband":
        d = rng.uniform(1.0, 50.0, size=n)
        m = int(round(0.05 * n))
        idx = rng.choice(n, size=m, replace=False)
        d[idx] = rng.uniform(1.0, 1.49, size=m)
        return d
    raise ValueError(f"unknown spectrum kind {kind!r}")


def _spectral_norm(B: np.ndarray, rng: np.random.Generator) -> float:
    n = B.shape[0]
    if n <= 2048:
        return float(np.linalg.norm(B, 2))
    # Block power iteration on B^H B (16 vectors, 60 sweeps): converges to well
    # below 1e-6 relative for these random symmetric B; the exact value only sets
    # the coupling strength beta.
    V = rng.standard_normal((n, 16)) + 1j * rng.standard_normal((n, 16))
    for _ in range(60):
        V, _ = np.linalg.qr(B.conj().T @ (B @ V))
    s = np.linalg.svd(B @ V, compute_uv=False)
    return float(s[0])


def make_problem(n: int, seed: int = 0, spec: str = "uniform:1:10", beta: float = 0.3,
                 real: bool = False, b_zero: bool = False) -> BSEProblem:
    """Draw A = Q diag(d) Q^*, B = G + G^T with ||B||_2 = beta * min(d).

    ``real`` gives a real orthogonal Q and a real G (A, B real symmetric);
    ``b_zero`` sets B = 0 (then the spectrum of H is exactly +-d).
    """
    rng = np.random.default_rng(seed)
    d = spectrum(spec, n, rng)
    Qm = haar_unitary(n, rng, real=real)
    A = (Qm * d[None, :]) @ Qm.conj().T
    A = 0.5 * (A + A.conj().T)
    if b_zero:
        B = np.zeros((n, n), dtype=np.complex128)
    else:
        if real:
            G = rng.standard_normal((n, n)) + 0j
        else:
            G = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
        B = G + G.T
        B *= beta * d.min() / _spectral_norm(B, rng)
    return BSEProblem(A=np.ascontiguousarray(A, dtype=np.complex128),
                      B=np.ascontiguousarray(B, dtype=np.complex128),
                      d=d, beta=beta, seed=seed, real=real)


def make_problem_device(n: int, seed: int = 0, spec: str = "uniform:1:10", beta: float = 0.3, device="cuda"):
    """The generator of ``make_problem`` for large n, assembled on a GPU with torch:
    returns (A, B, d) with A, B (n, n) complex128 torch tensors on ``device`` (row-major
    storage as above) and d the planted spectrum (numpy).

    Same recipe, cheaper arithmetic: the complex Gaussian Z and G are drawn with torch's
    CPU generator seeded by ``seed`` (the planted d with numpy's, as above); Q is the
    Haar-unitary factor of Z (QR with the phases of diag(R) moved into Q) and
    A = Q diag(d) Q^* are computed in complex64 on the device, then A is taken to
    complex128 and symmetrised, (A + A^*)/2.  So A is hermitian to the last bit and
    equals Q diag(d) Q^* to FP32 accuracy (its eigenvalues are d up to ~1e-6 ||A||),
    which is all the solver's checks at these sizes use: they test residuals, the
    S-Rayleigh quotient and inertia counts of A and B as given, never d itself.
    B = G + G^T (complex128) scaled to ||B||_2 = beta * min(d) with ||B||_2 from 30
    steps of block power iteration on B^* B (8 vectors).  Used for n >= 8192, where the
    host QR of ``make_problem`` takes minutes."""
    import torch
    rng = np.random.default_rng(seed)
    d = spectrum(spec, n, rng)
    gen = torch.Generator(device="cpu").manual_seed(int(seed) * 7919 + 17)
    Z = torch.complex(torch.randn((n, n), generator=gen, dtype=torch.float32),
                      torch.randn((n, n), generator=gen, dtype=torch.float32)).to(device)
    with torch.no_grad():
        prev_tf32 = torch.backends.cuda.matmul.allow_tf32
        torch.backends.cuda.matmul.allow_tf32 = False
        try:
            Qm, R = torch.linalg.qr(Z)
            del Z
            dr = torch.diagonal(R)
            Qm = Qm * (dr / dr.abs())[None, :]
            del R
            dt = torch.from_numpy(d.astype(np.float32)).to(device)
            A32 = (Qm * dt[None, :].to(Qm.dtype)) @ Qm.conj().T
            del Qm
        finally:
            torch.backends.cuda.matmul.allow_tf32 = prev_tf32
        A = A32.to(torch.complex128)
        del A32
        A = 0.5 * (A + A.conj().T)
        G = torch.complex(torch.randn((n, n), generator=gen, dtype=torch.float64),
                          torch.randn((n, n), generator=gen, dtype=torch.float64)).to(device)
        B = G + G.T
        del G
        V = torch.complex(torch.randn((n, 8), generator=gen, dtype=torch.float64),
                          torch.randn((n, 8), generator=gen, dtype=torch.float64)).to(device)
        for _ in range(30):
            V, _ = torch.linalg.qr(B.conj().T @ (B @ V))
        s = torch.linalg.svdvals(B @ V)[0].item()
        B *= beta * float(d.min()) / s
    return A.contiguous(), B.contiguous(), d


def start_block(n: int, k: int, seed: int) -> np.ndarray:
    """Raw complex Gaussian start block, shape (k, 2n): re, im ~ N(0, 1).

    This is the ``randn`` draw of the initial search space; the method itself
    scales its lower half by gamma.
    """
    rng = np.random.default_rng(seed + 1_000_003)
    return rng.standard_normal((k, 2 * n)) + 1j * rng.standard_normal((k, 2 * n))


def lanczos_starts(n: int, nvec: int, seed: int) -> np.ndarray:
    """Random start vectors of the Lanczos bound estimate, shape (nvec, 2n)."""
    rng = np.random.default_rng(seed + 2_000_029)
    return rng.standard_normal((nvec, 2 * n)) + 1j * rng.standard_normal((nvec, 2 * n))


def loss_weights(nev: int, seed: int) -> np.ndarray:
    """w ~ N(0, 1) for the scalar loss L = sum_i w_i lambda_i."""
    rng = np.random.default_rng(seed + 3_000_017)
    return rng.standard_normal(nev)


# Workloads with the sizes and spectra of the paper-scale experiments (the
# paper's Yambo matrices are not available; these synthetic problems stand in).
WORKLOADS = {
    "n512": dict(n=512, spec="uniform:1:10", beta=0.3, nev=20, nex=10, deg=20,
                 deg_min=20, deg_max=20, tol=1e-10),
    "n4096": dict(n=4096, spec="groups8", beta=0.3, nev=200, nex=60, deg=20,
                  deg_min=20, deg_max=36, tol=1e-10),
    "n16384": dict(n=16384, spec="gapband", beta=0.3, nev=1000, nex=300, deg=20,
                   deg_min=8, deg_max=36, tol=1e-10),
    "n8192grad": dict(n=8192, spec="uniform:1:10", beta=0.3, nev=100, nex=40, deg=20,
                      deg_min=20, deg_max=20, tol=1e-10),
    "n32768": dict(n=32768, spec="uniform:0.5:60", beta=0.4, nev=2000, nex=500, deg=20,
                   deg_min=8, deg_max=40, tol=1e-10),
}
