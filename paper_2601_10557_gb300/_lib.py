"""ctypes binding of libchase_bse.so (argument marshalling only).

Every numerical step runs inside the CUDA library; this module checks tensor
layouts, passes raw device pointers and the current CUDA stream, and turns
status codes into exceptions.  Tensors follow the library's storage
convention: A, B are (n, n) complex128 row-major; a block of k 2n-vectors is a
(k, 2n) complex128 tensor (the column-major 2n x k block of the C ABI).
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libchase_bse.so")

FP64 = 0
MIXED_BF16X3 = 1
MIXED_BF16X6 = 2
MIXED_FP16X3 = 3
# "mixed" is the default tensor-core scheme (FP16 pieces, FP32-class products)
FP64_TC = 4
_PREC = {"fp64": FP64, "mixed": MIXED_FP16X3, "fp16x3": MIXED_FP16X3, "bf16x3": MIXED_BF16X3,
         "bf16x6": MIXED_BF16X6, "fp64_tc": FP64_TC}


class ChaseBSEError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: status {status} ({strerror(status)})")


class Opts(ctypes.Structure):
    _fields_ = [
        ("size", ctypes.c_uint32),
        ("precision", ctypes.c_int32),
        ("maxiter", ctypes.c_int32),
        ("deg_min", ctypes.c_int32),
        ("deg_max", ctypes.c_int32),
        ("lanczos_steps", ctypes.c_int32),
        ("lanczos_vecs", ctypes.c_int32),
        ("fp64_products", ctypes.c_int32),
        ("gamma", ctypes.c_double),
        ("switch_tol", ctypes.c_double),
        ("seed", ctypes.c_uint64),
        ("W0", ctypes.c_void_p),
        ("V0", ctypes.c_void_p),
        ("stream", ctypes.c_void_p),
        ("rr", ctypes.c_int32),
        ("h2", ctypes.c_int32),
    ]


class Stats(ctypes.Structure):
    _fields_ = [
        ("size", ctypes.c_uint32),
        ("iterations", ctypes.c_int32),
        ("converged", ctypes.c_int32),
        ("householder", ctypes.c_int32),
        ("mu1", ctypes.c_double),
        ("mu_nevex", ctypes.c_double),
        ("muN", ctypes.c_double),
        ("rho_hat", ctypes.c_double),
        ("ms_total", ctypes.c_double),
        ("ms_lanczos", ctypes.c_double),
        ("ms_filter", ctypes.c_double),
        ("ms_qr", ctypes.c_double),
        ("ms_rr", ctypes.c_double),
        ("ms_resid", ctypes.c_double),
        ("filter_flops", ctypes.c_double),
        ("filter_flops_fp64", ctypes.c_double),
        ("ms_filter_fp64", ctypes.c_double),
        ("ms_filter_mixed", ctypes.c_double),
        ("filter_launches", ctypes.c_int64),
        ("max_residual", ctypes.c_double),
        ("lanczos_mu1", ctypes.c_double),
        ("lanczos_mu_nevex", ctypes.c_double),
        ("lanczos_muN", ctypes.c_double),
        ("fallback_rr", ctypes.c_int32),
        ("ms_h2", ctypes.c_double),
    ]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_ if name != "size"}


_lib: Optional[ctypes.CDLL] = None

EXPORTS = ["chase_bse_solve", "chase_bse_filter", "chase_bse_rr", "chase_bse_residuals", "chase_bse_grad",
           "chase_bse_strerror", "chase_bse_version", "chase_bse_has_mixed", "chase_bse_launch_count",
           "chase_bse_residuals_noalloc", "chase_bse_dgemm_sliced", "chase_bse_trim_memory",
           "chase_bse_alloc_count", "chase_bse_degrees", "chase_bse_eigh", "chase_bse_filter_cols",
           "chase_bse_set_wait_limit", "chase_bse_gemm_timer", "chase_bse_gemm_time", "chase_bse_rr_fallback",
           "chase_bse_eig_general", "chase_bse_h2_blocks", "chase_bse_filter_h2"]

# 2n * k limit of chase_bse_residuals_noalloc (its fixed device scratch, complex128 entries)
NOALLOC_MAX_ENTRIES = 1 << 19


def lib() -> ctypes.CDLL:
    """Load the CUDA library; fails loudly when it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                           "`python -c 'import __graft_entry__ as g; g.build()'`")
    L = ctypes.CDLL(LIB_PATH)
    vp, i64, i32, dbl = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_double
    L.chase_bse_solve.argtypes = [vp, vp, i64, i64, i64, i32, dbl, ctypes.POINTER(Opts), vp, vp,
                                  ctypes.POINTER(Stats)]
    L.chase_bse_filter.argtypes = [vp, vp, i64, vp, i64, ctypes.POINTER(ctypes.c_int32), dbl, dbl, dbl, i32, vp]
    L.chase_bse_rr.argtypes = [vp, vp, i64, vp, i64, ctypes.POINTER(ctypes.c_double), vp, vp]
    L.chase_bse_residuals.argtypes = [vp, vp, i64, vp, vp, i64, vp, vp]
    L.chase_bse_residuals_noalloc.argtypes = [vp, vp, i64, vp, vp, i64, vp, vp]
    L.chase_bse_grad.argtypes = [vp, vp, i64, i64, vp, vp, vp]
    L.chase_bse_dgemm_sliced.argtypes = [vp, i64, vp, i64, i64, i64, i64, dbl, vp, i64, vp]
    L.chase_bse_degrees.argtypes = [vp, vp, vp, vp, i64, dbl, dbl, dbl, i32, i32, vp]
    L.chase_bse_eigh.argtypes = [vp, i64, vp, vp, i32, dbl, vp]
    L.chase_bse_filter_cols.argtypes = [vp, vp, i64, vp, i64, ctypes.POINTER(ctypes.c_int32),
                                        ctypes.POINTER(ctypes.c_int32), dbl, dbl, dbl, vp]
    L.chase_bse_rr_fallback.argtypes = [vp, vp, i64, vp, i64, ctypes.POINTER(ctypes.c_double), vp,
                                        ctypes.POINTER(ctypes.c_int64), vp]
    L.chase_bse_eig_general.argtypes = [vp, i64, vp, vp, vp]
    L.chase_bse_h2_blocks.argtypes = [vp, vp, i64, vp, vp, vp]
    L.chase_bse_filter_h2.argtypes = [vp, vp, i64, vp, i64, ctypes.POINTER(ctypes.c_int32), dbl, dbl, dbl, i32, vp]
    L.chase_bse_set_wait_limit.argtypes = [ctypes.c_uint64]
    L.chase_bse_set_wait_limit.restype = None
    L.chase_bse_gemm_timer.argtypes = [ctypes.c_int32]
    L.chase_bse_gemm_timer.restype = None
    L.chase_bse_gemm_time.argtypes = [ctypes.c_int32, ctypes.POINTER(ctypes.c_double),
                                      ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64)]
    L.chase_bse_gemm_time.restype = ctypes.c_int
    L.chase_bse_strerror.argtypes = [ctypes.c_int]
    L.chase_bse_strerror.restype = ctypes.c_char_p
    L.chase_bse_launch_count.restype = ctypes.c_int64
    L.chase_bse_alloc_count.restype = ctypes.c_int64
    L.chase_bse_trim_memory.restype = None
    for name in ["chase_bse_solve", "chase_bse_filter", "chase_bse_rr", "chase_bse_residuals", "chase_bse_grad",
                 "chase_bse_version", "chase_bse_has_mixed", "chase_bse_residuals_noalloc",
                 "chase_bse_dgemm_sliced", "chase_bse_degrees", "chase_bse_eigh", "chase_bse_filter_cols",
                 "chase_bse_rr_fallback", "chase_bse_eig_general", "chase_bse_h2_blocks", "chase_bse_filter_h2"]:
        getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


def launch_count() -> int:
    """Kernels launched by the library so far (diagnostics)."""
    return int(lib().chase_bse_launch_count())


def alloc_count() -> int:
    """Device allocations requested by the library so far (diagnostics)."""
    return int(lib().chase_bse_alloc_count())


def trim_memory() -> None:
    """Return the device memory the library keeps cached between calls to the driver."""
    lib().chase_bse_trim_memory()


def has_mixed() -> bool:
    return bool(lib().chase_bse_has_mixed())


def strerror(status: int) -> str:
    return lib().chase_bse_strerror(int(status)).decode()


def _check(status: int, where: str, ok=(0,)):
    if status not in ok:
        raise ChaseBSEError(status, where)
    return status


def _stream(stream) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


def _mat(X: torch.Tensor, name: str, n: Optional[int] = None) -> torch.Tensor:
    if not (isinstance(X, torch.Tensor) and X.is_cuda and X.dtype == torch.complex128 and X.dim() == 2):
        raise ValueError(f"{name} must be a CUDA complex128 matrix")
    if not X.is_contiguous():
        raise ValueError(f"{name} must be contiguous (row-major)")
    if n is not None and X.shape != (n, n):
        raise ValueError(f"{name} must be {n} x {n}")
    return X


def _block(W: torch.Tensor, name: str, n2: int) -> torch.Tensor:
    if not (isinstance(W, torch.Tensor) and W.is_cuda and W.dtype == torch.complex128 and W.dim() == 2):
        raise ValueError(f"{name} must be a CUDA complex128 tensor of shape (k, 2n)")
    if W.shape[1] != n2 or not W.is_contiguous():
        raise ValueError(f"{name} must be contiguous with shape (k, {n2})")
    return W


def _ptr(t: Optional[torch.Tensor]):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def solve(A: torch.Tensor, B: torch.Tensor, nev: int, nex: int, deg: int = 20, tol: float = 1e-10, *,
          precision: str = "fp64", W0: Optional[torch.Tensor] = None, V0: Optional[torch.Tensor] = None,
          maxiter: int = 25, deg_min: Optional[int] = None, deg_max: Optional[int] = None,
          lanczos_steps: int = 26, lanczos_vecs: int = 4, gamma: float = 1e-3, switch_tol: float = 1e-8,
          seed: int = 0, stream=None, allow_partial: bool = False, fp64_products: str = "tensor",
          rr: str = "oblique", h2: str = "implicit"):
    """chase_bse_solve: returns (evals (nev,) float64, evecs (nev, 2n) complex128, stats dict).

    precision: "fp64" (FP64 pipe), "fp64_tc" (FP64-accurate throughout, every large
    product a sliced tensor-core GEMM), "mixed" (= "fp16x3"), "bf16x6", "bf16x3".
    fp64_products ("tensor" or "fp64"): in mixed precision, where the FP64-accurate
    products of QR and Rayleigh-Ritz run (sliced tensor-core GEMM or FP64 pipe).
    rr: "oblique" (Algorithm 2, the non-hermitian fallback only where Q^* S H Q is not
    positive definite) or "fallback" (the non-hermitian fallback in every iteration).
    h2: "implicit" (H applied twice per filter step, the paper's method) or "explicit"
    (mixed precision only: the blocks of H^2 formed once, one product per step)."""
    if h2 not in ("implicit", "explicit"):
        raise ValueError("h2 must be 'implicit' or 'explicit'")
    if fp64_products not in ("tensor", "fp64"):
        raise ValueError("fp64_products must be 'tensor' or 'fp64'")
    if rr not in ("oblique", "fallback"):
        raise ValueError("rr must be 'oblique' or 'fallback'")
    A = _mat(A, "A")
    n = A.shape[0]
    B = _mat(B, "B", n)
    nevex = nev + nex
    if W0 is not None:
        W0 = _block(W0, "W0", 2 * n)
        if W0.shape[0] != nevex:
            raise ValueError("W0 must have nev + nex rows")
    if V0 is not None:
        V0 = _block(V0, "V0", 2 * n)
        lanczos_vecs = V0.shape[0]
    o = Opts(size=ctypes.sizeof(Opts), precision=_PREC[precision], maxiter=maxiter,
             deg_min=deg if deg_min is None else deg_min, deg_max=deg if deg_max is None else deg_max,
             lanczos_steps=lanczos_steps, lanczos_vecs=lanczos_vecs, gamma=gamma, switch_tol=switch_tol,
             seed=seed, W0=_ptr(W0), V0=_ptr(V0), stream=ctypes.c_void_p(_stream(stream)),
             fp64_products=0 if fp64_products == "tensor" else 1, rr=0 if rr == "oblique" else 1,
             h2=0 if h2 == "implicit" else 1)
    evals = torch.zeros(nev, dtype=torch.float64, device=A.device)
    evecs = torch.zeros((nev, 2 * n), dtype=torch.complex128, device=A.device)
    st = Stats(size=ctypes.sizeof(Stats))
    status = lib().chase_bse_solve(_ptr(A), _ptr(B), n, nev, nex, deg, tol, ctypes.byref(o), _ptr(evals),
                                   _ptr(evecs), ctypes.byref(st))
    _check(status, "chase_bse_solve", ok=(0, 1) if allow_partial else (0,))
    d = st.as_dict()
    d["status"] = status
    return evals, evecs, d


def filter(A: torch.Tensor, B: torch.Tensor, W: torch.Tensor, degs, mu1: float, mu_nevex: float, muN: float,
           precision: str = "fp64", stream=None) -> torch.Tensor:
    """chase_bse_filter, in place on W (k, 2n); returns W."""
    A = _mat(A, "A")
    n = A.shape[0]
    B = _mat(B, "B", n)
    W = _block(W, "W", 2 * n)
    k = W.shape[0]
    d = (ctypes.c_int32 * max(k, 1))(*[int(x) for x in degs])
    if len(degs) != k:
        raise ValueError("one degree per vector")
    _check(lib().chase_bse_filter(_ptr(A), _ptr(B), n, _ptr(W), k, d, mu1, mu_nevex, muN, _PREC[precision],
                                  ctypes.c_void_p(_stream(stream))), "chase_bse_filter")
    return W


def filter_cols(A: torch.Tensor, B: torch.Tensor, W: torch.Tensor, degs, precs, mu1: float, mu_nevex: float,
                muN: float, stream=None) -> torch.Tensor:
    """chase_bse_filter_cols: the filter with a precision per column ("fp64" or "fp64_tc",
    not both, or one tensor-core scheme name), in place on W (k, 2n); returns W."""
    A = _mat(A, "A")
    n = A.shape[0]
    B = _mat(B, "B", n)
    W = _block(W, "W", 2 * n)
    k = W.shape[0]
    if len(degs) != k or len(precs) != k:
        raise ValueError("one degree and one precision per vector")
    d = (ctypes.c_int32 * max(k, 1))(*[int(x) for x in degs])
    p = (ctypes.c_int32 * max(k, 1))(*[_PREC[x] for x in precs])
    _check(lib().chase_bse_filter_cols(_ptr(A), _ptr(B), n, _ptr(W), k, d, p, mu1, mu_nevex, muN,
                                       ctypes.c_void_p(_stream(stream))), "chase_bse_filter_cols")
    return W


def rayleigh_ritz_fallback(A: torch.Tensor, B: torch.Tensor, Q: torch.Tensor, stream=None):
    """chase_bse_rr_fallback: the non-hermitian fallback Rayleigh-Ritz on Q (k, 2n) with
    orthonormal rows-as-vectors; returns (ritz numpy (m,), W (m, 2n)) for the m Ritz pairs
    with positive real part, ascending."""
    import numpy as np
    A = _mat(A, "A")
    n = A.shape[0]
    B = _mat(B, "B", n)
    Q = _block(Q, "Q", 2 * n)
    k = Q.shape[0]
    ritz = (ctypes.c_double * k)()
    W = torch.zeros((k, 2 * n), dtype=torch.complex128, device=A.device)
    npos = ctypes.c_int64(0)
    _check(lib().chase_bse_rr_fallback(_ptr(A), _ptr(B), n, _ptr(Q), k, ritz, _ptr(W), ctypes.byref(npos),
                                       ctypes.c_void_p(_stream(stream))), "chase_bse_rr_fallback")
    m = int(npos.value)
    return np.array(ritz[:m]), W[:m]


def eig_general(G: torch.Tensor, stream=None):
    """chase_bse_eig_general: eigenpairs of a general complex matrix.  G is a (k, k)
    complex128 device tensor holding the matrix in row-major order (G[i, j] = g_ij);
    returns (lam (k,) complex128, V (k, k)) with G V = V diag(lam), unit columns of V
    (V[:, j] is the j-th eigenvector)."""
    if G.dtype != torch.complex128 or G.dim() != 2 or G.shape[0] != G.shape[1] or not G.is_cuda:
        raise ValueError("G must be a square complex128 CUDA tensor")
    k = G.shape[0]
    Gc = G.t().contiguous()  # column-major storage of G
    lam = torch.zeros(k, dtype=torch.complex128, device=G.device)
    Vc = torch.zeros((k, k), dtype=torch.complex128, device=G.device)  # column-major V
    _check(lib().chase_bse_eig_general(_ptr(Gc), k, _ptr(lam), _ptr(Vc), ctypes.c_void_p(_stream(stream))),
           "chase_bse_eig_general")
    return lam, Vc.t()


def h2_blocks(A: torch.Tensor, B: torch.Tensor, stream=None):
    """chase_bse_h2_blocks: (P, Q) with H^2 = [[P, Q], [conj Q, conj P]], (n, n) complex128
    row-major like A and B (FP64-accurate)."""
    A = _mat(A, "A")
    n = A.shape[0]
    B = _mat(B, "B", n)
    P = torch.empty((n, n), dtype=torch.complex128, device=A.device)
    Q = torch.empty((n, n), dtype=torch.complex128, device=A.device)
    _check(lib().chase_bse_h2_blocks(_ptr(A), _ptr(B), n, _ptr(P), _ptr(Q), ctypes.c_void_p(_stream(stream))),
           "chase_bse_h2_blocks")
    return P, Q


def filter_h2(A: torch.Tensor, B: torch.Tensor, W: torch.Tensor, degs, mu1: float, mu_nevex: float, muN: float,
              precision: str = "mixed", stream=None) -> torch.Tensor:
    """chase_bse_filter_h2: the tensor-core filter with H^2 applied from its blocks (the
    explicit-H^2 variant), in place on W (k, 2n); returns W."""
    A = _mat(A, "A")
    n = A.shape[0]
    B = _mat(B, "B", n)
    W = _block(W, "W", 2 * n)
    k = W.shape[0]
    d = (ctypes.c_int32 * max(k, 1))(*[int(x) for x in degs])
    _check(lib().chase_bse_filter_h2(_ptr(A), _ptr(B), n, _ptr(W), k, d, mu1, mu_nevex, muN, _PREC[precision],
                                     ctypes.c_void_p(_stream(stream))), "chase_bse_filter_h2")
    return W


def set_wait_limit(ns: int) -> None:
    """Bound (ns) of the cooperative kernels' grid-barrier waits; 0 = the default 2 s."""
    lib().chase_bse_set_wait_limit(int(ns))


def gemm_timer(enable: bool) -> None:
    """chase_bse_gemm_timer: start (True) or stop (False) the event record of the
    filter's H applications; both clear it."""
    lib().chase_bse_gemm_timer(1 if enable else 0)


def gemm_time(kind: str = "tensor"):
    """chase_bse_gemm_time: (total device ms, total algorithmic flops, launches) of the
    recorded H applications of ``kind`` ("tensor": the tensor-core filter GEMM, "fp64":
    the FP64 H application, "sliced": the FP64-accurate sliced H application) since the
    record was started or last read; clears that kind's record."""
    ms = ctypes.c_double(0.0)
    fl = ctypes.c_double(0.0)
    cnt = ctypes.c_int64(0)
    _check(lib().chase_bse_gemm_time({"tensor": 0, "fp64": 1, "sliced": 2}[kind], ctypes.byref(ms), ctypes.byref(fl),
                                     ctypes.byref(cnt)), "chase_bse_gemm_time")
    return float(ms.value), float(fl.value), int(cnt.value)


def rayleigh_ritz(A: torch.Tensor, B: torch.Tensor, Q: torch.Tensor, stream=None):
    """chase_bse_rr: returns (ritz numpy (k/2,), Wpos (k/2, 2n))."""
    import numpy as np
    A = _mat(A, "A")
    n = A.shape[0]
    B = _mat(B, "B", n)
    Q = _block(Q, "Q", 2 * n)
    k = Q.shape[0]
    ritz = (ctypes.c_double * (k // 2))()
    Wpos = torch.zeros((k // 2, 2 * n), dtype=torch.complex128, device=A.device)
    _check(lib().chase_bse_rr(_ptr(A), _ptr(B), n, _ptr(Q), k, ritz, _ptr(Wpos), ctypes.c_void_p(_stream(stream))),
           "chase_bse_rr")
    return np.array(ritz[:]), Wpos


def residuals(A: torch.Tensor, B: torch.Tensor, W: torch.Tensor, lam: torch.Tensor, stream=None) -> torch.Tensor:
    A = _mat(A, "A")
    n = A.shape[0]
    B = _mat(B, "B", n)
    W = _block(W, "W", 2 * n)
    lam = lam.to(device=A.device, dtype=torch.float64).contiguous()
    res = torch.zeros(W.shape[0], dtype=torch.float64, device=A.device)
    _check(lib().chase_bse_residuals(_ptr(A), _ptr(B), n, _ptr(W), _ptr(lam), W.shape[0], _ptr(res),
                                     ctypes.c_void_p(_stream(stream))), "chase_bse_residuals")
    return res


def residuals_noalloc(A: torch.Tensor, B: torch.Tensor, W: torch.Tensor, lam: torch.Tensor, out: torch.Tensor,
                      stream=None) -> torch.Tensor:
    """chase_bse_residuals_noalloc: residual norms into the caller's `out`
    (float64, k entries) without any device allocation by the library; the
    scratch is a fixed per-device array of NOALLOC_MAX_ENTRIES complex128
    entries shared by all calls (see include/chase_bse.h)."""
    A = _mat(A, "A")
    n = A.shape[0]
    B = _mat(B, "B", n)
    W = _block(W, "W", 2 * n)
    k = W.shape[0]
    if 2 * n * k > NOALLOC_MAX_ENTRIES:
        raise ValueError(f"2n*k = {2 * n * k} exceeds the fixed scratch of {NOALLOC_MAX_ENTRIES} entries")
    if not (lam.is_cuda and lam.dtype == torch.float64 and lam.is_contiguous() and lam.numel() == k):
        raise ValueError("lam must be a contiguous CUDA float64 tensor with one entry per vector")
    if not (out.is_cuda and out.dtype == torch.float64 and out.is_contiguous() and out.numel() == k):
        raise ValueError("out must be a contiguous CUDA float64 tensor with one entry per vector")
    _check(lib().chase_bse_residuals_noalloc(_ptr(A), _ptr(B), n, _ptr(W), _ptr(lam), k, _ptr(out),
                                             ctypes.c_void_p(_stream(stream))), "chase_bse_residuals_noalloc")
    return out


def dgemm_sliced(A: torch.Tensor, B: torch.Tensor, alpha: float = 1.0, stream=None) -> torch.Tensor:
    """chase_bse_dgemm_sliced: alpha * A @ B.T for float64 CUDA matrices A (M, K), B (N, K)."""
    for t, nm in ((A, "A"), (B, "B")):
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.dim() == 2
                and t.is_contiguous()):
            raise ValueError(f"{nm} must be a contiguous CUDA float64 matrix")
    M, K = A.shape
    N = B.shape[0]
    if B.shape[1] != K:
        raise ValueError("A and B must have the same number of columns")
    C = torch.empty((N, M), dtype=torch.float64, device=A.device)  # column-major M x N
    _check(lib().chase_bse_dgemm_sliced(_ptr(A), K, _ptr(B), K, M, N, K, float(alpha), _ptr(C), M,
                                        ctypes.c_void_p(_stream(stream))), "chase_bse_dgemm_sliced")
    return C.T


def degrees(ritz, res, prev_res, prev_deg, tol: float, mu_nevex: float, muN: float, deg_min: int,
            deg_max: int):
    """chase_bse_degrees: the solver's per-vector degree rule (host only); returns a list."""
    import numpy as np
    ritz = np.ascontiguousarray(ritz, dtype=np.float64)
    k = len(ritz)
    res = np.ascontiguousarray(res, dtype=np.float64)
    prev_res = np.ascontiguousarray(prev_res, dtype=np.float64)
    prev_deg = np.ascontiguousarray(prev_deg, dtype=np.int32)
    if not (len(res) == len(prev_res) == len(prev_deg) == k):
        raise ValueError("ritz, res, prev_res and prev_deg must have the same length")
    out = np.zeros(k, dtype=np.int32)
    _check(lib().chase_bse_degrees(ritz.ctypes.data, res.ctypes.data, prev_res.ctypes.data, prev_deg.ctypes.data,
                                   k, tol, mu_nevex, muN, deg_min, deg_max, out.ctypes.data), "chase_bse_degrees")
    return out.tolist()


EIGH_METHODS = {"jacobi": 0, "mixed": 1, "block": 2}


def eigh(G: torch.Tensor, method: str = "mixed", thr: float = 2e-16, stream=None):
    """chase_bse_eigh: (theta (k,), V (k, k)) with G V = V diag(theta) for a hermitian CUDA
    complex128 matrix G (k even); the columns of V (k, k) are the eigenvectors."""
    if not (isinstance(G, torch.Tensor) and G.is_cuda and G.dtype == torch.complex128 and G.dim() == 2
            and G.shape[0] == G.shape[1]):
        raise ValueError("G must be a square CUDA complex128 matrix")
    k = G.shape[0]
    Gc = G.transpose(0, 1).contiguous()  # column-major storage of G
    theta = torch.empty(k, dtype=torch.float64, device=G.device)
    Vt = torch.empty((k, k), dtype=torch.complex128, device=G.device)  # column-major V
    _check(lib().chase_bse_eigh(_ptr(Gc), k, _ptr(theta), _ptr(Vt), EIGH_METHODS[method], thr,
                                ctypes.c_void_p(_stream(stream))), "chase_bse_eigh")
    return theta, Vt.transpose(0, 1)


def grad(V: torch.Tensor, w: torch.Tensor, stream=None):
    """chase_bse_grad: (gA, gB), each (n, n) complex128 row-major."""
    n2 = V.shape[1]
    V = _block(V, "V", n2)
    n = n2 // 2
    w = w.to(device=V.device, dtype=torch.float64).contiguous()
    gA = torch.empty((n, n), dtype=torch.complex128, device=V.device)
    gB = torch.empty((n, n), dtype=torch.complex128, device=V.device)
    _check(lib().chase_bse_grad(_ptr(V), _ptr(w), n, V.shape[0], _ptr(gA), _ptr(gB),
                                ctypes.c_void_p(_stream(stream))), "chase_bse_grad")
    return gA, gB


class BSEEigvals(torch.autograd.Function):
    """lambda_1..lambda_nev of H(A, B) with a hand-written backward.

    backward(g) calls chase_bse_grad with w = g, which folds
    d lambda_i = (S v_i)^* dH v_i / (v_i^* S v_i) into hermitian dL/dA and
    symmetric dL/dB (PyTorch's convention dL = Re sum conj(G) dZ).
    """

    @staticmethod
    def forward(ctx, A, B, nev, nex, deg, tol, kwargs):
        evals, evecs, stats = solve(A.detach(), B.detach(), nev, nex, deg, tol, **(kwargs or {}))
        ctx.save_for_backward(evecs)
        ctx.stats = stats
        return evals

    @staticmethod
    def backward(ctx, g):
        (evecs,) = ctx.saved_tensors
        gA, gB = grad(evecs, g.contiguous())
        return gA, gB, None, None, None, None, None


def eigvals(A, B, nev, nex, deg=20, tol=1e-10, **kwargs):
    """Differentiable wrapper around chase_bse_solve (eigenvalues only)."""
    return BSEEigvals.apply(A, B, nev, nex, deg, tol, kwargs)
