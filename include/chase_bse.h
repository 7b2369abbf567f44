/*
 * chase_bse.h -- C ABI of a GB300 (sm_103a) implementation of ChASE for
 * pseudo-hermitian Bethe-Salpeter Hamiltonians (arXiv 2601.10557).
 *
 * Problem (Section 1, eq. introduction::hamiltonian_definition):
 *     H = [[A, B], [-conj(B), -conj(A)]],  A = A^* (n x n),  B = B^T (n x n),
 * with S H = [[A, B], [conj(B), conj(A)]] hermitian positive definite
 * (eq. introduction::quasi_hermitian_condition).  The library computes the nev
 * smallest positive eigenvalues of H and their right eigenvectors with the
 * Chebyshev-filtered subspace iteration of Algorithm 3.  H is never formed:
 * every product with H reads only the stored A and B.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Complex numbers are complex128: two interleaved doubles (re, im).
 * - A and B are n x n, stored ROW-MAJOR (element (i, j) at offset i*n + j).
 *   Because A is hermitian and B symmetric this is also the column-major
 *   storage of conj(A) and of B.  Only A's hermitian part and B's symmetric
 *   part are assumed; the library does not symmetrise.
 * - Blocks of 2n-vectors (W, Q, V, ...) are 2n x k COLUMN-MAJOR with leading
 *   dimension 2n: vector j occupies the 2n consecutive complex numbers starting
 *   at offset j*2n (a torch tensor of shape (k, 2n)).
 * - Pointers marked "device" must be CUDA device (or managed) memory on the
 *   current device; the caller owns every buffer passed in.  Workspace is
 *   allocated by the library with stream-ordered allocation on `stream` and
 *   released before the call returns.
 * - `stream` is a cudaStream_t (NULL = legacy default stream).  Entry points
 *   that return results to host memory synchronise that stream.
 * - Status codes: 0 OK; 1 NOT_CONVERGED (partial results are written); negative
 *   values are errors (see chase_bse_status).  No C++ exception crosses the ABI.
 *   chase_bse_strerror() turns a status into a static string.
 */
#ifndef CHASE_BSE_H
#define CHASE_BSE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum chase_bse_status {
  CHASE_BSE_OK = 0,
  CHASE_BSE_NOT_CONVERGED = 1,   /* maxiter reached; stats->converged pairs valid      */
  CHASE_BSE_BAD_ARG = -1,        /* invalid size, NULL pointer, bad option            */
  CHASE_BSE_CUDA_ERROR = -2,     /* a CUDA runtime call or kernel launch failed       */
  CHASE_BSE_OOM = -3,            /* workspace allocation failed                       */
  CHASE_BSE_NOT_DEFINITE = -4,   /* Cholesky of Q^* S H Q failed: S H not HPD (in a
                                    solve: and the non-hermitian fallback found fewer
                                    Ritz values with positive real part than needed) */
  CHASE_BSE_QR_FAILED = -5,      /* search space rank-deficient even for Householder  */
  CHASE_BSE_DEVICE_TIMEOUT = -6, /* a bounded device-side wait gave up                */
  CHASE_BSE_UNSUPPORTED = -7,    /* feature needs a device this build cannot run on   */
  CHASE_BSE_NONFINITE = -8       /* an input (A, B, W0, V0) holds a NaN or an Inf      */
} chase_bse_status;

typedef enum chase_bse_precision {
  CHASE_BSE_FP64 = 0,          /* every product in FP64 (DFMA)                         */
  CHASE_BSE_MIXED_BF16X3 = 1,  /* filter products on tcgen05 tensor cores from BF16
                                  pieces, x = x0 + x1, 3 products, FP32 accumulation
                                  (about 16-bit accurate); everything else FP64      */
  CHASE_BSE_MIXED_BF16X6 = 2,  /* as above with 3 pieces and 6 products (FP32 class) */
  CHASE_BSE_MIXED_FP16X3 = 3,  /* filter products from FP16 pieces x = x0 + x1 (11 +
                                  11 bits, every operand row scaled by a power of two
                                  into FP16's range), 3 products, FP32 accumulation:
                                  FP32-class accuracy at the cost of BF16X3; the
                                  default mixed precision                            */
  CHASE_BSE_FP64_TC = 4        /* FP64-accurate throughout, with every large product
                                  (the filter's H applications, QR, Rayleigh-Ritz,
                                  Lanczos) an FP64-accurate sliced GEMM on the tensor
                                  cores (see chase_bse_dgemm_sliced); needs compute
                                  capability 10.3                                    */
} chase_bse_precision;
/* In chase_bse_solve the mixed filter runs, from the second iteration on, on the
 * correction q(H^2) r2 with r2 = (H^2 - lambda^2) v of each Ritz pair (FP64
 * residual), q the divided difference of the filter polynomial, so that its
 * rounding error scales with the residual; a column whose residual is below
 * switch_tol and stops decreasing is moved to the FP64 filter. */

/* Options of chase_bse_solve.  Zero-initialise, set `size`, then override. */
typedef struct chase_bse_opts {
  uint32_t size;           /* sizeof(chase_bse_opts)                                  */
  int32_t precision;       /* chase_bse_precision (default FP64)                      */
  int32_t maxiter;         /* outer iterations (default 25, Section 6)                */
  int32_t deg_min;         /* per-vector degree clamp (default: deg)                  */
  int32_t deg_max;         /* (default: deg)                                          */
  int32_t lanczos_steps;   /* even number of Lanczos steps (default 26, Section 4.1)  */
  int32_t lanczos_vecs;    /* start vectors of the bound estimate (default 4, <= 64)  */
  int32_t fp64_products;   /* mixed mode: 0 = the FP64 products of QR and Rayleigh-Ritz
                              on the tensor cores, FP64-accurate (see
                              chase_bse_dgemm_sliced; default), 1 = on the FP64 pipe */
  double gamma;            /* lower-half scale of the start block (default 1e-3,
                              Section 4.6)                                            */
  double switch_tol;       /* mixed mode: a column below this residual whose residual
                              stops decreasing moves to the FP64 filter (default 1e-8) */
  uint64_t seed;           /* counter-based generator seed when W0/V0 are NULL        */
  const void* W0;          /* device, 2n x (nev+nex) raw start block, or NULL         */
  const void* V0;          /* device, 2n x lanczos_vecs Lanczos start vectors, or NULL*/
  void* stream;            /* cudaStream_t                                            */
  int32_t rr;              /* Rayleigh-Ritz step: 0 = Algorithm 2, with the non-hermitian
                              fallback (see chase_bse_rr_fallback) in an iteration where
                              Q^* S H Q is not positive definite (default); 1 = the
                              fallback in every iteration                             */
  int32_t h2;              /* mixed precision only: 0 = the filter applies H twice per
                              step (Section 4.2, default); 1 = the explicit-H^2 variant,
                              not the paper's method: the blocks of H^2 are formed once
                              (chase_bse_h2_blocks) and applied with one tensor-core
                              product per step                                        */
} chase_bse_opts;

/* Statistics of chase_bse_solve (host struct, filled when non-NULL). */
typedef struct chase_bse_stats {
  uint32_t size;           /* sizeof(chase_bse_stats), set by the caller              */
  int32_t iterations;
  int32_t converged;       /* eigenpairs written                                      */
  int32_t householder;     /* iterations that fell back to Householder QR            */
  double mu1, mu_nevex, muN, rho_hat;   /* final filter bounds, residual scale       */
  double ms_total, ms_lanczos, ms_filter, ms_qr, ms_rr, ms_resid;
  double filter_flops;     /* algorithmic: sum over H^2 steps of 64 n^2 k_active    */
  double filter_flops_fp64;/* the part run by the FP64 filter                        */
  double ms_filter_fp64;   /* time of the FP64 filter launches                        */
  double ms_filter_mixed;  /* time of the tensor-core filter launches                 */
  int64_t filter_launches; /* GEMM launches of the filter                             */
  double max_residual;     /* largest scaled residual of the returned pairs           */
  double lanczos_mu1, lanczos_mu_nevex, lanczos_muN;  /* the bounds of Section 4.1 as the
                              Lanczos estimate returned them, before any update     */
  int32_t fallback_rr;     /* iterations that ran the non-hermitian fallback RR       */
  double ms_h2;            /* explicit-H^2 variant: time to form the blocks of H^2    */
} chase_bse_stats;

/* Full solve (Algorithm 3).
 *   A, B     device, n x n complex128 row-major (see conventions)
 *   n        block size (H is 2n x 2n), n >= 1
 *   nev      wanted pairs, 1 <= nev; nev + nex <= n
 *   nex      extra search vectors
 *   deg      Chebyshev degree (H^2 steps) of the first iteration, >= 1
 *   tol      residual tolerance on ||H v - lambda v||_2 / rho_hat, ||v|| = 1
 *   opts     NULL for defaults
 *   evals    device, nev doubles: ascending positive eigenvalues
 *   evecs    device, 2n x nev complex128 column-major: unit right eigenvectors,
 *            phase-fixed so the largest-magnitude entry of the upper half is real
 *            and positive
 *   stats    host, may be NULL
 * Returns OK, NOT_CONVERGED (the first stats->converged entries are valid), or
 * an error; NONFINITE (nothing computed) when A, B, opts->W0 or opts->V0 hold a
 * NaN or an Inf.  Synchronises opts->stream. */
int chase_bse_solve(const void* A, const void* B, int64_t n, int64_t nev, int64_t nex,
                    int32_t deg, double tol, const chase_bse_opts* opts, double* evals,
                    void* evecs, chase_bse_stats* stats);

/* The blocks of H^2 = [[P, Q], [conj Q, conj P]] for H = [[A, B], [-conj B, -conj A]]:
 * P = A A - B conj(B), Q = A B - B conj(A), as the top block row
 * [A | -B] [[A, B], [conj B, conj A]] in FP64-accurate sliced tensor-core GEMMs (see
 * chase_bse_dgemm_sliced; 32 n^3 flops).  No counterpart in the paper's method, which
 * applies H twice: the operand of the explicit-H^2 variant.
 *   P, Q   device, n x n complex128 each, row-major like A and B
 * Needs compute capability 10.3 (UNSUPPORTED otherwise).  Synchronises `stream`. */
int chase_bse_h2_blocks(const void* A, const void* B, int64_t n, void* P, void* Q, void* stream);

/* The tensor-core filter of chase_bse_filter in the explicit-H^2 variant (not the paper's
 * method): the blocks of H^2 are formed for the call (chase_bse_h2_blocks) and each step
 * applies H^2 with one product instead of two applications of H.  precision: one of the
 * MIXED schemes; other arguments as chase_bse_filter. */
int chase_bse_filter_h2(const void* A, const void* B, int64_t n, void* W, int64_t k,
                        const int32_t* degs, double mu1, double mu_nevex, double muN,
                        int32_t precision, void* stream);

/* Chebyshev filter on H^2 (Section 4.2, eq. three-term_recurrence_pseudo-hermitian),
 * scaled three-term recurrence with a = mu_nevex^2, b = muN^2, c = (a+b)/2,
 * e = (b-a)/2, sigma_1 = e/(mu1^2 - c):
 *   Y_1 = (sigma_1/e)(H^2 Y_0 - c Y_0),
 *   Y_{j+1} = (2 sigma_{j+1}/e)(H^2 Y_j - c Y_j) - sigma_j sigma_{j+1} Y_{j-1},
 *   sigma_{j+1} = 1/(2/sigma_1 - sigma_j).
 *   W        device, 2n x k complex128, in: Y_0, out: column i = Y_{degs[i]}
 *   degs     host, k ints >= 1 (any order)
 *   precision chase_bse_precision (FP64_TC: the FP64 recurrence with both H
 *            applications of a step as sliced tensor-core GEMMs; the sliced form of
 *            H, 7 * 8 n^2 bytes, is built for the call)
 * 0 < mu1 < mu_nevex < muN.  k = 0 is a no-op.  Asynchronous on `stream` except
 * for workspace bookkeeping; the result is ready when the stream reaches it. */
int chase_bse_filter(const void* A, const void* B, int64_t n, void* W, int64_t k,
                     const int32_t* degs, double mu1, double mu_nevex, double muN,
                     int32_t precision, void* stream);

/* chase_bse_filter with a precision per column (the precision groups of a mixed solve,
 * where a column that nears the tolerance moves to the FP64 filter): precs (host, k
 * entries) are chase_bse_precision codes; the FP64 (or FP64_TC) columns run the FP64
 * filter and the others the tensor-core filter, which takes one scheme per call (all
 * mixed entries equal, and FP64 and FP64_TC not both present, else BAD_ARG).  Same
 * arguments otherwise. */
int chase_bse_filter_cols(const void* A, const void* B, int64_t n, void* W, int64_t k,
                          const int32_t* degs, const int32_t* precs, double mu1,
                          double mu_nevex, double muN, void* stream);

/* Oblique Rayleigh-Ritz with hermitian spectral equivalence (Algorithm 2):
 * T = S H Q, M = Q^* T = L L^*, G = L^{-1}(I - 2 Q_2^* Q_2) L^{-*}, G y = theta y,
 * ritz = 1/theta for the k/2 positive theta, Wpos = Q L^{-*} Y_+ (unit columns).
 *   Q     device, 2n x k complex128 with orthonormal columns, k even
 *   ritz  host, k/2 doubles, ascending
 *   Wpos  device, 2n x k/2 complex128 (may not alias Q)
 * Returns NOT_DEFINITE when Q^* S H Q is not positive definite and QR_FAILED
 * when fewer than k/2 eigenvalues of G are positive (range(Q) is not closed
 * under W -> K conj(W), e.g. after an exactly rank-deficient search space).
 * Synchronises `stream`. */
int chase_bse_rr(const void* A, const void* B, int64_t n, const void* Q, int64_t k,
                 double* ritz, void* Wpos, void* stream);

/* Residual norms ||H w_j - lambda_j w_j||_2 (Section 4.5).
 *   W      device, 2n x k; lambda device, k doubles; res device, k doubles. */
int chase_bse_residuals(const void* A, const void* B, int64_t n, const void* W,
                        const double* lambda, int64_t k, double* res, void* stream);

/* chase_bse_residuals for callers that cannot let a library allocate device
 * memory (the paper has no counterpart): for example an application whose own
 * memory pool owns the whole device, a program with a fixed device-memory
 * budget, or a latency-critical loop in which an allocation or a free may
 * synchronise the device.  Same arguments and results as chase_bse_residuals;
 * the 2n x k scratch block lives in a fixed array of
 * CHASE_BSE_NOALLOC_MAX_ENTRIES complex128 entries (8 MiB) that every device
 * using the library holds until the process exits, and the call performs no
 * allocation or free: its H product runs as one launch over the whole K range,
 * without the split-K partial sums of chase_bse_residuals (slower when 2n * k is
 * small, identical results up to the order of the FP64 sums).
 *   - 2n * k > CHASE_BSE_NOALLOC_MAX_ENTRIES returns BAD_ARG; nothing runs.
 *   - The first call on a device looks up the array's device address (once per
 *     device, with that device current); make that first call before any stream
 *     capture.  The address is kept for the life of the process: after a
 *     cudaDeviceReset of that device, reload the library (a new process).
 *   - All calls share the array, which keeps the last call's contents: calls
 *     whose kernels overlap on the GPU (different streams, or different host
 *     threads, without ordering between them) race on it and give wrong
 *     results.  Order them on one stream or synchronise between them. */
#define CHASE_BSE_NOALLOC_MAX_ENTRIES ((int64_t)1 << 19)
int chase_bse_residuals_noalloc(const void* A, const void* B, int64_t n, const void* W,
                                const double* lambda, int64_t k, double* res, void* stream);

/* Eigenvalue gradient of L = sum_i w_i lambda_i (left eigenvector u = S v,
 * Theorem SH_HPD): with V = [X; Y], s_i = |x_i|^2 - |y_i|^2, c_i = w_i / s_i,
 *   gA = sum_i c_i (x_i x_i^* + conj(y_i) y_i^T)   (hermitian)
 *   gB = sum_i c_i (x_i y_i^* + conj(y_i) x_i^T)   (symmetric)
 * under the convention dL = Re sum conj(G) .* dZ.
 *   V      device, 2n x nev right eigenvectors (any normalisation)
 *   w      device, nev doubles
 *   gA, gB device, n x n complex128, written ROW-MAJOR like A and B.
 * On compute capability 10.3 the two rank-2nev products run as FP64-accurate
 * sliced GEMMs on the tensor cores (see chase_bse_dgemm_sliced), elsewhere on
 * the FP64 pipe. */
int chase_bse_grad(const void* V, const double* w, int64_t n, int64_t nev, void* gA,
                   void* gB, void* stream);

/* Non-hermitian fallback Rayleigh-Ritz (Section 4.4, last paragraph), for a search space
 * where Q^* S Q is singular or Q^* S H Q is not positive definite, so that Algorithm 2's
 * hermitian equivalence does not apply: with M = Q^* S Q, the dual basis
 *   Q_L = (S Q - Q (M - diag M)) diag(M)^{-1}    (Q_L^* Q = I; M itself may be singular),
 * G = Q_L^* H Q (not hermitian), G Z = Z diag(lam) by a complex Schur decomposition
 * (see chase_bse_eig_general); the Ritz pairs are those with Re lam > 0, ascending.
 *   Q      device, 2n x k complex128 with orthonormal columns, 1 <= k <= 2n, k <= 32768
 *   ritz   host, k doubles: Re lam of the returned pairs, ascending
 *   W      device, 2n x k complex128: columns 0 .. *npos - 1 receive Q Z_+ (unit norm)
 *   npos   host: the number of pairs returned
 * Returns QR_FAILED when a diagonal entry of M is zero (relative to the largest) or not
 * real, NOT_CONVERGED when the QR iteration does not converge.  Synchronises `stream`. */
int chase_bse_rr_fallback(const void* A, const void* B, int64_t n, const void* Q, int64_t k,
                          double* ritz, void* W, int64_t* npos, void* stream);

/* Dense eigensolver for a general complex matrix (the eigenproblem of the fallback
 * Rayleigh-Ritz step; the paper calls a library routine): Householder reduction to
 * Hessenberg form, shifted QR iteration to the complex Schur form G = Z T Z^*, and the
 * eigenvectors of T by back substitution: G V = V diag(lam).
 *   G    device, k x k complex128 column-major (not modified), 0 <= k <= 32768
 *   lam  device, k complex128 eigenvalues, in the order of V's columns (unsorted)
 *   V    device, k x k complex128, unit columns
 * Returns NOT_CONVERGED when an eigenvalue needs more than 30 k QR sweeps in all.
 * Synchronises `stream`. */
int chase_bse_eig_general(const void* G, int64_t k, void* lam, void* V, void* stream);

/* Dense hermitian eigensolver of the Rayleigh-Ritz step (Algorithm 2, the HEEVD call
 * G y = theta y), as the solver runs it: G V = V diag(theta).
 *   G       device, k x k complex128 column-major, hermitian (not modified)
 *   theta   device, k doubles: the eigenvalues, in the order of V's columns (unsorted)
 *   V       device, k x k complex128: unit eigenvectors as columns
 *   k       even, >= 2
 *   method  0: FP64 Jacobi with scalar rotations (one round of k/2 disjoint rotations
 *              per grid barrier); 1: mixed precision as in a mixed solve (FP32 block
 *              Jacobi, two Ogita-Aishima refinement steps in FP64-accurate tensor-core
 *              GEMMs, FP64 Jacobi on the indices still coupled; needs compute
 *              capability 10.3); 2: FP64 block Jacobi (blocks of 32 indices)
 *   thr     rotations stop when every |g_pq| <= thr sqrt|g_pp g_qq| (thr >= 2e-16;
 *           the mixed method's FP32 phase stops at 2e-6)
 * Returns BAD_ARG, UNSUPPORTED (method 1 on another device), DEVICE_TIMEOUT.
 * Synchronises `stream`. */
int chase_bse_eigh(const void* G, int64_t k, double* theta, void* V, int32_t method, double thr,
                   void* stream);

/* FP64-accurate real GEMM on the BF16 tensor cores, the building block of the
 * mixed solve's QR and Rayleigh-Ritz products (the paper has no counterpart: it
 * serves the GB300, whose FP64 pipe runs at 1/64 of its FP32 rate).
 *   C[r + c * ldc] = alpha * sum_k A[r * lda + k] * B[c * ldb + k]
 * for r < M, c < N: A is M x K and B is N x K, both row-major (K contiguous), C is
 * column-major.  A, B, C device pointers (FP64); K even; lda, ldb >= K; ldc >= M.
 * Each row of A and of B is scaled by a power of two and cut into 7 signed 8-bit
 * digits; digit products of equal weight are summed exactly in the tensor cores'
 * FP32 accumulators over 128-long K chunks and folded into 64-bit integers, so
 * that the error is about 2^-56 K max|A_r.| max|B_c.| (FP64 class) plus the
 * final rounding.  M = 0 or N = 0 is a no-op.  Returns UNSUPPORTED on a device
 * other than compute capability 10.3, DEVICE_TIMEOUT if a bounded device-side
 * wait gave up.  Synchronises `stream`. */
int chase_bse_dgemm_sliced(const double* A, int64_t lda, const double* B, int64_t ldb,
                           int64_t M, int64_t N, int64_t K, double alpha, double* C,
                           int64_t ldc, void* stream);

/* Per-vector Chebyshev degrees for the next filter (host only, no GPU work): the
 * degree rule the solver applies after each Rayleigh-Ritz step.  The paper sets the
 * degree of each vector from its convergence rate (Section 6; the formula it cites is
 * not printed); this library's reading, with a = mu_nevex^2, b = muN^2,
 * c = (a+b)/2, e = (b-a)/2 and t_i = (ritz_i^2 - c)/e:
 *   rho_i = 1/(|t_i| + sqrt(t_i^2 - 1))   (1 when |t_i| <= 1), the predicted
 *           damping of the residual per H^2 step, replaced by the observed rate
 *           (res_i/prev_res_i)^(1/prev_deg_i) when that is slower (0 < res_i <
 *           prev_res_i, prev_res_i finite);
 *   degs_i = deg_min if res_i <= tol, deg_max if rho_i >= 1, else
 *            clamp(ceil(ln(tol/res_i)/ln(rho_i)) + 1, deg_min, deg_max).
 *   ritz, res, prev_res, prev_deg, degs: host arrays of k entries (prev_res may
 *   hold +inf for "no history"); 1 <= deg_min <= deg_max; 0 < mu_nevex < muN.
 * Returns BAD_ARG on invalid arguments. */
int chase_bse_degrees(const double* ritz, const double* res, const double* prev_res,
                      const int32_t* prev_deg, int64_t k, double tol, double mu_nevex,
                      double muN, int32_t deg_min, int32_t deg_max, int32_t* degs);

/* Static description of a status code. */
const char* chase_bse_strerror(int status);

/* Library version, and 1 when the mixed-precision (tcgen05) filter is compiled in. */
int chase_bse_version(void);
int chase_bse_has_mixed(void);

/* Device memory (no counterpart in the paper): the library allocates its
 * workspaces stream-ordered from its own memory pool on each device and keeps
 * freed memory cached for the next allocation (a solve allocates the same
 * workspaces every iteration).  This call returns the cached memory of the
 * current device to the driver; memory still in use by a call in flight is
 * not affected. */
void chase_bse_trim_memory(void);

/* Diagnostics (no counterpart in the paper): the number of CUDA kernels this
 * library has launched since it was loaded, summed over all threads. */
int64_t chase_bse_launch_count(void);

/* Testing and diagnostics (no counterpart in the paper): the bound, in nanoseconds of
 * %globaltimer, of every grid-barrier wait of the cooperative kernels (Cholesky, the
 * Jacobi eigensolvers); 0 restores the default of 2 s.  A wait that runs out makes the
 * kernel record an error and leave at its next barrier; the call then returns
 * DEVICE_TIMEOUT and the device stays usable.  Applies to calls made after it. */
void chase_bse_set_wait_limit(uint64_t ns);

/* Diagnostics (no counterpart in the paper): the number of device allocations
 * (stream-ordered, from the library's pool) the library has requested since it
 * was loaded, summed over all threads. */
int64_t chase_bse_alloc_count(void);

/* Diagnostics (no counterpart in the paper): device time of the filter's H
 * applications (the step of Algorithm 2 that applies H to a block of vectors).
 * chase_bse_gemm_timer(1) clears the record and starts bracketing every such launch
 * made afterwards, by any thread, with a pair of CUDA events recorded on the launch's
 * stream: kind 0 the tensor-core GEMM of a mixed-precision filter, kind 1 the FP64 H
 * application (with its K-split reduction where one is used), kind 2 the FP64-accurate
 * sliced H application (its vector slicing, GEMM and recombination).  chase_bse_gemm_timer(0)
 * stops and clears.  chase_bse_gemm_time waits for the recorded launches of `kind`
 * (blocking the host), writes into *total_ms the sum of their event-to-event device
 * times in milliseconds, into *flops the sum of their algorithmic flops (32 n^2 k for
 * k vectors: H is 2n x 2n complex, 8 real flops per complex multiply-add) and into
 * *launches their number, and clears that kind's record.  Returns BAD_ARG for a NULL
 * pointer or a kind other than 0, 1 or 2. */
void chase_bse_gemm_timer(int32_t enable);
int chase_bse_gemm_time(int32_t kind, double* total_ms, double* flops, int64_t* launches);

#ifdef __cplusplus
}
#endif
#endif /* CHASE_BSE_H */
