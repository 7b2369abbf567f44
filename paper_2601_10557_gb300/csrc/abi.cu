// extern "C" entry points declared in include/chase_bse.h.
#include <exception>
#include <vector>

#include "dense_kernels.cuh"
#include "solver.cuh"
#include "tc_dgemm.cuh"

using cb::cplx;

#define CB_GUARD(body)                 \
  try {                                \
    body                               \
  } catch (const std::bad_alloc&) {    \
    return CHASE_BSE_OOM;              \
  } catch (...) {                      \
    return CHASE_BSE_CUDA_ERROR;       \
  }

static int degrees_host(const double* ritz, const double* res, const double* prev_res, const int32_t* prev_deg,
                        int64_t k, double tol, double mu_nevex, double muN, int32_t deg_min, int32_t deg_max,
                        int32_t* degs) {
  std::vector<double> r(ritz, ritz + k);
  std::vector<double> q(res, res + k);
  std::vector<double> p(prev_res, prev_res + k);
  std::vector<int> pd(prev_deg, prev_deg + k);
  std::vector<int> d;
  cb::degrees_update(r, q, p, pd, tol, mu_nevex, muN, deg_min, deg_max, d);
  for (int64_t i = 0; i < k; ++i) degs[i] = d[i];
  return CHASE_BSE_OK;
}

// Filter call of the ABI: with tc64 the FP64 columns apply H by sliced tensor-core GEMMs
// (the sliced form of H is cut for this call).
static int filter_call(const cplx* A, const cplx* B, int64_t n, cplx* W, int64_t k, const int* degs, const int* prec,
                       double mu1, double mu_nevex, double muN, int scheme, bool tc64, cudaStream_t s) {
  if (!tc64) return cb::filter(A, B, n, W, k, degs, prec, mu1, mu_nevex, muN, scheme, nullptr, nullptr, s, nullptr);
  cb::Workspace ws(s);
  cb::SlicedOp ph;
  CB_TRY(cb::sliced_alloc(ws, ph, 2 * n, 2 * n, s));
  CB_TRY(cb::slice_hamiltonian(A, B, n, ph, s));
  CB_TRY(cb::filter(A, B, n, W, k, degs, prec, mu1, mu_nevex, muN, scheme, nullptr, nullptr, s, nullptr, &ph));
  // the workspace (and the sliced H) is released on the stream after the filter
  return CHASE_BSE_OK;
}

static int eigh_impl(const cplx* G, int64_t k, double* theta, cplx* V, int method, double thr, cudaStream_t s) {
  cb::Workspace ws(s);
  cplx *Gc, *rot;
  double* red;
  CB_TRY(ws.alloc(&Gc, k * k));
  CB_TRY(ws.alloc(&rot, 2 * k));
  CB_TRY(ws.alloc(&red, 2));
  CB_CUDA(cudaMemcpyAsync(Gc, G, sizeof(cplx) * k * k, cudaMemcpyDeviceToDevice, s));
  int sw = 0, sw32 = 0;
  int st = CHASE_BSE_OK;
  if (method == 0) st = cb::jacobi_eigh(Gc, k, V, theta, rot, red, 40, &sw, s, thr);
  else if (method == 1) st = cb::jacobi_eigh_mixed(Gc, k, V, theta, rot, red, &sw32, &sw, s, thr);
  else st = cb::jacobi_block(Gc, k, V, theta, false, thr, 0.5 * thr, 40, &sw, s);
  if (cb::verbose()) fprintf(stderr, "[chase_bse] eigh method %d k %ld sweeps %d (FP32 %d)\n", method, (long)k, sw, sw32);
  if (st != CHASE_BSE_OK) return st;
  CB_CUDA(cudaStreamSynchronize(s));
  return CHASE_BSE_OK;
}

extern "C" {

int chase_bse_version(void) { return 100; }

int64_t chase_bse_launch_count(void) { return cb::launch_count(); }

int64_t chase_bse_alloc_count(void) { return cb::alloc_count(); }

void chase_bse_set_wait_limit(uint64_t ns) { cb::set_wait_limit_ns(ns); }

void chase_bse_gemm_timer(int32_t enable) { cb::timer_enable(enable != 0); }

int chase_bse_gemm_time(int32_t kind, double* total_ms, double* flops, int64_t* launches) {
  if (!total_ms || !flops || !launches || kind < 0 || kind > 2) return CHASE_BSE_BAD_ARG;
  return cb::timer_read(kind, total_ms, flops, launches);
}

int chase_bse_has_mixed(void) { return cb::mixed_available() ? 1 : 0; }

void chase_bse_trim_memory(void) { cb::pool_trim(); }

const char* chase_bse_strerror(int status) {
  switch (status) {
    case CHASE_BSE_OK: return "ok";
    case CHASE_BSE_NOT_CONVERGED: return "not converged within maxiter (partial results written)";
    case CHASE_BSE_BAD_ARG: return "invalid argument";
    case CHASE_BSE_CUDA_ERROR: return "CUDA error";
    case CHASE_BSE_OOM: return "device workspace allocation failed";
    case CHASE_BSE_NOT_DEFINITE: return "S H is not positive definite on the search space";
    case CHASE_BSE_QR_FAILED: return "orthonormalisation failed";
    case CHASE_BSE_DEVICE_TIMEOUT: return "a bounded device-side wait gave up";
    case CHASE_BSE_UNSUPPORTED: return "not supported on this device";
    case CHASE_BSE_NONFINITE: return "an input holds a NaN or an Inf";
    default: return "unknown status";
  }
}

int chase_bse_solve(const void* A, const void* B, int64_t n, int64_t nev, int64_t nex, int32_t deg, double tol,
                    const chase_bse_opts* opts, double* evals, void* evecs, chase_bse_stats* stats) {
  CB_GUARD(return cb::solve((const cplx*)A, (const cplx*)B, n, nev, nex, deg, tol, opts, evals, (cplx*)evecs,
                            stats);)
}

int chase_bse_filter(const void* A, const void* B, int64_t n, void* W, int64_t k, const int32_t* degs, double mu1,
                     double mu_nevex, double muN, int32_t precision, void* stream) {
  if (k == 0) return CHASE_BSE_OK;
  if (!A || !B || !W || !degs || n < 1 || k < 0 || !(mu1 > 0) || !(mu_nevex > mu1) || !(muN > mu_nevex))
    return CHASE_BSE_BAD_ARG;
  if (precision != CHASE_BSE_FP64 && precision != CHASE_BSE_MIXED_BF16X3 && precision != CHASE_BSE_MIXED_BF16X6 &&
      precision != CHASE_BSE_MIXED_FP16X3 && precision != CHASE_BSE_FP64_TC)
    return CHASE_BSE_BAD_ARG;
  for (int64_t i = 0; i < k; ++i)
    if (degs[i] < 1) return CHASE_BSE_BAD_ARG;
  if (precision == CHASE_BSE_FP64_TC && !cb::mixed_available()) return CHASE_BSE_UNSUPPORTED;
  CB_GUARD({
    const bool fp64 = precision == CHASE_BSE_FP64 || precision == CHASE_BSE_FP64_TC;
    std::vector<int> prec(k, fp64 ? 0 : 1);
    return filter_call((const cplx*)A, (const cplx*)B, n, (cplx*)W, k, degs, prec.data(), mu1, mu_nevex, muN,
                       fp64 ? (int)CHASE_BSE_MIXED_FP16X3 : precision, precision == CHASE_BSE_FP64_TC,
                       (cudaStream_t)stream);
  })
}

int chase_bse_filter_cols(const void* A, const void* B, int64_t n, void* W, int64_t k, const int32_t* degs,
                          const int32_t* precs, double mu1, double mu_nevex, double muN, void* stream) {
  if (k == 0) return CHASE_BSE_OK;
  if (!A || !B || !W || !degs || !precs || n < 1 || k < 0 || !(mu1 > 0) || !(mu_nevex > mu1) ||
      !(muN > mu_nevex))
    return CHASE_BSE_BAD_ARG;
  int scheme = 0;
  bool dfma = false, tc64 = false;
  for (int64_t i = 0; i < k; ++i) {
    if (degs[i] < 1) return CHASE_BSE_BAD_ARG;
    const int p = precs[i];
    if (p == CHASE_BSE_FP64) {
      dfma = true;
      continue;
    }
    if (p == CHASE_BSE_FP64_TC) {
      tc64 = true;
      continue;
    }
    if (p != CHASE_BSE_MIXED_BF16X3 && p != CHASE_BSE_MIXED_BF16X6 && p != CHASE_BSE_MIXED_FP16X3)
      return CHASE_BSE_BAD_ARG;
    if (scheme != 0 && p != scheme) return CHASE_BSE_BAD_ARG;
    scheme = p;
  }
  if (dfma && tc64) return CHASE_BSE_BAD_ARG;
  if (tc64 && !cb::mixed_available()) return CHASE_BSE_UNSUPPORTED;
  CB_GUARD({
    std::vector<int> prec(k);
    for (int64_t i = 0; i < k; ++i)
      prec[i] = (precs[i] == CHASE_BSE_FP64 || precs[i] == CHASE_BSE_FP64_TC) ? 0 : 1;
    return filter_call((const cplx*)A, (const cplx*)B, n, (cplx*)W, k, degs, prec.data(), mu1, mu_nevex, muN,
                       scheme == 0 ? CHASE_BSE_MIXED_FP16X3 : scheme, tc64, (cudaStream_t)stream);
  })
}

int chase_bse_rr(const void* A, const void* B, int64_t n, const void* Q, int64_t k, double* ritz, void* Wpos,
                 void* stream) {
  if (!A || !B || !Q || !ritz || !Wpos || n < 1 || k < 2 || (k % 2) != 0 || k > 2 * n) return CHASE_BSE_BAD_ARG;
  CB_GUARD(return cb::rayleigh_ritz((const cplx*)A, (const cplx*)B, n, (const cplx*)Q, k, ritz, (cplx*)Wpos,
                                    (cudaStream_t)stream);)
}

int chase_bse_residuals(const void* A, const void* B, int64_t n, const void* W, const double* lambda, int64_t k,
                        double* res, void* stream) {
  if (k == 0) return CHASE_BSE_OK;
  if (!A || !B || !W || !lambda || !res || n < 1 || k < 0) return CHASE_BSE_BAD_ARG;
  CB_GUARD(return cb::residuals((const cplx*)A, (const cplx*)B, n, (const cplx*)W, lambda, k, res,
                                (cudaStream_t)stream);)
}

int chase_bse_grad(const void* V, const double* w, int64_t n, int64_t nev, void* gA, void* gB, void* stream) {
  if (!V || !w || !gA || !gB || n < 1 || nev < 1) return CHASE_BSE_BAD_ARG;
  CB_GUARD(return cb::gradient((const cplx*)V, w, n, nev, (cplx*)gA, (cplx*)gB, (cudaStream_t)stream);)
}

int chase_bse_degrees(const double* ritz, const double* res, const double* prev_res, const int32_t* prev_deg,
                      int64_t k, double tol, double mu_nevex, double muN, int32_t deg_min, int32_t deg_max,
                      int32_t* degs) {
  if (k < 0 || (k > 0 && (!ritz || !res || !prev_res || !prev_deg || !degs)) || !(tol > 0) || deg_min < 1 ||
      deg_max < deg_min || !(mu_nevex > 0) || !(muN > mu_nevex))
    return CHASE_BSE_BAD_ARG;
  CB_GUARD(return degrees_host(ritz, res, prev_res, prev_deg, k, tol, mu_nevex, muN, deg_min, deg_max, degs);)
}

int chase_bse_eigh(const void* G, int64_t k, double* theta, void* V, int32_t method, double thr, void* stream) {
  if (!G || !theta || !V || k < 2 || (k % 2) != 0 || method < 0 || method > 2 || !(thr >= 2e-16))
    return CHASE_BSE_BAD_ARG;
  if (method == 1 && !cb::mixed_available()) return CHASE_BSE_UNSUPPORTED;
  CB_GUARD(return eigh_impl((const cplx*)G, k, theta, (cplx*)V, method, thr, (cudaStream_t)stream);)
}

int chase_bse_h2_blocks(const void* A, const void* B, int64_t n, void* P, void* Q, void* stream) {
  if (!A || !B || !P || !Q || n < 1) return CHASE_BSE_BAD_ARG;
  if (!cb::mixed_available()) return CHASE_BSE_UNSUPPORTED;
  CB_GUARD(return cb::form_h2((const cplx*)A, (const cplx*)B, n, (cplx*)P, (cplx*)Q, (cudaStream_t)stream);)
}

int chase_bse_filter_h2(const void* A, const void* B, int64_t n, void* W, int64_t k, const int32_t* degs, double mu1,
                        double mu_nevex, double muN, int32_t precision, void* stream) {
  if (k == 0) return CHASE_BSE_OK;
  if (!A || !B || !W || !degs || n < 1 || k < 0 || !(mu1 > 0) || !(mu_nevex > mu1) || !(muN > mu_nevex))
    return CHASE_BSE_BAD_ARG;
  if (precision != CHASE_BSE_MIXED_BF16X3 && precision != CHASE_BSE_MIXED_BF16X6 &&
      precision != CHASE_BSE_MIXED_FP16X3)
    return CHASE_BSE_BAD_ARG;
  for (int64_t i = 0; i < k; ++i)
    if (degs[i] < 1) return CHASE_BSE_BAD_ARG;
  if (!cb::mixed_available()) return CHASE_BSE_UNSUPPORTED;
  CB_GUARD({
    cudaStream_t s = (cudaStream_t)stream;
    cb::Workspace ws(s);
    cplx* P2 = nullptr;
    cplx* Q2 = nullptr;
    CB_TRY(ws.alloc(&P2, n * n));
    CB_TRY(ws.alloc(&Q2, n * n));
    CB_TRY(cb::form_h2((const cplx*)A, (const cplx*)B, n, P2, Q2, s));
    std::vector<int> prec(k, 1);
    return cb::filter((const cplx*)A, (const cplx*)B, n, (cplx*)W, k, degs, prec.data(), mu1, mu_nevex, muN,
                      precision, nullptr, nullptr, s, nullptr, nullptr, P2, Q2);
  })
}

int chase_bse_eig_general(const void* G, int64_t k, void* lam, void* V, void* stream) {
  if (k == 0) return CHASE_BSE_OK;
  if (!G || !lam || !V || k < 0 || k > ((int64_t)1 << 15)) return CHASE_BSE_BAD_ARG;
  CB_GUARD(return cb::geev((const cplx*)G, k, (cplx*)lam, (cplx*)V, (cudaStream_t)stream);)
}

int chase_bse_rr_fallback(const void* A, const void* B, int64_t n, const void* Q, int64_t k, double* ritz, void* W,
                          int64_t* npos, void* stream) {
  if (!A || !B || !Q || !ritz || !W || !npos || n < 1 || k < 1 || k > 2 * n || k > ((int64_t)1 << 15))
    return CHASE_BSE_BAD_ARG;
  CB_GUARD(return cb::rayleigh_ritz_fallback((const cplx*)A, (const cplx*)B, n, (const cplx*)Q, k, ritz, (cplx*)W,
                                             npos, (cudaStream_t)stream);)
}

int chase_bse_dgemm_sliced(const double* A, int64_t lda, const double* B, int64_t ldb, int64_t M, int64_t N,
                           int64_t K, double alpha, double* C, int64_t ldc, void* stream) {
  if (M == 0 || N == 0) return CHASE_BSE_OK;
  if (!A || !B || !C || M < 0 || N < 0 || K < 2 || (K % 2) != 0 || lda < K || ldb < K || ldc < M)
    return CHASE_BSE_BAD_ARG;
  if (!cb::mixed_available()) return CHASE_BSE_UNSUPPORTED;
  CB_GUARD({
    cudaStream_t s = (cudaStream_t)stream;
    cb::Workspace ws(s);
    cb::SlicedOp a;
    cb::SlicedOp b;
    CB_TRY(cb::sliced_alloc(ws, a, M, K, s));
    CB_TRY(cb::sliced_alloc(ws, b, N, K, s));
    CB_TRY(cb::slice_rows(A, lda, 0, a, s));
    CB_TRY(cb::slice_rows(B, ldb, 0, b, s));
    return cb::sliced_gemm(a, b, alpha, C, 1, ldc, false, s);
  })
}

}  // extern "C"
