// Host-side stages of the solver (each runs its kernels on one stream).
#pragma once
#include <vector>
#include "common.cuh"

namespace cb {

struct FilterStats {
  double flops = 0, flops_fp64 = 0, ms_fp64 = 0, ms_mixed = 0;
  int64_t launches = 0;
};

// Tensor-core filter schemes (split products, tc_filter.cu); the values equal the
// chase_bse_precision codes that select them.
enum FilterScheme : int { SCHEME_BF16X3 = 1, SCHEME_BF16X6 = 2, SCHEME_FP16X3 = 3 };

// Chebyshev filter on H^2, in place on W (2n x k); degs/prec are per column
// (host).  prec[i] = 0: FP64 path, 1: tensor-core path with `scheme`
// (FilterScheme).  With ritz (host, per column) and R (device, 2n x k, the FP64
// residual vectors H w - ritz w) the tensor-core columns use the correction form.
// With ph (the sliced operand of slice_hamiltonian) the FP64 columns apply H by
// FP64-accurate sliced GEMMs on the tensor cores instead of the FP64 pipe.  With P2, Q2
// (the blocks of H^2, see form_h2) the tensor-core columns apply H^2 from its blocks
// (the explicit-H^2 variant).
struct SlicedOp;
int filter(const cplx* A, const cplx* B, int64_t n, cplx* W, int64_t k, const int* degs, const int* prec,
           double mu1, double mu_nevex, double muN, int scheme, const double* ritz, const cplx* R, cudaStream_t s,
           FilterStats* fs, const SlicedOp* ph = nullptr, const cplx* P2 = nullptr, const cplx* Q2 = nullptr);

// The blocks of H^2 = [[P2, Q2], [conj Q2, conj P2]]: P2 = A A - B conj(B),
// Q2 = A B - B conj(A) (row-major n x n, like A and B), as the top block row
// [A | -B] [[A, B], [conj B, conj A]], FP64-accurate sliced GEMMs (tc_dgemm.cu).
int form_h2(const cplx* A, const cplx* B, int64_t n, cplx* P2, cplx* Q2, cudaStream_t s);

// Lanczos bounds: mu1, mu_nevex, muN and rho_hat (max |theta|); with ph (the sliced
// operand of slice_hamiltonian) H is applied on the tensor cores, FP64-accurate.
int lanczos_bounds(const cplx* A, const cplx* B, int64_t n, const cplx* V0, int64_t nvec, int steps,
                   int64_t nevex, double out[4], cudaStream_t s, const SlicedOp* ph = nullptr);

// Orthonormal Q (2n x m) of X (2n x m; X is preserved).  *used_hh set to 1 if
// the Householder fallback ran.
int qr(const cplx* X, int64_t n2, int64_t m, cplx* Q, int* used_hh, cudaStream_t s);

// Algorithm 2 on Q (2n x k): ritz (host, k/2 ascending) and Wpos (2n x k/2).
// With R and res (device), also the residual vectors R = H Wpos - Wpos diag(ritz)
// and their norms, from H Wpos = S T Z+ (T = S H Q of the Rayleigh-Ritz step: no extra H product).
int rayleigh_ritz(const cplx* A, const cplx* B, int64_t n, const cplx* Q, int64_t k, double* ritz_host,
                  cplx* Wpos, cudaStream_t s, cplx* R = nullptr, double* res = nullptr);

// res[j] = ||H w_j - lambda_j w_j||_2 (device lambda and res); the residual
// vectors are kept in Rout when it is not NULL (2n x k).
int residuals(const cplx* A, const cplx* B, int64_t n, const cplx* W, const double* lambda, int64_t k,
              double* res, cudaStream_t s, cplx* Rout = nullptr);

int solve(const cplx* A, const cplx* B, int64_t n, int64_t nev, int64_t nex, int deg, double tol,
          const chase_bse_opts* opts, double* evals, cplx* evecs, chase_bse_stats* stats);

// The per-vector degree rule (see chase_bse_degrees): host only.
void degrees_update(const std::vector<double>& ritz, const std::vector<double>& res,
                    const std::vector<double>& prev_res, const std::vector<int>& prev_deg, double tol, double mu_ne,
                    double muN, int dmin, int dmax, std::vector<int>& degs);

// Eigen-decomposition of a general complex k x k matrix G (column-major; not
// modified): G V = V diag(lam), unit columns (geev.cu).  NOT_CONVERGED if the shifted
// QR iteration needs more than 30 k sweeps.
int geev(const cplx* G, int64_t k, cplx* lam, cplx* V, cudaStream_t s);

// Non-hermitian fallback Rayleigh-Ritz (Section 4.4, last paragraph; geev.cu): the dual
// basis of Q, G = Q_L^* H Q, and the Ritz pairs with positive real part (ascending):
// ritz_host[0 .. *npos), W (2n x *npos) = Q Z_+ with unit columns.
int rayleigh_ritz_fallback(const cplx* A, const cplx* B, int64_t n, const cplx* Q, int64_t k, double* ritz_host,
                           cplx* W, int64_t* npos, cudaStream_t s);

int gradient(const cplx* V, const double* w, int64_t n, int64_t nev, cplx* gA, cplx* gB, cudaStream_t s);

// Mixed-precision (tcgen05) filter on a column group whose columns are sorted
// by descending degree; defined in the tensor-core translation unit.
// scheme: a FilterScheme.
// With P2, Q2 (the blocks of H^2, see form_h2) the filter applies H^2 from its blocks.
int filter_mixed_sorted(const cplx* A, const cplx* B, int64_t n, cplx* Y0, int64_t k, const int* degs_sorted,
                        double mu1, double mu_nevex, double muN, cplx* out, int scheme, cudaStream_t s,
                        FilterStats* fs, const cplx* P2 = nullptr, const cplx* Q2 = nullptr);
// Correction form (see tc_filter.cu): V holds Ritz vectors, ritz their values,
// R = H V - V diag(ritz) (FP64); out = p(H^2) V.
int filter_mixed_correction_sorted(const cplx* A, const cplx* B, int64_t n, cplx* V, int64_t k,
                                   const int* degs_sorted, const double* ritz_sorted, const cplx* R, double mu1,
                                   double mu_nevex, double muN, cplx* out, int scheme, cudaStream_t s,
                                   FilterStats* fs, const cplx* P2 = nullptr, const cplx* Q2 = nullptr);
bool mixed_available();

}  // namespace cb
