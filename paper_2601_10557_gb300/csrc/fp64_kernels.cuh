// FP64 kernels: H-application GEMM with fused epilogues and a generic complex GEMM.
#pragma once
#include "common.cuh"

namespace cb {

// ---- H application --------------------------------------------------------
// H W for W = [X; Y] (2n x k, column-major, ld 2n) reading only A and B
// (row-major).  With P = [A | B] (n x 2n) and W_hat = [[X, conj(Y)], [Y, conj(X)]]:
//   P W_hat = [H W_top, -conj(H W_bottom)],
// so one pass over P yields both halves (the block structure of Section 1).
enum HopMode : int {
  HOP_STORE = 0,   // out = H W               (sflip: out = S H W)
  HOP_CHEB = 1,    // out = alpha (H W - c Wc) + beta Wp
  HOP_RESID = 2    // out = H W - W diag(lambda)
};

struct HopArgs {
  const cplx* A;
  const cplx* B;
  int64_t n;
  const cplx* W;     // 2n x k input
  int64_t k;         // active columns (prefix)
  cplx* out;         // 2n x k output (ld 2n)
  int mode;
  int sflip;         // HOP_STORE: negate the lower half (T = S H Q)
  double alpha, beta, c;
  const cplx* Wc;    // HOP_CHEB: current iterate (ld 2n)
  const cplx* Wp;    // HOP_CHEB: previous iterate (ld 2n), unused if beta == 0
  const double* lambda;  // HOP_RESID
  int no_split;      // 1: one launch over the whole K range (no split-K partials, allocates nothing)
};

int hop_fp64(const HopArgs& a, cudaStream_t s);

// Top half of H applied to J-fixed vectors q = [x; conj(x)] (J = K conj):
// H q = [y; -conj(y)] with y = A x + B conj(x).  X and Y are n x k (ld n).
int hop_top_fp64(const cplx* A, const cplx* B, int64_t n, const cplx* X, int64_t k, cplx* Y, cudaStream_t s);

// ---- generic complex GEMM (column-major, BLAS semantics) --------------------
// C = alpha op(A) op(B) + beta C, op in {'N', 'T', 'C'}; beta == 0 ignores C.
int zgemm(char opA, char opB, int64_t M, int64_t N, int64_t K, cplx alpha, const cplx* A,
          int64_t lda, const cplx* B, int64_t ldb, cplx beta, cplx* C, int64_t ldc,
          cudaStream_t s);

}  // namespace cb
