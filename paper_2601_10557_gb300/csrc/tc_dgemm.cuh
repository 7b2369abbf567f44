// FP64-accurate real GEMM on BF16 tensor cores (sm_103a), for the FP64 products of
// the QR and Rayleigh-Ritz steps.
//
// GB300 executes FP64 at 1/64 of its FP32 rate (about 1.2 TFLOP/s), so the
// Gram matrices, the Rayleigh-Ritz product H Q and the back-transforms would
// dominate the solve on the FP64 pipe.  Here each operand row is scaled by a
// power of two 2^-e (|x| < 2^e on the row) and cut into S = 7 signed 8-bit
// digits d_t in [-128, 128] (exact BF16 integers):
//     x = 2^(e-7) * sum_t d_t 2^(-8t) + O(2^(e-56)).
// The digit products of equal weight w = t + u < S are summed by tcgen05.mma into
// FP32 TMEM accumulators over 128-long K chunks; each such sum is an integer below
// 2^24 and therefore exact.  The epilogue folds them into two 64-bit integers (the
// weights 2^0 .. 2^-24 and 2^-32 .. 2^-48), so the only rounding is the final
// conversion to FP64 and the dropped digits beyond 2^-56 of the row scales (error
// about 2^-56 K |x|max |y|max).
#pragma once
#include <cuda.h>
#include <cuda_bf16.h>

#include "common.cuh"

namespace cb {

constexpr int SLICES = 7;

// One operand in sliced form: SLICES planes of rows_pad x kpad BF16 digits
// (K contiguous), rows_pad a multiple of 128, kpad of 32, and a per-row exponent.
struct SlicedOp {
  __nv_bfloat16* planes = nullptr;
  int* exps = nullptr;
  int64_t rows = 0, rows_pad = 0, K = 0, kpad = 0;
  CUtensorMap map_a;  // 128-row boxes (operand A: rows of C)
  CUtensorMap map_b;  // 32-row boxes (operand B: columns of C)
};

// Allocate the planes of an operand with `rows` rows of length K (from ws).
int sliced_alloc(Workspace& ws, SlicedOp& op, int64_t rows, int64_t K, cudaStream_t s);

// Rows of a real FP64 matrix, row r at src + r * ld (K values); mode 0 takes
// them as they are, mode 1 maps each pair (a, b) to (b, -a), mode 2 to (a, -b).
int slice_rows(const double* src, int64_t ld, int mode, SlicedOp& op, cudaStream_t s);

// The real form of the rows of the complex n x m matrix X (column-major, ld):
// row 2i = (Re X_il, -Im X_il)_l, row 2i+1 = (Im X_il, Re X_il)_l, so that with
// B rows (Re Z_lj, Im Z_lj)_l the product gives (Re, Im) of (X Z)_ij in rows 2i,
// 2i+1.  `tmp` holds 4 n m doubles.
int slice_complex_rows(const cplx* X, int64_t ldx, int64_t n, int64_t m, double* tmp, SlicedOp& op,
                       cudaStream_t s);

// Rows of the complex matrix M (column-major, ld), conjugated, as (re, im) pairs:
// the B operand of X M^* (op.rows = rows of M, op.K = 2 x columns of M).
int slice_conj_rows(const cplx* M, int64_t ld, SlicedOp& op, cudaStream_t s);
// The same rows without conjugation: the B operand of X M^T.
int slice_plain_rows(const cplx* M, int64_t ld, SlicedOp& op, cudaStream_t s);

// Rows of the real 2n x 2n matrix P' with [Re y; Im y] interleaved = P' [Re x; Im x]
// interleaved for y = A x + B conj(x) (A, B row-major complex n x n).
int slice_hamiltonian(const cplx* A, const cplx* B, int64_t n, SlicedOp& op, cudaStream_t s);

// out = H W for a general 2n x k block W (column-major, ld 2n), from the sliced
// P' of slice_hamiltonian: each w = [x; y] is the sum of the J-fixed vectors
// [a; conj(a)] and -i [c; conj(c)], a = (x + conj(y))/2, c = i (x - conj(y))/2,
// and H [z; conj(z)] = [P'z; -conj(P'z)].
int hop_sliced(const SlicedOp& ph, const cplx* W, int64_t n, int64_t k, cplx* out, cudaStream_t s);

// C[r][c] = alpha * sum_k a[r][k] b[c][k] for r < a.rows, c < b.rows, written to
// out[r * rs + c * cs]; with neg_odd the rows r odd are negated (complex
// conjugate of a real-form result).
int sliced_gemm(const SlicedOp& a, const SlicedOp& b, double alpha, double* out, int64_t rs, int64_t cs,
                bool neg_odd, cudaStream_t s);

}  // namespace cb
