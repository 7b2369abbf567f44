// Small dense FP64 kernels: Cholesky, triangular inverse, Jacobi eigensolver,
// Householder QR, Lanczos pieces and column utilities.  Matrices are
// column-major complex128 unless stated otherwise.
#pragma once
#include <utility>
#include <vector>

#include "common.cuh"

namespace cb {

// Blocked Cholesky G = L L^* in place (lower triangle; strict upper zeroed).
// *info_host = 0 on success, j+1 if the j-th pivot is not positive (or NaN).
int cholesky(cplx* G, int64_t k, int* info_dev, int* info_host, cudaStream_t s, bool real = false);
// out = in^* (k x k)
int conj_transpose(const cplx* in, int64_t k, cplx* out, cudaStream_t s);
// X = L^{-1} for lower-triangular L (k x k); T is k*32 complex scratch; real: L has
// zero imaginary parts.
int tri_inverse(const cplx* L, int64_t k, cplx* X, cplx* T, cudaStream_t s, bool real = false);

// red[0] = ||offdiag(G)||_F^2, red[1] = ||G||_F^2 (device)
int offdiag_norms(const cplx* G, int64_t k, double* red, cudaStream_t s);
// Cyclic Jacobi on hermitian G (k x k, k even, overwritten by its diagonal form);
// V receives the eigenvectors (columns).  theta[k] (device) gets diag(G).
// rot is k/2 * 4 complex scratch, red 2 doubles scratch; rotations stop below the
// relative threshold thr (>= 2e-16).
int jacobi_eigh(cplx* G, int64_t k, cplx* V, double* theta, cplx* rot, double* red,
                int max_sweeps, int* sweeps_out, cudaStream_t s, double thr = 2e-16);

// As jacobi_eigh, for G far from diagonal: FP32 Jacobi sweeps first, then the FP32
// eigenvectors made unitary in FP64 (Newton-Schulz on the tensor cores), G1 = V1^* G V1
// and FP64 Jacobi on G1 (jacobi_mixed.cu).  Falls back to jacobi_eigh for small k or a
// nearly diagonal G.  Needs the tensor cores (compute capability 10.3).
int jacobi_eigh_mixed(cplx* G, int64_t k, cplx* V, double* theta, cplx* rot, double* red, int* sweeps32_out,
                      int* sweeps64_out, cudaStream_t s, double thr);

// Block Jacobi (jacobi_block.cu): blocks of 32 indices paired round-robin, each pair's
// 64 x 64 sub-problem swept in shared memory, coalesced 64 x 64 tile updates of G and V;
// FP32 (fp32) or FP64 arithmetic.  G (k x k, hermitian, FP64) is not modified; V (k x k)
// receives the eigenvectors and theta (device, optional) the diagonal of the rotated G.
// Rotations stop when every |g_pq| <= thr sqrt|g_pp g_qq| or <= floor_rel ||G||_F.
int jacobi_block(const cplx* G, int64_t k, cplx* V, double* theta, bool fp32, double thr, double floor_rel,
                 int max_sweeps, int* sweeps_out, cudaStream_t s);

// The pairs i < j with |g_ij| > t sqrt|g_ii g_jj| and |g_ij| > floor_abs (at most cap
// of them, else OOM).
int coupled_pairs(const cplx* G, int64_t k, double t, double floor_abs, std::vector<std::pair<int, int>>& out,
                  int cap, cudaStream_t s);
// For disjoint index sets (set j = idx[off[j] .. off[j+1]), at most 64 each): FP64 Jacobi
// on G[set, set] (one CTA per set), its eigenvectors into those rows and columns of V2
// (k x k, preset to the identity) and its eigenvalues into theta.
int cluster_eig(const cplx* G, int64_t k, const std::vector<int>& idx, const std::vector<int>& off, double thr,
                double floor_abs, cplx* V2, double* theta, cudaStream_t s);

// Unblocked Householder QR: Q (N x m, column-major, ld N) receives the
// orthonormal factor of X (N x m), which is destroyed.  Vs: N*m, Us: N*m,
// wrow: m complex scratch.
int householder_qr(cplx* X, int64_t N, int64_t m, cplx* Q, cplx* Vs, cplx* Us, cplx* wrow,
                   cudaStream_t s);

// ---- utilities ----
int scale_lower(cplx* W, int64_t n, int64_t k, double gamma, cudaStream_t s);
// X = [S Yp, S K conj(Yp), Wf, K conj(Wf)]  (2n x (2L + 2kf))
int build_qr_input(cplx* X, const cplx* Yp, int64_t L, const cplx* Wf, int64_t kf, int64_t n,
                   cudaStream_t s);
int gather_cols(cplx* dst, const cplx* src, const int* idx, int64_t rows, int64_t m, cudaStream_t s);
// J-fixed basis (J = K conj) of span[S Y+, S Y-, W+, W-], top halves only (n x 2(L + kf)),
// in pairs per vector: locked top(Sy + J Sy), top(i (Sy - J Sy)); active top(w + J w),
// top(i (w - J w)).
int build_jfixed(cplx* Xt, const cplx* Yp, int64_t L, const cplx* W, int64_t kf, int64_t n, cudaStream_t s);
// out = U^* M U and Z = U Z' for U = blockdiag([[1, 1], [-i, i]] / sqrt 2) (k even)
int pair_transform(const cplx* M, cplx* out, int64_t k, cudaStream_t s);
int pair_apply(const cplx* Zp, cplx* Z, int64_t k, int64_t h, cudaStream_t s);
// out = 2 Re(C) (mode 0) or 2 i Im(C) (mode 1), k x k
int re_im_part(const cplx* C, cplx* out, int64_t k, int mode, cudaStream_t s);
// dst = conj(src), rows x m with leading dimensions lds, ldd
int conj_copy(cplx* dst, int64_t ldd, const cplx* src, int64_t lds, int64_t rows, int64_t m, cudaStream_t s);
// dst[:, j] = src_j[:, j] with src_j = bufs[sel[j]]  (collect filter outputs)
int collect_cols(cplx* dst, const cplx* b0, const cplx* b1, const cplx* b2, const int* sel,
                 int64_t rows, int64_t m, cudaStream_t s);
int scatter_cols(cplx* dst, const cplx* src, const int* idx, int64_t rows, int64_t m, cudaStream_t s);
int col_norms(const cplx* X, int64_t rows, int64_t m, double* out, cudaStream_t s);
int normalize_cols(cplx* X, int64_t rows, int64_t m, cudaStream_t s);
// Given W (2n x m, unnormalised Ritz vectors), HZ = S H W (2n x m) and ritz (device):
// nrm_j = ||W_j||, W_j /= nrm_j, R_j = S HZ_j / nrm_j - ritz_j W_j.
int normalize_and_residual(cplx* W, const cplx* SHW, const double* ritz, int64_t n, int64_t m, cplx* R,
                           cudaStream_t s);
int set_identity(cplx* M, int64_t k, cudaStream_t s);
// *count_host = the number of entries of X (total) with a NaN or Inf part
int count_nonfinite(const cplx* X, int64_t total, int* count_dev, int* count_host, cudaStream_t s);
// R[:, j] = HV[:, j] - lam[j] V[:, j] (n2 x m; lam device)
int residual_from_hv(const cplx* HV, const cplx* V, const double* lam, int64_t n2, int64_t m, cplx* R,
                     cudaStream_t s);
int hermitize(cplx* G, int64_t k, cudaStream_t s);
int diag_real(const cplx* G, int64_t k, double* out, cudaStream_t s);
int phase_fix(cplx* V, int64_t n, int64_t m, cudaStream_t s);
int copy_cols(cplx* dst, int64_t ldd, const cplx* src, int64_t lds, int64_t rows, int64_t m,
              cudaStream_t s);
// Lanczos pieces (per column c of nvec): out[c] = Re(x_c^* S y_c)
int sdot_real(const cplx* X, const cplx* Y, int64_t n, int64_t nvec, double* out, cudaStream_t s);
// Wv = U - alpha V - beta_prev Vp (beta_prev may be NULL)
int lanczos_axpy(cplx* Wv, const cplx* U, const cplx* V, const cplx* Vp, const double* alpha,
                 const double* beta_prev, int64_t n, int64_t nvec, cudaStream_t s);
// beta = sqrt(max(nrm2, 0)); V = Wv / beta; U = Y / beta
int lanczos_normalise(double* beta, const double* nrm2, const cplx* Wv, const cplx* Y, cplx* V,
                      cplx* U, int64_t n, int64_t nvec, cudaStream_t s);
// Counter-based standard normal draws (Philox4x32-10 + Box-Muller): out[i] = N(0,1) + i N(0,1)
int randn_complex(cplx* out, int64_t count, uint64_t seed, uint64_t stream_id, cudaStream_t s);
// Gradient helpers: Uc = [conj(X) c, Y c], U2 = [X, conj(Y)], Ub = [X c, conj(Y) c], U3 = [conj(Y), X]
int grad_prepare(const cplx* V, const double* w, int64_t n, int64_t nev, double* cbuf, cplx* Uc,
                 cplx* U2, cplx* Ub, cplx* U3, cudaStream_t s);

}  // namespace cb
