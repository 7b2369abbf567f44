// Dense eigensolver for a general (non-hermitian) complex k x k matrix, for the
// non-hermitian fallback of the Rayleigh-Ritz step (Section 4.4, last paragraph):
// there the projected matrix G = Q_L^* H Q is not hermitian and has no hermitian
// equivalent, so its eigenpairs come from a complex Schur decomposition:
//   1. Householder reduction to upper Hessenberg form, G = Z Hs Z^*;
//   2. implicitly shifted QR iteration (one Wilkinson shift per sweep, exceptional
//      shifts after 10 and 20 sweeps without deflation, deflation on negligible
//      subdiagonal entries), accumulating the rotations into Z: G = Z T Z^*,
//      T upper triangular;
//   3. eigenvectors of T by back substitution, (T - t_ii I) x = 0 with x_i = 1,
//      then V = Z X with unit columns.
// The textbook algorithm (Golub and Van Loan, Matrix Computations, sections 7.4-7.6),
// one CTA of 1024 threads per stage: the Householder and Givens updates of a step are
// spread over the threads, the steps themselves are sequential.  Meant for the
// fallback path (k up to a few thousand), not for speed.
#include <algorithm>
#include <cmath>
#include <vector>

#include "dense_kernels.cuh"
#include "fp64_kernels.cuh"
#include "solver.cuh"

namespace cb {
namespace gv {

constexpr int THREADS = 1024;
constexpr double EPS = 1.1102230246251565e-16;  // 2^-53
constexpr double TINY = 1e-300;

__device__ __forceinline__ double cabs1(cplx a) { return fabs(a.x) + fabs(a.y); }
__device__ __forceinline__ cplx cdivz(cplx a, cplx b) {
  // a / b, scaled by the larger component of b (Smith's method)
  if (fabs(b.x) >= fabs(b.y)) {
    const double r = b.y / b.x, d = b.x + r * b.y;
    return mk((a.x + a.y * r) / d, (a.y - a.x * r) / d);
  }
  const double r = b.x / b.y, d = b.y + r * b.x;
  return mk((a.x * r + a.y) / d, (a.y * r - a.x) / d);
}
__device__ __forceinline__ cplx csqrtz(cplx z) {
  const double r = hypot(z.x, z.y);
  if (r == 0.0) return mk(0.0, 0.0);
  const double t = sqrt(0.5 * (r + fabs(z.x)));
  if (z.x >= 0.0) return mk(t, z.y / (2.0 * t));
  return mk(fabs(z.y) / (2.0 * t), copysign(t, z.y));
}

// block sum of one double per thread (all threads of the block call it)
__device__ double block_sum(double v, double* red) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  if (w == 0) {
    v = lane < (int)(blockDim.x >> 5) ? red[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) red[0] = v;
  }
  __syncthreads();
  return red[0];
}

// Householder reduction of G (k x k, column-major, in place) to upper Hessenberg form;
// Z (k x k) receives the accumulated unitary factor (G_in = Z Hs Z^*).  v: k scratch.
// Reflector of step j: H_j = I - tau v v^*, v = [0 (j+1); 1; u], chosen so that
// H_j^* G[j+1:, j] = beta e_1 (beta real); G <- H_j^* G H_j, Z <- Z H_j.
__global__ void __launch_bounds__(THREADS) hess_kernel(cplx* G, cplx* Z, int k, cplx* v) {
  __shared__ double red[32];
  __shared__ cplx s_tau;
  __shared__ int s_skip;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int i = tid; i < k * k; i += THREADS) Z[i] = mk((i % k) == (i / k) ? 1.0 : 0.0, 0.0);
  for (int j = 0; j + 2 < k; ++j) {
    double part = 0.0;
    for (int r = j + 2 + tid; r < k; r += THREADS) part += cabs2(G[r + (int64_t)j * k]);
    const double xnorm2 = block_sum(part, red);
    if (tid == 0) {
      const cplx alpha = G[(j + 1) + (int64_t)j * k];
      if (xnorm2 == 0.0 && alpha.y == 0.0) {
        s_skip = 1;
      } else {
        s_skip = 0;
        const double nrm = sqrt(alpha.x * alpha.x + alpha.y * alpha.y + xnorm2);
        const double beta = alpha.x >= 0.0 ? -nrm : nrm;
        s_tau = mk((beta - alpha.x) / beta, -alpha.y / beta);
        v[j + 1] = mk(1.0, 0.0);
        G[(j + 1) + (int64_t)j * k] = mk(beta, 0.0);
        // the scale 1 / (alpha - beta) of the rest of the vector, kept in v[j] for the others
        v[j] = cdivz(mk(1.0, 0.0), mk(alpha.x - beta, alpha.y));
      }
    }
    __syncthreads();
    if (s_skip) continue;
    const cplx scal = v[j];
    for (int r = j + 2 + tid; r < k; r += THREADS) {
      v[r] = cmul(G[r + (int64_t)j * k], scal);
      G[r + (int64_t)j * k] = mk(0.0, 0.0);
    }
    __syncthreads();
    const cplx tau = s_tau, ctau = cconj(s_tau);
    // left: G[j+1:, c] -= conj(tau) v (v^* G[j+1:, c]) for c > j (one warp per column)
    for (int c = j + 1 + warp; c < k; c += THREADS / 32) {
      cplx* col = G + (int64_t)c * k;
      cplx w = mk(0.0, 0.0);
      for (int r = j + 1 + lane; r < k; r += 32) cfma(w, cconj(v[r]), col[r]);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        w.x += __shfl_xor_sync(0xffffffffu, w.x, o);
        w.y += __shfl_xor_sync(0xffffffffu, w.y, o);
      }
      const cplx f = cmul(ctau, w);
      for (int r = j + 1 + lane; r < k; r += 32) col[r] = csub(col[r], cmul(v[r], f));
    }
    __syncthreads();
    // right: M[r, j+1:] -= tau (M[r, j+1:] v) v^* for every row r, M = G and Z
    for (int r = tid; r < 2 * k; r += THREADS) {
      cplx* M = r < k ? G : Z;
      const int rr = r < k ? r : r - k;
      cplx w = mk(0.0, 0.0);
      for (int c = j + 1; c < k; ++c) cfma(w, M[rr + (int64_t)c * k], v[c]);
      const cplx f = cmul(tau, w);
      for (int c = j + 1; c < k; ++c) M[rr + (int64_t)c * k] = csub(M[rr + (int64_t)c * k], cmul(f, cconj(v[c])));
    }
    __syncthreads();
  }
}

// Givens rotation [c s; -conj(s) c] with [c s; -conj(s) c] [f; g] = [r; 0], c real.
__device__ void givens(cplx f, cplx g, double& c, cplx& s) {
  const double af = hypot(f.x, f.y), ag = hypot(g.x, g.y);
  if (ag == 0.0) {
    c = 1.0;
    s = mk(0.0, 0.0);
    return;
  }
  if (af == 0.0) {
    c = 0.0;
    s = mk(g.x / ag, -g.y / ag);  // conj(g) / |g|
    return;
  }
  const double nrm = hypot(af, ag);
  c = af / nrm;
  const cplx ph = mk(f.x / af, f.y / af);
  s = cscale(cmul(ph, cconj(g)), 1.0 / nrm);
}

// Shifted QR iteration on the upper Hessenberg G (in place -> upper triangular T),
// rotations accumulated into Z.  err[0] = 1 if an eigenvalue needs more than 30 k
// sweeps in all.
__global__ void __launch_bounds__(THREADS) hqr_kernel(cplx* G, cplx* Z, int k, int* err) {
  __shared__ double s_c;
  __shared__ cplx s_s;
  __shared__ int s_lo;
  const int tid = threadIdx.x;
  auto at = [&](int r, int c) -> cplx& { return G[r + (int64_t)c * k]; };
  int hi = k - 1, its = 0;
  long total = 0;
  const long limit = 30L * k + 30;
  while (hi > 0) {
    if (tid == 0) {
      int l = hi;
      while (l > 0) {
        double tst = cabs1(at(l - 1, l - 1)) + cabs1(at(l, l));
        if (tst == 0.0) tst = cabs1(at(l - 1, l)) + cabs1(at(l, l - 1)) + TINY;
        if (cabs1(at(l, l - 1)) <= EPS * tst) {
          at(l, l - 1) = mk(0.0, 0.0);
          break;
        }
        --l;
      }
      s_lo = l;
    }
    __syncthreads();
    const int lo = s_lo;
    __syncthreads();
    if (lo == hi) {
      --hi;
      its = 0;
      continue;
    }
    if (++total > limit) {
      if (tid == 0) err[0] = 1;
      return;
    }
    ++its;
    if (tid == 0) {
      cplx mu;
      const cplx a = at(hi - 1, hi - 1), b = at(hi - 1, hi), cc = at(hi, hi - 1), d = at(hi, hi);
      if (its == 10 || its == 20) {
        // exceptional shift
        mu = cadd(d, mk(0.75 * cabs1(cc), 0.0));
      } else {
        // the eigenvalue of the trailing 2 x 2 block closer to d
        const cplx hd = cscale(csub(a, d), 0.5);
        const cplx disc = csqrtz(cadd(cmul(hd, hd), cmul(b, cc)));
        const cplx m1 = cadd(cscale(cadd(a, d), 0.5), disc), m2 = csub(cscale(cadd(a, d), 0.5), disc);
        mu = cabs1(csub(m1, d)) <= cabs1(csub(m2, d)) ? m1 : m2;
      }
      double c;
      cplx s;
      givens(csub(at(lo, lo), mu), at(lo + 1, lo), c, s);
      s_c = c;
      s_s = s;
    }
    for (int i = lo; i < hi; ++i) {
      __syncthreads();
      const double c = s_c;
      const cplx s = s_s, cs = cconj(s);
      // rows i, i+1 (columns from the bulge on, through the whole Schur form)
      const int c0 = i > lo ? i - 1 : lo;
      for (int col = c0 + tid; col < k; col += THREADS) {
        const cplx x = at(i, col), y = at(i + 1, col);
        at(i, col) = cadd(cscale(x, c), cmul(s, y));
        // the bulge entry (i+1, i-1) is annihilated: store the exact zero
        at(i + 1, col) = (i > lo && col == i - 1) ? mk(0.0, 0.0) : csub(cscale(y, c), cmul(cs, x));
      }
      __syncthreads();
      // columns i, i+1 of G (rows 0 .. min(i+2, hi)) and of Z (all rows)
      const int rmax = min(i + 2, hi);
      for (int r = tid; r <= rmax + k; r += THREADS) {
        cplx* M = r <= rmax ? G : Z;
        const int rr = r <= rmax ? r : r - rmax - 1;
        if (rr >= k) continue;
        cplx& x = M[rr + (int64_t)i * k];
        cplx& y = M[rr + (int64_t)(i + 1) * k];
        const cplx xv = x, yv = y;
        x = cadd(cscale(xv, c), cmul(cs, yv));
        y = csub(cscale(yv, c), cmul(s, xv));
      }
      __syncthreads();
      if (tid == 0 && i + 1 < hi) {
        double c2;
        cplx s2;
        givens(at(i + 1, i), at(i + 2, i), c2, s2);
        s_c = c2;
        s_s = s2;
      }
    }
    __syncthreads();
  }
}

// Eigenvectors of the upper triangular T: column i of X solves (T - t_ii I) x = 0 with
// x_i = 1 and x_r = 0 below i (one thread per eigenvector).  Near-zero pivots are
// replaced by smin = max(EPS * max|t_rr|, TINY).
__global__ void trevc_kernel(const cplx* T, int k, cplx* X) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= k) return;
  double tmax = 0.0;
  for (int r = 0; r < k; ++r) tmax = fmax(tmax, cabs1(T[r + (int64_t)r * k]));
  const double smin = fmax(EPS * tmax, TINY);
  cplx* x = X + (int64_t)i * k;
  for (int r = i + 1; r < k; ++r) x[r] = mk(0.0, 0.0);
  x[i] = mk(1.0, 0.0);
  const cplx lam = T[i + (int64_t)i * k];
  for (int r = i - 1; r >= 0; --r) {
    cplx sum = mk(0.0, 0.0);
    for (int c = r + 1; c <= i; ++c) cfma(sum, T[r + (int64_t)c * k], x[c]);
    cplx d = csub(T[r + (int64_t)r * k], lam);
    if (cabs1(d) < smin) d = mk(smin, 0.0);
    x[r] = cdivz(mk(-sum.x, -sum.y), d);
  }
}

__global__ void diag_kernel(const cplx* T, int k, cplx* lam) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < k) lam[i] = T[i + (int64_t)i * k];
}

// out = S Q (rows n .. 2n-1 negated), 2n x k
__global__ void sflip_kernel(const cplx* Q, int64_t n, int64_t k, cplx* out) {
  const int64_t total = 2 * n * k;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const cplx q = Q[i];
    out[i] = (i % (2 * n)) >= n ? mk(-q.x, -q.y) : q;
  }
}
// D[i] = M[i, i]; M's diagonal set to zero (k x k)
__global__ void split_diag_kernel(cplx* M, int64_t k, cplx* D) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < k) {
    D[i] = M[i + i * k];
    M[i + i * k] = mk(0.0, 0.0);
  }
}
// column j of X divided by the real number d[j].x
__global__ void scale_cols_kernel(cplx* X, int64_t rows, int64_t k, const cplx* d) {
  const int64_t total = rows * k;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x)
    X[i] = cscale(X[i], 1.0 / d[i / rows].x);
}

}  // namespace gv

int geev(const cplx* G, int64_t k, cplx* lam, cplx* V, cudaStream_t s) {
  if (k <= 0) return CHASE_BSE_OK;
  if (k > (int64_t)1 << 15) return CHASE_BSE_BAD_ARG;
  Workspace ws(s);
  cplx *T, *Z, *X, *v;
  int* err;
  CB_TRY(ws.alloc(&T, k * k));
  CB_TRY(ws.alloc(&Z, k * k));
  CB_TRY(ws.alloc(&X, k * k));
  CB_TRY(ws.alloc(&v, k));
  CB_TRY(ws.alloc(&err, 1));
  CB_CUDA(cudaMemsetAsync(err, 0, sizeof(int), s));
  CB_CUDA(cudaMemcpyAsync(T, G, sizeof(cplx) * k * k, cudaMemcpyDeviceToDevice, s));
  gv::hess_kernel<<<1, gv::THREADS, 0, s>>>(T, Z, (int)k, v);
  count_launch();
  CB_LAUNCH();
  gv::hqr_kernel<<<1, gv::THREADS, 0, s>>>(T, Z, (int)k, err);
  count_launch();
  CB_LAUNCH();
  gv::diag_kernel<<<cdiv(k, 256), 256, 0, s>>>(T, (int)k, lam);
  count_launch();
  gv::trevc_kernel<<<cdiv(k, 128), 128, 0, s>>>(T, (int)k, X);
  count_launch();
  CB_LAUNCH();
  CB_TRY(zgemm('N', 'N', k, k, k, mk(1.0, 0.0), Z, k, X, k, mk(0.0, 0.0), V, k, s));
  CB_TRY(normalize_cols(V, k, k, s));
  int herr = 0;
  CB_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s));
  CB_CUDA(cudaStreamSynchronize(s));
  return herr ? CHASE_BSE_NOT_CONVERGED : CHASE_BSE_OK;
}

// Non-hermitian fallback Rayleigh-Ritz (Section 4.4, last paragraph) on Q (2n x k,
// orthonormal columns): M = Q^* S Q, the dual basis Q_L = (S Q - Q (M - diag M))
// diag(M)^{-1} (Q_L^* Q = I whenever diag(M) has no zero, M itself may be singular),
// G = Q_L^* H Q, G Z = Z diag(lam) by geev, and the Ritz pairs with positive real
// part in ascending order: ritz_host[0 .. *npos) and W = Q Z_+ (2n x *npos, unit
// columns).  A zero (or non-real) diagonal entry of M returns QR_FAILED.
int rayleigh_ritz_fallback(const cplx* A, const cplx* B, int64_t n, const cplx* Q, int64_t k, double* ritz_host,
                           cplx* W, int64_t* npos, cudaStream_t s) {
  *npos = 0;
  if (k <= 0) return CHASE_BSE_OK;
  const int64_t n2 = 2 * n;
  Workspace ws(s);
  cplx *SQ, *M, *D, *HQ, *G, *lam, *Z, *Zp;
  int* didx;
  CB_TRY(ws.alloc(&SQ, n2 * k));
  CB_TRY(ws.alloc(&M, k * k));
  CB_TRY(ws.alloc(&D, k));
  CB_TRY(ws.alloc(&HQ, n2 * k));
  CB_TRY(ws.alloc(&G, k * k));
  CB_TRY(ws.alloc(&lam, k));
  CB_TRY(ws.alloc(&Z, k * k));
  CB_TRY(ws.alloc(&Zp, k * k));
  CB_TRY(ws.alloc(&didx, k));
  const unsigned gb = (unsigned)std::min<int64_t>((n2 * k + 255) / 256, 8192);
  gv::sflip_kernel<<<gb, 256, 0, s>>>(Q, n, k, SQ);
  count_launch();
  CB_LAUNCH();
  CB_TRY(zgemm('C', 'N', k, k, n2, mk(1.0, 0.0), Q, n2, SQ, n2, mk(0.0, 0.0), M, k, s));
  gv::split_diag_kernel<<<cdiv(k, 256), 256, 0, s>>>(M, k, D);
  count_launch();
  CB_LAUNCH();
  std::vector<cplx> dh(k);
  CB_CUDA(cudaMemcpyAsync(dh.data(), D, sizeof(cplx) * k, cudaMemcpyDeviceToHost, s));
  CB_CUDA(cudaStreamSynchronize(s));
  double dmax = 0.0;
  for (const cplx& d : dh) dmax = std::max(dmax, std::fabs(d.x));
  for (const cplx& d : dh)
    if (!(std::fabs(d.x) > 1e-14 * dmax) || !(std::fabs(d.y) <= 1e-10 * std::fabs(d.x))) return CHASE_BSE_QR_FAILED;
  // Q_L = (S Q - Q Moff) diag(d)^{-1}, built in SQ
  CB_TRY(zgemm('N', 'N', n2, k, k, mk(-1.0, 0.0), Q, n2, M, k, mk(1.0, 0.0), SQ, n2, s));
  gv::scale_cols_kernel<<<gb, 256, 0, s>>>(SQ, n2, k, D);
  count_launch();
  CB_LAUNCH();
  HopArgs h{};
  h.A = A; h.B = B; h.n = n; h.W = Q; h.k = k; h.out = HQ; h.mode = HOP_STORE;
  CB_TRY(hop_fp64(h, s));
  CB_TRY(zgemm('C', 'N', k, k, n2, mk(1.0, 0.0), SQ, n2, HQ, n2, mk(0.0, 0.0), G, k, s));
  const int st = geev(G, k, lam, Z, s);
  if (st != CHASE_BSE_OK) return st;
  std::vector<cplx> lh(k);
  CB_CUDA(cudaMemcpyAsync(lh.data(), lam, sizeof(cplx) * k, cudaMemcpyDeviceToHost, s));
  CB_CUDA(cudaStreamSynchronize(s));
  std::vector<int> pos;
  for (int64_t i = 0; i < k; ++i)
    if (lh[i].x > 0.0) pos.push_back((int)i);
  std::stable_sort(pos.begin(), pos.end(), [&](int a, int b) { return lh[a].x < lh[b].x; });
  const int64_t m = (int64_t)pos.size();
  *npos = m;
  if (m == 0) return CHASE_BSE_OK;
  for (int64_t i = 0; i < m; ++i) ritz_host[i] = lh[pos[i]].x;
  CB_CUDA(cudaMemcpyAsync(didx, pos.data(), sizeof(int) * m, cudaMemcpyHostToDevice, s));
  CB_TRY(gather_cols(Zp, Z, didx, k, m, s));
  CB_TRY(zgemm('N', 'N', n2, m, k, mk(1.0, 0.0), Q, n2, Zp, k, mk(0.0, 0.0), W, n2, s));
  CB_TRY(normalize_cols(W, n2, m, s));
  CB_CUDA(cudaStreamSynchronize(s));  // pos must outlive the copy
  return CHASE_BSE_OK;
}

}  // namespace cb
