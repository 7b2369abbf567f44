// FP64 kernels of the ChASE-BSE library.
//
// On GB300 the FP64 pipe runs at ~1/64 of the FP32 rate (measured: 1.20 TFLOP/s
// with DFMA, 1.05 TFLOP/s with DMMA mma.sync.m8n8k4), so an FP64 product of an
// n x 2n matrix with even a handful of vectors is bound by the FP64 pipe, not by
// HBM.  The kernels below therefore use plain DFMA with register tiles and keep
// the shared-memory staging simple; what matters is enough independent FMAs in
// flight per SM sub-partition.
#include "fp64_kernels.cuh"

namespace cb {

// ---------------------------------------------------------------------------
// H application.  One CTA computes a BM-row slice of P W_hat for BNW columns of
// W, i.e. 2*BNW complex outputs per row: the top half (H W)_top = P W and the
// bottom half (H W)_bot = -conj(P [conj(Y); conj(X)]).  The K loop runs over
// the 2n columns of P = [A | B]; the second operand is built on the fly from W
// with the half-swap and conjugation, so W_hat is never stored.
// Epilogue of the H application for output row i (< n) of column j: C1 = (P w)_i,
// C2 = (P u)_i, so (H w)_top(i) = C1 and (H w)_bot(i) = -conj(C2).
__device__ __forceinline__ void hop_epilogue(const HopArgs& a, int64_t i, int64_t j, cplx c1, cplx c2) {
  const int64_t n = a.n, n2 = 2 * a.n;
  const cplx top = c1;
  const cplx bot = mk(-c2.x, c2.y);  // -conj(C2)
  const int64_t ot = j * n2 + i, ob = j * n2 + n + i;
  if (a.mode == HOP_STORE) {
    a.out[ot] = top;
    a.out[ob] = a.sflip ? mk(-bot.x, -bot.y) : bot;
  } else if (a.mode == HOP_CHEB) {
    cplx t = csub(top, cscale(a.Wc[ot], a.c));
    cplx b = csub(bot, cscale(a.Wc[ob], a.c));
    t = cscale(t, a.alpha);
    b = cscale(b, a.alpha);
    if (a.beta != 0.0) {
      t = cadd(t, cscale(a.Wp[ot], a.beta));
      b = cadd(b, cscale(a.Wp[ob], a.beta));
    }
    a.out[ot] = t;
    a.out[ob] = b;
  } else {  // HOP_RESID
    const double lam = a.lambda[j];
    a.out[ot] = csub(top, cscale(a.W[ot], lam));
    a.out[ob] = csub(bot, cscale(a.W[ob], lam));
  }
}

// part != NULL: K split over blockIdx.z in chunks of kchunk columns of P.
template <int BM, int BNW, int TM, int TNW, int BK>
__global__ void __launch_bounds__((BM / TM) * (BNW / TNW))
hop_kernel(HopArgs a, cplx* part, int64_t kchunk) {
  constexpr int TY = BM / TM;
  constexpr int TX = BNW / TNW;
  constexpr int NT = TX * TY;
  __shared__ cplx Ps[BK][BM];
  __shared__ cplx W1s[BK][BNW];
  __shared__ cplx W2s[BK][BNW];
  const int tid = threadIdx.x;
  const int ty = tid % TY;
  const int tx = tid / TY;
  const int64_t n = a.n, n2 = 2 * a.n;
  const int64_t row0 = (int64_t)blockIdx.x * BM;
  const int64_t col0 = (int64_t)blockIdx.y * BNW;

  cplx acc1[TM][TNW], acc2[TM][TNW];
#pragma unroll
  for (int r = 0; r < TM; ++r)
#pragma unroll
    for (int c = 0; c < TNW; ++c) { acc1[r][c] = mk(0, 0); acc2[r][c] = mk(0, 0); }

  const int64_t kbeg = part ? (int64_t)blockIdx.z * kchunk : 0;
  const int64_t kend = part ? (kbeg + kchunk < n2 ? kbeg + kchunk : n2) : n2;
  for (int64_t kb = kbeg; kb < kend; kb += BK) {
    for (int idx = tid; idx < BM * BK; idx += NT) {
      const int r = idx / BK, cc = idx % BK;
      const int64_t gi = row0 + r, gl = kb + cc;
      cplx v = mk(0, 0);
      if (gi < n && gl < kend) v = (gl < n) ? a.A[gi * n + gl] : a.B[gi * n + (gl - n)];
      Ps[cc][r] = v;
    }
    for (int idx = tid; idx < BNW * BK; idx += NT) {
      const int j = idx / BK, l = idx % BK;
      const int64_t gj = col0 + j, gl = kb + l;
      cplx v1 = mk(0, 0), v2 = mk(0, 0);
      if (gj < a.k && gl < kend) {
        const cplx* w = a.W + gj * n2;
        v1 = w[gl];
        v2 = cconj(w[gl < n ? gl + n : gl - n]);
      }
      W1s[l][j] = v1;
      W2s[l][j] = v2;
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < BK; ++kk) {
      cplx p[TM], w1[TNW], w2[TNW];
#pragma unroll
      for (int r = 0; r < TM; ++r) p[r] = Ps[kk][ty + TY * r];
#pragma unroll
      for (int c = 0; c < TNW; ++c) { w1[c] = W1s[kk][tx + TX * c]; w2[c] = W2s[kk][tx + TX * c]; }
#pragma unroll
      for (int r = 0; r < TM; ++r)
#pragma unroll
        for (int c = 0; c < TNW; ++c) { cfma(acc1[r][c], p[r], w1[c]); cfma(acc2[r][c], p[r], w2[c]); }
    }
    __syncthreads();
  }

#pragma unroll
  for (int r = 0; r < TM; ++r) {
#pragma unroll
    for (int c = 0; c < TNW; ++c) {
      const int64_t i = row0 + ty + TY * r;
      const int64_t j = col0 + tx + TX * c;
      if (i >= n || j >= a.k) continue;
      if (part) {  // split K: raw partial sums of P W and P U for this K chunk
        cplx* p = part + (int64_t)blockIdx.z * (2 * n * a.k) + j * n2;
        p[i] = acc1[r][c];
        p[n + i] = acc2[r][c];
      } else {
        hop_epilogue(a, i, j, acc1[r][c], acc2[r][c]);
      }
    }
  }
}

template <int BM, int BNW>
__global__ void hop_reduce_kernel(HopArgs a, const cplx* part, int nsplit) {
  const int64_t n = a.n, n2 = 2 * n, total = n * a.k;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = idx % n, j = idx / n;
    cplx c1 = mk(0, 0), c2 = mk(0, 0);
    for (int z = 0; z < nsplit; ++z) {
      const cplx* p = part + (int64_t)z * (2 * n * a.k) + j * n2;
      c1 = cadd(c1, p[i]);
      c2 = cadd(c2, p[n + i]);
    }
    hop_epilogue(a, i, j, c1, c2);
  }
}

static int num_sms() {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                 cudaSuccess || sms <= 0)
      sms = 148;
  }
  return sms;
}

// Number of K chunks so that a small output grid still fills the GPU (two CTAs per
// SM); 1 when the grid is large enough or K too short to split.
static int64_t split_count(int64_t tiles, int64_t K, int64_t min_chunk) {
  const int64_t want = 2 * (int64_t)num_sms();
  if (tiles >= want || K < 2 * min_chunk) return 1;
  int64_t s = (want + tiles - 1) / tiles;
  if (s > K / min_chunk) s = K / min_chunk;
  return s < 1 ? 1 : s;
}

template <int BM, int BNW, int TM, int TNW>
static int hop_launch(const HopArgs& a, cudaStream_t s) {
  const int64_t tiles = (int64_t)cdiv(a.n, BM) * cdiv(a.k, BNW);
  const int64_t n2 = 2 * a.n;
  const int64_t nsplit = a.no_split ? 1 : split_count(tiles, n2, 256);
  if (nsplit <= 1) {
    dim3 grid(cdiv(a.n, BM), cdiv(a.k, BNW));
    const int64_t tid = timer_begin(1, 32.0 * (double)a.n * (double)a.n * (double)a.k, s);
    hop_kernel<BM, BNW, TM, TNW, 16><<<grid, (BM / TM) * (BNW / TNW), 0, s>>>(a, nullptr, 0);
    timer_end(tid, s);
    count_launch();
    CB_LAUNCH();
    return CHASE_BSE_OK;
  }
  const int64_t kchunk = ((n2 + nsplit - 1) / nsplit + 15) / 16 * 16;
  const int64_t ns = (n2 + kchunk - 1) / kchunk;
  cplx* part = nullptr;
  CB_CUDA(dalloc(&part, sizeof(cplx) * ns * 2 * a.n * a.k, s));
  dim3 grid(cdiv(a.n, BM), cdiv(a.k, BNW), (unsigned)ns);
  // the split product and its reduction: one H application
  const int64_t tid = timer_begin(1, 32.0 * (double)a.n * (double)a.n * (double)a.k, s);
  hop_kernel<BM, BNW, TM, TNW, 16><<<grid, (BM / TM) * (BNW / TNW), 0, s>>>(a, part, kchunk);
  count_launch();
  const int64_t total = a.n * a.k;
  const unsigned rb = (unsigned)((total + 255) / 256 < 8192 ? (total + 255) / 256 : 8192);
  hop_reduce_kernel<BM, BNW><<<rb, 256, 0, s>>>(a, part, (int)ns);
  timer_end(tid, s);
  count_launch();
  cudaError_t e = cudaGetLastError();
  cudaFreeAsync(part, s);
  if (e != cudaSuccess) return CHASE_BSE_CUDA_ERROR;
  return CHASE_BSE_OK;
}

// y = [A | B] [x; conj(x)] for k vectors x (n x k, ld n).  part != NULL: K split.
template <int BM, int BNW, int TM, int TNW, int BK>
__global__ void __launch_bounds__((BM / TM) * (BNW / TNW))
hop_top_kernel(const cplx* __restrict__ A, const cplx* __restrict__ B, int64_t n, const cplx* __restrict__ X,
               int64_t k, cplx* Y, cplx* part, int64_t kchunk) {
  constexpr int TY = BM / TM;
  constexpr int TX = BNW / TNW;
  constexpr int NT = TX * TY;
  __shared__ cplx Ps[BK][BM];
  __shared__ cplx Ws[BK][BNW];
  const int tid = threadIdx.x;
  const int ty = tid % TY;
  const int tx = tid / TY;
  const int64_t n2 = 2 * n;
  const int64_t row0 = (int64_t)blockIdx.x * BM;
  const int64_t col0 = (int64_t)blockIdx.y * BNW;
  const int64_t kbeg = part ? (int64_t)blockIdx.z * kchunk : 0;
  const int64_t kend = part ? (kbeg + kchunk < n2 ? kbeg + kchunk : n2) : n2;
  cplx acc[TM][TNW];
#pragma unroll
  for (int r = 0; r < TM; ++r)
#pragma unroll
    for (int c = 0; c < TNW; ++c) acc[r][c] = mk(0, 0);
  for (int64_t kb = kbeg; kb < kend; kb += BK) {
    for (int idx = tid; idx < BM * BK; idx += NT) {
      const int r = idx / BK, cc = idx % BK;
      const int64_t gi = row0 + r, gl = kb + cc;
      cplx v = mk(0, 0);
      if (gi < n && gl < kend) v = (gl < n) ? A[gi * n + gl] : B[gi * n + (gl - n)];
      Ps[cc][r] = v;
    }
    for (int idx = tid; idx < BNW * BK; idx += NT) {
      const int j = idx / BK, l = idx % BK;
      const int64_t gj = col0 + j, gl = kb + l;
      cplx v = mk(0, 0);
      if (gj < k && gl < kend) v = (gl < n) ? X[gj * n + gl] : cconj(X[gj * n + (gl - n)]);
      Ws[l][j] = v;
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < BK; ++kk) {
      cplx p[TM], w[TNW];
#pragma unroll
      for (int r = 0; r < TM; ++r) p[r] = Ps[kk][ty + TY * r];
#pragma unroll
      for (int c = 0; c < TNW; ++c) w[c] = Ws[kk][tx + TX * c];
#pragma unroll
      for (int r = 0; r < TM; ++r)
#pragma unroll
        for (int c = 0; c < TNW; ++c) cfma(acc[r][c], p[r], w[c]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < TM; ++r)
#pragma unroll
    for (int c = 0; c < TNW; ++c) {
      const int64_t i = row0 + ty + TY * r, j = col0 + tx + TX * c;
      if (i >= n || j >= k) continue;
      if (part) part[(int64_t)blockIdx.z * n * k + j * n + i] = acc[r][c];
      else Y[j * n + i] = acc[r][c];
    }
}

__global__ void sum_parts_kernel(const cplx* part, int nsplit, int64_t total, cplx* Y) {
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    cplx v = mk(0, 0);
    for (int z = 0; z < nsplit; ++z) v = cadd(v, part[(int64_t)z * total + idx]);
    Y[idx] = v;
  }
}

int hop_top_fp64(const cplx* A, const cplx* B, int64_t n, const cplx* X, int64_t k, cplx* Y, cudaStream_t s) {
  if (k <= 0 || n <= 0) return CHASE_BSE_OK;
  constexpr int BM = 64, BNW = 64, TM = 4, TNW = 4;
  const int64_t tiles = (int64_t)cdiv(n, BM) * cdiv(k, BNW);
  const int64_t n2 = 2 * n;
  const int64_t nsplit = split_count(tiles, n2, 256);
  dim3 grid(cdiv(n, BM), cdiv(k, BNW));
  if (nsplit <= 1) {
    hop_top_kernel<BM, BNW, TM, TNW, 16><<<grid, 256, 0, s>>>(A, B, n, X, k, Y, nullptr, 0);
    count_launch();
    CB_LAUNCH();
    return CHASE_BSE_OK;
  }
  const int64_t kchunk = ((n2 + nsplit - 1) / nsplit + 15) / 16 * 16;
  const int64_t ns = (n2 + kchunk - 1) / kchunk;
  cplx* part = nullptr;
  CB_CUDA(dalloc(&part, sizeof(cplx) * ns * n * k, s));
  grid.z = (unsigned)ns;
  hop_top_kernel<BM, BNW, TM, TNW, 16><<<grid, 256, 0, s>>>(A, B, n, X, k, Y, part, kchunk);
  count_launch();
  const int64_t total = n * k;
  sum_parts_kernel<<<(unsigned)((total + 255) / 256 < 8192 ? (total + 255) / 256 : 8192), 256, 0, s>>>(
      part, (int)ns, total, Y);
  count_launch();
  cudaError_t e = cudaGetLastError();
  cudaFreeAsync(part, s);
  if (e != cudaSuccess) return CHASE_BSE_CUDA_ERROR;
  return CHASE_BSE_OK;
}

int hop_fp64(const HopArgs& a, cudaStream_t s) {
  if (a.k <= 0 || a.n <= 0) return CHASE_BSE_OK;
  if (a.k <= 4) return hop_launch<64, 4, 1, 1>(a, s);
  return hop_launch<64, 32, 4, 2>(a, s);
}

// ---------------------------------------------------------------------------
// Generic complex GEMM, column-major.
__device__ __forceinline__ cplx load_op(const cplx* X, int64_t ld, char op, int64_t r, int64_t c) {
  // element (r, c) of op(X)
  if (op == 'N') return X[r + c * ld];
  const cplx v = X[c + r * ld];
  return op == 'C' ? cconj(v) : v;
}

// kchunk > 0: K split over blockIdx.z; block z writes alpha * its partial product to
// C + z * ldc * N (beta ignored).
template <int BM, int BN, int TM, int TN, int BK>
__global__ void __launch_bounds__((BM / TM) * (BN / TN))
zgemm_kernel(char opA, char opB, int64_t M, int64_t N, int64_t K, cplx alpha, const cplx* __restrict__ A,
             int64_t lda, const cplx* __restrict__ B, int64_t ldb, cplx beta, cplx* C, int64_t ldc, int64_t kchunk) {
  constexpr int TY = BM / TM;
  constexpr int TX = BN / TN;
  constexpr int NT = TX * TY;
  __shared__ cplx As[BK][BM];
  __shared__ cplx Bs[BK][BN];
  const int tid = threadIdx.x;
  const int ty = tid % TY;
  const int tx = tid / TY;
  const int64_t row0 = (int64_t)blockIdx.x * BM;
  const int64_t col0 = (int64_t)blockIdx.y * BN;
  cplx acc[TM][TN];
#pragma unroll
  for (int r = 0; r < TM; ++r)
#pragma unroll
    for (int c = 0; c < TN; ++c) acc[r][c] = mk(0, 0);

  const int64_t kbeg = kchunk ? (int64_t)blockIdx.z * kchunk : 0;
  const int64_t kend = kchunk ? (kbeg + kchunk < K ? kbeg + kchunk : K) : K;
  if (kchunk) {
    C += (int64_t)blockIdx.z * ldc * N;
    beta = mk(0, 0);
  }
  for (int64_t kb = kbeg; kb < kend; kb += BK) {
    for (int idx = tid; idx < BM * BK; idx += NT) {
      int r, l;
      if (opA == 'N') { r = idx % BM; l = idx / BM; } else { l = idx % BK; r = idx / BK; }
      const int64_t gr = row0 + r, gl = kb + l;
      As[l][r] = (gr < M && gl < kend) ? load_op(A, lda, opA, gr, gl) : mk(0, 0);
    }
    for (int idx = tid; idx < BN * BK; idx += NT) {
      int c, l;
      if (opB == 'N') { l = idx % BK; c = idx / BK; } else { c = idx % BN; l = idx / BN; }
      const int64_t gc = col0 + c, gl = kb + l;
      Bs[l][c] = (gc < N && gl < kend) ? load_op(B, ldb, opB, gl, gc) : mk(0, 0);
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < BK; ++kk) {
      cplx av[TM], bv[TN];
#pragma unroll
      for (int r = 0; r < TM; ++r) av[r] = As[kk][ty + TY * r];
#pragma unroll
      for (int c = 0; c < TN; ++c) bv[c] = Bs[kk][tx + TX * c];
#pragma unroll
      for (int r = 0; r < TM; ++r)
#pragma unroll
        for (int c = 0; c < TN; ++c) cfma(acc[r][c], av[r], bv[c]);
    }
    __syncthreads();
  }
  const bool use_beta = (beta.x != 0.0 || beta.y != 0.0);
#pragma unroll
  for (int r = 0; r < TM; ++r) {
#pragma unroll
    for (int c = 0; c < TN; ++c) {
      const int64_t i = row0 + ty + TY * r, j = col0 + tx + TX * c;
      if (i >= M || j >= N) continue;
      cplx v = cmul(alpha, acc[r][c]);
      if (use_beta) v = cadd(v, cmul(beta, C[i + j * ldc]));
      C[i + j * ldc] = v;
    }
  }
}

// C = alpha * sum_z part[z] + beta * C
__global__ void zgemm_reduce_kernel(const cplx* part, int nsplit, int64_t M, int64_t N, cplx beta, cplx* C,
                                    int64_t ldc) {
  const int64_t total = M * N;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = idx % M, j = idx / M;
    cplx v = mk(0, 0);
    for (int z = 0; z < nsplit; ++z) v = cadd(v, part[(int64_t)z * M * N + idx]);
    if (beta.x != 0.0 || beta.y != 0.0) v = cadd(v, cmul(beta, C[i + j * ldc]));
    C[i + j * ldc] = v;
  }
}

template <int BM, int BN, int TM, int TN>
static int zgemm_launch(char opA, char opB, int64_t M, int64_t N, int64_t K, cplx alpha, const cplx* A, int64_t lda,
                        const cplx* B, int64_t ldb, cplx beta, cplx* C, int64_t ldc, cudaStream_t s) {
  const int64_t tiles = (int64_t)cdiv(M, BM) * cdiv(N, BN);
  const int64_t nsplit = split_count(tiles, K, 512);
  dim3 grid(cdiv(M, BM), cdiv(N, BN));
  if (nsplit <= 1) {
    zgemm_kernel<BM, BN, TM, TN, 8><<<grid, 256, 0, s>>>(opA, opB, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, 0);
    count_launch();
    CB_LAUNCH();
    return CHASE_BSE_OK;
  }
  const int64_t kchunk = ((K + nsplit - 1) / nsplit + 7) / 8 * 8;
  const int64_t ns = (K + kchunk - 1) / kchunk;
  cplx* part = nullptr;
  CB_CUDA(dalloc(&part, sizeof(cplx) * ns * M * N, s));
  grid.z = (unsigned)ns;
  zgemm_kernel<BM, BN, TM, TN, 8><<<grid, 256, 0, s>>>(opA, opB, M, N, K, alpha, A, lda, B, ldb, beta, part, M,
                                                       kchunk);
  count_launch();
  const int64_t total = M * N;
  const unsigned rb = (unsigned)((total + 255) / 256 < 8192 ? (total + 255) / 256 : 8192);
  zgemm_reduce_kernel<<<rb, 256, 0, s>>>(part, (int)ns, M, N, beta, C, ldc);
  count_launch();
  cudaError_t e = cudaGetLastError();
  cudaFreeAsync(part, s);
  if (e != cudaSuccess) return CHASE_BSE_CUDA_ERROR;
  return CHASE_BSE_OK;
}

int zgemm(char opA, char opB, int64_t M, int64_t N, int64_t K, cplx alpha, const cplx* A, int64_t lda,
          const cplx* B, int64_t ldb, cplx beta, cplx* C, int64_t ldc, cudaStream_t s) {
  if (M <= 0 || N <= 0) return CHASE_BSE_OK;
  if (K < 0) K = 0;  // K = 0: C = beta C (empty K loop)
  if (M <= 16 || N <= 16) return zgemm_launch<32, 32, 2, 2>(opA, opB, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, s);
  return zgemm_launch<64, 64, 4, 4>(opA, opB, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, s);
}

}  // namespace cb
