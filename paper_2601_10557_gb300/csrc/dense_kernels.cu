// Small dense FP64 kernels (see dense_kernels.cuh).
#include <cuda_pipeline.h>

#include <mutex>

#include "dense_kernels.cuh"
#include "fp64_kernels.cuh"
#include "coop.cuh"

namespace cb {

static inline unsigned gs(int64_t total) {
  const int64_t b = (total + 255) / 256;
  return (unsigned)(b < 8192 ? (b > 0 ? b : 1) : 8192);
}

namespace {
constexpr int NB = 32;  // Cholesky / triangular-inverse block size

__device__ double block_sum(double v, double* sh) {
  // blockDim.x is a multiple of 32, at most 1024
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  const int nw = blockDim.x >> 5;
  v = (threadIdx.x < nw) ? sh[threadIdx.x] : 0.0;
  if (w == 0)
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if (threadIdx.x == 0) sh[0] = v;
  __syncthreads();
  v = sh[0];
  __syncthreads();
  return v;
}
}  // namespace

// ---------------------------------------------------------------- Cholesky
__global__ void chol_diag_kernel(cplx* G, int64_t ld, int64_t j0, int nb, int* info) {
  __shared__ cplx a[NB][NB + 1];
  const int t = threadIdx.x;
  for (int idx = t; idx < nb * nb; idx += blockDim.x) {
    const int r = idx % nb, c = idx / nb;
    a[r][c] = G[(j0 + r) + (j0 + c) * ld];
  }
  __syncthreads();
  for (int c = 0; c < nb; ++c) {
    if (t == 0) {
      double d = a[c][c].x;
      if (!(d > 0.0)) {
        atomicCAS(info, 0, (int)(j0 + c + 1));
        d = 1.0;
      }
      a[c][c] = mk(sqrt(d), 0.0);
    }
    __syncthreads();
    const double inv = 1.0 / a[c][c].x;
    for (int r = c + 1 + t; r < nb; r += blockDim.x) a[r][c] = cscale(a[r][c], inv);
    __syncthreads();
    const int m = nb - c - 1;
    for (int idx = t; idx < m * m; idx += blockDim.x) {
      const int r = c + 1 + idx % m, q = c + 1 + idx / m;
      if (q <= r) a[r][q] = csub(a[r][q], cmul(a[r][c], cconj(a[q][c])));
    }
    __syncthreads();
  }
  for (int idx = t; idx < nb * nb; idx += blockDim.x) {
    const int r = idx % nb, c = idx / nb;
    G[(j0 + r) + (j0 + c) * ld] = (r >= c) ? a[r][c] : mk(0, 0);
  }
}

__global__ void chol_panel_kernel(cplx* G, int64_t ld, int64_t k, int64_t j0, int nb) {
  __shared__ cplx L11[NB][NB + 1];
  for (int idx = threadIdx.x; idx < nb * nb; idx += blockDim.x) {
    const int r = idx % nb, c = idx / nb;
    L11[r][c] = G[(j0 + r) + (j0 + c) * ld];
  }
  __syncthreads();
  const int64_t r = j0 + nb + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= k) return;
  cplx x[NB];
#pragma unroll
  for (int c = 0; c < NB; ++c) x[c] = (c < nb) ? G[r + (j0 + c) * ld] : mk(0, 0);
#pragma unroll
  for (int c = 0; c < NB; ++c) {
    if (c < nb) {
      cplx v = x[c];
#pragma unroll
      for (int q = 0; q < NB; ++q)
        if (q < c) v = csub(v, cmul(x[q], cconj(L11[c][q])));
      x[c] = cscale(v, 1.0 / L11[c][c].x);
    }
  }
#pragma unroll
  for (int c = 0; c < NB; ++c)
    if (c < nb) G[r + (j0 + c) * ld] = x[c];
}

__global__ void zero_upper_kernel(cplx* G, int64_t k) {
  const int64_t total = k * k;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = i % k, c = i / k;
    if (r < c) G[i] = mk(0, 0);
  }
}

// Right-looking blocked Cholesky (NB-wide block columns) in one cooperative
// kernel: per block column, CTA 0 factors the diagonal block, then every CTA
// takes panel rows (forward substitution against L_JJ^*, as in chol_panel_kernel)
// and finally tiles of the trailing update A22 -= L21 L21^*, with a grid barrier
// after each phase.
// acc - a conj(b); REAL: the operands have zero imaginary parts (4x fewer FP64 instructions)
template <bool REAL>
__device__ __forceinline__ cplx msub_conj(cplx acc, cplx a, cplx b) {
  if (REAL) return mk(fma(-a.x, b.x, acc.x), 0.0);
  return csub(acc, cmul(a, cconj(b)));
}
template <bool REAL>
__device__ __forceinline__ cplx scale_re(cplx a, double s) {
  return REAL ? mk(a.x * s, 0.0) : cscale(a, s);
}

template <bool REAL>
__global__ void chol_coop_kernel(cplx* G, int64_t k, int* info, GridSync* gsync, int* err) {
  __shared__ cplx buf[2][NB][NB + 1];
  auto& a = buf[0];   // diagonal block (phases 1, 2)
  auto& pi = buf[0];  // panel rows of tile row I (phase 3)
  auto& pk = buf[1];  // panel rows of tile column K (phase 3)
  __shared__ double dinv[NB];
  const int t = threadIdx.x;
  const int64_t nb = (k + NB - 1) / NB;
  for (int64_t J = 0; J < nb; ++J) {
    const int64_t j0 = J * NB;
    const int jb = (int)((k - j0) < NB ? (k - j0) : NB);
    if (blockIdx.x == 0) {
      for (int idx = t; idx < jb * jb; idx += blockDim.x) {
        const int r = idx % jb, c = idx / jb;
        a[r][c] = __ldcg(G + (j0 + r) + (j0 + c) * k);
      }
      __syncthreads();
      for (int c = 0; c < jb; ++c) {
        if (t == 0) {
          double d = a[c][c].x;
          if (!(d > 0.0)) {
            atomicCAS(info, 0, (int)(j0 + c + 1));
            d = 1.0;
          }
          const double sd = sqrt(d);
          a[c][c] = mk(sd, 0.0);
          dinv[c] = 1.0 / sd;
        }
        __syncthreads();
        const double inv = dinv[c];
        for (int r = c + 1 + t; r < jb; r += blockDim.x) a[r][c] = scale_re<REAL>(a[r][c], inv);
        __syncthreads();
        const int m = jb - c - 1;
        for (int idx = t; idx < m * m; idx += blockDim.x) {
          const int r = c + 1 + idx % m, q = c + 1 + idx / m;
          if (q <= r) a[r][q] = msub_conj<REAL>(a[r][q], a[r][c], a[q][c]);
        }
        __syncthreads();
      }
      for (int idx = t; idx < jb * jb; idx += blockDim.x) {
        const int r = idx % jb, c = idx / jb;
        G[(j0 + r) + (j0 + c) * k] = (r >= c) ? a[r][c] : mk(0, 0);
      }
    }
    if (!grid_barrier(gsync, err)) return;
    const int64_t rest = k - j0 - jb;
    if (rest > 0) {
      // panel: rows i >= j0 + jb solve x L_JJ^* = a_i (forward substitution)
      for (int idx = t; idx < jb * jb; idx += blockDim.x) {
        const int r = idx % jb, c = idx / jb;
        a[r][c] = __ldcg(G + (j0 + r) + (j0 + c) * k);
      }
      __syncthreads();
      if (t < jb) dinv[t] = 1.0 / a[t][t].x;
      __syncthreads();
      // consecutive rows on consecutive CTAs: the FP64 work spreads over all SMs
      for (int64_t i = j0 + jb + blockIdx.x + (int64_t)gridDim.x * t; i < k; i += (int64_t)gridDim.x * blockDim.x) {
        cplx x[NB];
#pragma unroll
        for (int c = 0; c < NB; ++c) x[c] = (c < jb) ? __ldcg(G + i + (j0 + c) * k) : mk(0, 0);
#pragma unroll
        for (int c = 0; c < NB; ++c) {
          if (c < jb) {
            cplx v = x[c];
#pragma unroll
            for (int q = 0; q < NB; ++q)
              if (q < c) v = msub_conj<REAL>(v, x[q], a[c][q]);
            x[c] = scale_re<REAL>(v, dinv[c]);
          }
        }
#pragma unroll
        for (int c = 0; c < NB; ++c)
          if (c < jb) G[i + (j0 + c) * k] = x[c];
      }
      if (!grid_barrier(gsync, err)) return;
      // trailing update, NB x NB tiles (I, K) with K <= I over the lower triangle
      const int64_t T = (rest + NB - 1) / NB;
      for (int64_t tile = blockIdx.x; tile < T * (T + 1) / 2; tile += gridDim.x) {
        int64_t I = (int64_t)((sqrt(8.0 * (double)tile + 1.0) - 1.0) * 0.5);
        while (I * (I + 1) / 2 > tile) --I;
        while ((I + 1) * (I + 2) / 2 <= tile) ++I;
        const int64_t K = tile - I * (I + 1) / 2;
        const int64_t i0 = j0 + jb + I * NB, c0 = j0 + jb + K * NB;
        const int ib = (int)((k - i0) < NB ? (k - i0) : NB), cbk = (int)((k - c0) < NB ? (k - c0) : NB);
        __syncthreads();
        for (int idx = t; idx < NB * jb; idx += blockDim.x) {
          const int r = idx % NB, q = idx / NB;
          pi[r][q] = (r < ib) ? __ldcg(G + (i0 + r) + (j0 + q) * k) : mk(0, 0);
          pk[r][q] = (r < cbk) ? __ldcg(G + (c0 + r) + (j0 + q) * k) : mk(0, 0);
        }
        __syncthreads();
        for (int idx = t; idx < ib * cbk; idx += blockDim.x) {
          const int r = idx % ib, c = idx / ib;
          if (I == K && c > r) continue;
          cplx acc = __ldcg(G + (i0 + r) + (c0 + c) * k);
          for (int q = 0; q < jb; ++q) acc = msub_conj<REAL>(acc, pi[r][q], pk[c][q]);
          G[(i0 + r) + (c0 + c) * k] = acc;
        }
      }
      if (!grid_barrier(gsync, err)) return;
    }
  }
}

static int coop_grid(const void* kern, int threads, int* grid_out) {
  int dev = 0, sms = 0, per_sm = 0, coop = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, 0);
  if (!coop || per_sm < 1 || sms < 1) return 0;
  *grid_out = sms;  // one CTA per SM: fewer barrier arrivals
  return 1;
}

int cholesky(cplx* G, int64_t k, int* info_dev, int* info_host, cudaStream_t s, bool real) {
  CB_CUDA(cudaMemsetAsync(info_dev, 0, sizeof(int), s));
  int grid = 0;
  const void* kern = real ? (const void*)chol_coop_kernel<true> : (const void*)chol_coop_kernel<false>;
  if (coop_grid(kern, 256, &grid)) {
    GridSync* gsync = nullptr;
    int* err = nullptr;
    CB_CUDA(dalloc(&gsync, sizeof(GridSync), s));
    CB_CUDA(dalloc(&err, sizeof(int), s));
    CB_CUDA(gsync_init(gsync, s));
    CB_CUDA(cudaMemsetAsync(err, 0, sizeof(int), s));
    int64_t kk = k;
    void* args[] = {&G, &kk, &info_dev, &gsync, &err};
    const cudaError_t le = cudaLaunchCooperativeKernel(kern, dim3(grid), dim3(256), args, 0, s);
    if (le != cudaSuccess) cudaGetLastError();
    count_launch();
    zero_upper_kernel<<<cdiv(k * k, 256) < 4096 ? cdiv(k * k, 256) : 4096, 256, 0, s>>>(G, k);
    count_launch();
    int herr = 0;
    CB_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s));
    CB_CUDA(cudaMemcpyAsync(info_host, info_dev, sizeof(int), cudaMemcpyDeviceToHost, s));
    cudaFreeAsync(gsync, s);
    cudaFreeAsync(err, s);
    CB_CUDA(cudaStreamSynchronize(s));
    if (le != cudaSuccess) return CHASE_BSE_CUDA_ERROR;
    return herr ? CHASE_BSE_DEVICE_TIMEOUT : CHASE_BSE_OK;
  }
  for (int64_t j0 = 0; j0 < k; j0 += NB) {
    const int nb = (int)((k - j0) < NB ? (k - j0) : NB);
    chol_diag_kernel<<<1, 256, 0, s>>>(G, k, j0, nb, info_dev);
    count_launch();
    CB_LAUNCH();
    const int64_t rest = k - j0 - nb;
    if (rest > 0) {
      chol_panel_kernel<<<cdiv(rest, 128), 128, 0, s>>>(G, k, k, j0, nb);
      count_launch();
      CB_LAUNCH();
      cplx* L21 = G + (j0 + nb) + j0 * k;
      cplx* A22 = G + (j0 + nb) + (j0 + nb) * k;
      CB_TRY(zgemm('N', 'C', rest, rest, nb, mk(-1, 0), L21, k, L21, k, mk(1, 0), A22, k, s));
    }
  }
  zero_upper_kernel<<<cdiv(k * k, 256) < 4096 ? cdiv(k * k, 256) : 4096, 256, 0, s>>>(G, k);
  count_launch();
  CB_LAUNCH();
  CB_CUDA(cudaMemcpyAsync(info_host, info_dev, sizeof(int), cudaMemcpyDeviceToHost, s));
  CB_CUDA(cudaStreamSynchronize(s));
  return CHASE_BSE_OK;
}

// ------------------------------------------------------ triangular inverse
__global__ void inv_diag_blocks_kernel(const cplx* L, int64_t k, cplx* X) {
  __shared__ cplx a[NB][NB + 1];
  const int64_t j0 = (int64_t)blockIdx.x * NB;
  const int nb = (int)((k - j0) < NB ? (k - j0) : NB);
  for (int idx = threadIdx.x; idx < nb * nb; idx += blockDim.x) {
    const int r = idx % nb, c = idx / nb;
    a[r][c] = L[(j0 + r) + (j0 + c) * k];
  }
  __syncthreads();
  const int c = threadIdx.x;
  if (c >= nb) return;
  cplx x[NB];
#pragma unroll
  for (int r = 0; r < NB; ++r) {
    if (r < nb) {
      cplx v = (r == c) ? mk(1, 0) : mk(0, 0);
#pragma unroll
      for (int q = 0; q < NB; ++q)
        if (q < r && q >= c) v = csub(v, cmul(a[r][q], x[q]));
      // a[r][r] is real and positive (Cholesky factor)
      x[r] = (r >= c) ? cscale(v, 1.0 / a[r][r].x) : mk(0, 0);
    }
  }
#pragma unroll
  for (int r = 0; r < NB; ++r)
    if (r < nb) X[(j0 + r) + (j0 + c) * k] = x[r];
}

// X = L^{-1} by block forward substitution on TCB columns per CTA:
// X_I = L_II^{-1} (E_I - sum_{J < I} L_IJ X_J) for the block rows I below the
// columns' diagonal block, with the inverted diagonal blocks already in X.  The
// CTA keeps its TCB columns of X in shared memory; 256 threads = 32 rows x TCB
// columns x 2 halves of each dot product.  REAL: L has zero imaginary parts.
constexpr int TCB = 4;
template <bool REAL>
__global__ void trinv_cols_kernel(const cplx* __restrict__ L, int64_t k, cplx* X) {
  extern __shared__ cplx xs[];  // k x TCB, xs[l * TCB + c]
  __shared__ cplx red[2][NB][TCB];
  __shared__ cplx rhs[NB][TCB];
  const int t = threadIdx.x, r = t & 31, c = (t >> 5) & (TCB - 1), h = t / (32 * TCB);
  const int64_t c0 = (int64_t)blockIdx.x * TCB;
  const int64_t I0 = c0 / NB, nb = (k + NB - 1) / NB;
  const int64_t lo = I0 * NB, hi0 = ((I0 + 1) * NB < k) ? (I0 + 1) * NB : k;
  for (int64_t idx = t; idx < hi0 * TCB; idx += blockDim.x) {
    const int64_t l = idx / TCB;
    const int cc = (int)(idx % TCB);
    xs[idx] = (l >= lo && c0 + cc < k) ? X[l + (c0 + cc) * k] : mk(0, 0);
  }
  __syncthreads();
  for (int64_t I = I0 + 1; I < nb; ++I) {
    const int64_t i0 = I * NB;
    const int ib = (int)((k - i0) < NB ? (k - i0) : NB);
    const int64_t mid = lo + (i0 - lo) / 2;
    const int64_t from = h ? mid : lo, to = h ? i0 : mid;
    cplx acc = mk(0, 0);
    if (r < ib) {
      const cplx* Lr = L + i0 + r;
      if (REAL) {
        double a = 0.0;
        for (int64_t l = from; l < to; ++l) a = fma(Lr[l * k].x, xs[l * TCB + c].x, a);
        acc = mk(a, 0.0);
      } else {
        for (int64_t l = from; l < to; ++l) acc = cadd(acc, cmul(Lr[l * k], xs[l * TCB + c]));
      }
    }
    red[h][r][c] = acc;
    __syncthreads();
    if (h == 0) rhs[r][c] = mk(-(red[0][r][c].x + red[1][r][c].x), -(red[0][r][c].y + red[1][r][c].y));
    __syncthreads();
    if (h == 0 && r < ib) {
      cplx v = mk(0, 0);
      for (int q = 0; q <= r; ++q) {
        const cplx d = X[(i0 + r) + (i0 + q) * k];
        if (REAL) v.x = fma(d.x, rhs[q][c].x, v.x);
        else v = cadd(v, cmul(d, rhs[q][c]));
      }
      xs[(i0 + r) * TCB + c] = v;
      if (c0 + c < k) X[(i0 + r) + (c0 + c) * k] = v;
    }
    __syncthreads();
  }
}

int tri_inverse(const cplx* L, int64_t k, cplx* X, cplx* T, cudaStream_t s, bool real) {
  CB_CUDA(cudaMemsetAsync(X, 0, sizeof(cplx) * k * k, s));
  const int64_t nblk = (k + NB - 1) / NB;
  inv_diag_blocks_kernel<<<(unsigned)nblk, NB, 0, s>>>(L, k, X);
  count_launch();
  CB_LAUNCH();
  const size_t smem = sizeof(cplx) * (size_t)k * TCB;
  if (smem <= 200 * 1024) {
    static bool attr = false;
    if (!attr) {
      CB_CUDA(cudaFuncSetAttribute(trinv_cols_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
      CB_CUDA(cudaFuncSetAttribute(trinv_cols_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
      attr = true;
    }
    const unsigned grid = (unsigned)((k + TCB - 1) / TCB);
    if (real) trinv_cols_kernel<true><<<grid, 64 * TCB, smem, s>>>(L, k, X);
    else trinv_cols_kernel<false><<<grid, 64 * TCB, smem, s>>>(L, k, X);
    count_launch();
    CB_LAUNCH();
    return CHASE_BSE_OK;
  }
  for (int64_t b = 1; b < nblk; ++b) {
    const int64_t i0 = b * NB;
    const int64_t nbi = (k - i0) < NB ? (k - i0) : NB;
    // T = L[i0:i0+nbi, 0:i0] * X[0:i0, 0:i0]
    CB_TRY(zgemm('N', 'N', nbi, i0, i0, mk(1, 0), L + i0, k, X, k, mk(0, 0), T, nbi, s));
    // X[i0:i0+nbi, 0:i0] = -X_bb * T
    CB_TRY(zgemm('N', 'N', nbi, i0, nbi, mk(-1, 0), X + i0 + i0 * k, k, T, nbi, mk(0, 0), X + i0, k, s));
  }
  return CHASE_BSE_OK;
}

// ------------------------------------------------------------------ Jacobi
// Round-robin (circle) ordering: position 0 holds index 0, position p > 0 holds
// ((p - 1 + r) mod (k - 1)) + 1; slot s pairs positions s and k - 1 - s.
__device__ __forceinline__ void jpair(int64_t slot, int r, int64_t k, int64_t& p, int64_t& q) {
  auto pl = [&](int64_t pos) -> int64_t { return pos == 0 ? 0 : ((pos - 1 + r) % (k - 1)) + 1; };
  const int64_t a = pl(slot), b = pl(k - 1 - slot);
  p = a < b ? a : b;
  q = a < b ? b : a;
}

// Rotation of pair (p, q) of round r.  Entries negligible next to their diagonal
// (|a_pq| <= 1e-17 sqrt|a_pp a_qq|) or to the matrix (|a_pq| <= 1e-18 ||G||_F)
// are skipped (threshold Jacobi); a sweep that applies no rotation ends the
// iteration.  |a_pq| is formed with hypot: squaring entries that have become tiny
// would underflow and make the rotation non-unitary.
__global__ void jacobi_rot_kernel(const cplx* G, int64_t k, int r, cplx* rot, const double* red, int* applied) {
  const int64_t slot = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (slot >= k / 2) return;
  int64_t p, q;
  jpair(slot, r, k, p, q);
  const double app = G[p + p * k].x, aqq = G[q + q * k].x;
  const cplx apq = G[p + q * k];
  const double rr = hypot(apq.x, apq.y);
  const double normG = sqrt(red[1]);
  cplx J00 = mk(1, 0), J01 = mk(0, 0), J10 = mk(0, 0), J11 = mk(1, 0);
  if (rr > 2e-16 * sqrt(fabs(app * aqq)) && rr > 1e-16 * normG && rr > 1e-300) {
    atomicAdd(applied, 1);
    const cplx ec = mk(apq.x / rr, -apq.y / rr);  // conj(e^{i phi})
    const double tau = (aqq - app) / (2.0 * rr);
    const double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + hypot(1.0, tau));
    const double c = 1.0 / hypot(1.0, t), sn = t * c;
    J00 = mk(c, 0);
    J01 = mk(sn, 0);
    J10 = cscale(ec, -sn);
    J11 = cscale(ec, c);
  }
  rot[4 * slot + 0] = J00;
  rot[4 * slot + 1] = J01;
  rot[4 * slot + 2] = J10;
  rot[4 * slot + 3] = J11;
}

__global__ void jacobi_apply_kernel(cplx* G, cplx* V, int64_t k, int r, const cplx* __restrict__ rot) {
  const int64_t half = k / 2;
  const int64_t nG = half * half, nV = k * half;
  for (int64_t item = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; item < nG + nV;
       item += (int64_t)gridDim.x * blockDim.x) {
    if (item < nG) {
      const int64_t a = item % half, b = item / half;
      int64_t pa, qa, pb, qb;
      jpair(a, r, k, pa, qa);
      jpair(b, r, k, pb, qb);
      const cplx A00 = rot[4 * a], A01 = rot[4 * a + 1], A10 = rot[4 * a + 2], A11 = rot[4 * a + 3];
      const cplx B00 = rot[4 * b], B01 = rot[4 * b + 1], B10 = rot[4 * b + 2], B11 = rot[4 * b + 3];
      const cplx x00 = G[pa + pb * k], x01 = G[pa + qb * k], x10 = G[qa + pb * k], x11 = G[qa + qb * k];
      // J_a^* X
      const cplx y00 = cadd(cmul(cconj(A00), x00), cmul(cconj(A10), x10));
      const cplx y01 = cadd(cmul(cconj(A00), x01), cmul(cconj(A10), x11));
      const cplx y10 = cadd(cmul(cconj(A01), x00), cmul(cconj(A11), x10));
      const cplx y11 = cadd(cmul(cconj(A01), x01), cmul(cconj(A11), x11));
      // (.) J_b
      G[pa + pb * k] = cadd(cmul(y00, B00), cmul(y01, B10));
      G[pa + qb * k] = cadd(cmul(y00, B01), cmul(y01, B11));
      G[qa + pb * k] = cadd(cmul(y10, B00), cmul(y11, B10));
      G[qa + qb * k] = cadd(cmul(y10, B01), cmul(y11, B11));
    } else {
      const int64_t it = item - nG;
      const int64_t i = it % k, b = it / k;
      int64_t pb, qb;
      jpair(b, r, k, pb, qb);
      const cplx B00 = rot[4 * b], B01 = rot[4 * b + 1], B10 = rot[4 * b + 2], B11 = rot[4 * b + 3];
      const cplx v0 = V[i + pb * k], v1 = V[i + qb * k];
      V[i + pb * k] = cadd(cmul(v0, B00), cmul(v1, B10));
      V[i + qb * k] = cadd(cmul(v0, B01), cmul(v1, B11));
    }
  }
}

__global__ void offdiag_norm_kernel(const cplx* G, int64_t k, double* red) {
  __shared__ double sh[32];
  double off = 0.0, tot = 0.0;
  for (int64_t i = threadIdx.x; i < k * k; i += blockDim.x) {
    const double v = cabs2(G[i]);
    tot += v;
    if (i % k != i / k) off += v;
  }
  off = block_sum(off, sh);
  tot = block_sum(tot, sh);
  if (threadIdx.x == 0) { red[0] = off; red[1] = tot; }
}

// ---- Jacobi sweeps with one grid barrier per round ------------------------
// A rotation of pair (p, q), p < q, is (c, s, e) with c, s real and |e| = 1:
// J = [[c, s], [-s e, c e]] on columns (p, q); G <- J^* G J and V <- V J.
struct Rot {
  double c, s, er, ei;
};

// 2^-E for a normal m = f 2^E, f in [1, 2) (exact power of two, from the bits)
__device__ __forceinline__ double pow2_inv_exp(double m) {
  const int e = (__double2hiint(m) >> 20) & 0x7ff;
  return __hiloint2double((2046 - e) << 20, 0);
}
// Thresholds of the Jacobi rotations, evaluated once per pair in FP32 on values
// scaled by sn = 2^-E(||G||_F) (all entries are then at most 1 in magnitude):
// rotate when |a_pq| > t sqrt|a_pp a_qq| and |a_pq| > (t/2) ||G||_F, with
// t2a = t^2, t2b = t^2/4 (t = 2e-16 diagonalises to the rounding level).  The
// sweeps and the convergence count use this same predicate.
__device__ __forceinline__ bool jacobi_active(double app, double aqq, cplx apq, double sn, float n2s, float t2a,
                                              float t2b) {
  const float xr = (float)(apq.x * sn), xi = (float)(apq.y * sn);
  const float a1 = (float)(app * sn), a2 = (float)(aqq * sn);
  const float r2 = fmaf(xr, xr, xi * xi);
  return r2 > t2a * fabsf(a1 * a2) && r2 > t2b * n2s && r2 > 0.0f;
}

// Rotation annihilating a_pq (identity below the thresholds).  GB300 issues an
// FP64 warp instruction at 1/64 of the FP32 rate, so the serial chain is kept
// short: t = tan(angle) from an FP32 estimate plus one Newton step on
// t^2 + 2 tau t - 1 = 0 (FP64 class), and c = (1 + t^2)^(-1/2) and 1/|a_pq| from
// FP32 reciprocal square roots refined by two FP64 Newton steps, so that
// c^2 + s^2 = 1 and |e| = 1 hold to FP64 rounding.  a_pq is first scaled by an
// exact power of two to magnitude in [1, 2).
__device__ Rot jacobi_rotation(double app, double aqq, cplx apq, double sn, float n2s, float t2a, float t2b,
                               int* applied) {
  Rot R{1.0, 0.0, 1.0, 0.0};
  if (!jacobi_active(app, aqq, apq, sn, n2s, t2a, t2b)) return R;
  atomicAdd(applied, 1);
  const double sc = pow2_inv_exp(fmax(fabs(apq.x), fabs(apq.y)));
  const double xr = apq.x * sc, xi = apq.y * sc;
  const double r2 = fma(xr, xr, xi * xi);  // in [1, 8)
  double ri = (double)rsqrtf((float)r2);   // 1 / (sc |a_pq|)
  ri = ri * fma(-0.5 * r2, ri * ri, 1.5);
  ri = ri * fma(-0.5 * r2, ri * ri, 1.5);
  R.er = xr * ri;  // e = conj(a_pq) / |a_pq|
  R.ei = -xi * ri;
  const double tau = 0.5 * (aqq - app) * ri * sc;  // (a_qq - a_pp) / (2 |a_pq|), below ~1e16
  const float tf = (float)tau;
  double t = (double)(copysignf(1.0f, tf) / (fabsf(tf) + sqrtf(fmaf(tf, tf, 1.0f))));
  if (fabs(tau) < 1e15) {
    const double f = fma(t, t + 2.0 * tau, -1.0);
    t -= f * (double)(1.0f / (float)(2.0 * (t + tau)));
  }
  const double h = fma(t, t, 1.0);
  double c = (double)rsqrtf((float)h);
  c = c * fma(-0.5 * h, c * c, 1.5);
  c = c * fma(-0.5 * h, c * c, 1.5);
  R.c = c;
  R.s = t * c;
  return R;
}

// rotations written by other CTAs earlier in the same launch: read through L2
__device__ __forceinline__ Rot ld_rot(const Rot* r) {
  const double2 u = __ldcg(reinterpret_cast<const double2*>(r));
  const double2 v = __ldcg(reinterpret_cast<const double2*>(r) + 1);
  return Rot{u.x, u.y, v.x, v.y};
}

// Z = A^* X B for the 2 x 2 block X of rows (pa, qa) and columns (pb, qb).
__device__ __forceinline__ void rot_block(const Rot& A, const Rot& B, const cplx x[4], cplx z[4]) {
  const cplx ea = mk(A.er, -A.ei);  // conj(e_A)
  const cplx w0 = cmul(ea, x[2]), w1 = cmul(ea, x[3]);
  const cplx y00 = mk(A.c * x[0].x - A.s * w0.x, A.c * x[0].y - A.s * w0.y);
  const cplx y01 = mk(A.c * x[1].x - A.s * w1.x, A.c * x[1].y - A.s * w1.y);
  const cplx y10 = mk(A.s * x[0].x + A.c * w0.x, A.s * x[0].y + A.c * w0.y);
  const cplx y11 = mk(A.s * x[1].x + A.c * w1.x, A.s * x[1].y + A.c * w1.y);
  const cplx eb = mk(B.er, B.ei);
  const cplx u0 = cmul(y01, eb), u1 = cmul(y11, eb);
  z[0] = mk(B.c * y00.x - B.s * u0.x, B.c * y00.y - B.s * u0.y);
  z[1] = mk(B.s * y00.x + B.c * u0.x, B.s * y00.y + B.c * u0.y);
  z[2] = mk(B.c * y10.x - B.s * u1.x, B.c * y10.y - B.s * u1.y);
  z[3] = mk(B.s * y10.x + B.c * u1.x, B.s * y10.y + B.c * u1.y);
}
// Diagonal entry i (0: p, 1: q) of J^* X J for the hermitian diagonal block X of (p, q):
// c^2 x_pp + s^2 x_qq -+ 2 c s Re(e x_pq).
__device__ __forceinline__ double rot_diag(const Rot& A, const cplx* G, int k, int p, int q, int i) {
  const double xpp = __ldcg(G + p + (int64_t)p * k).x, xqq = __ldcg(G + q + (int64_t)q * k).x;
  if (A.s == 0.0) return i == 0 ? xpp : xqq;
  const cplx xpq = __ldcg(G + p + (int64_t)q * k);
  const double re = A.er * xpq.x - A.ei * xpq.y;  // Re(e x_pq)
  const double cc = A.c * A.c, ss = A.s * A.s, cs2 = 2.0 * A.c * A.s;
  return i == 0 ? fma(cc, xpp, fma(ss, xqq, -cs2 * re)) : fma(ss, xpp, fma(cc, xqq, cs2 * re));
}
__device__ __forceinline__ void load_block(const cplx* G, int k, int p0, int q0, int p1, int q1, cplx x[4]) {
  x[0] = __ldcg(G + p0 + (int64_t)p1 * k);
  x[1] = __ldcg(G + p0 + (int64_t)q1 * k);
  x[2] = __ldcg(G + q0 + (int64_t)p1 * k);
  x[3] = __ldcg(G + q0 + (int64_t)q1 * k);
}

// One sweep (k - 1 rounds) on G, ping-ponging between Ga (input) and Gb; the
// rotations of every round go to rots[r * k/2 + slot] for the V pass.  Round r
// updates the 2 x 2 blocks (a, b), a >= b, of the pairs of slots a and b (and
// writes the mirrored block); the thread whose block holds the pivot a_xy of a
// pair of round r + 1 also recomputes the two new diagonal entries and writes
// that pair's rotation, so each round needs one grid barrier.
__global__ void jacobi_sweep_kernel(cplx* Ga, cplx* Gb, int k, Rot* rots, const double* red, int* applied,
                                    GridSync* gsync, int* err, float t2a, float t2b) {
  const int half = k / 2;
  const int64_t nblk = (int64_t)half * (half + 1) / 2;
  const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
  const double normG = sqrt(red[1]);
  const double sn = pow2_inv_exp(normG);
  const float n2s = (float)((normG * sn) * (normG * sn));
  // items interleaved over the CTAs: the FP64 work spreads over all SMs
  const int64_t first = (int64_t)threadIdx.x * gridDim.x + blockIdx.x;
  for (int64_t sl = first; sl < half; sl += nthreads) {
    int p, q;
    jpair32((int)sl, 0, k, p, q);
    rots[sl] = jacobi_rotation(__ldcg(Ga + p + (int64_t)p * k).x, __ldcg(Ga + q + (int64_t)q * k).x,
                               __ldcg(Ga + p + (int64_t)q * k), sn, n2s, t2a, t2b, applied);
  }
  if (!grid_barrier(gsync, err)) return;
  for (int r = 0; r < k - 1; ++r) {
    const cplx* Gi = (r & 1) ? Gb : Ga;
    cplx* Go = (r & 1) ? Ga : Gb;
    const Rot* R = rots + (int64_t)r * half;
    for (int64_t item = first; item < nblk; item += nthreads) {
      int a = (int)((sqrtf(8.0f * (float)item + 1.0f) - 1.0f) * 0.5f);
      while ((int64_t)a * (a + 1) / 2 > item) --a;
      while ((int64_t)(a + 1) * (a + 2) / 2 <= item) ++a;
      const int b = (int)(item - (int64_t)a * (a + 1) / 2);
      int pa, qa, pb, qb;
      jpair32(a, r, k, pa, qa);
      jpair32(b, r, k, pb, qb);
      const Rot A = ld_rot(R + a), B = ld_rot(R + b);
      cplx x[4], z[4];
      load_block(Gi, k, pa, qa, pb, qb, x);
      if (A.s == 0.0 && B.s == 0.0) {
        z[0] = x[0]; z[1] = x[1]; z[2] = x[2]; z[3] = x[3];
      } else {
        rot_block(A, B, x, z);
      }
      Go[pa + (int64_t)pb * k] = z[0];
      Go[pa + (int64_t)qb * k] = z[1];
      Go[qa + (int64_t)pb * k] = z[2];
      Go[qa + (int64_t)qb * k] = z[3];
      if (a == b) continue;
      Go[pb + (int64_t)pa * k] = cconj(z[0]);
      Go[qb + (int64_t)pa * k] = cconj(z[1]);
      Go[pb + (int64_t)qa * k] = cconj(z[2]);
      Go[qb + (int64_t)qa * k] = cconj(z[3]);
      if (r + 1 >= k - 1) continue;
#pragma unroll
      for (int ix = 0; ix < 2; ++ix) {
        const int xi = ix == 0 ? pa : qa;
        const int pos = jpos(xi, r + 1, k);
        const int yi = jat(k - 1 - pos, r + 1, k);
        if (yi != pb && yi != qb) continue;
        const int iy = (yi == pb) ? 0 : 1;
        const cplx zxy = z[2 * ix + iy];
        const double dx = rot_diag(A, Gi, k, pa, qa, ix), dy = rot_diag(B, Gi, k, pb, qb, iy);
        const int slot = pos < k - 1 - pos ? pos : k - 1 - pos;
        rots[(int64_t)(r + 1) * half + slot] =
            xi < yi ? jacobi_rotation(dx, dy, zxy, sn, n2s, t2a, t2b, applied)
                    : jacobi_rotation(dy, dx, cconj(zxy), sn, n2s, t2a, t2b, applied);
      }
    }
    if (!grid_barrier(gsync, err)) return;
  }
}

// V <- V J_0 J_1 ... J_{k-2} for the stored rotations of one sweep: one warp per
// row of V (rows are independent), the row in shared memory.
constexpr int VROWS = 2;
__global__ void jacobi_vpass_kernel(cplx* V, int k, const Rot* rots) {
  extern __shared__ cplx vrow[];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t i = (int64_t)blockIdx.x * VROWS + w;
  if (i >= k) return;  // whole warp; no block-wide synchronisation below
  cplx* v = vrow + (int64_t)w * k;
  for (int j = lane; j < k; j += 32) v[j] = V[i + (int64_t)j * k];
  __syncwarp();
  const int half = k / 2;
  for (int r = 0; r < k - 1; ++r) {
    const Rot* R = rots + (int64_t)r * half;
    for (int sl = lane; sl < half; sl += 32) {
      const Rot B = R[sl];
      if (B.s == 0.0) continue;  // identity
      int p, q;
      jpair32(sl, r, k, p, q);
      const cplx vp = v[p], u = cmul(v[q], mk(B.er, B.ei));
      v[p] = mk(B.c * vp.x - B.s * u.x, B.c * vp.y - B.s * u.y);
      v[q] = mk(B.s * vp.x + B.c * u.x, B.s * vp.y + B.c * u.y);
    }
    __syncwarp();
  }
  for (int j = lane; j < k; j += 32) V[i + (int64_t)j * k] = v[j];
}

// The same with the rotations of each round staged in shared memory by cp.async while
// the previous round is applied (the per-round L2 latency is hidden); R rows of V
// per CTA (one warp each) share the staged rotations.
template <int R>
__global__ void jacobi_vpass_staged_kernel(cplx* V, int k, const Rot* rots) {
  extern __shared__ __align__(16) unsigned char vs_raw[];
  const int half = k / 2;
  Rot* rb = reinterpret_cast<Rot*>(vs_raw);                       // [2][half]
  cplx* vrow = reinterpret_cast<cplx*>(rb + 2 * (int64_t)half);   // [R][k]
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t i = (int64_t)blockIdx.x * R + w;
  const bool active = i < k;
  cplx* v = vrow + (int64_t)w * k;
  if (active)
    for (int j = lane; j < k; j += 32) v[j] = V[i + (int64_t)j * k];
  // a round's rotations are half * 32 bytes: 16-byte pieces over the CTA
  auto stage = [&](int r, int buf) {
    const char* src = reinterpret_cast<const char*>(rots + (int64_t)r * half);
    char* dst = reinterpret_cast<char*>(rb + (int64_t)buf * half);
    for (int c = threadIdx.x; c < 2 * half; c += blockDim.x)
      __pipeline_memcpy_async(dst + 16 * c, src + 16 * c, 16);
    __pipeline_commit();
  };
  stage(0, 0);
  for (int r = 0; r < k - 1; ++r) {
    __pipeline_wait_prior(0);
    __syncthreads();  // round r staged; round r - 1 done with the other buffer
    if (r + 1 < k - 1) stage(r + 1, (r + 1) & 1);
    const Rot* Rr = rb + (int64_t)(r & 1) * half;
    if (active) {
      for (int sl = lane; sl < half; sl += 32) {
        const Rot B = Rr[sl];
        if (B.s == 0.0) continue;  // identity
        int p, q;
        jpair32(sl, r, k, p, q);
        const cplx vp = v[p], u = cmul(v[q], mk(B.er, B.ei));
        v[p] = mk(B.c * vp.x - B.s * u.x, B.c * vp.y - B.s * u.y);
        v[q] = mk(B.s * vp.x + B.c * u.x, B.s * vp.y + B.c * u.y);
      }
    }
    __syncwarp();
  }
  if (active)
    for (int j = lane; j < k; j += 32) V[i + (int64_t)j * k] = v[j];
}

// Number of pairs p < q that a sweep would rotate (the thresholds of jacobi_rotation).
__global__ void jacobi_count_kernel(const cplx* G, int k, const double* red, int* count, float t2a, float t2b) {
  const double normG = sqrt(red[1]);
  const double sn = pow2_inv_exp(normG);
  const float n2s = (float)((normG * sn) * (normG * sn));
  const int64_t total = (int64_t)k * k;
  int local = 0;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int p = (int)(idx % k), q = (int)(idx / k);
    if (p >= q) continue;
    if (jacobi_active(G[p + (int64_t)p * k].x, G[q + (int64_t)q * k].x, G[idx], sn, n2s, t2a, t2b)) ++local;
  }
  if (local) atomicAdd(count, local);
}

// A non-blocking stream per device, created on first use, for the captured sweeps.
static cudaStream_t jacobi_stream() {
  static std::mutex mu;
  static cudaStream_t streams[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  std::lock_guard<std::mutex> lock(mu);
  if (!streams[dev] && cudaStreamCreateWithFlags(&streams[dev], cudaStreamNonBlocking) != cudaSuccess)
    return nullptr;
  return streams[dev];
}

int offdiag_norms(const cplx* G, int64_t k, double* red, cudaStream_t s) {
  offdiag_norm_kernel<<<1, 1024, 0, s>>>(G, k, red);
  count_launch();
  CB_LAUNCH();
  return CHASE_BSE_OK;
}

int jacobi_eigh(cplx* G, int64_t k, cplx* V, double* theta, cplx* rot, double* red, int max_sweeps,
                int* sweeps_out, cudaStream_t s, double thr) {
  if (!(thr >= 2e-16)) thr = 2e-16;
  float t2a = (float)(thr * thr), t2b = (float)(0.25 * thr * thr);
  if (k % 2 != 0) return CHASE_BSE_BAD_ARG;
  CB_TRY(set_identity(V, k, s));
  int sweeps = 0;
  const int64_t half = k / 2;
  const int64_t items = half * half + k * half;
  const unsigned gapply = (unsigned)((items + 255) / 256 < 2048 ? (items + 255) / 256 : 2048);
  double hred[2] = {0, 0};
  int* applied = nullptr;
  CB_CUDA(dalloc(&applied, sizeof(int), s));
  offdiag_norm_kernel<<<1, 1024, 0, s>>>(G, k, red);  // red[1] = ||G||_F^2 (invariant)
  count_launch();
  // Preferred: one cooperative launch per sweep (one grid barrier per round),
  // then the V pass over the stored rotations.
  {
    int dev = 0, sms = 0, per_sm = 0, coop = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, jacobi_sweep_kernel, 512, 0);
    // one CTA per SM: every SM's FP64 pipe takes part, one barrier arrival each
    const unsigned grid = (unsigned)(sms > 0 ? sms : 1);
    const size_t vsmem = sizeof(cplx) * (size_t)VROWS * (size_t)k;
    const size_t staged_smem = sizeof(Rot) * 2 * (size_t)half + sizeof(cplx) * 4 * (size_t)k;
    if (coop && per_sm >= 1 && k <= (1 << 20) && vsmem <= 200 * 1024) {
      static bool attr = false;
      if (!attr) {
        CB_CUDA(cudaFuncSetAttribute(jacobi_vpass_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
        CB_CUDA(cudaFuncSetAttribute(jacobi_vpass_staged_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     200 * 1024));
        attr = true;
      }
      GridSync* gsync = nullptr;
      int *err = nullptr, *cnt = nullptr;
      cplx* G2 = nullptr;
      Rot* rots = nullptr;
      CB_CUDA(dalloc(&gsync, sizeof(GridSync), s));
      CB_CUDA(dalloc(&err, sizeof(int), s));
      CB_CUDA(dalloc(&cnt, sizeof(int), s));
      CB_CUDA(dalloc(&G2, sizeof(cplx) * k * k, s));
      CB_CUDA(dalloc(&rots, sizeof(Rot) * (size_t)(k - 1) * half + sizeof(Rot), s));
      CB_CUDA(gsync_init(gsync, s));
      CB_CUDA(cudaMemsetAsync(err, 0, sizeof(int), s));
      int herr = 0, status = CHASE_BSE_OK;
      int hc[2] = {1, 1};
      int ki = (int)k;
      cplx *Ga = G, *Gb = G2;
      // a matrix that is diagonal to the thresholds needs no sweep
      CB_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int), s));
      jacobi_count_kernel<<<gs(k * k), 256, 0, s>>>(Ga, ki, red, cnt, t2a, t2b);
      count_launch();
      CB_CUDA(cudaMemcpyAsync(&hc[1], cnt, sizeof(int), cudaMemcpyDeviceToHost, s));
      CB_CUDA(cudaStreamSynchronize(s));
      for (; hc[1] > 0 && sweeps < max_sweeps; ++sweeps) {
        CB_CUDA(cudaMemsetAsync(applied, 0, sizeof(int), s));
        CB_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int), s));
        void* args[] = {&Ga, &Gb, &ki, &rots, &red, &applied, &gsync, &err, &t2a, &t2b};
        if (cudaLaunchCooperativeKernel((const void*)jacobi_sweep_kernel, dim3(grid), dim3(512), args, 0, s) !=
            cudaSuccess) {
          cudaGetLastError();
          status = CHASE_BSE_CUDA_ERROR;
          break;
        }
        count_launch();
        if (staged_smem <= 200 * 1024)
          jacobi_vpass_staged_kernel<4><<<(unsigned)((k + 3) / 4), 128, staged_smem, s>>>(V, ki, rots);
        else
          jacobi_vpass_kernel<<<(unsigned)((k + VROWS - 1) / VROWS), 32 * VROWS, vsmem, s>>>(V, ki, rots);
        count_launch();
        std::swap(Ga, Gb);  // the last round (k - 2, even) wrote Gb
        jacobi_count_kernel<<<gs(k * k), 256, 0, s>>>(Ga, ki, red, cnt, t2a, t2b);
        count_launch();
        CB_CUDA(cudaMemcpyAsync(&hc[0], applied, sizeof(int), cudaMemcpyDeviceToHost, s));
        CB_CUDA(cudaMemcpyAsync(&hc[1], cnt, sizeof(int), cudaMemcpyDeviceToHost, s));
        CB_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s));
        CB_CUDA(cudaStreamSynchronize(s));
        if (herr) {
          status = CHASE_BSE_DEVICE_TIMEOUT;
          break;
        }
      }
      if (status == CHASE_BSE_OK && Ga != G)
        CB_CUDA(cudaMemcpyAsync(G, Ga, sizeof(cplx) * k * k, cudaMemcpyDeviceToDevice, s));
      cudaFreeAsync(rots, s);
      cudaFreeAsync(G2, s);
      cudaFreeAsync(cnt, s);
      cudaFreeAsync(gsync, s);
      cudaFreeAsync(err, s);
      cudaFreeAsync(applied, s);
      if (status != CHASE_BSE_OK) return status;
      if (sweeps_out) *sweeps_out = sweeps;
      CB_TRY(diag_real(G, k, theta, s));
      CB_CUDA(cudaMemcpyAsync(hred, red, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
      CB_CUDA(cudaStreamSynchronize(s));
      if (hred[1] != hred[1]) return CHASE_BSE_CUDA_ERROR;  // NaN in G
      return CHASE_BSE_OK;
    }
  }
  // Otherwise one sweep (k - 1 rounds, two launches each) is captured once into a CUDA graph
  // on a library stream and replayed per sweep: the rounds are short, so launch
  // overhead would otherwise dominate.  The library stream is ordered after and
  // before the caller's stream with events.
  cudaStream_t js = jacobi_stream();
  if (!js) return CHASE_BSE_CUDA_ERROR;
  cudaEvent_t ev;
  CB_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
  CB_CUDA(cudaEventRecord(ev, s));
  CB_CUDA(cudaStreamWaitEvent(js, ev, 0));
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  CB_CUDA(cudaStreamBeginCapture(js, cudaStreamCaptureModeThreadLocal));
  cudaMemsetAsync(applied, 0, sizeof(int), js);
  for (int r = 0; r < k - 1; ++r) {
    jacobi_rot_kernel<<<cdiv(half, 128), 128, 0, js>>>(G, k, r, rot, red, applied);
    jacobi_apply_kernel<<<gapply, 256, 0, js>>>(G, V, k, r, rot);
  }
  CB_CUDA(cudaStreamEndCapture(js, &graph));
  CB_CUDA(cudaGraphInstantiate(&exec, graph, 0));
  int happ = 1;
  int status = CHASE_BSE_OK;
  for (; sweeps < max_sweeps; ++sweeps) {
    if (cudaGraphLaunch(exec, js) != cudaSuccess) { status = CHASE_BSE_CUDA_ERROR; break; }
    for (int64_t i = 0; i < 2 * (k - 1); ++i) count_launch();
    if (cudaMemcpyAsync(&happ, applied, sizeof(int), cudaMemcpyDeviceToHost, js) != cudaSuccess ||
        cudaStreamSynchronize(js) != cudaSuccess) {
      status = CHASE_BSE_CUDA_ERROR;
      break;
    }
    if (happ == 0) {
      ++sweeps;
      break;
    }
  }
  cudaGraphExecDestroy(exec);
  cudaGraphDestroy(graph);
  CB_CUDA(cudaEventRecord(ev, js));
  CB_CUDA(cudaStreamWaitEvent(s, ev, 0));
  cudaEventDestroy(ev);
  CB_CUDA(cudaMemcpyAsync(hred, red, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
  CB_CUDA(cudaStreamSynchronize(s));
  cudaFreeAsync(applied, s);
  if (status != CHASE_BSE_OK) return status;
  if (sweeps_out) *sweeps_out = sweeps;
  CB_TRY(diag_real(G, k, theta, s));
  if (hred[1] != hred[1]) return CHASE_BSE_CUDA_ERROR;  // NaN in G
  return CHASE_BSE_OK;
}

// --------------------------------------------------------------- Householder
__global__ void hh_reflector_kernel(cplx* X, int64_t N, int64_t j, cplx* Vs, cplx* Us) {
  __shared__ double sh[32];
  const cplx* x = X + j * N;
  double ss = 0.0;
  for (int64_t r = j + threadIdx.x; r < N; r += blockDim.x) ss += cabs2(x[r]);
  ss = block_sum(ss, sh);
  const double xn = sqrt(ss);
  const cplx alpha = x[j];
  const double aa = sqrt(cabs2(alpha));
  cplx beta = mk(0, 0);
  double tau = 0.0;
  if (xn > 0.0) {
    const cplx ph = aa > 0.0 ? cscale(alpha, 1.0 / aa) : mk(1, 0);
    beta = cscale(ph, -xn);
    tau = 2.0 / (2.0 * ss + 2.0 * xn * aa);
  }
  cplx* v = Vs + j * N;
  cplx* u = Us + j * N;
  for (int64_t r = threadIdx.x; r < N; r += blockDim.x) {
    cplx vr = mk(0, 0);
    if (r >= j && xn > 0.0) vr = (r == j) ? csub(alpha, beta) : x[r];
    v[r] = vr;
    u[r] = cscale(vr, tau);
  }
}

// wrow[c] = sum_{r >= j} conj(v[r]) X[r, c] for c in [c0, m)
__global__ void hh_row_kernel(const cplx* X, int64_t N, int64_t j, int64_t c0, const cplx* v, cplx* wrow) {
  __shared__ double sh[32];
  const int64_t c = c0 + blockIdx.x;
  double re = 0.0, im = 0.0;
  for (int64_t r = j + threadIdx.x; r < N; r += blockDim.x) {
    const cplx p = cmul(cconj(v[r]), X[r + c * N]);
    re += p.x;
    im += p.y;
  }
  re = block_sum(re, sh);
  im = block_sum(im, sh);
  if (threadIdx.x == 0) wrow[c] = mk(re, im);
}

// X[r, c] -= u[r] wrow[c] for r >= j, c in [c0, m)
__global__ void hh_update_kernel(cplx* X, int64_t N, int64_t m, int64_t j, int64_t c0, const cplx* u,
                                 const cplx* wrow) {
  const int64_t rows = N - j, cols = m - c0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < rows * cols; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = j + i % rows, c = c0 + i / rows;
    X[r + c * N] = csub(X[r + c * N], cmul(u[r], wrow[c]));
  }
}

__global__ void set_diag_rect_kernel(cplx* Q, int64_t N, int64_t m) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c < m) Q[c + c * N] = mk(1, 0);
}

int householder_qr(cplx* X, int64_t N, int64_t m, cplx* Q, cplx* Vs, cplx* Us, cplx* wrow, cudaStream_t s) {
  if (m > N || m <= 0) return CHASE_BSE_BAD_ARG;
  for (int64_t j = 0; j < m; ++j) {
    hh_reflector_kernel<<<1, 1024, 0, s>>>(X, N, j, Vs, Us);
    count_launch();
    if (j + 1 < m) {
      hh_row_kernel<<<(unsigned)(m - j - 1), 256, 0, s>>>(X, N, j, j + 1, Vs + j * N, wrow);
      count_launch();
      const int64_t tot = (N - j) * (m - j - 1);
      hh_update_kernel<<<cdiv(tot, 256) < 4096 ? cdiv(tot, 256) : 4096, 256, 0, s>>>(X, N, m, j, j + 1,
                                                                                     Us + j * N, wrow);
                                                                                     count_launch();
    }
  }
  CB_LAUNCH();
  // Q = H_0 H_1 ... H_{m-1} [I; 0], accumulated backwards
  CB_CUDA(cudaMemsetAsync(Q, 0, sizeof(cplx) * N * m, s));
  set_diag_rect_kernel<<<cdiv(m, 256), 256, 0, s>>>(Q, N, m);
  count_launch();
  for (int64_t j = m - 1; j >= 0; --j) {
    hh_row_kernel<<<(unsigned)(m - j), 256, 0, s>>>(Q, N, j, j, Vs + j * N, wrow);
    count_launch();
    const int64_t tot = (N - j) * (m - j);
    hh_update_kernel<<<cdiv(tot, 256) < 4096 ? cdiv(tot, 256) : 4096, 256, 0, s>>>(Q, N, m, j, j, Us + j * N, wrow);
    count_launch();
  }
  CB_LAUNCH();
  return CHASE_BSE_OK;
}

// ----------------------------------------------------------------- utilities
#define GRID_STRIDE(i, total) \
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < (total); i += (int64_t)gridDim.x * blockDim.x)

__global__ void scale_lower_kernel(cplx* W, int64_t n, int64_t k, double g) {
  GRID_STRIDE(i, n * k) {
    const int64_t r = i % n, c = i / n;
    W[c * 2 * n + n + r] = cscale(W[c * 2 * n + n + r], g);
  }
}
int scale_lower(cplx* W, int64_t n, int64_t k, double gamma, cudaStream_t s) {
  if (n * k == 0) return CHASE_BSE_OK;
  scale_lower_kernel<<<gs(n * k), 256, 0, s>>>(W, n, k, gamma);
  count_launch();
  CB_LAUNCH();
  return CHASE_BSE_OK;
}

__global__ void build_qr_input_kernel(cplx* X, const cplx* Yp, int64_t L, const cplx* Wf, int64_t kf, int64_t n) {
  const int64_t n2 = 2 * n, cols = 2 * L + 2 * kf;
  GRID_STRIDE(i, n2 * cols) {
    const int64_t r = i % n2, c = i / n2;
    cplx v;
    if (c < L) {                       // S Y+
      v = Yp[c * n2 + r];
      if (r >= n) v = mk(-v.x, -v.y);
    } else if (c < 2 * L) {            // S K conj(Y+)
      const cplx* y = Yp + (c - L) * n2;
      v = (r < n) ? cconj(y[r + n]) : mk(-y[r - n].x, y[r - n].y);
    } else if (c < 2 * L + kf) {       // W+
      v = Wf[(c - 2 * L) * n2 + r];
    } else {                           // K conj(W+)
      const cplx* w = Wf + (c - 2 * L - kf) * n2;
      v = cconj(r < n ? w[r + n] : w[r - n]);
    }
    X[i] = v;
  }
}
int build_qr_input(cplx* X, const cplx* Yp, int64_t L, const cplx* Wf, int64_t kf, int64_t n, cudaStream_t s) {
  const int64_t tot = 2 * n * (2 * L + 2 * kf);
  if (tot == 0) return CHASE_BSE_OK;
  build_qr_input_kernel<<<gs(tot), 256, 0, s>>>(X, Yp, L, Wf, kf, n);
  count_launch();
  CB_LAUNCH();
  return CHASE_BSE_OK;
}

__global__ void build_jfixed_kernel(cplx* Xt, const cplx* Yp, int64_t L, const cplx* W, int64_t kf, int64_t n) {
  const int64_t n2 = 2 * n, cols = 2 * (L + kf);
  GRID_STRIDE(idx, n * cols) {
    const int64_t r = idx % n, c = idx / n;
    cplx v;
    // columns in pairs (v1, v2) per vector, so that pair j spans {u_j, J u_j}
    if (c < 2 * L) {
      const cplx* y = Yp + (c / 2) * n2;
      const cplx yt = y[r], ybc = cconj(y[n + r]);
      // S y = [yt; -yb], J S y = [-conj(yb); conj(yt)]
      v = (c % 2 == 0) ? csub(yt, ybc) : cmul(mk(0, 1), cadd(yt, ybc));
    } else {
      const int64_t a = c - 2 * L;
      const cplx* w = W + (a / 2) * n2;
      const cplx wt = w[r], wbc = cconj(w[n + r]);
      // J w = [conj(wb); conj(wt)]
      v = (a % 2 == 0) ? cadd(wt, wbc) : cmul(mk(0, 1), csub(wt, wbc));
    }
    Xt[c * n + r] = v;
  }
}
int build_jfixed(cplx* Xt, const cplx* Yp, int64_t L, const cplx* W, int64_t kf, int64_t n, cudaStream_t s) {
  const int64_t tot = n * 2 * (L + kf);
  if (tot == 0) return CHASE_BSE_OK;
  build_jfixed_kernel<<<gs(tot), 256, 0, s>>>(Xt, Yp, L, W, kf, n);
  count_launch();
  CB_LAUNCH();
  return CHASE_BSE_OK;
}
// Pairwise unitary U = blockdiag(u), u = [[1, 1], [-i, i]] / sqrt(2): maps a J-fixed
// pair (w + Jw, i (w - Jw)) to directions along (w, Jw).
__global__ void pair_transform_kernel(const cplx* M, cplx* out, int64_t k) {
  // out = U^* M U, one thread per 2x2 block
  const int64_t h = k / 2;
  GRID_STRIDE(idx, h * h) {
    const int64_t a = idx % h, b = idx / h;
    const cplx m00 = M[2 * a + 2 * b * k], m10 = M[2 * a + 1 + 2 * b * k];
    const cplx m01 = M[2 * a + (2 * b + 1) * k], m11 = M[2 * a + 1 + (2 * b + 1) * k];
    // M U: columns (m_.0 - i m_.1)/sqrt2, (m_.0 + i m_.1)/sqrt2
    const double r = 0.70710678118654752440;
    const cplx i1 = mk(0, 1);
    const cplx p00 = cscale(csub(m00, cmul(i1, m01)), r), p01 = cscale(cadd(m00, cmul(i1, m01)), r);
    const cplx p10 = cscale(csub(m10, cmul(i1, m11)), r), p11 = cscale(cadd(m10, cmul(i1, m11)), r);
    // U^* (.): rows (p_0. + i p_1.)/sqrt2, (p_0. - i p_1.)/sqrt2
    out[2 * a + 2 * b * k] = cscale(cadd(p00, cmul(i1, p10)), r);
    out[2 * a + (2 * b + 1) * k] = cscale(cadd(p01, cmul(i1, p11)), r);
    out[2 * a + 1 + 2 * b * k] = cscale(csub(p00, cmul(i1, p10)), r);
    out[2 * a + 1 + (2 * b + 1) * k] = cscale(csub(p01, cmul(i1, p11)), r);
  }
}
int pair_transform(const cplx* M, cplx* out, int64_t k, cudaStream_t s) {
  if (k == 0) return CHASE_BSE_OK;
  pair_transform_kernel<<<gs(k * k / 4), 256, 0, s>>>(M, out, k);
  count_launch();
  CB_LAUNCH();
  return CHASE_BSE_OK;
}
// Z = U Z' (k x h): rows 2a, 2a+1 of Z from rows of Z'
__global__ void pair_apply_kernel(const cplx* Zp, cplx* Z, int64_t k, int64_t h) {
  GRID_STRIDE(idx, (k / 2) * h) {
    const int64_t a = idx % (k / 2), j = idx / (k / 2);
    const cplx z0 = Zp[2 * a + j * k], z1 = Zp[2 * a + 1 + j * k];
    const double r = 0.70710678118654752440;
    Z[2 * a + j * k] = cscale(cadd(z0, z1), r);
    Z[2 * a + 1 + j * k] = cscale(cmul(mk(0, 1), csub(z1, z0)), r);
  }
}
int pair_apply(const cplx* Zp, cplx* Z, int64_t k, int64_t h, cudaStream_t s) {
  if (k * h == 0) return CHASE_BSE_OK;
  pair_apply_kernel<<<gs(k * h / 2), 256, 0, s>>>(Zp, Z, k, h);
  count_launch();
  CB_LAUNCH();
  return CHASE_BSE_OK;
}

// out = in^* (k x k, column-major)
__global__ void conj_transpose_kernel(const cplx* in, int64_t k, cplx* out) {
  __shared__ cplx tile[32][33];
  const int64_t r0 = (int64_t)blockIdx.x * 32, c0 = (int64_t)blockIdx.y * 32;
  for (int j = threadIdx.y; j < 32; j += 8) {
    const int64_t r = r0 + threadIdx.x, c = c0 + j;
    if (r < k && c < k) tile[j][threadIdx.x] = in[r + c * k];
  }
  __syncthreads();
  for (int j = threadIdx.y; j < 32; j += 8) {
    const int64_t r = c0 + threadIdx.x, c = r0 + j;  // out[r, c] = conj(in[c, r])
    if (r < k && c < k) out[r + c * k] = cconj(tile[threadIdx.x][j]);
  }
}
int conj_transpose(const cplx* in, int64_t k, cplx* out, cudaStream_t s) {
  if (k == 0) return CHASE_BSE_OK;
  conj_transpose_kernel<<<dim3(cdiv(k, 32), cdiv(k, 32)), dim3(32, 8), 0, s>>>(in, k, out);
  count_launch();
  CB_LAUNCH();
  return CHASE_BSE_OK;
}
__global__ void re_im_part_kernel(const cplx* C, cplx* out, int64_t k, int mode) {
  GRID_STRIDE(i, k * k) { out[i] = (mode == 0) ? mk(2.0 * C[i].x, 0.0) : mk(0.0, 2.0 * C[i].y); }
}
int re_im_part(const cplx* C, cplx* out, int64_t k, int mode, cudaStream_t s) {
  if (k == 0) return CHASE_BSE_OK;
  re_im_part_kernel<<<gs(k * k), 256, 0, s>>>(C, out, k, mode);
  count_launch();
  CB_LAUNCH();
  return CHASE_BSE_OK;
}
__global__ void conj_copy_kernel(cplx* dst, int64_t ldd, const cplx* src, int64_t lds, int64_t rows, int64_t m) {
  GRID_STRIDE(i, rows * m) {
    const int64_t r = i % rows, c = i / rows;
    dst[r + c * ldd] = cconj(src[r + c * lds]);
  }
}
int conj_copy(cplx* dst, int64_t ldd, const cplx* src, int64_t lds, int64_t rows, int64_t m, cudaStream_t s) {
  if (rows * m == 0) return CHASE_BSE_OK;
  conj_copy_kernel<<<gs(rows * m), 256, 0, s>>>(dst, ldd, src, lds, rows, m);
  count_launch();
  CB_LAUNCH();
  return CHASE_BSE_OK;
}

__global__ void gather_cols_kernel(cplx* dst, const cplx* src, const int* idx, int64_t rows, int64_t m) {
  GRID_STRIDE(i, rows * m) {
    const int64_t r = i % rows, c = i / rows;
    dst[i] = src[(int64_t)idx[c] * rows + r];
  }
}
int gather_cols(cplx* dst, const cplx* src, const int* idx, int64_t rows, int64_t m, cudaStream_t s) {
  if (rows * m == 0) return CHASE_BSE_OK;
  gather_cols_kernel<<<gs(rows * m), 256, 0, s>>>(dst, src, idx, rows, m);
  count_launch();
  CB_LAUNCH();
  return CHASE_BSE_OK;
}
__global__ void scatter_cols_kernel(cplx* dst, const cplx* src, const int* idx, int64_t rows, int64_t m) {
  GRID_STRIDE(i, rows * m) {
    const int64_t r = i % rows, c = i / rows;
    dst[(int64_t)idx[c] * rows + r] = src[i];
  }
}
int scatter_cols(cplx* dst, const cplx* src, const int* idx, int64_t rows, int64_t m, cudaStream_t s) {
  if (rows * m == 0) return CHASE_BSE_OK;
  scatter_cols_kernel<<<gs(rows * m), 256, 0, s>>>(dst, src, idx, rows, m);
  count_launch();
  CB_LAUNCH();
  return CHASE_BSE_OK;
}
__global__ void collect_cols_kernel(cplx* dst, const cplx* b0, const cplx* b1, const cplx* b2, const int* sel,
                                    int64_t rows, int64_t m) {
  GRID_STRIDE(i, rows * m) {
    const int64_t c = i / rows;
    const int q = sel[c];
    const cplx* b = q == 0 ? b0 : (q == 1 ? b1 : b2);
    dst[i] = b[i];
  }
}
int collect_cols(cplx* dst, const cplx* b0, const cplx* b1, const cplx* b2, const int* sel, int64_t rows,
                 int64_t m, cudaStream_t s) {
  if (rows * m == 0) return CHASE_BSE_OK;
  collect_cols_kernel<<<gs(rows * m), 256, 0, s>>>(dst, b0, b1, b2, sel, rows, m);
  count_launch();
  CB_LAUNCH();
  return CHASE_BSE_OK;
}

__global__ void col_norms_kernel(const cplx* X, int64_t rows, double* out) {
  __shared__ double sh[32];
  const cplx* x = X + (int64_t)blockIdx.x * rows;
  double ss = 0.0;
  for (int64_t r = threadIdx.x; r < rows; r += blockDim.x) ss += cabs2(x[r]);
  ss = block_sum(ss, sh);
  if (threadIdx.x == 0) out[blockIdx.x] = sqrt(ss);
}
int col_norms(const cplx* X, int64_t rows, int64_t m, double* out, cudaStream_t s) {
  if (m == 0) return CHASE_BSE_OK;
  col_norms_kernel<<<(unsigned)m, 256, 0, s>>>(X, rows, out);
  count_launch();
  CB_LAUNCH();
  return CHASE_BSE_OK;
}
__global__ void normalize_cols_kernel(cplx* X, int64_t rows) {
  __shared__ double sh[32];
  cplx* x = X + (int64_t)blockIdx.x * rows;
  double ss = 0.0;
  for (int64_t r = threadIdx.x; r < rows; r += blockDim.x) ss += cabs2(x[r]);
  ss = block_sum(ss, sh);
  const double inv = ss > 0.0 ? 1.0 / sqrt(ss) : 0.0;
  for (int64_t r = threadIdx.x; r < rows; r += blockDim.x) x[r] = cscale(x[r], inv);
}
int normalize_cols(cplx* X, int64_t rows, int64_t m, cudaStream_t s) {
  if (m == 0) return CHASE_BSE_OK;
  normalize_cols_kernel<<<(unsigned)m, 256, 0, s>>>(X, rows);
  count_launch();
  CB_LAUNCH();
  return CHASE_BSE_OK;
}
__global__ void normalize_and_residual_kernel(cplx* W, const cplx* SHW, const double* ritz, int64_t n, cplx* R) {
  __shared__ double sh[32];
  const int64_t j = blockIdx.x, n2 = 2 * n;
  cplx* w = W + j * n2;
  const cplx* h = SHW + j * n2;
  cplx* r = R + j * n2;
  double ss = 0.0;
  for (int64_t i = threadIdx.x; i < n2; i += blockDim.x) ss += cabs2(w[i]);
  ss = block_sum(ss, sh);
  const double inv = ss > 0.0 ? 1.0 / sqrt(ss) : 0.0;
  const double lam = ritz[j];
  for (int64_t i = threadIdx.x; i < n2; i += blockDim.x) {
    const cplx wn = cscale(w[i], inv);
    cplx hw = cscale(h[i], inv);
    if (i >= n) hw = mk(-hw.x, -hw.y);  // undo S
    w[i] = wn;
    r[i] = csub(hw, cscale(wn, lam));
  }
}
int normalize_and_residual(cplx* W, const cplx* SHW, const double* ritz, int64_t n, int64_t m, cplx* R,
                           cudaStream_t s) {
  if (m == 0) return CHASE_BSE_OK;
  normalize_and_residual_kernel<<<(unsigned)m, 256, 0, s>>>(W, SHW, ritz, n, R);
  count_launch();
  CB_LAUNCH();
  return CHASE_BSE_OK;
}

__global__ void count_nonfinite_kernel(const cplx* X, int64_t total, int* count) {
  int local = 0;
  GRID_STRIDE(i, total) {
    const cplx v = X[i];
    if (!isfinite(v.x) || !isfinite(v.y)) ++local;
  }
  if (local) atomicAdd(count, local);
}
int count_nonfinite(const cplx* X, int64_t total, int* count_dev, int* count_host, cudaStream_t s) {
  CB_CUDA(cudaMemsetAsync(count_dev, 0, sizeof(int), s));
  if (total > 0) {
    count_nonfinite_kernel<<<gs(total), 256, 0, s>>>(X, total, count_dev);
    count_launch();
    CB_LAUNCH();
  }
  CB_CUDA(cudaMemcpyAsync(count_host, count_dev, sizeof(int), cudaMemcpyDeviceToHost, s));
  CB_CUDA(cudaStreamSynchronize(s));
  return CHASE_BSE_OK;
}

// R[:, j] = HV[:, j] - lam[j] V[:, j]
__global__ void residual_from_hv_kernel(const cplx* HV, const cplx* V, const double* lam, int64_t n2, int64_t m,
                                        cplx* R) {
  GRID_STRIDE(idx, n2 * m) { R[idx] = csub(HV[idx], cscale(V[idx], lam[idx / n2])); }
}
int residual_from_hv(const cplx* HV, const cplx* V, const double* lam, int64_t n2, int64_t m, cplx* R,
                     cudaStream_t s) {
  if (m == 0) return CHASE_BSE_OK;
  residual_from_hv_kernel<<<gs(n2 * m), 256, 0, s>>>(HV, V, lam, n2, m, R);
  count_launch();
  CB_LAUNCH();
  return CHASE_BSE_OK;
}

__global__ void set_identity_kernel(cplx* M, int64_t k) {
  GRID_STRIDE(i, k * k) { M[i] = (i % k == i / k) ? mk(1, 0) : mk(0, 0); }
}
int set_identity(cplx* M, int64_t k, cudaStream_t s) {
  if (k == 0) return CHASE_BSE_OK;
  set_identity_kernel<<<gs(k * k), 256, 0, s>>>(M, k);
  count_launch();
  CB_LAUNCH();
  return CHASE_BSE_OK;
}
__global__ void hermitize_kernel(cplx* G, int64_t k) {
  GRID_STRIDE(i, k * k) {
    const int64_t r = i % k, c = i / k;
    if (r > c) {
      const cplx a = G[r + c * k], b = G[c + r * k];
      const cplx m = mk(0.5 * (a.x + b.x), 0.5 * (a.y - b.y));  // (a + conj(b)) / 2
      G[r + c * k] = m;
      G[c + r * k] = cconj(m);
    } else if (r == c) {
      G[i].y = 0.0;
    }
  }
}
int hermitize(cplx* G, int64_t k, cudaStream_t s) {
  if (k == 0) return CHASE_BSE_OK;
  hermitize_kernel<<<gs(k * k), 256, 0, s>>>(G, k);
  count_launch();
  CB_LAUNCH();
  return CHASE_BSE_OK;
}
__global__ void diag_real_kernel(const cplx* G, int64_t k, double* out) {
  GRID_STRIDE(i, k) { out[i] = G[i + i * k].x; }
}
int diag_real(const cplx* G, int64_t k, double* out, cudaStream_t s) {
  if (k == 0) return CHASE_BSE_OK;
  diag_real_kernel<<<gs(k), 256, 0, s>>>(G, k, out);
  count_launch();
  CB_LAUNCH();
  return CHASE_BSE_OK;
}
// largest |v_i| over the upper half (smallest index on ties); v <- v |v_i| / v_i
__global__ void phase_fix_kernel(cplx* V, int64_t n) {
  __shared__ double bv[1024];
  __shared__ int64_t bi[1024];
  cplx* v = V + (int64_t)blockIdx.x * 2 * n;
  double best = -1.0;
  int64_t besti = 0;
  for (int64_t r = threadIdx.x; r < n; r += blockDim.x) {
    const double a = cabs2(v[r]);
    if (a > best) { best = a; besti = r; }
  }
  bv[threadIdx.x] = best;
  bi[threadIdx.x] = besti;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      const double a = bv[threadIdx.x + o];
      const int64_t ia = bi[threadIdx.x + o];
      if (a > bv[threadIdx.x] || (a == bv[threadIdx.x] && ia < bi[threadIdx.x])) {
        bv[threadIdx.x] = a;
        bi[threadIdx.x] = ia;
      }
    }
    __syncthreads();
  }
  const cplx p = v[bi[0]];
  const double a = sqrt(cabs2(p));
  const cplx f = a > 0.0 ? mk(p.x / a, -p.y / a) : mk(1, 0);  // |p| / p
  __syncthreads();
  for (int64_t r = threadIdx.x; r < 2 * n; r += blockDim.x) v[r] = cmul(v[r], f);
}
int phase_fix(cplx* V, int64_t n, int64_t m, cudaStream_t s) {
  if (m == 0) return CHASE_BSE_OK;
  phase_fix_kernel<<<(unsigned)m, 1024, 0, s>>>(V, n);
  count_launch();
  CB_LAUNCH();
  return CHASE_BSE_OK;
}
__global__ void copy_cols_kernel(cplx* dst, int64_t ldd, const cplx* src, int64_t lds, int64_t rows, int64_t m) {
  GRID_STRIDE(i, rows * m) {
    const int64_t r = i % rows, c = i / rows;
    dst[r + c * ldd] = src[r + c * lds];
  }
}
int copy_cols(cplx* dst, int64_t ldd, const cplx* src, int64_t lds, int64_t rows, int64_t m, cudaStream_t s) {
  if (rows * m == 0) return CHASE_BSE_OK;
  copy_cols_kernel<<<gs(rows * m), 256, 0, s>>>(dst, ldd, src, lds, rows, m);
  count_launch();
  CB_LAUNCH();
  return CHASE_BSE_OK;
}

// ------------------------------------------------------------------ Lanczos
__global__ void sdot_real_kernel(const cplx* X, const cplx* Y, int64_t n, double* out) {
  __shared__ double sh[32];
  const int64_t c = blockIdx.x;
  const cplx* x = X + c * 2 * n;
  const cplx* y = Y + c * 2 * n;
  double acc = 0.0;
  for (int64_t r = threadIdx.x; r < 2 * n; r += blockDim.x) {
    const double d = x[r].x * y[r].x + x[r].y * y[r].y;  // Re(conj(x) y)
    acc += (r < n) ? d : -d;
  }
  acc = block_sum(acc, sh);
  if (threadIdx.x == 0) out[c] = acc;
}
int sdot_real(const cplx* X, const cplx* Y, int64_t n, int64_t nvec, double* out, cudaStream_t s) {
  sdot_real_kernel<<<(unsigned)nvec, 1024, 0, s>>>(X, Y, n, out);
  count_launch();
  CB_LAUNCH();
  return CHASE_BSE_OK;
}
__global__ void lanczos_axpy_kernel(cplx* Wv, const cplx* U, const cplx* V, const cplx* Vp, const double* alpha,
                                    const double* beta_prev, int64_t n, int64_t nvec) {
  GRID_STRIDE(i, 2 * n * nvec) {
    const int64_t c = i / (2 * n);
    cplx w = csub(U[i], cscale(V[i], alpha[c]));
    if (beta_prev) w = csub(w, cscale(Vp[i], beta_prev[c]));
    Wv[i] = w;
  }
}
int lanczos_axpy(cplx* Wv, const cplx* U, const cplx* V, const cplx* Vp, const double* alpha,
                 const double* beta_prev, int64_t n, int64_t nvec, cudaStream_t s) {
  lanczos_axpy_kernel<<<gs(2 * n * nvec), 256, 0, s>>>(Wv, U, V, Vp, alpha, beta_prev, n, nvec);
  count_launch();
  CB_LAUNCH();
  return CHASE_BSE_OK;
}
__global__ void lanczos_beta_kernel(double* beta, const double* nrm2, int64_t nvec) {
  const int64_t c = threadIdx.x;
  if (c < nvec) beta[c] = sqrt(nrm2[c] > 0.0 ? nrm2[c] : 0.0);
}
__global__ void lanczos_scale_kernel(const double* beta, const cplx* Wv, const cplx* Y, cplx* V, cplx* U,
                                     int64_t n, int64_t nvec) {
  GRID_STRIDE(i, 2 * n * nvec) {
    const int64_t c = i / (2 * n);
    const double b = beta[c];
    const double inv = b > 0.0 ? 1.0 / b : 0.0;
    V[i] = cscale(Wv[i], inv);
    U[i] = cscale(Y[i], inv);
  }
}
int lanczos_normalise(double* beta, const double* nrm2, const cplx* Wv, const cplx* Y, cplx* V, cplx* U,
                      int64_t n, int64_t nvec, cudaStream_t s) {
  lanczos_beta_kernel<<<1, 64, 0, s>>>(beta, nrm2, nvec);
  count_launch();
  lanczos_scale_kernel<<<gs(2 * n * nvec), 256, 0, s>>>(beta, Wv, Y, V, U, n, nvec);
  count_launch();
  CB_LAUNCH();
  return CHASE_BSE_OK;
}

// ------------------------------------------------- counter-based normals
// Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11): 10 rounds of the
// multiply-xor round with multipliers 0xD2511F53 / 0xCD9E8D57 and Weyl key
// increments 0x9E3779B9 / 0xBB67AE85.  Two uniforms -> one complex normal by
// Box-Muller (re, im independent N(0, 1)).
__device__ __forceinline__ uint4 philox4x32_10(uint4 ctr, uint2 key) {
#pragma unroll
  for (int i = 0; i < 10; ++i) {
    const unsigned lo0 = 0xD2511F53u * ctr.x, hi0 = __umulhi(0xD2511F53u, ctr.x);
    const unsigned lo1 = 0xCD9E8D57u * ctr.z, hi1 = __umulhi(0xCD9E8D57u, ctr.z);
    ctr = make_uint4(hi1 ^ ctr.y ^ key.x, lo1, hi0 ^ ctr.w ^ key.y, lo0);
    key.x += 0x9E3779B9u;
    key.y += 0xBB67AE85u;
  }
  return ctr;
}
__global__ void randn_complex_kernel(cplx* out, int64_t count, uint64_t seed, uint64_t sid) {
  GRID_STRIDE(i, count) {
    const uint4 r = philox4x32_10(make_uint4((unsigned)i, (unsigned)(i >> 32), (unsigned)sid, (unsigned)(sid >> 32)),
                                  make_uint2((unsigned)seed, (unsigned)(seed >> 32)));
    const double u1 = ((double)r.x + (double)r.y * 4294967296.0 + 1.0) / 18446744073709551616.0;  // (0, 1]
    const double u2 = ((double)r.z + (double)r.w * 4294967296.0) / 18446744073709551616.0;        // [0, 1)
    const double rad = sqrt(-2.0 * log(u1));
    double sn, cs;
    sincospi(2.0 * u2, &sn, &cs);
    out[i] = mk(rad * cs, rad * sn);
  }
}
int randn_complex(cplx* out, int64_t count, uint64_t seed, uint64_t sid, cudaStream_t s) {
  if (count == 0) return CHASE_BSE_OK;
  randn_complex_kernel<<<gs(count), 256, 0, s>>>(out, count, seed, sid);
  count_launch();
  CB_LAUNCH();
  return CHASE_BSE_OK;
}

// ------------------------------------------------------------------ gradient
__global__ void grad_coef_kernel(const cplx* V, const double* w, int64_t n, double* cbuf) {
  __shared__ double sh[32];
  const int64_t m = blockIdx.x;
  const cplx* v = V + m * 2 * n;
  double acc = 0.0;
  for (int64_t r = threadIdx.x; r < 2 * n; r += blockDim.x) acc += (r < n) ? cabs2(v[r]) : -cabs2(v[r]);
  acc = block_sum(acc, sh);
  if (threadIdx.x == 0) cbuf[m] = w[m] / acc;  // c_m = w_m / (|x|^2 - |y|^2)
}
__global__ void grad_pack_kernel(const cplx* V, const double* cbuf, int64_t n, int64_t nev, cplx* Uc, cplx* U2,
                                 cplx* Ub, cplx* U3) {
  GRID_STRIDE(i, n * nev) {
    const int64_t r = i % n, m = i / n;
    const cplx x = V[m * 2 * n + r], y = V[m * 2 * n + n + r];
    const double c = cbuf[m];
    const int64_t a = r + m * n, b = r + (m + nev) * n;
    Uc[a] = cscale(cconj(x), c);
    Uc[b] = cscale(y, c);
    U2[a] = x;
    U2[b] = cconj(y);
    Ub[a] = cscale(x, c);
    Ub[b] = cscale(cconj(y), c);
    U3[a] = cconj(y);
    U3[b] = x;
  }
}
int grad_prepare(const cplx* V, const double* w, int64_t n, int64_t nev, double* cbuf, cplx* Uc, cplx* U2,
                 cplx* Ub, cplx* U3, cudaStream_t s) {
  grad_coef_kernel<<<(unsigned)nev, 256, 0, s>>>(V, w, n, cbuf);
  count_launch();
  grad_pack_kernel<<<gs(n * nev), 256, 0, s>>>(V, cbuf, n, nev, Uc, U2, Ub, U3);
  count_launch();
  CB_LAUNCH();
  return CHASE_BSE_OK;
}

}  // namespace cb
