// Mixed-precision eigensolver for the small hermitian problem of the oblique
// Rayleigh-Ritz step (G y = theta y in Algorithm 2), for G far from diagonal.
//
// GB300 runs FP32 at 64x its FP64 rate, so the bulk of the Jacobi work (the early
// sweeps, which rotate every pair) runs in FP32; FP64 accuracy is then recovered
// with FP64-accurate tensor-core GEMMs (sliced GEMM) and, if needed, a short FP64 Jacobi:
//   1. FP32 Jacobi on G (scaled to ||G||_F ~ 1) until every |g_pq| is below
//      2e-6 sqrt|g_pp g_qq| or 1e-8 ||G|| (the FP32 rotations need not be exactly
//      unitary);
//   2. two steps of the iterative refinement of Ogita and Aishima (2018, Japan J.
//      Indust. Appl. Math.) on X = the FP32 eigenvectors in FP64: with
//      R = I - X^* X and S = X^* G X, lam_i = s_ii / (1 - r_ii) and
//      X <- X (I + E), E_ij = (s_ij + lam_j r_ij) / (lam_j - lam_i) where that
//      correction is small (a pair test symmetric in i and j; the published method
//      separates clusters by a norm bound delta), else r_ij / 2, E_ii = r_ii / 2
//      (the first-order terms of X = X^ (I + E), X^* X = I, X^* G X diagonal);
//      each step squares the error of the separated pairs (a third step can
//      amplify the noise of nearly equal pairs, so there are two), and all the
//      arithmetic is in FP64-accurate tensor-core GEMMs;
//   3. G1 = X^* G X, hermitised;
//   4. FP64 Jacobi on G1 (what the refinement left: near-degenerate pairs, often
//      nothing), V = X V2.
// The FP32 sweep has the FP64 sweep's structure: one cooperative kernel per sweep,
// one grid barrier per round, G ping-ponged, the next round's rotations formed by
// the threads that produce their pivots, V updated afterwards over the stored
// rotations.
#include <cuda_pipeline.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <vector>

#include "coop.cuh"
#include "dense_kernels.cuh"
#include "solver.cuh"
#include "tc_dgemm.cuh"

namespace cb {
namespace jm {

struct Rot32 {
  float c, s, er, ei;
};

__device__ __forceinline__ float2 mkf(float r, float i) { return make_float2(r, i); }
__device__ __forceinline__ float2 cmulf(float2 a, float2 b) {
  return mkf(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// rotate when |g_pq| > t sqrt|g_pp g_qq| (t2 = t^2) and |g_pq| > 1e-8 ||G|| (n2 = ||G||^2,
// G scaled to ||G||_F ~ 1): the FP32 phase hands over eigenvectors accurate relative to
// the diagonal, which the first-order refinement needs for nearly equal pairs
__device__ __forceinline__ bool active32(float app, float aqq, float2 apq, float t2, float n2) {
  const float r2 = fmaf(apq.x, apq.x, apq.y * apq.y);
  return r2 > t2 * fabsf(app * aqq) && r2 > 1e-16f * n2 && r2 > 0.0f;
}
__device__ Rot32 rotation32(float app, float aqq, float2 apq, float t2, float n2, int* applied) {
  Rot32 R{1.0f, 0.0f, 1.0f, 0.0f};
  if (!active32(app, aqq, apq, t2, n2)) return R;
  atomicAdd(applied, 1);
  const float ri = rsqrtf(fmaf(apq.x, apq.x, apq.y * apq.y));
  R.er = apq.x * ri;  // e = conj(g_pq) / |g_pq|
  R.ei = -apq.y * ri;
  const float tau = 0.5f * (aqq - app) * ri;
  const float t = copysignf(1.0f, tau) / (fabsf(tau) + sqrtf(fmaf(tau, tau, 1.0f)));
  R.c = rsqrtf(fmaf(t, t, 1.0f));
  R.s = t * R.c;
  return R;
}
__device__ __forceinline__ void rot_block32(const Rot32& A, const Rot32& B, const float2 x[4], float2 z[4]) {
  const float2 ea = mkf(A.er, -A.ei);
  const float2 w0 = cmulf(ea, x[2]), w1 = cmulf(ea, x[3]);
  const float2 y00 = mkf(A.c * x[0].x - A.s * w0.x, A.c * x[0].y - A.s * w0.y);
  const float2 y01 = mkf(A.c * x[1].x - A.s * w1.x, A.c * x[1].y - A.s * w1.y);
  const float2 y10 = mkf(A.s * x[0].x + A.c * w0.x, A.s * x[0].y + A.c * w0.y);
  const float2 y11 = mkf(A.s * x[1].x + A.c * w1.x, A.s * x[1].y + A.c * w1.y);
  const float2 eb = mkf(B.er, B.ei);
  const float2 u0 = cmulf(y01, eb), u1 = cmulf(y11, eb);
  z[0] = mkf(B.c * y00.x - B.s * u0.x, B.c * y00.y - B.s * u0.y);
  z[1] = mkf(B.s * y00.x + B.c * u0.x, B.s * y00.y + B.c * u0.y);
  z[2] = mkf(B.c * y10.x - B.s * u1.x, B.c * y10.y - B.s * u1.y);
  z[3] = mkf(B.s * y10.x + B.c * u1.x, B.s * y10.y + B.c * u1.y);
}
__device__ __forceinline__ float rot_diag32(const Rot32& A, const float2* G, int k, int p, int q, int i) {
  const float xpp = __ldcg(&G[p + (int64_t)p * k].x), xqq = __ldcg(&G[q + (int64_t)q * k].x);
  if (A.s == 0.0f) return i == 0 ? xpp : xqq;
  const float2 xpq = __ldcg(G + p + (int64_t)q * k);
  const float re = A.er * xpq.x - A.ei * xpq.y;
  const float cc = A.c * A.c, ss = A.s * A.s, cs2 = 2.0f * A.c * A.s;
  return i == 0 ? fmaf(cc, xpp, fmaf(ss, xqq, -cs2 * re)) : fmaf(ss, xpp, fmaf(cc, xqq, cs2 * re));
}
__device__ __forceinline__ Rot32 ld_rot32(const Rot32* r) {
  const float4 u = __ldcg(reinterpret_cast<const float4*>(r));
  return Rot32{u.x, u.y, u.z, u.w};
}
__device__ __forceinline__ void load_block32(const float2* G, int k, int p0, int q0, int p1, int q1, float2 x[4]) {
  x[0] = __ldcg(G + p0 + (int64_t)p1 * k);
  x[1] = __ldcg(G + p0 + (int64_t)q1 * k);
  x[2] = __ldcg(G + q0 + (int64_t)p1 * k);
  x[3] = __ldcg(G + q0 + (int64_t)q1 * k);
}

__global__ void sweep32_kernel(float2* Ga, float2* Gb, int k, Rot32* rots, float t2, float n2, int* applied,
                               GridSync* gsync, int* err) {
  const int half = k / 2;
  const int64_t nblk = (int64_t)half * (half + 1) / 2;
  const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
  const int64_t first = (int64_t)threadIdx.x * gridDim.x + blockIdx.x;
  for (int64_t sl = first; sl < half; sl += nthreads) {
    int p, q;
    jpair32((int)sl, 0, k, p, q);
    rots[sl] = rotation32(__ldcg(&Ga[p + (int64_t)p * k].x), __ldcg(&Ga[q + (int64_t)q * k].x),
                          __ldcg(Ga + p + (int64_t)q * k), t2, n2, applied);
  }
  if (!grid_barrier(gsync, err)) return;
  for (int r = 0; r < k - 1; ++r) {
    const float2* Gi = (r & 1) ? Gb : Ga;
    float2* Go = (r & 1) ? Ga : Gb;
    const Rot32* R = rots + (int64_t)r * half;
    for (int64_t item = first; item < nblk; item += nthreads) {
      int a = (int)((sqrtf(8.0f * (float)item + 1.0f) - 1.0f) * 0.5f);
      while ((int64_t)a * (a + 1) / 2 > item) --a;
      while ((int64_t)(a + 1) * (a + 2) / 2 <= item) ++a;
      const int b = (int)(item - (int64_t)a * (a + 1) / 2);
      int pa, qa, pb, qb;
      jpair32(a, r, k, pa, qa);
      jpair32(b, r, k, pb, qb);
      const Rot32 A = ld_rot32(R + a), B = ld_rot32(R + b);
      float2 x[4], z[4];
      load_block32(Gi, k, pa, qa, pb, qb, x);
      if (A.s == 0.0f && B.s == 0.0f) {
        z[0] = x[0]; z[1] = x[1]; z[2] = x[2]; z[3] = x[3];
      } else {
        rot_block32(A, B, x, z);
      }
      Go[pa + (int64_t)pb * k] = z[0];
      Go[pa + (int64_t)qb * k] = z[1];
      Go[qa + (int64_t)pb * k] = z[2];
      Go[qa + (int64_t)qb * k] = z[3];
      if (a == b) continue;
      Go[pb + (int64_t)pa * k] = mkf(z[0].x, -z[0].y);
      Go[qb + (int64_t)pa * k] = mkf(z[1].x, -z[1].y);
      Go[pb + (int64_t)qa * k] = mkf(z[2].x, -z[2].y);
      Go[qb + (int64_t)qa * k] = mkf(z[3].x, -z[3].y);
      if (r + 1 >= k - 1) continue;
#pragma unroll
      for (int ix = 0; ix < 2; ++ix) {
        const int xi = ix == 0 ? pa : qa;
        const int pos = jpos(xi, r + 1, k);
        const int yi = jat(k - 1 - pos, r + 1, k);
        if (yi != pb && yi != qb) continue;
        const int iy = (yi == pb) ? 0 : 1;
        const float2 zxy = z[2 * ix + iy];
        const float dx = rot_diag32(A, Gi, k, pa, qa, ix), dy = rot_diag32(B, Gi, k, pb, qb, iy);
        const int slot = pos < k - 1 - pos ? pos : k - 1 - pos;
        rots[(int64_t)(r + 1) * half + slot] = xi < yi ? rotation32(dx, dy, zxy, t2, n2, applied)
                                                       : rotation32(dy, dx, mkf(zxy.x, -zxy.y), t2, n2, applied);
      }
    }
    if (!grid_barrier(gsync, err)) return;
  }
}

// V (FP32) <- V J_0 ... J_{k-2}; each round's rotations staged in shared memory.
template <int R>
__global__ void vpass32_kernel(float2* V, int k, const Rot32* rots) {
  extern __shared__ __align__(16) unsigned char vs_raw[];
  const int half = k / 2;
  Rot32* rb = reinterpret_cast<Rot32*>(vs_raw);
  float2* vrow = reinterpret_cast<float2*>(rb + 2 * (int64_t)half);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t i = (int64_t)blockIdx.x * R + w;
  const bool active = i < k;
  float2* v = vrow + (int64_t)w * k;
  if (active)
    for (int j = lane; j < k; j += 32) v[j] = V[i + (int64_t)j * k];
  auto stage = [&](int r, int buf) {
    const char* src = reinterpret_cast<const char*>(rots + (int64_t)r * half);
    char* dst = reinterpret_cast<char*>(rb + (int64_t)buf * half);
    for (int c = threadIdx.x; c < half; c += blockDim.x) __pipeline_memcpy_async(dst + 16 * c, src + 16 * c, 16);
    __pipeline_commit();
  };
  stage(0, 0);
  for (int r = 0; r < k - 1; ++r) {
    __pipeline_wait_prior(0);
    __syncthreads();
    if (r + 1 < k - 1) stage(r + 1, (r + 1) & 1);
    const Rot32* Rr = rb + (int64_t)(r & 1) * half;
    if (active) {
      for (int sl = lane; sl < half; sl += 32) {
        const Rot32 B = Rr[sl];
        if (B.s == 0.0f) continue;
        int p, q;
        jpair32(sl, r, k, p, q);
        const float2 vp = v[p], u = cmulf(v[q], mkf(B.er, B.ei));
        v[p] = mkf(B.c * vp.x - B.s * u.x, B.c * vp.y - B.s * u.y);
        v[q] = mkf(B.s * vp.x + B.c * u.x, B.s * vp.y + B.c * u.y);
      }
    }
    __syncwarp();
  }
  if (active)
    for (int j = lane; j < k; j += 32) V[i + (int64_t)j * k] = v[j];
}

__global__ void count32_kernel(const float2* G, int k, float t2, float n2, int* count) {
  const int64_t total = (int64_t)k * k;
  int local = 0;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int p = (int)(idx % k), q = (int)(idx / k);
    if (p >= q) continue;
    if (active32(G[p + (int64_t)p * k].x, G[q + (int64_t)q * k].x, G[idx], t2, n2)) ++local;
  }
  if (local) atomicAdd(count, local);
}

// G32 = G * 2^-e (exact scaling; 2^e > ||G||_F >= 2^(e-1)), V32 = I
__global__ void to32_kernel(const cplx* G, int64_t k, int e, float2* G32, float2* V32) {
  const int64_t total = k * k;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const cplx g = G[i];
    G32[i] = mkf((float)ldexp(g.x, -e), (float)ldexp(g.y, -e));
    V32[i] = mkf((i % k) == (i / k) ? 1.0f : 0.0f, 0.0f);
  }
}
__global__ void to64_kernel(const float2* V32, int64_t total, cplx* V) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x)
    V[i] = mk((double)V32[i].x, (double)V32[i].y);
}

// lam_i = S_ii / (X^* X)_ii  (= s_ii / (1 - r_ii) with R = I - X^* X)
__global__ void oa_lambda_kernel(const cplx* S, const cplx* S1, int64_t k, double* lam) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < k) lam[i] = S[i + i * k].x / S1[i + i * k].x;
}
// E_ij = (S_ij + lam_j R_ij) / (lam_j - lam_i) when that first-order correction is small
// for the pair (|S_ij| + max(|lam_i|, |lam_j|) |R_ij| <= 1e-2 |lam_j - lam_i|, a test
// symmetric in i and j so that E + E^* = R still holds), R_ij / 2 otherwise (R = I - S1):
// the first-order terms of X = X^ (I + E) with X^* X = I and X^* G X diagonal.  Pairs
// of nearly equal lam are only re-orthogonalised; the FP64 Jacobi afterwards separates
// them.
__global__ void oa_correction_kernel(const cplx* S, const cplx* S1, const double* lam, int64_t k, cplx* E) {
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < k * k;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = idx % k, j = idx / k;
    const cplx r1 = S1[idx];
    const cplx r = (i == j) ? mk(1.0 - r1.x, -r1.y) : mk(-r1.x, -r1.y);
    const double gap = lam[j] - lam[i];
    const cplx sv = S[idx];
    const double bound = sqrt(cabs2(sv)) + fmax(fabs(lam[i]), fabs(lam[j])) * sqrt(cabs2(r));
    if (i != j && bound <= 1e-2 * fabs(gap)) {
      E[idx] = mk((sv.x + lam[j] * r.x) / gap, (sv.y + lam[j] * r.y) / gap);
    } else {
      E[idx] = mk(0.5 * r.x, 0.5 * r.y);
    }
  }
}
// flags[i] = 1 for every index i of a pair (i, j) that the FP64 Jacobi would still
// rotate: |g_ij| > t sqrt|g_ii g_jj| and |g_ij| > (t/2) ||G||_F
__global__ void mark_active_kernel(const cplx* G, int64_t k, double t2, double n2, int* flags) {
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < k * k;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = idx % k, q = idx / k;
    if (p >= q) continue;
    const double r2 = cabs2(G[idx]);
    if (r2 > t2 * fabs(G[p + p * k].x * G[q + q * k].x) && r2 > 0.25 * t2 * n2) {
      flags[p] = 1;
      flags[q] = 1;
    }
  }
}
// sub = G[act, act] (m x m)
__global__ void gather_sub_kernel(const cplx* G, int64_t k, const int* act, int64_t m, cplx* sub) {
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < m * m;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = idx % m, j = idx / m;
    sub[idx] = G[act[i] + (int64_t)act[j] * k];
  }
}
// V2 = I with V2[act, act] = Vs; theta[act[i]] = ts[i]
__global__ void scatter_sub_kernel(const cplx* Vs, const double* ts, const int* act, int64_t m, int64_t k, cplx* V2,
                                   double* theta) {
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < m * m;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = idx % m, j = idx / m;
    V2[act[i] + (int64_t)act[j] * k] = Vs[idx];
    if (i == j) theta[act[i]] = ts[i];
  }
}

__global__ void add_kernel(cplx* X, const cplx* D, int64_t total) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x)
    X[i] = cadd(X[i], D[i]);
}

static unsigned gsz(int64_t total) {
  const int64_t b = (total + 255) / 256;
  return (unsigned)std::min<int64_t>(std::max<int64_t>(b, 1), 8192);
}

// out = X^* Y (k x k complex, column-major): real and imaginary parts as two sliced GEMMs
static int gemm_hn(const cplx* X, const cplx* Y, int64_t k, cplx* out, Workspace& ws, SlicedOp& sx, SlicedOp& sy,
                   cudaStream_t s) {
  (void)ws;
  CB_TRY(slice_rows(reinterpret_cast<const double*>(X), 2 * k, 0, sx, s));
  CB_TRY(slice_rows(reinterpret_cast<const double*>(Y), 2 * k, 0, sy, s));
  CB_TRY(sliced_gemm(sx, sy, 1.0, reinterpret_cast<double*>(out), 2, 2 * k, false, s));
  CB_TRY(slice_rows(reinterpret_cast<const double*>(Y), 2 * k, 1, sy, s));  // (Im y, -Re y)
  return sliced_gemm(sx, sy, 1.0, reinterpret_cast<double*>(out) + 1, 2, 2 * k, false, s);
}
// out = X M (k x k complex): real-form rows of X against the columns of M
static int gemm_nn(const cplx* X, const cplx* M, int64_t k, cplx* out, double* tmp, SlicedOp& sr, SlicedOp& sc,
                   cudaStream_t s) {
  CB_TRY(slice_complex_rows(X, k, k, k, tmp, sr, s));
  CB_TRY(slice_rows(reinterpret_cast<const double*>(M), 2 * k, 0, sc, s));
  return sliced_gemm(sr, sc, 1.0, reinterpret_cast<double*>(out), 1, 2 * k, false, s);
}

}  // namespace jm

int jacobi_eigh_mixed(cplx* G, int64_t k, cplx* V, double* theta, cplx* rot, double* red, int* sweeps32_out,
                      int* sweeps64_out, cudaStream_t s, double thr) {
  using namespace jm;
  if (sweeps32_out) *sweeps32_out = 0;
  int dev = 0, sms = 0, coop = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sweep32_kernel, 512, 0);
  double hred[2] = {0.0, 0.0};
  CB_TRY(offdiag_norms(G, k, red, s));
  CB_CUDA(cudaMemcpyAsync(hred, red, sizeof(hred), cudaMemcpyDeviceToHost, s));
  CB_CUDA(cudaStreamSynchronize(s));
  const double ratio = hred[1] > 0.0 ? std::sqrt(hred[0] / hred[1]) : 0.0;
  const size_t vsm = sizeof(Rot32) * (size_t)k + sizeof(float2) * 4 * (size_t)k;  // 2 rounds + 4 rows
  // near-diagonal G, small k or no cooperative launch: FP64 Jacobi alone
  if (k < 128 || k % 2 || ratio < 1e-4 || !coop || per_sm < 1 || !mixed_available() || vsm > 200 * 1024)
    return jacobi_eigh(G, k, V, theta, rot, red, 40, sweeps64_out, s, thr);
  Workspace ws(s);
  float2 *Ga, *Gb, *V32;
  Rot32* rots;
  GridSync* gsync;
  int *err, *cnt, *applied;
  CB_TRY(ws.alloc(&Ga, k * k));
  CB_TRY(ws.alloc(&Gb, k * k));
  CB_TRY(ws.alloc(&V32, k * k));
  CB_TRY(ws.alloc(&rots, (size_t)(k - 1) * (k / 2) + 1));
  CB_TRY(ws.alloc(&gsync, 1));
  CB_TRY(ws.alloc(&err, 1));
  CB_TRY(ws.alloc(&cnt, 1));
  CB_TRY(ws.alloc(&applied, 1));
  CB_CUDA(cudaMemsetAsync(gsync, 0, sizeof(GridSync), s));
  CB_CUDA(cudaMemsetAsync(err, 0, sizeof(int), s));
  // the FP32 phase: G scaled to ||G||_F in [0.5, 1)
  const double nrm = std::sqrt(hred[1]);
  int e = 0;
  if (nrm > 0.0) std::frexp(nrm, &e);
  to32_kernel<<<gsz(k * k), 256, 0, s>>>(G, k, e, Ga, V32);
  count_launch();
  CB_LAUNCH();
  static bool attr = false;
  if (!attr) {
    CB_CUDA(cudaFuncSetAttribute(vpass32_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    attr = true;
  }
  float n2 = (float)std::pow(std::ldexp(nrm, -e), 2.0);
  float t2 = 4e-12f;  // (2e-6)^2
  int ki = (int)k, herr = 0, hc = 1, sw = 0;
  float2 *ga = Ga, *gb = Gb;
  for (; hc > 0 && sw < 30; ++sw) {
    CB_CUDA(cudaMemsetAsync(applied, 0, sizeof(int), s));
    CB_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int), s));
    void* args[] = {&ga, &gb, &ki, &rots, &t2, &n2, &applied, &gsync, &err};
    if (cudaLaunchCooperativeKernel((const void*)sweep32_kernel, dim3(sms), dim3(512), args, 0, s) != cudaSuccess) {
      cudaGetLastError();
      return CHASE_BSE_CUDA_ERROR;
    }
    count_launch();
    vpass32_kernel<4><<<(unsigned)((k + 3) / 4), 128, vsm, s>>>(V32, ki, rots);
    count_launch();
    std::swap(ga, gb);
    count32_kernel<<<gsz(k * k), 256, 0, s>>>(ga, ki, t2, n2, cnt);
    count_launch();
    CB_CUDA(cudaMemcpyAsync(&hc, cnt, sizeof(int), cudaMemcpyDeviceToHost, s));
    CB_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s));
    CB_CUDA(cudaStreamSynchronize(s));
    if (herr) return CHASE_BSE_DEVICE_TIMEOUT;
  }
  if (sweeps32_out) *sweeps32_out = sw;
  // FP64: V1 = unitary factor of V32 (two Newton-Schulz steps), G1 = V1^* G V1
  cplx *X, *Y, *S, *G1, *V2;
  double* tmp;
  CB_TRY(ws.alloc(&X, k * k));
  CB_TRY(ws.alloc(&Y, k * k));
  CB_TRY(ws.alloc(&S, k * k));
  CB_TRY(ws.alloc(&G1, k * k));
  CB_TRY(ws.alloc(&V2, k * k));
  CB_TRY(ws.alloc(&tmp, 4 * k * k));
  SlicedOp sa, sb, sr;
  CB_TRY(sliced_alloc(ws, sa, k, 2 * k, s));
  CB_TRY(sliced_alloc(ws, sb, k, 2 * k, s));
  CB_TRY(sliced_alloc(ws, sr, 2 * k, 2 * k, s));
  to64_kernel<<<gsz(k * k), 256, 0, s>>>(V32, k * k, X);
  count_launch();
  CB_LAUNCH();
  // two steps of the Ogita-Aishima refinement: R = I - X^* X, S = X^* G X,
  // lam_i = s_ii / (1 - r_ii), X <- X (I + E) with the first-order correction E
  double* lamd;
  CB_TRY(ws.alloc(&lamd, k));
  for (int it = 0; it < 2; ++it) {
    CB_TRY(gemm_hn(X, X, k, S, ws, sa, sb, s));   // S = X^* X
    CB_TRY(gemm_nn(G, X, k, Y, tmp, sr, sb, s));  // Y = G X
    CB_TRY(gemm_hn(X, Y, k, G1, ws, sa, sb, s));  // G1 = X^* G X
    oa_lambda_kernel<<<(unsigned)((k + 255) / 256), 256, 0, s>>>(G1, S, k, lamd);
    count_launch();
    oa_correction_kernel<<<gsz(k * k), 256, 0, s>>>(G1, S, lamd, k, Y);
    count_launch();
    CB_LAUNCH();
    CB_TRY(gemm_nn(X, Y, k, S, tmp, sr, sb, s));  // S = X E
    add_kernel<<<gsz(k * k), 256, 0, s>>>(X, S, k * k);
    count_launch();
    CB_LAUNCH();
  }
  CB_TRY(gemm_nn(G, X, k, Y, tmp, sr, sb, s));  // Y = G V1
  CB_TRY(gemm_hn(X, Y, k, G1, ws, sa, sb, s));  // G1 = V1^* G V1
  CB_TRY(hermitize(G1, k, s));
  // What the refinement left (pairs of nearly equal eigenvalues) couples few indices:
  // the FP64 Jacobi runs on the sub-problem of the indices in a pair above the
  // threshold; the couplings between those and the others are below it.
  int* flags;
  CB_TRY(ws.alloc(&flags, k));
  CB_CUDA(cudaMemsetAsync(flags, 0, sizeof(int) * k, s));
  CB_TRY(offdiag_norms(G1, k, red, s));
  double g1[2];
  CB_CUDA(cudaMemcpyAsync(g1, red, sizeof(g1), cudaMemcpyDeviceToHost, s));
  CB_CUDA(cudaStreamSynchronize(s));
  const double tt = std::max(thr, 2e-16);
  mark_active_kernel<<<gsz(k * k), 256, 0, s>>>(G1, k, tt * tt, g1[1], flags);
  count_launch();
  CB_LAUNCH();
  std::vector<int> hf(k);
  CB_CUDA(cudaMemcpyAsync(hf.data(), flags, sizeof(int) * k, cudaMemcpyDeviceToHost, s));
  CB_CUDA(cudaStreamSynchronize(s));
  std::vector<int> act;
  for (int64_t i = 0; i < k; ++i)
    if (hf[i]) act.push_back((int)i);
  if (act.size() % 2)  // the Jacobi pairs indices: add one inactive index
    for (int64_t i = 0; i < k; ++i)
      if (!hf[i]) {
        act.push_back((int)i);
        break;
      }
  const int64_t m = (int64_t)act.size();
  if (verbose()) fprintf(stderr, "[chase_bse] jacobi k %ld: FP32 %d sweeps, FP64 on %ld active indices\n", (long)k,
                         sw, (long)m);
  if (m > k / 2) {  // most indices still coupled: the whole problem
    CB_TRY(jacobi_eigh(G1, k, V2, theta, rot, red, 40, sweeps64_out, s, thr));
    return jm::gemm_nn(X, V2, k, V, tmp, sr, sb, s);  // V = V1 V2
  }
  CB_TRY(diag_real(G1, k, theta, s));
  if (m == 0) {
    if (sweeps64_out) *sweeps64_out = 0;
    CB_CUDA(cudaMemcpyAsync(V, X, sizeof(cplx) * k * k, cudaMemcpyDeviceToDevice, s));
    return CHASE_BSE_OK;
  }
  int* actd;
  cplx *sub, *Vs;
  double* ts;
  CB_TRY(ws.alloc(&actd, m));
  CB_TRY(ws.alloc(&sub, m * m));
  CB_TRY(ws.alloc(&Vs, m * m));
  CB_TRY(ws.alloc(&ts, m));
  CB_CUDA(cudaMemcpyAsync(actd, act.data(), sizeof(int) * m, cudaMemcpyHostToDevice, s));
  gather_sub_kernel<<<gsz(m * m), 256, 0, s>>>(G1, k, actd, m, sub);
  count_launch();
  CB_LAUNCH();
  CB_TRY(jacobi_eigh(sub, m, Vs, ts, rot, red, 40, sweeps64_out, s, thr));
  CB_TRY(set_identity(V2, k, s));
  scatter_sub_kernel<<<gsz(m * m), 256, 0, s>>>(Vs, ts, actd, m, k, V2, theta);
  count_launch();
  CB_LAUNCH();
  CB_CUDA(cudaStreamSynchronize(s));  // act (host) outlives its copy
  return jm::gemm_nn(X, V2, k, V, tmp, sr, sb, s);  // V = V1 V2
}

}  // namespace cb
