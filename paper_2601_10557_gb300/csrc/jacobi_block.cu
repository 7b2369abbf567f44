// Block Jacobi eigensolver for the small hermitian problem G y = theta y of the
// Rayleigh-Ritz step (Algorithm 2), in FP32 or FP64.
//
// The indices (padded to a multiple of 64 with decoupled zero rows) are cut into
// blocks of 32; the blocks are paired round-robin, so a sweep has nb - 1 rounds
// (nb = k/32) instead of the k - 1 rounds of the scalar method.  One round is one
// cooperative kernel phase pair:
//   A  every block pair (I, J) runs one cyclic Jacobi sweep on its 64 x 64 sub-problem
//      S = G[I u J, I u J] in shared memory (63 inner rounds of 32 disjoint rotations,
//      the scalar method's rotation and threshold) and writes the accumulated unitary
//      U (64 x 64);
//   B  every 64 x 64 tile G[P_g, P_h] (g <= h, P = the pairs' index sets) becomes
//      U_g^* G[P_g, P_h] U_h, its mirror the conjugate transpose; and every 64 x 64
//      tile of V's columns P_g becomes V[rows, P_g] U_g.
// A grid barrier separates A from B and B from the next round's A.  Every access is
// a coalesced 32-element column segment of a block, instead of the scattered 2 x 2
// blocks of a scalar round, and the arithmetic of B is dense 64 x 64 products.  A
// rotation whose pivot is below the threshold is the identity, so a sweep on a
// matrix that is already diagonal leaves it unchanged.
#include <algorithm>
#include <cstdio>
#include <cmath>
#include <utility>
#include <vector>

#include "coop.cuh"
#include "dense_kernels.cuh"

namespace cb {
namespace bj {

constexpr int BS = 32;        // indices per block
constexpr int PS = 2 * BS;    // indices of a block pair
constexpr int THREADS = 256;

template <class R>
struct Cx;
template <>
struct Cx<float> {
  using T = float2;
  __device__ static T mk(float r, float i) { return make_float2(r, i); }
};
template <>
struct Cx<double> {
  using T = double2;
  __device__ static T mk(double r, double i) { return make_double2(r, i); }
};

template <class R>
struct BRot {
  R c, s, er, ei;
};

// Rotation J = [[c, s], [-s e, c e]] on (p, q) with G <- J^* G J annihilating g_pq
// (e = conj(g_pq)/|g_pq|, t = tan = sign(tau)/(|tau| + sqrt(1 + tau^2)),
// tau = (g_qq - g_pp)/(2 |g_pq|)); the identity unless |g_pq|^2 > t2 |g_pp g_qq| and
// |g_pq|^2 > f2 (f2: the absolute floor).
template <class R>
__device__ BRot<R> rotation(R app, R aqq, R pr, R pi, R t2, R f2) {
  BRot<R> Q{R(1), R(0), R(1), R(0)};
  const R r2 = pr * pr + pi * pi;
  if (!(r2 > t2 * fabs(app * aqq)) || !(r2 > f2) || !(r2 > R(0))) return Q;
  const R r = sqrt(r2);
  Q.er = pr / r;
  Q.ei = -pi / r;
  const R tau = R(0.5) * (aqq - app) / r;
  const R t = copysign(R(1), tau) / (fabs(tau) + sqrt(R(1) + tau * tau));
  Q.c = R(1) / sqrt(R(1) + t * t);
  Q.s = t * Q.c;
  return Q;
}

template <class R>
struct Params {
  typename Cx<R>::T* G;  // kp x kp, column-major, hermitian
  typename Cx<R>::T* V;  // kp x kp
  typename Cx<R>::T* U;  // nb/2 matrices of PS x PS
  int kp, nb;
  R t2, f2;
  GridSync* gsync;
  int* err;
  int* rotated;  // nb/2 flags: pair g of the current round applied a rotation
  int* nrot;     // rotated pairs, summed over the sweep
};

// global index of local index l (< 64) of the pair (I, J)
__device__ __forceinline__ int gidx(int l, int I, int J) { return l < BS ? BS * I + l : BS * J + (l - BS); }

// Phase A: one inner sweep on the sub-problem of pair g of round r.
template <class R>
__device__ void solve_pair(const Params<R>& P, int r, int g, typename Cx<R>::T* S, typename Cx<R>::T* Uu,
                           BRot<R>* rot) {
  using C = typename Cx<R>::T;
  int I, J;
  jpair32(g, r, P.nb, I, J);
  const int tid = threadIdx.x;
  constexpr int LD = PS + 1;
  for (int e = tid; e < PS * PS; e += THREADS) {
    const int i = e % PS, j = e / PS;
    S[i + j * LD] = __ldcg(P.G + gidx(i, I, J) + (int64_t)gidx(j, I, J) * P.kp);
    Uu[i + j * LD] = Cx<R>::mk(i == j ? R(1) : R(0), R(0));
  }
  __shared__ int any;
  if (tid == 0) any = 0;
  __syncthreads();
  for (int ir = 0; ir < PS - 1; ++ir) {
    if (tid < BS) {
      int p, q;
      jpair32(tid, ir, PS, p, q);
      const C x = S[p + q * LD];
      rot[tid] = rotation<R>(S[p + p * LD].x, S[q + q * LD].x, x.x, x.y, P.t2, P.f2);
      if (rot[tid].s != R(0)) any = 1;
    }
    __syncthreads();
    // S <- J^* S J on every 2 x 2 block (slots a, b)
    for (int item = tid; item < BS * BS; item += THREADS) {
      const int a = item / BS, b = item % BS;
      const BRot<R> A = rot[a], B = rot[b];
      if (A.s == R(0) && B.s == R(0)) continue;
      int pa, qa, pb, qb;
      jpair32(a, ir, PS, pa, qa);
      jpair32(b, ir, PS, pb, qb);
      const C x0 = S[pa + pb * LD], x1 = S[pa + qb * LD], x2 = S[qa + pb * LD], x3 = S[qa + qb * LD];
      // rows: [x0 x1; x2 x3] <- A^* [..]: row p' = c row p - s conj(e) row q, row q' = s row p + c conj(e) row q
      const R ar = A.er, ai = -A.ei;  // conj(e_A)
      const C w2 = Cx<R>::mk(ar * x2.x - ai * x2.y, ar * x2.y + ai * x2.x);
      const C w3 = Cx<R>::mk(ar * x3.x - ai * x3.y, ar * x3.y + ai * x3.x);
      const C y0 = Cx<R>::mk(A.c * x0.x - A.s * w2.x, A.c * x0.y - A.s * w2.y);
      const C y1 = Cx<R>::mk(A.c * x1.x - A.s * w3.x, A.c * x1.y - A.s * w3.y);
      const C y2 = Cx<R>::mk(A.s * x0.x + A.c * w2.x, A.s * x0.y + A.c * w2.y);
      const C y3 = Cx<R>::mk(A.s * x1.x + A.c * w3.x, A.s * x1.y + A.c * w3.y);
      // columns: col p' = c col p - s e col q... with J: col p' = c col p - s e col q, col q' = s col p + c e col q
      const R br = B.er, bi = B.ei;
      const C u1 = Cx<R>::mk(br * y1.x - bi * y1.y, br * y1.y + bi * y1.x);
      const C u3 = Cx<R>::mk(br * y3.x - bi * y3.y, br * y3.y + bi * y3.x);
      S[pa + pb * LD] = Cx<R>::mk(B.c * y0.x - B.s * u1.x, B.c * y0.y - B.s * u1.y);
      S[pa + qb * LD] = Cx<R>::mk(B.s * y0.x + B.c * u1.x, B.s * y0.y + B.c * u1.y);
      S[qa + pb * LD] = Cx<R>::mk(B.c * y2.x - B.s * u3.x, B.c * y2.y - B.s * u3.y);
      S[qa + qb * LD] = Cx<R>::mk(B.s * y2.x + B.c * u3.x, B.s * y2.y + B.c * u3.y);
    }
    // Uu <- Uu J (rows independent)
    for (int item = tid; item < PS * BS; item += THREADS) {
      const int i = item / BS, sl = item % BS;
      const BRot<R> B = rot[sl];
      if (B.s == R(0)) continue;
      int p, q;
      jpair32(sl, ir, PS, p, q);
      const C vp = Uu[i + p * LD], vq = Uu[i + q * LD];
      const C u = Cx<R>::mk(B.er * vq.x - B.ei * vq.y, B.er * vq.y + B.ei * vq.x);
      Uu[i + p * LD] = Cx<R>::mk(B.c * vp.x - B.s * u.x, B.c * vp.y - B.s * u.y);
      Uu[i + q * LD] = Cx<R>::mk(B.s * vp.x + B.c * u.x, B.s * vp.y + B.c * u.y);
    }
    __syncthreads();
  }
  // U stays exactly the identity when no rotation was applied: phase B then skips the
  // tiles of pairs that both kept the identity (a tile with one rotated pair still reads
  // this U)
  C* Ug = P.U + (int64_t)g * PS * PS;
  for (int e = tid; e < PS * PS; e += THREADS) Ug[e] = Uu[(e % PS) + (e / PS) * LD];
  if (tid == 0) {
    P.rotated[g] = any;
    if (any) atomicAdd(P.nrot, 1);
  }
  __syncthreads();
}

// out (64 x 64, ld LD) = op(X) * Y with X, Y 64 x 64 (ld LD) in shared memory;
// op(X) = X (conjx = false) or X^* (conjx = true).  Each thread owns a 4 x 4 tile.
template <class R>
__device__ __forceinline__ void mm64(const typename Cx<R>::T* X, const typename Cx<R>::T* Y, bool conjx,
                                     typename Cx<R>::T acc[4][4]) {
  using C = typename Cx<R>::T;
  constexpr int LD = PS + 1;
  const int tr = threadIdx.x % 16, tc = threadIdx.x / 16;  // rows tr + 16 i, columns tc + 16 j
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = Cx<R>::mk(R(0), R(0));
  for (int l = 0; l < PS; ++l) {
    C xa[4], yb[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int row = tr + 16 * i;
      if (conjx) {
        const C v = X[l + row * LD];
        xa[i] = Cx<R>::mk(v.x, -v.y);
      } else {
        xa[i] = X[row + l * LD];
      }
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) yb[j] = Y[l + (tc + 16 * j) * LD];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        acc[i][j].x = fma(xa[i].x, yb[j].x, acc[i][j].x);
        acc[i][j].x = fma(-xa[i].y, yb[j].y, acc[i][j].x);
        acc[i][j].y = fma(xa[i].x, yb[j].y, acc[i][j].y);
        acc[i][j].y = fma(xa[i].y, yb[j].x, acc[i][j].y);
      }
  }
}

template <class R>
__device__ void load_u(const Params<R>& P, int g, typename Cx<R>::T* Us) {
  constexpr int LD = PS + 1;
  const typename Cx<R>::T* Ug = P.U + (int64_t)g * PS * PS;
  for (int e = threadIdx.x; e < PS * PS; e += THREADS) Us[(e % PS) + (e / PS) * LD] = __ldcg(Ug + e);
}

// Phase B, G tile (g, h), g <= h: G[P_g, P_h] <- U_g^* G[P_g, P_h] U_h (and the mirror).
template <class R>
__device__ void update_tile(const Params<R>& P, int r, int g, int h, typename Cx<R>::T* T, typename Cx<R>::T* Ua,
                            typename Cx<R>::T* Ub) {
  using C = typename Cx<R>::T;
  constexpr int LD = PS + 1;
  int Ig, Jg, Ih, Jh;
  jpair32(g, r, P.nb, Ig, Jg);
  jpair32(h, r, P.nb, Ih, Jh);
  for (int e = threadIdx.x; e < PS * PS; e += THREADS) {
    const int i = e % PS, j = e / PS;
    T[i + j * LD] = __ldcg(P.G + gidx(i, Ig, Jg) + (int64_t)gidx(j, Ih, Jh) * P.kp);
  }
  load_u<R>(P, g, Ua);
  load_u<R>(P, h, Ub);
  __syncthreads();
  C acc[4][4];
  mm64<R>(T, Ub, false, acc);  // W = T U_h
  __syncthreads();
  const int tr = threadIdx.x % 16, tc = threadIdx.x / 16;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) T[(tr + 16 * i) + (tc + 16 * j) * LD] = acc[i][j];
  __syncthreads();
  mm64<R>(Ua, T, true, acc);  // U_g^* W
  __syncthreads();
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) T[(tr + 16 * i) + (tc + 16 * j) * LD] = acc[i][j];
  __syncthreads();
  for (int e = threadIdx.x; e < PS * PS; e += THREADS) {
    const int i = e % PS, j = e / PS;
    P.G[gidx(i, Ig, Jg) + (int64_t)gidx(j, Ih, Jh) * P.kp] = T[i + j * LD];
  }
  if (g != h) {
    for (int e = threadIdx.x; e < PS * PS; e += THREADS) {
      const int j = e % PS, i = e / PS;  // element (j of P_h, i of P_g) = conj(T[i, j])
      const C v = T[i + j * LD];
      P.G[gidx(j, Ih, Jh) + (int64_t)gidx(i, Ig, Jg) * P.kp] = Cx<R>::mk(v.x, -v.y);
    }
  }
  __syncthreads();
}

// Phase B, V tile: rows [64 c, 64 c + 64) of V's columns P_g <- times U_g.
template <class R>
__device__ void update_v(const Params<R>& P, int r, int c, int g, typename Cx<R>::T* T, typename Cx<R>::T* Ua) {
  using C = typename Cx<R>::T;
  constexpr int LD = PS + 1;
  int Ig, Jg;
  jpair32(g, r, P.nb, Ig, Jg);
  for (int e = threadIdx.x; e < PS * PS; e += THREADS) {
    const int i = e % PS, j = e / PS;
    T[i + j * LD] = __ldcg(P.V + (int64_t)PS * c + i + (int64_t)gidx(j, Ig, Jg) * P.kp);
  }
  load_u<R>(P, g, Ua);
  __syncthreads();
  C acc[4][4];
  mm64<R>(T, Ua, false, acc);
  const int tr = threadIdx.x % 16, tc = threadIdx.x / 16;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
      P.V[(int64_t)PS * c + tr + 16 * i + (int64_t)gidx(tc + 16 * j, Ig, Jg) * P.kp] = acc[i][j];
  __syncthreads();
}

template <class R>
__global__ void __launch_bounds__(THREADS, 1) bj_sweep_kernel(Params<R> P) {
  using C = typename Cx<R>::T;
  constexpr int LD = PS + 1;
  extern __shared__ __align__(16) unsigned char sm_raw[];
  C* T = reinterpret_cast<C*>(sm_raw);
  C* Ua = T + PS * LD;
  C* Ub = Ua + PS * LD;
  BRot<R>* rot = reinterpret_cast<BRot<R>*>(Ub + PS * LD);
  const int half = P.nb / 2;
  const int ntile = half * (half + 1) / 2;
  const int nvt = (P.kp / PS) * half;
  for (int r = 0; r < P.nb - 1; ++r) {
    for (int g = blockIdx.x; g < half; g += gridDim.x) solve_pair<R>(P, r, g, T, Ua, rot);
    if (!grid_barrier(P.gsync, P.err)) return;
    for (int item = blockIdx.x; item < ntile + nvt; item += gridDim.x) {
      if (item < ntile) {
        int g = 0, rem = item;  // item -> (g, h), g <= h, row by row of the upper triangle
        while (rem >= half - g) {
          rem -= half - g;
          ++g;
        }
        // U_g^* T U_h = T when neither pair rotated
        if (__ldcg(P.rotated + g) || __ldcg(P.rotated + g + rem)) update_tile<R>(P, r, g, g + rem, T, Ua, Ub);
      } else {
        const int v = item - ntile;
        if (__ldcg(P.rotated + v % half)) update_v<R>(P, r, v / half, v % half, T, Ua);
      }
    }
    if (!grid_barrier(P.gsync, P.err)) return;
  }
}

// couplings still above the thresholds (upper triangle)
template <class R>
__global__ void bj_count_kernel(const typename Cx<R>::T* G, int kp, R t2, R f2, int* count) {
  const int64_t total = (int64_t)kp * kp;
  int local = 0;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int p = (int)(idx % kp), q = (int)(idx / kp);
    if (p >= q) continue;
    const auto x = G[idx];
    const R r2 = x.x * x.x + x.y * x.y;
    if (r2 > t2 * fabs(G[p + (int64_t)p * kp].x * G[q + (int64_t)q * kp].x) && r2 > f2) ++local;
  }
  if (local) atomicAdd(count, local);
}

// Gp (kp x kp) = G * 2^-e padded with zeros, V = I
template <class R>
__global__ void bj_pad_kernel(const cplx* G, int64_t k, int64_t kp, int e, typename Cx<R>::T* Gp,
                              typename Cx<R>::T* V) {
  const int64_t total = kp * kp;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = idx % kp, j = idx / kp;
    cplx g = mk(0, 0);
    if (i < k && j < k) g = G[i + j * k];
    Gp[idx] = Cx<R>::mk((R)ldexp(g.x, -e), (R)ldexp(g.y, -e));
    V[idx] = Cx<R>::mk(i == j ? R(1) : R(0), R(0));
  }
}
// V (k x k, FP64) = the leading block of Vp; theta = 2^e diag(Gp) (leading k)
template <class R>
__global__ void bj_out_kernel(const typename Cx<R>::T* Vp, const typename Cx<R>::T* Gp, int64_t k, int64_t kp,
                              int e, cplx* V, double* theta) {
  const int64_t total = k * k;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = idx % k, j = idx / k;
    const auto v = Vp[i + j * kp];
    V[idx] = mk((double)v.x, (double)v.y);
    if (theta && i == j) theta[i] = ldexp((double)Gp[i + i * kp].x, e);
  }
}

static unsigned gsz(int64_t total) {
  const int64_t b = (total + 255) / 256;
  return (unsigned)std::min<int64_t>(std::max<int64_t>(b, 1), 8192);
}

// t: relative threshold (rotate when |g_pq| > t sqrt|g_pp g_qq|), f: absolute floor
// (and |g_pq| > f ||G||_F)
template <class R>
static int run(const cplx* G, int64_t k, cplx* V, double* theta, double t, double f, int max_sweeps,
               int* sweeps_out, cudaStream_t s) {
  using C = typename Cx<R>::T;
  if (sweeps_out) *sweeps_out = 0;
  if (k <= 0) return CHASE_BSE_OK;
  const int64_t kp = ((k + PS - 1) / PS) * PS;
  const int nb = (int)(kp / BS);
  int dev = 0, sms = 0, coop = 0;
  CB_CUDA(cudaGetDevice(&dev));
  CB_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  CB_CUDA(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
  if (!coop) return CHASE_BSE_UNSUPPORTED;
  const size_t smem = sizeof(C) * 3 * PS * (PS + 1) + sizeof(BRot<R>) * BS;
  static bool attr = false;
  if (!attr) {
    CB_CUDA(cudaFuncSetAttribute(bj_sweep_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    attr = true;
  }
  int per_sm = 0;
  CB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, bj_sweep_kernel<R>, THREADS, smem));
  if (per_sm < 1) return CHASE_BSE_UNSUPPORTED;
  Workspace ws(s);
  C *Gp, *Vp, *U;
  GridSync* gsync;
  int *err, *cnt, *rotated, *nrot;
  double* red;
  CB_TRY(ws.alloc(&rotated, nb / 2));
  CB_TRY(ws.alloc(&nrot, 1));
  CB_TRY(ws.alloc(&Gp, kp * kp));
  CB_TRY(ws.alloc(&Vp, kp * kp));
  CB_TRY(ws.alloc(&U, (int64_t)(nb / 2) * PS * PS));
  CB_TRY(ws.alloc(&gsync, 1));
  CB_TRY(ws.alloc(&err, 1));
  CB_TRY(ws.alloc(&cnt, 1));
  CB_TRY(ws.alloc(&red, 2));
  CB_CUDA(gsync_init(gsync, s));
  CB_CUDA(cudaMemsetAsync(err, 0, sizeof(int), s));
  // scale G to ||G||_F in [1/2, 1): exact, and FP32 keeps its range
  CB_TRY(offdiag_norms(G, k, red, s));
  double hred[2] = {0.0, 0.0};
  CB_CUDA(cudaMemcpyAsync(hred, red, sizeof(hred), cudaMemcpyDeviceToHost, s));
  CB_CUDA(cudaStreamSynchronize(s));
  int e = 0;
  if (hred[1] > 0.0) std::frexp(std::sqrt(hred[1]), &e);
  bj_pad_kernel<R><<<gsz(kp * kp), 256, 0, s>>>(G, k, kp, e, Gp, Vp);
  count_launch();
  CB_LAUNCH();
  const double n2 = hred[1] > 0.0 ? std::pow(std::ldexp(std::sqrt(hred[1]), -e), 2.0) : 0.0;
  Params<R> P{};
  P.G = Gp;
  P.V = Vp;
  P.U = U;
  P.kp = (int)kp;
  P.nb = nb;
  P.t2 = (R)(t * t);
  P.f2 = (R)(f * f * n2);
  P.gsync = gsync;
  P.err = err;
  P.rotated = rotated;
  P.nrot = nrot;
  const unsigned grid = (unsigned)std::min<int64_t>((int64_t)sms, std::max<int64_t>(1, (int64_t)nb * nb));
  int hc = 1, herr = 0, sw = 0;
  CB_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int), s));
  bj_count_kernel<R><<<gsz(kp * kp), 256, 0, s>>>(Gp, (int)kp, P.t2, P.f2, cnt);
  count_launch();
  CB_CUDA(cudaMemcpyAsync(&hc, cnt, sizeof(int), cudaMemcpyDeviceToHost, s));
  CB_CUDA(cudaStreamSynchronize(s));
  for (; hc > 0 && sw < max_sweeps; ++sw) {
    CB_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int), s));
    CB_CUDA(cudaMemsetAsync(nrot, 0, sizeof(int), s));
    void* args[] = {&P};
    if (cudaLaunchCooperativeKernel((const void*)bj_sweep_kernel<R>, dim3(grid), dim3(THREADS), args, smem, s) !=
        cudaSuccess) {
      cudaGetLastError();
      return CHASE_BSE_CUDA_ERROR;
    }
    count_launch();
    bj_count_kernel<R><<<gsz(kp * kp), 256, 0, s>>>(Gp, (int)kp, P.t2, P.f2, cnt);
    count_launch();
    CB_CUDA(cudaMemcpyAsync(&hc, cnt, sizeof(int), cudaMemcpyDeviceToHost, s));
    CB_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s));
    int hn = 0;
    if (verbose()) CB_CUDA(cudaMemcpyAsync(&hn, nrot, sizeof(int), cudaMemcpyDeviceToHost, s));
    CB_CUDA(cudaStreamSynchronize(s));
    if (herr) return CHASE_BSE_DEVICE_TIMEOUT;
    if (verbose())
      fprintf(stderr, "[chase_bse] block jacobi k %ld sweep %d: %d of %d block pairs rotated, %d couplings left\n",
              (long)k, sw + 1, hn, (nb - 1) * (nb / 2), hc);
  }
  if (sweeps_out) *sweeps_out = sw;
  bj_out_kernel<R><<<gsz(k * k), 256, 0, s>>>(Vp, Gp, k, kp, e, V, theta);
  count_launch();
  CB_LAUNCH();
  CB_CUDA(cudaStreamSynchronize(s));
  return CHASE_BSE_OK;
}

// Eigen-decomposition of the sub-problems G[c, c] of disjoint index sets c (at most 64
// indices each; the clusters of nearly equal eigenvalues that the refinement leaves
// coupled), one CTA per set: cyclic Jacobi sweeps in shared memory (zero padding is
// decoupled) until a sweep applies no rotation, at most 40 sweeps.  Writes the set's
// rows and columns of V2 (preset to the identity) and its entries of theta.
__global__ void __launch_bounds__(THREADS) cluster_eig_kernel(const cplx* G, int64_t k, const int* idx,
                                                               const int* off, double t2, double f2, cplx* V2,
                                                               double* theta) {
  using R = double;
  using C = double2;
  constexpr int LD = PS + 1;
  extern __shared__ __align__(16) unsigned char sm_raw[];
  C* S = reinterpret_cast<C*>(sm_raw);
  C* Uu = S + PS * LD;
  BRot<R>* rot = reinterpret_cast<BRot<R>*>(Uu + PS * LD);
  __shared__ int applied;
  const int j = blockIdx.x;
  const int o = off[j], c = off[j + 1] - o;
  const int tid = threadIdx.x;
  for (int e = tid; e < PS * PS; e += THREADS) {
    const int a = e % PS, b = e / PS;
    S[a + b * LD] = (a < c && b < c) ? G[idx[o + a] + (int64_t)idx[o + b] * k] : make_double2(0.0, 0.0);
    Uu[a + b * LD] = make_double2(a == b ? 1.0 : 0.0, 0.0);
  }
  __syncthreads();
  for (int sweep = 0; sweep < 40; ++sweep) {
    if (tid == 0) applied = 0;
    __syncthreads();
    for (int ir = 0; ir < PS - 1; ++ir) {
      if (tid < BS) {
        int p, q;
        jpair32(tid, ir, PS, p, q);
        const C x = S[p + q * LD];
        rot[tid] = rotation<R>(S[p + p * LD].x, S[q + q * LD].x, x.x, x.y, (R)t2, (R)f2);
        if (rot[tid].s != 0.0) atomicAdd(&applied, 1);
      }
      __syncthreads();
      for (int item = tid; item < BS * BS; item += THREADS) {
        const int a = item / BS, b = item % BS;
        const BRot<R> A = rot[a], B = rot[b];
        if (A.s == 0.0 && B.s == 0.0) continue;
        int pa, qa, pb, qb;
        jpair32(a, ir, PS, pa, qa);
        jpair32(b, ir, PS, pb, qb);
        const C x0 = S[pa + pb * LD], x1 = S[pa + qb * LD], x2 = S[qa + pb * LD], x3 = S[qa + qb * LD];
        const R ar = A.er, ai = -A.ei;
        const C w2 = make_double2(ar * x2.x - ai * x2.y, ar * x2.y + ai * x2.x);
        const C w3 = make_double2(ar * x3.x - ai * x3.y, ar * x3.y + ai * x3.x);
        const C y0 = make_double2(A.c * x0.x - A.s * w2.x, A.c * x0.y - A.s * w2.y);
        const C y1 = make_double2(A.c * x1.x - A.s * w3.x, A.c * x1.y - A.s * w3.y);
        const C y2 = make_double2(A.s * x0.x + A.c * w2.x, A.s * x0.y + A.c * w2.y);
        const C y3 = make_double2(A.s * x1.x + A.c * w3.x, A.s * x1.y + A.c * w3.y);
        const R br = B.er, bi = B.ei;
        const C u1 = make_double2(br * y1.x - bi * y1.y, br * y1.y + bi * y1.x);
        const C u3 = make_double2(br * y3.x - bi * y3.y, br * y3.y + bi * y3.x);
        S[pa + pb * LD] = make_double2(B.c * y0.x - B.s * u1.x, B.c * y0.y - B.s * u1.y);
        S[pa + qb * LD] = make_double2(B.s * y0.x + B.c * u1.x, B.s * y0.y + B.c * u1.y);
        S[qa + pb * LD] = make_double2(B.c * y2.x - B.s * u3.x, B.c * y2.y - B.s * u3.y);
        S[qa + qb * LD] = make_double2(B.s * y2.x + B.c * u3.x, B.s * y2.y + B.c * u3.y);
      }
      for (int item = tid; item < PS * BS; item += THREADS) {
        const int i = item / BS, sl = item % BS;
        const BRot<R> B = rot[sl];
        if (B.s == 0.0) continue;
        int p, q;
        jpair32(sl, ir, PS, p, q);
        const C vp = Uu[i + p * LD], vq = Uu[i + q * LD];
        const C u = make_double2(B.er * vq.x - B.ei * vq.y, B.er * vq.y + B.ei * vq.x);
        Uu[i + p * LD] = make_double2(B.c * vp.x - B.s * u.x, B.c * vp.y - B.s * u.y);
        Uu[i + q * LD] = make_double2(B.s * vp.x + B.c * u.x, B.s * vp.y + B.c * u.y);
      }
      __syncthreads();
    }
    if (applied == 0) break;
    __syncthreads();
  }
  for (int e = tid; e < c * c; e += THREADS) {
    const int a = e % c, b = e / c;
    V2[idx[o + a] + (int64_t)idx[o + b] * k] = Uu[a + b * LD];
  }
  for (int a = tid; a < c; a += THREADS) theta[idx[o + a]] = S[a + a * LD].x;
}

// Pairs i < j with |g_ij|^2 > t2 |g_ii g_jj| and > f2, appended to pairs (at most cap of
// them; *count may exceed cap, meaning the list is incomplete).
__global__ void coupled_pairs_kernel(const cplx* G, int64_t k, double t2, double f2, int2* pairs, int cap,
                                     int* count) {
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < k * k;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = idx % k, j = idx / k;
    if (i >= j) continue;
    const double r2 = cabs2(G[idx]);
    if (r2 > t2 * fabs(G[i + i * k].x * G[j + j * k].x) && r2 > f2) {
      const int slot = atomicAdd(count, 1);
      if (slot < cap) pairs[slot] = make_int2((int)i, (int)j);
    }
  }
}

}  // namespace bj

int coupled_pairs(const cplx* G, int64_t k, double t, double floor_abs, std::vector<std::pair<int, int>>& out,
                  int cap, cudaStream_t s) {
  out.clear();
  Workspace ws(s);
  int2* pairs;
  int* cnt;
  CB_TRY(ws.alloc(&pairs, cap));
  CB_TRY(ws.alloc(&cnt, 1));
  CB_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int), s));
  bj::coupled_pairs_kernel<<<bj::gsz(k * k), 256, 0, s>>>(G, k, t * t, floor_abs * floor_abs, pairs, cap, cnt);
  count_launch();
  CB_LAUNCH();
  int hc = 0;
  CB_CUDA(cudaMemcpyAsync(&hc, cnt, sizeof(int), cudaMemcpyDeviceToHost, s));
  CB_CUDA(cudaStreamSynchronize(s));
  if (hc > cap) return CHASE_BSE_OOM;  // the list does not fit: the caller falls back
  std::vector<int2> h(hc);
  if (hc > 0) {
    CB_CUDA(cudaMemcpyAsync(h.data(), pairs, sizeof(int2) * hc, cudaMemcpyDeviceToHost, s));
    CB_CUDA(cudaStreamSynchronize(s));
  }
  out.reserve(hc);
  for (const int2& p : h) out.push_back({p.x, p.y});
  return CHASE_BSE_OK;
}

int cluster_eig(const cplx* G, int64_t k, const std::vector<int>& idx, const std::vector<int>& off, double thr,
                double floor_abs, cplx* V2, double* theta, cudaStream_t s) {
  const int ncl = (int)off.size() - 1;
  if (ncl <= 0) return CHASE_BSE_OK;
  for (int j = 0; j < ncl; ++j)
    if (off[j + 1] - off[j] > bj::PS) return CHASE_BSE_BAD_ARG;
  Workspace ws(s);
  int *di, *doff;
  CB_TRY(ws.alloc(&di, (int64_t)idx.size()));
  CB_TRY(ws.alloc(&doff, (int64_t)off.size()));
  CB_CUDA(cudaMemcpyAsync(di, idx.data(), sizeof(int) * idx.size(), cudaMemcpyHostToDevice, s));
  CB_CUDA(cudaMemcpyAsync(doff, off.data(), sizeof(int) * off.size(), cudaMemcpyHostToDevice, s));
  const size_t smem = sizeof(double2) * 2 * bj::PS * (bj::PS + 1) + sizeof(bj::BRot<double>) * bj::BS;
  static bool attr = false;
  if (!attr) {
    CB_CUDA(cudaFuncSetAttribute(bj::cluster_eig_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    attr = true;
  }
  bj::cluster_eig_kernel<<<(unsigned)ncl, bj::THREADS, smem, s>>>(G, k, di, doff, thr * thr, floor_abs * floor_abs,
                                                                  V2, theta);
  count_launch();
  CB_LAUNCH();
  CB_CUDA(cudaStreamSynchronize(s));  // the host vectors outlive their copies
  return CHASE_BSE_OK;
}

int jacobi_block(const cplx* G, int64_t k, cplx* V, double* theta, bool fp32, double thr, double floor_rel,
                 int max_sweeps, int* sweeps_out, cudaStream_t s) {
  if (fp32) return bj::run<float>(G, k, V, theta, thr, floor_rel, max_sweeps, sweeps_out, s);
  return bj::run<double>(G, k, V, theta, std::max(thr, 2e-16), floor_rel, max_sweeps, sweeps_out, s);
}

}  // namespace cb
