// Mixed-precision eigensolver for the small hermitian problem of the oblique
// Rayleigh-Ritz step (G y = theta y in Algorithm 2), for G far from diagonal.
//
// GB300 runs FP32 at 64x its FP64 rate, so the bulk of the Jacobi work (the early
// sweeps, which rotate every pair) runs in FP32; FP64 accuracy is then recovered
// with FP64-accurate tensor-core GEMMs (sliced GEMM) and, if needed, a short FP64 Jacobi:
//   1. FP32 block Jacobi (jacobi_block.cu) on G (scaled to ||G||_F ~ 1) until every
//      |g_pq| is below 2e-6 sqrt|g_pp g_qq| or 1e-8 ||G|| (the FP32 rotations need
//      not be exactly unitary);
//   2. on X = the FP32 eigenvectors in FP64, two Newton-Schulz steps
//      X <- X (I + (I - X^* X)/2) (the FP32 products leave X unitary only to
//      ~1e-3), then three times a step of the iterative refinement of Ogita and
//      Aishima (2018, Japan J. Indust. Appl. Math.): with R = I - X^* X and
//      S = X^* G X, lam_i = s_ii / (1 - r_ii) and X <- X (I + E),
//      E_ij = (s_ij + lam_j r_ij) / (lam_j - lam_i) where that correction is small
//      (a pair test symmetric in i and j; the published method separates clusters
//      by a norm bound delta), else r_ij / 2, E_ii = r_ii / 2 (the first-order terms
//      of X = X^ (I + E), X^* X = I, X^* G X diagonal), each followed by two
//      Newton-Schulz steps (a refinement step squares the couplings of the separated
//      pairs but moves X away from unitarity by about the square of its
//      corrections); all the arithmetic is in FP64-accurate tensor-core GEMMs;
//   3. G1 = X^* G X, hermitised;
//   4. FP64 Jacobi on each cluster of indices of G1 still coupled above the
//      threshold (at least 1e-13 sqrt|g_ii g_jj|: what the refinement left, nearly
//      equal eigenvalues), one CTA per cluster, V = X V2.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "coop.cuh"
#include "dense_kernels.cuh"
#include "solver.cuh"
#include "tc_dgemm.cuh"

namespace cb {
namespace jm {

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

// E = (I - S) / 2 (the Newton-Schulz step toward the unitary factor: X <- X (I + E))
__global__ void ns_correction_kernel(const cplx* S, int64_t k, cplx* E) {
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < k * k;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const cplx v = S[idx];
    E[idx] = (idx % k == idx / k) ? mk(0.5 * (1.0 - v.x), -0.5 * v.y) : mk(-0.5 * v.x, -0.5 * v.y);
  }
}

// out[0] = max |S - I| (mode 0) or max |offdiag(S)| (mode 1), as float bits (diagnostics)
__global__ void max_dev_kernel(const cplx* S, int64_t k, int mode, unsigned* out) {
  float m = 0.0f;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < k * k;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const bool d = (idx % k) == (idx / k);
    if (mode == 1 && d) continue;
    cplx v = S[idx];
    if (d) v.x -= 1.0;
    m = fmaxf(m, (float)sqrt(cabs2(v)));
  }
  atomicMax(out, __float_as_uint(m));
}

// diagnostics: cnt[b] = pairs i < j with |g_ij| > 10^-(3 + 2b) sqrt|g_ii g_jj|, b < 6
__global__ void coupling_hist_kernel(const cplx* G, int64_t k, int* cnt) {
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < k * k;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = idx % k, j = idx / k;
    if (i >= j) continue;
    const double r = sqrt(cabs2(G[idx]) / fabs(G[i + i * k].x * G[j + j * k].x));
    double t = 1e-3;
    for (int b = 0; b < 6; ++b, t *= 1e-2)
      if (r > t) atomicAdd(cnt + b, 1);
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
  int dev = 0, coop = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
  double hred[2] = {0.0, 0.0};
  CB_TRY(offdiag_norms(G, k, red, s));
  CB_CUDA(cudaMemcpyAsync(hred, red, sizeof(hred), cudaMemcpyDeviceToHost, s));
  CB_CUDA(cudaStreamSynchronize(s));
  const double ratio = hred[1] > 0.0 ? std::sqrt(hred[0] / hred[1]) : 0.0;
  // near-diagonal G, small k or no cooperative launch: FP64 Jacobi alone
  if (k < 128 || k % 2 || ratio < 1e-4 || !coop || !mixed_available())
    return jacobi_eigh(G, k, V, theta, rot, red, 40, sweeps64_out, s, thr);
  Workspace ws(s);
  cplx *X, *Y, *S, *G1, *V2;
  double* tmp;
  CB_TRY(ws.alloc(&X, k * k));
  // the FP32 phase: block Jacobi (G scaled to ||G||_F in [1/2, 1)) until every
  // |g_pq| <= 2e-6 sqrt|g_pp g_qq| or <= 1e-8 ||G||_F; X = its eigenvectors in FP64
  int sw = 0;
  CB_TRY(jacobi_block(G, k, X, nullptr, true, 2e-6, 1e-8, 30, &sw, s));
  if (sweeps32_out) *sweeps32_out = sw;
  CB_TRY(ws.alloc(&Y, k * k));
  CB_TRY(ws.alloc(&S, k * k));
  CB_TRY(ws.alloc(&G1, k * k));
  CB_TRY(ws.alloc(&V2, k * k));
  CB_TRY(ws.alloc(&tmp, 4 * k * k));
  SlicedOp sa, sb, sr;
  CB_TRY(sliced_alloc(ws, sa, k, 2 * k, s));
  CB_TRY(sliced_alloc(ws, sb, k, 2 * k, s));
  CB_TRY(sliced_alloc(ws, sr, 2 * k, 2 * k, s));
  // Refinement in FP64-accurate tensor-core GEMMs.  The FP32 block Jacobi leaves X
  // diagonalising G to ~2e-6 but unitary only to ~1e-3 (its FP32 products accumulate
  // over the rounds), and a refinement step that corrects the couplings moves X away
  // from unitarity by about the square of its corrections, so the steps alternate:
  //   two Newton-Schulz steps X <- X (I + (I - X^* X)/2) (orthogonality error squared),
  //   then three times an Ogita-Aishima step (R = I - X^* X, S = X^* G X,
  //   lam_i = s_ii / (1 - r_ii), X <- X (I + E) with the first-order correction E)
  //   followed by two Newton-Schulz steps (corrections up to 1e-2 leave X unitary only
  //   to ~1e-4; two steps take that to the rounding level).
  double* lamd;
  CB_TRY(ws.alloc(&lamd, k));
  unsigned* dev_d = nullptr;
  if (verbose()) CB_TRY(ws.alloc(&dev_d, 1));
  auto report = [&](const cplx* M, int mode, const char* tag) {
    if (!dev_d) return;
    cudaMemsetAsync(dev_d, 0, sizeof(unsigned), s);
    max_dev_kernel<<<gsz(k * k), 256, 0, s>>>(M, k, mode, dev_d);
    unsigned h = 0;
    cudaMemcpyAsync(&h, dev_d, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
    cudaStreamSynchronize(s);
    float f;
    memcpy(&f, &h, sizeof(f));
    fprintf(stderr, "[chase_bse] refine k %ld %s %.2e\n", (long)k, tag, (double)f);
  };
  int* hist_d = nullptr;
  if (verbose()) CB_TRY(ws.alloc(&hist_d, 6));
  auto hist = [&](const cplx* M, const char* tag) {
    if (!hist_d) return;
    cudaMemsetAsync(hist_d, 0, 6 * sizeof(int), s);
    coupling_hist_kernel<<<gsz(k * k), 256, 0, s>>>(M, k, hist_d);
    int h[6];
    cudaMemcpyAsync(h, hist_d, sizeof(h), cudaMemcpyDeviceToHost, s);
    cudaStreamSynchronize(s);
    fprintf(stderr, "[chase_bse] refine k %ld %s pairs > 1e-3 %d, 1e-5 %d, 1e-7 %d, 1e-9 %d, 1e-11 %d, 1e-13 %d\n",
            (long)k, tag, h[0], h[1], h[2], h[3], h[4], h[5]);
  };
  auto ns_step = [&]() -> int {
    CB_TRY(gemm_hn(X, X, k, S, ws, sa, sb, s));  // S = X^* X
    report(S, 0, "ns: |X^*X - I|");
    ns_correction_kernel<<<gsz(k * k), 256, 0, s>>>(S, k, Y);
    count_launch();
    CB_LAUNCH();
    CB_TRY(gemm_nn(X, Y, k, S, tmp, sr, sb, s));  // S = X E
    add_kernel<<<gsz(k * k), 256, 0, s>>>(X, S, k * k);
    count_launch();
    CB_LAUNCH();
    return CHASE_BSE_OK;
  };
  auto oa_step = [&]() -> int {
    CB_TRY(gemm_hn(X, X, k, S, ws, sa, sb, s));   // S = X^* X
    CB_TRY(gemm_nn(G, X, k, Y, tmp, sr, sb, s));  // Y = G X
    CB_TRY(gemm_hn(X, Y, k, G1, ws, sa, sb, s));  // G1 = X^* G X
    report(S, 0, "oa: |X^*X - I|");
    report(G1, 1, "oa: |offdiag X^*GX|");
    hist(G1, "oa");
    oa_lambda_kernel<<<(unsigned)((k + 255) / 256), 256, 0, s>>>(G1, S, k, lamd);
    count_launch();
    oa_correction_kernel<<<gsz(k * k), 256, 0, s>>>(G1, S, lamd, k, Y);
    count_launch();
    CB_LAUNCH();
    CB_TRY(gemm_nn(X, Y, k, S, tmp, sr, sb, s));  // S = X E
    add_kernel<<<gsz(k * k), 256, 0, s>>>(X, S, k * k);
    count_launch();
    CB_LAUNCH();
    return CHASE_BSE_OK;
  };
  CB_TRY(ns_step());
  CB_TRY(ns_step());
  for (int it = 0; it < 3; ++it) {
    CB_TRY(oa_step());
    CB_TRY(ns_step());
    CB_TRY(ns_step());
  }
  CB_TRY(gemm_nn(G, X, k, Y, tmp, sr, sb, s));  // Y = G V1
  CB_TRY(gemm_hn(X, Y, k, G1, ws, sa, sb, s));  // G1 = V1^* G V1
  CB_TRY(hermitize(G1, k, s));
  if (dev_d) {
    CB_TRY(gemm_hn(X, X, k, S, ws, sa, sb, s));
    report(S, 0, "final: |X^*X - I|");
    report(G1, 1, "final: |offdiag X^*GX|");
    hist(G1, "final");
  }
  // What the refinement left coupled are clusters of nearly equal eigenvalues (pairs
  // whose coupling is not small against their gap, which the refinement only
  // re-orthogonalises).  The pairs above max(thr, 1e-13) sqrt|g_ii g_jj| (below that,
  // the level the FP64-accurate products resolve) are listed, their connected
  // components found on the host, and each component's sub-problem is solved by FP64
  // Jacobi: one CTA per component of at most 64 indices, FP64 block Jacobi on a
  // gathered sub-problem for larger ones.
  CB_TRY(offdiag_norms(G1, k, red, s));
  double g1[2];
  CB_CUDA(cudaMemcpyAsync(g1, red, sizeof(g1), cudaMemcpyDeviceToHost, s));
  CB_CUDA(cudaStreamSynchronize(s));
  const double tt = std::max(thr, 2e-16);
  const double ta = std::max(tt, 1e-13);
  const double floor_abs = 0.5 * ta * std::sqrt(g1[1]);
  CB_TRY(diag_real(G1, k, theta, s));
  std::vector<std::pair<int, int>> pairs;
  const int ps = coupled_pairs(G1, k, ta, floor_abs, pairs, 1 << 22, s);
  if (ps == CHASE_BSE_OOM) {  // too many coupled pairs to list: the whole problem
    CB_TRY(jacobi_block(G1, k, V2, theta, false, tt, 0.5 * tt, 40, sweeps64_out, s));
    return jm::gemm_nn(X, V2, k, V, tmp, sr, sb, s);  // V = V1 V2
  }
  CB_TRY(ps);
  if (pairs.empty()) {
    if (sweeps64_out) *sweeps64_out = 0;
    CB_CUDA(cudaMemcpyAsync(V, X, sizeof(cplx) * k * k, cudaMemcpyDeviceToDevice, s));
    CB_CUDA(cudaStreamSynchronize(s));
    return CHASE_BSE_OK;
  }
  // connected components (union-find with path halving)
  std::vector<int> parent(k);
  for (int64_t i = 0; i < k; ++i) parent[i] = (int)i;
  auto find = [&](int x) {
    while (parent[x] != x) {
      parent[x] = parent[parent[x]];
      x = parent[x];
    }
    return x;
  };
  for (const auto& pr : pairs) {
    const int a = find(pr.first), b = find(pr.second);
    if (a != b) parent[a < b ? b : a] = a < b ? a : b;
  }
  std::vector<std::vector<int>> comps;
  std::vector<int> cid(k, -1);
  for (int64_t i = 0; i < k; ++i) {
    const int r = find((int)i);
    if (cid[r] < 0) {
      cid[r] = (int)comps.size();
      comps.emplace_back();
    }
    comps[cid[r]].push_back((int)i);
  }
  std::vector<int> sidx, soff{0};
  int64_t clustered = 0, largest = 0;
  std::vector<const std::vector<int>*> big;
  for (const auto& c : comps) {
    if (c.size() < 2) continue;
    clustered += (int64_t)c.size();
    largest = std::max<int64_t>(largest, (int64_t)c.size());
    if (c.size() <= 64) {
      sidx.insert(sidx.end(), c.begin(), c.end());
      soff.push_back((int)sidx.size());
    } else {
      big.push_back(&c);
    }
  }
  if (verbose())
    fprintf(stderr, "[chase_bse] jacobi k %ld: FP32 %d sweeps, %zu coupled pairs, %ld clustered indices, largest %ld\n",
            (long)k, sw, pairs.size(), (long)clustered, (long)largest);
  CB_TRY(set_identity(V2, k, s));
  CB_TRY(cluster_eig(G1, k, sidx, soff, tt, floor_abs, V2, theta, s));
  int sw64 = 0;
  for (const std::vector<int>* c : big) {
    const int64_t m = (int64_t)c->size();
    int* actd;
    cplx *sub, *Vs;
    double* ts;
    Workspace cws(s);
    CB_TRY(cws.alloc(&actd, m));
    CB_TRY(cws.alloc(&sub, m * m));
    CB_TRY(cws.alloc(&Vs, m * m));
    CB_TRY(cws.alloc(&ts, m));
    CB_CUDA(cudaMemcpyAsync(actd, c->data(), sizeof(int) * m, cudaMemcpyHostToDevice, s));
    gather_sub_kernel<<<gsz(m * m), 256, 0, s>>>(G1, k, actd, m, sub);
    count_launch();
    CB_LAUNCH();
    int w = 0;
    CB_TRY(jacobi_block(sub, m, Vs, ts, false, tt, 0.5 * tt, 40, &w, s));
    sw64 = std::max(sw64, w);
    scatter_sub_kernel<<<gsz(m * m), 256, 0, s>>>(Vs, ts, actd, m, k, V2, theta);
    count_launch();
    CB_LAUNCH();
    CB_CUDA(cudaStreamSynchronize(s));  // c (host) outlives its copy
  }
  if (sweeps64_out) *sweeps64_out = sw64;
  return jm::gemm_nn(X, V2, k, V, tmp, sr, sb, s);  // V = V1 V2
}

}  // namespace cb
