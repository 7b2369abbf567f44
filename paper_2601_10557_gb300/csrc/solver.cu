// Host driver of the pseudo-hermitian ChASE solver (Algorithm 3) and its stages.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <numeric>
#include <mutex>
#include <vector>

#include "dense_kernels.cuh"
#include "fp64_kernels.cuh"
#include "solver.cuh"
#include "tc_dgemm.cuh"

namespace cb {

namespace {
std::mutex g_pool_mu;
cudaMemPool_t g_pools[64] = {};
}  // namespace

static std::atomic<uint64_t> g_wait_limit{0};
uint64_t wait_limit_ns() { return g_wait_limit.load(std::memory_order_relaxed); }
void set_wait_limit_ns(uint64_t ns) { g_wait_limit.store(ns, std::memory_order_relaxed); }

static std::atomic<int64_t> g_allocs{0};
int64_t alloc_count() { return g_allocs.load(std::memory_order_relaxed); }

cudaError_t dalloc(void** p, size_t bytes, cudaStream_t s) {
  g_allocs.fetch_add(1, std::memory_order_relaxed);
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaMallocAsync(p, bytes, s);
  cudaMemPool_t pool;
  {
    std::lock_guard<std::mutex> lock(g_pool_mu);
    if (!g_pools[dev]) {
      cudaMemPoolProps props{};
      props.allocType = cudaMemAllocationTypePinned;
      props.location.type = cudaMemLocationTypeDevice;
      props.location.id = dev;
      e = cudaMemPoolCreate(&g_pools[dev], &props);
      if (e != cudaSuccess) {
        g_pools[dev] = nullptr;
        return e;
      }
      uint64_t thr = UINT64_MAX;
      cudaMemPoolSetAttribute(g_pools[dev], cudaMemPoolAttrReleaseThreshold, &thr);
    }
    pool = g_pools[dev];
  }
  return cudaMallocFromPoolAsync(p, bytes, pool, s);
}

void pool_trim() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return;
  std::lock_guard<std::mutex> lock(g_pool_mu);
  if (g_pools[dev]) cudaMemPoolTrimTo(g_pools[dev], 0);
}

static std::atomic<int64_t> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
int64_t launch_count() { return g_launches.load(std::memory_order_relaxed); }

// Device-time record of the filter's H applications (diagnostics).  While it is
// on, every launch of the tensor-core filter GEMM (kind 0), of the FP64 H
// application (kind 1) and every sliced H application (kind 2) is bracketed by a
// pair of CUDA events on its stream.
// Completed pairs are harvested without blocking at the next bracket, so the
// record holds at most a few launches in flight.
namespace {
struct TimerPair {
  cudaEvent_t a, b;
  int kind;
  int64_t id;
  double flops;
  bool closed;  // the end event has been recorded
};
std::mutex g_timer_mu;
bool g_timer_on = false;
std::vector<TimerPair> g_timer_open;   // recorded, not yet harvested
std::vector<TimerPair> g_timer_spare;  // harvested, events reusable
constexpr int kTimerKinds = 3;
double g_timer_ms[kTimerKinds] = {};
double g_timer_flops[kTimerKinds] = {};
int64_t g_timer_n[kTimerKinds] = {};
int64_t g_timer_next = 0;

void timer_harvest(bool wait) {
  size_t keep = 0;
  for (size_t i = 0; i < g_timer_open.size(); ++i) {
    TimerPair& t = g_timer_open[i];
    if (!t.closed) {
      g_timer_open[keep++] = t;
      continue;
    }
    cudaError_t q = wait ? cudaEventSynchronize(t.b) : cudaEventQuery(t.b);
    if (q == cudaSuccess) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, t.a, t.b) == cudaSuccess) {
        g_timer_ms[t.kind] += ms;
        g_timer_flops[t.kind] += t.flops;
        g_timer_n[t.kind] += 1;
      }
      g_timer_spare.push_back(t);
    } else {
      if (q != cudaErrorNotReady) cudaGetLastError();
      g_timer_open[keep++] = t;
    }
  }
  g_timer_open.resize(keep);
}
}  // namespace

int64_t timer_begin(int kind, double flops, cudaStream_t s) {
  std::lock_guard<std::mutex> lock(g_timer_mu);
  if (!g_timer_on) return -1;
  timer_harvest(false);
  TimerPair t{};
  if (!g_timer_spare.empty()) {
    t = g_timer_spare.back();
    g_timer_spare.pop_back();
  } else if (cudaEventCreate(&t.a) != cudaSuccess || cudaEventCreate(&t.b) != cudaSuccess) {
    cudaGetLastError();
    return -1;
  }
  t.kind = kind;
  t.flops = flops;
  t.id = g_timer_next++;
  t.closed = false;
  if (cudaEventRecord(t.a, s) != cudaSuccess) {
    cudaGetLastError();
    g_timer_spare.push_back(t);
    return -1;
  }
  g_timer_open.push_back(t);
  return t.id;
}

void timer_end(int64_t id, cudaStream_t s) {
  if (id < 0) return;
  std::lock_guard<std::mutex> lock(g_timer_mu);
  for (size_t i = g_timer_open.size(); i-- > 0;) {
    if (g_timer_open[i].id == id) {
      if (cudaEventRecord(g_timer_open[i].b, s) == cudaSuccess)
        g_timer_open[i].closed = true;
      else
        cudaGetLastError();
      return;
    }
  }
}

void timer_enable(bool on) {
  std::lock_guard<std::mutex> lock(g_timer_mu);
  timer_harvest(true);
  for (const TimerPair& t : g_timer_open) g_timer_spare.push_back(t);  // brackets never closed
  g_timer_open.clear();
  g_timer_on = on;
  for (int i = 0; i < kTimerKinds; ++i) {
    g_timer_ms[i] = 0.0;
    g_timer_flops[i] = 0.0;
    g_timer_n[i] = 0;
  }
}

int timer_read(int kind, double* ms, double* flops, int64_t* launches) {
  std::lock_guard<std::mutex> lock(g_timer_mu);
  timer_harvest(true);
  *ms = g_timer_ms[kind];
  *flops = g_timer_flops[kind];
  *launches = g_timer_n[kind];
  g_timer_ms[kind] = 0.0;
  g_timer_flops[kind] = 0.0;
  g_timer_n[kind] = 0;
  return CHASE_BSE_OK;
}

bool verbose() {
  static int v = -1;
  if (v < 0) {
    const char* e = getenv("CHASE_BSE_VERBOSE");
    v = (e && e[0] && e[0] != '0') ? 1 : 0;
  }
  return v == 1;
}

// ------------------------------------------------------------------- filter
// nxt = alpha (HT - c cur) + beta prev over `total` entries (the recurrence step of the
// FP64 filter whose H applications ran as sliced tensor-core GEMMs)
__global__ void cheb_combine_kernel(cplx* nxt, const cplx* HT, const cplx* cur, const cplx* prev, double alpha,
                                    double beta, double c, int64_t total) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const cplx h = HT[i], y = cur[i];
    cplx z = mk(alpha * (h.x - c * y.x), alpha * (h.y - c * y.y));
    if (beta != 0.0) {
      const cplx p = prev[i];
      z.x = fma(beta, p.x, z.x);
      z.y = fma(beta, p.y, z.y);
    }
    nxt[i] = z;
  }
}

// FP64 three-term recurrence on H^2 over columns sorted by descending degree:
// at step j only the prefix of columns with deg >= j+1 is active.  Y_j lives in
// buffer j mod 3; a finished column keeps its last iterate in buffer deg mod 3.
// With ph (the sliced operand of slice_hamiltonian) both H applications of a step run
// as FP64-accurate sliced GEMMs on the tensor cores, else on the FP64 pipe (the second
// one with the recurrence fused).
static int filter_fp64_sorted(const cplx* A, const cplx* B, int64_t n, cplx* Y0, int64_t k, const int* degs,
                              double mu1, double mu_nevex, double muN, cplx* out, Workspace& ws, cudaStream_t s,
                              FilterStats* fs, const SlicedOp* ph) {
  const int64_t n2 = 2 * n;
  cplx *Y1, *Y2, *T, *HT = nullptr;
  CB_TRY(ws.alloc(&Y1, n2 * k));
  CB_TRY(ws.alloc(&Y2, n2 * k));
  CB_TRY(ws.alloc(&T, n2 * k));
  if (ph) CB_TRY(ws.alloc(&HT, n2 * k));
  cplx* Yb[3] = {Y0, Y1, Y2};
  const double a = mu_nevex * mu_nevex, b = muN * muN;
  const double c = 0.5 * (a + b), e = 0.5 * (b - a);
  const double sigma1 = e / (mu1 * mu1 - c);
  const double tau = 2.0 / sigma1;
  double sigma = sigma1;
  const int maxdeg = degs[0];
  cudaEvent_t e0, e1;
  CB_CUDA(cudaEventCreate(&e0));
  CB_CUDA(cudaEventCreate(&e1));
  CB_CUDA(cudaEventRecord(e0, s));
  for (int j = 0; j < maxdeg; ++j) {
    int64_t kj = 0;
    while (kj < k && degs[kj] >= j + 1) ++kj;
    cplx* cur = Yb[j % 3];
    cplx* nxt = Yb[(j + 1) % 3];
    cplx* prev = Yb[(j + 2) % 3];
    if (ph) {
      CB_TRY(hop_sliced(*ph, cur, n, kj, T, s));
    } else {
      HopArgs h{};
      h.A = A; h.B = B; h.n = n; h.W = cur; h.k = kj; h.out = T; h.mode = HOP_STORE;
      CB_TRY(hop_fp64(h, s));
    }
    double alpha, beta;
    if (j == 0) {
      alpha = sigma1 / e;
      beta = 0.0;
    } else {
      const double sn = 1.0 / (tau - sigma);
      alpha = 2.0 * sn / e;
      beta = -sigma * sn;
      sigma = sn;
    }
    if (ph) {
      CB_TRY(hop_sliced(*ph, T, n, kj, HT, s));
      const int64_t total = n2 * kj;
      const unsigned blocks = (unsigned)std::min<int64_t>((total + 255) / 256, 8192);
      cheb_combine_kernel<<<blocks, 256, 0, s>>>(nxt, HT, cur, prev, alpha, beta, c, total);
      count_launch();
      CB_LAUNCH();
    } else {
      HopArgs g{};
      g.A = A; g.B = B; g.n = n; g.W = T; g.k = kj; g.out = nxt; g.mode = HOP_CHEB;
      g.alpha = alpha; g.beta = beta; g.c = c; g.Wc = cur; g.Wp = prev;
      CB_TRY(hop_fp64(g, s));
    }
    if (fs) {
      fs->flops += 64.0 * (double)n * (double)n * (double)kj;
      fs->flops_fp64 += 64.0 * (double)n * (double)n * (double)kj;
      fs->launches += 2;
    }
  }
  CB_CUDA(cudaEventRecord(e1, s));
  std::vector<int> sel(k);
  for (int64_t i = 0; i < k; ++i) sel[i] = degs[i] % 3;
  int* dsel;
  CB_TRY(ws.alloc(&dsel, k));
  CB_CUDA(cudaMemcpyAsync(dsel, sel.data(), sizeof(int) * k, cudaMemcpyHostToDevice, s));
  CB_TRY(collect_cols(out, Yb[0], Yb[1], Yb[2], dsel, n2, k, s));
  if (fs) {
    CB_CUDA(cudaEventSynchronize(e1));
    float ms = 0;
    CB_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    fs->ms_fp64 += ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return CHASE_BSE_OK;
}

int filter(const cplx* A, const cplx* B, int64_t n, cplx* W, int64_t k, const int* degs, const int* prec,
           double mu1, double mu_nevex, double muN, int scheme, const double* ritz, const cplx* R, cudaStream_t s,
           FilterStats* fs, const SlicedOp* ph, const cplx* P2, const cplx* Q2) {
  if (k == 0) return CHASE_BSE_OK;
  const int64_t n2 = 2 * n;
  Workspace ws(s);
  // group 0: FP64 columns, group 1: mixed columns; each sorted by descending degree
  for (int grp = 0; grp < 2; ++grp) {
    std::vector<int> idx;
    for (int64_t i = 0; i < k; ++i)
      if ((prec ? prec[i] : 0) == grp) idx.push_back((int)i);
    if (idx.empty()) continue;
    std::stable_sort(idx.begin(), idx.end(), [&](int x, int y) { return degs[x] > degs[y]; });
    const int64_t m = (int64_t)idx.size();
    std::vector<int> ds(m);
    for (int64_t i = 0; i < m; ++i) ds[i] = degs[idx[i]];
    int* didx;
    cplx *Y0, *out;
    Workspace gws(s);
    CB_TRY(gws.alloc(&didx, m));
    CB_TRY(gws.alloc(&Y0, n2 * m));
    CB_TRY(gws.alloc(&out, n2 * m));
    CB_CUDA(cudaMemcpyAsync(didx, idx.data(), sizeof(int) * m, cudaMemcpyHostToDevice, s));
    CB_TRY(gather_cols(Y0, W, didx, n2, m, s));
    if (grp == 0) {
      CB_TRY(filter_fp64_sorted(A, B, n, Y0, m, ds.data(), mu1, mu_nevex, muN, out, gws, s, fs, ph));
    } else {
      if (!mixed_available()) return CHASE_BSE_UNSUPPORTED;
      if (ritz && R) {
        cplx* Rs;
        CB_TRY(gws.alloc(&Rs, n2 * m));
        CB_TRY(gather_cols(Rs, R, didx, n2, m, s));
        std::vector<double> rs(m);
        for (int64_t i = 0; i < m; ++i) rs[i] = ritz[idx[i]];
        CB_TRY(filter_mixed_correction_sorted(A, B, n, Y0, m, ds.data(), rs.data(), Rs, mu1, mu_nevex, muN, out,
                                              scheme, s, fs, P2, Q2));
      } else {
        CB_TRY(filter_mixed_sorted(A, B, n, Y0, m, ds.data(), mu1, mu_nevex, muN, out, scheme, s, fs, P2, Q2));
      }
    }
    CB_TRY(scatter_cols(W, out, didx, n2, m, s));
    // host vectors idx/ds must outlive the async copies: synchronise before they go
    CB_CUDA(cudaStreamSynchronize(s));
  }
  return CHASE_BSE_OK;
}

// ------------------------------------------------------------------ Lanczos
// Jacobi eigen-decomposition of a small real symmetric matrix (host; used only
// for the Lanczos tridiagonal matrices, at most a few dozen rows).
static void host_sym_eig(std::vector<double>& a, int m, std::vector<double>& w, std::vector<double>& v) {
  v.assign((size_t)m * m, 0.0);
  for (int i = 0; i < m; ++i) v[(size_t)i * m + i] = 1.0;
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int i = 0; i < m; ++i)
      for (int j = 0; j < m; ++j) {
        tot += a[(size_t)i * m + j] * a[(size_t)i * m + j];
        if (i != j) off += a[(size_t)i * m + j] * a[(size_t)i * m + j];
      }
    if (off <= 1e-30 * tot) break;
    for (int p = 0; p < m - 1; ++p)
      for (int q = p + 1; q < m; ++q) {
        const double apq = a[(size_t)p * m + q];
        if (apq == 0.0) continue;
        const double tau = (a[(size_t)q * m + q] - a[(size_t)p * m + p]) / (2.0 * apq);
        const double t = (tau >= 0 ? 1.0 : -1.0) / (std::fabs(tau) + std::sqrt(1.0 + tau * tau));
        const double c = 1.0 / std::sqrt(1.0 + t * t), sn = t * c;
        for (int r = 0; r < m; ++r) {  // columns p, q
          const double x = a[(size_t)r * m + p], y = a[(size_t)r * m + q];
          a[(size_t)r * m + p] = c * x - sn * y;
          a[(size_t)r * m + q] = sn * x + c * y;
        }
        for (int r = 0; r < m; ++r) {  // rows p, q
          const double x = a[(size_t)p * m + r], y = a[(size_t)q * m + r];
          a[(size_t)p * m + r] = c * x - sn * y;
          a[(size_t)q * m + r] = sn * x + c * y;
        }
        for (int r = 0; r < m; ++r) {
          const double x = v[(size_t)r * m + p], y = v[(size_t)r * m + q];
          v[(size_t)r * m + p] = c * x - sn * y;
          v[(size_t)r * m + q] = sn * x + c * y;
        }
      }
  }
  w.resize(m);
  for (int i = 0; i < m; ++i) w[i] = a[(size_t)i * m + i];
}

int lanczos_bounds(const cplx* A, const cplx* B, int64_t n, const cplx* V0, int64_t nvec, int steps,
                   int64_t nevex, double out[4], cudaStream_t s, const SlicedOp* ph) {
  const int64_t n2 = 2 * n, sz = n2 * nvec;
  Workspace ws(s);
  cplx *Vp, *V, *U, *Wv, *Y;
  double *alpha, *beta, *nrm2, *b0;
  CB_TRY(ws.alloc(&Vp, sz));
  CB_TRY(ws.alloc(&V, sz));
  CB_TRY(ws.alloc(&U, sz));
  CB_TRY(ws.alloc(&Wv, sz));
  CB_TRY(ws.alloc(&Y, sz));
  CB_TRY(ws.alloc(&alpha, (size_t)steps * nvec));
  CB_TRY(ws.alloc(&beta, (size_t)steps * nvec));
  CB_TRY(ws.alloc(&nrm2, nvec));
  CB_TRY(ws.alloc(&b0, nvec));
  CB_CUDA(cudaMemcpyAsync(Wv, V0, sizeof(cplx) * sz, cudaMemcpyDeviceToDevice, s));
  HopArgs h{};
  h.A = A; h.B = B; h.n = n; h.k = nvec; h.mode = HOP_STORE;
  h.W = Wv; h.out = Y;
  // H applied on the FP64 pipe, or (mixed mode) by the sliced tensor-core GEMM
  auto apply_h = [&]() { return ph ? hop_sliced(*ph, Wv, n, nvec, Y, s) : hop_fp64(h, s); };
  CB_TRY(apply_h());
  CB_TRY(sdot_real(Wv, Y, n, nvec, nrm2, s));
  CB_TRY(lanczos_normalise(b0, nrm2, Wv, Y, V, U, n, nvec, s));
  for (int j = 0; j < steps; ++j) {
    CB_TRY(sdot_real(U, U, n, nvec, alpha + (size_t)j * nvec, s));  // alpha_j = u^* S u, u = H v
    CB_TRY(lanczos_axpy(Wv, U, V, Vp, alpha + (size_t)j * nvec, j > 0 ? beta + (size_t)(j - 1) * nvec : nullptr, n,
                        nvec, s));
    h.W = Wv; h.out = Y;
    CB_TRY(apply_h());
    CB_TRY(sdot_real(Wv, Y, n, nvec, nrm2, s));
    std::swap(Vp, V);
    CB_TRY(lanczos_normalise(beta + (size_t)j * nvec, nrm2, Wv, Y, V, U, n, nvec, s));
  }
  std::vector<double> ha((size_t)steps * nvec), hb((size_t)steps * nvec);
  CB_CUDA(cudaMemcpyAsync(ha.data(), alpha, sizeof(double) * ha.size(), cudaMemcpyDeviceToHost, s));
  CB_CUDA(cudaMemcpyAsync(hb.data(), beta, sizeof(double) * hb.size(), cudaMemcpyDeviceToHost, s));
  CB_CUDA(cudaStreamSynchronize(s));
  double mu1 = INFINITY, muN = 0.0, rhat = 0.0;
  std::vector<std::pair<double, double>> pos;  // (theta, weight) over theta > 0
  for (int64_t cidx = 0; cidx < nvec; ++cidx) {
    int m = steps;
    for (int j = 0; j < steps; ++j)
      if (!(hb[(size_t)j * nvec + cidx] > 0.0) && j + 1 < steps) { m = j + 1; break; }
    std::vector<double> T((size_t)m * m, 0.0), w, v;
    for (int j = 0; j < m; ++j) {
      T[(size_t)j * m + j] = ha[(size_t)j * nvec + cidx];
      if (j + 1 < m) {
        T[(size_t)j * m + j + 1] = hb[(size_t)j * nvec + cidx];
        T[(size_t)(j + 1) * m + j] = hb[(size_t)j * nvec + cidx];
      }
    }
    host_sym_eig(T, m, w, v);
    double mx = 0.0;
    for (int i = 0; i < m; ++i) {
      mu1 = std::min(mu1, std::fabs(w[i]));
      mx = std::max(mx, std::fabs(w[i]));
      // weight tau_j / theta_j: the S H inner product weighs eigenvalue lambda by lambda
      if (w[i] > 0) pos.push_back({w[i], v[i] * v[i] / w[i]});  // v[i]: first row of eigenvectors
    }
    rhat = std::max(rhat, mx);
    muN = std::max(muN, mx + std::fabs(hb[(size_t)(m - 1) * nvec + cidx]));
  }
  std::sort(pos.begin(), pos.end());
  double tot = 0.0;
  for (auto& p : pos) tot += p.second;
  const double target = (double)nevex / (double)n;
  double mu_ne = pos.empty() ? mu1 : pos.back().first;
  double px = mu1, py = 0.0, cum = 0.0;
  for (auto& p : pos) {
    const double nx = p.first, ny = cum + p.second / tot;
    if (ny >= target) {
      mu_ne = (ny > py) ? px + (target - py) / (ny - py) * (nx - px) : nx;
      break;
    }
    px = nx;
    py = ny;
    cum = ny;
  }
  out[0] = mu1;
  out[1] = mu_ne;
  out[2] = muN;
  out[3] = rhat;
  if (!(mu1 > 0) || !(mu_ne > 0) || !(muN > mu_ne) || !std::isfinite(muN)) return CHASE_BSE_NOT_DEFINITE;
  return CHASE_BSE_OK;
}

// ----------------------------------------------------------------------- QR
int qr(const cplx* X, int64_t n2, int64_t m, cplx* Q, int* used_hh, cudaStream_t s) {
  *used_hh = 0;
  Workspace ws(s);
  cplx *G, *Linv, *T, *Q1;
  int* info_d;
  double* diag_d;
  CB_TRY(ws.alloc(&G, m * m));
  CB_TRY(ws.alloc(&Linv, m * m));
  CB_TRY(ws.alloc(&T, m * 32));
  CB_TRY(ws.alloc(&Q1, n2 * m));
  CB_TRY(ws.alloc(&info_d, 1));
  CB_TRY(ws.alloc(&diag_d, m));
  std::vector<double> dg(m);
  bool ok = true;
  const cplx* src = X;
  for (int pass = 0; pass < 2 && ok; ++pass) {
    cplx* dst = (pass == 0) ? Q1 : Q;
    CB_TRY(zgemm('C', 'N', m, m, n2, mk(1, 0), src, n2, src, n2, mk(0, 0), G, m, s));
    CB_TRY(hermitize(G, m, s));
    int info = 0;
    CB_TRY(cholesky(G, m, info_d, &info, s));
    if (info != 0) { ok = false; break; }
    if (pass == 0) {
      CB_TRY(diag_real(G, m, diag_d, s));
      CB_CUDA(cudaMemcpyAsync(dg.data(), diag_d, sizeof(double) * m, cudaMemcpyDeviceToHost, s));
      CB_CUDA(cudaStreamSynchronize(s));
      const double mx = *std::max_element(dg.begin(), dg.end());
      const double mn = *std::min_element(dg.begin(), dg.end());
      if (!(mn > 0.0) || (mx / mn) * (mx / mn) > 1e12) { ok = false; break; }
    }
    CB_TRY(tri_inverse(G, m, Linv, T, s));
    CB_TRY(zgemm('N', 'C', n2, m, m, mk(1, 0), src, n2, Linv, m, mk(0, 0), dst, n2, s));  // X L^{-*}
    src = Q1;
  }
  if (ok) return CHASE_BSE_OK;
  // Householder fallback
  *used_hh = 1;
  cplx *Xc, *Vs, *Us, *wrow;
  CB_TRY(ws.alloc(&Xc, n2 * m));
  CB_TRY(ws.alloc(&Vs, n2 * m));
  CB_TRY(ws.alloc(&Us, n2 * m));
  CB_TRY(ws.alloc(&wrow, m));
  CB_CUDA(cudaMemcpyAsync(Xc, X, sizeof(cplx) * n2 * m, cudaMemcpyDeviceToDevice, s));
  CB_TRY(householder_qr(Xc, n2, m, Q, Vs, Us, wrow, s));
  return CHASE_BSE_OK;
}

// --------------------------------------------------------------- Rayleigh-Ritz
int rayleigh_ritz(const cplx* A, const cplx* B, int64_t n, const cplx* Q, int64_t k, double* ritz_host,
                  cplx* Wpos, cudaStream_t s, cplx* R, double* res) {
  if (k <= 0 || (k % 2) != 0) return CHASE_BSE_BAD_ARG;
  const int64_t n2 = 2 * n, h = k / 2;
  Workspace ws(s);
  cplx *T, *M, *Linv, *M2, *Tmp, *G, *V, *Ypos, *Z, *rot, *scratch;
  double *theta, *red;
  int *info_d, *idx_d;
  CB_TRY(ws.alloc(&T, n2 * k));
  CB_TRY(ws.alloc(&M, k * k));
  CB_TRY(ws.alloc(&Linv, k * k));
  CB_TRY(ws.alloc(&M2, k * k));
  CB_TRY(ws.alloc(&Tmp, k * k));
  CB_TRY(ws.alloc(&G, k * k));
  CB_TRY(ws.alloc(&V, k * k));
  CB_TRY(ws.alloc(&Ypos, k * h));
  CB_TRY(ws.alloc(&Z, k * h));
  CB_TRY(ws.alloc(&rot, 2 * k));
  CB_TRY(ws.alloc(&scratch, k * 32));
  CB_TRY(ws.alloc(&theta, k));
  CB_TRY(ws.alloc(&red, 2));
  CB_TRY(ws.alloc(&info_d, 1));
  CB_TRY(ws.alloc(&idx_d, h));
  // Algorithm 2: T = S H Q, M = Q^* T
  HopArgs a{};
  a.A = A; a.B = B; a.n = n; a.W = Q; a.k = k; a.out = T; a.mode = HOP_STORE; a.sflip = 1;
  CB_TRY(hop_fp64(a, s));
  CB_TRY(zgemm('C', 'N', k, k, n2, mk(1, 0), Q, n2, T, n2, mk(0, 0), M, k, s));
  CB_TRY(hermitize(M, k, s));
  int info = 0;
  CB_TRY(cholesky(M, k, info_d, &info, s));  // M = L L^*
  if (info != 0) return CHASE_BSE_NOT_DEFINITE;
  CB_TRY(tri_inverse(M, k, Linv, scratch, s));
  // M2 = I - 2 Q_2^* Q_2 (= Q^* S Q)
  CB_TRY(set_identity(M2, k, s));
  CB_TRY(zgemm('C', 'N', k, k, n, mk(-2, 0), Q + n, n2, Q + n, n2, mk(1, 0), M2, k, s));
  // G = L^{-1} M2 L^{-*}
  CB_TRY(zgemm('N', 'N', k, k, k, mk(1, 0), Linv, k, M2, k, mk(0, 0), Tmp, k, s));
  CB_TRY(zgemm('N', 'C', k, k, k, mk(1, 0), Tmp, k, Linv, k, mk(0, 0), G, k, s));
  CB_TRY(hermitize(G, k, s));
  // G y = theta y
  int sweeps = 0;
  const auto tj = std::chrono::steady_clock::now();
  CB_TRY(jacobi_eigh(G, k, V, theta, rot, red, 40, &sweeps, s));
  if (verbose()) {
    cudaStreamSynchronize(s);
    fprintf(stderr, "[chase_bse] rr k %ld jacobi %d sweeps %.1f ms\n", (long)k, sweeps,
            std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - tj).count());
  }
  std::vector<double> th(k);
  CB_CUDA(cudaMemcpyAsync(th.data(), theta, sizeof(double) * k, cudaMemcpyDeviceToHost, s));
  CB_CUDA(cudaStreamSynchronize(s));
  // the k/2 largest theta; by Theorem positive-negative-symmetry_oblique_RR they are
  // exactly the positive half when range(Q) is closed under W -> K conj(W)
  std::vector<int> pos(k);
  std::iota(pos.begin(), pos.end(), 0);
  std::stable_sort(pos.begin(), pos.end(), [&](int x, int y) { return th[x] > th[y]; });
  pos.resize(h);
  if (!(th[pos[h - 1]] > 0.0)) return CHASE_BSE_QR_FAILED;  // search space lost its +- structure
  for (int64_t i = 0; i < h; ++i) ritz_host[i] = 1.0 / th[pos[i]];
  CB_CUDA(cudaMemcpyAsync(idx_d, pos.data(), sizeof(int) * h, cudaMemcpyHostToDevice, s));
  CB_TRY(gather_cols(Ypos, V, idx_d, k, h, s));
  // the back-substitution (read as z = L^{-*} y) and the half back-transform W+ = Q Z+
  CB_TRY(zgemm('C', 'N', k, h, k, mk(1, 0), Linv, k, Ypos, k, mk(0, 0), Z, k, s));
  CB_TRY(zgemm('N', 'N', n2, h, k, mk(1, 0), Q, n2, Z, k, mk(0, 0), Wpos, n2, s));
  if (R && res) {
    // Section 4.5 residuals on the positive half: H W+ = H Q Z+ = S T Z+
    cplx* SHW;
    CB_TRY(ws.alloc(&SHW, n2 * h));
    CB_TRY(zgemm('N', 'N', n2, h, k, mk(1, 0), T, n2, Z, k, mk(0, 0), SHW, n2, s));
    double* rz;
    CB_TRY(ws.alloc(&rz, h));
    CB_CUDA(cudaMemcpyAsync(rz, ritz_host, sizeof(double) * h, cudaMemcpyHostToDevice, s));
    CB_TRY(normalize_and_residual(Wpos, SHW, rz, n, h, R, s));
    CB_TRY(col_norms(R, n2, h, res, s));
  } else {
    CB_TRY(normalize_cols(Wpos, n2, h, s));
  }
  CB_CUDA(cudaStreamSynchronize(s));  // host vectors must outlive the copies
  return CHASE_BSE_OK;
}

// Stage timing printed in verbose mode (CHASE_BSE_VERBOSE=1).
struct StageTimer {
  cudaStream_t s;
  bool on;
  std::chrono::steady_clock::time_point t;
  char buf[512];
  int len = 0;
  StageTimer(cudaStream_t st, const char* name) : s(st), on(verbose()) {
    if (on) {
      cudaStreamSynchronize(s);
      t = std::chrono::steady_clock::now();
      len = snprintf(buf, sizeof(buf), "[chase_bse] %s:", name);
    }
  }
  void mark(const char* what) {
    if (!on) return;
    cudaStreamSynchronize(s);
    const auto now = std::chrono::steady_clock::now();
    len += snprintf(buf + len, sizeof(buf) - len, " %s %.1f", what,
                    std::chrono::duration<double, std::milli>(now - t).count());
    t = now;
  }
  ~StageTimer() {
    if (on) fprintf(stderr, "%s ms\n", buf);
  }
};

// ------------------------------------------------- J-fixed QR and Rayleigh-Ritz
// The search space [S Y+, S Y-, W+, W-] is closed under J = K conj, so it has an
// orthonormal basis of J-fixed vectors q = [x; conj(x)].  Inner products of
// J-fixed vectors are real (q_i^* q_j = 2 Re(x_i^* x_j)), so CholeskyQR runs on
// the top halves with real coefficients and keeps the basis J-fixed.  For such q,
// H q = [y; -conj(y)] with y = A x + B conj(x) (half an H application),
// Q^* S H Q = 2 Re(X^* Y) and Q^* S Q = 2 i Im(X^* X).  The Rayleigh-Ritz step is
// invariant to the choice of basis of the search space, so the results are
// those of Algorithm 2 on any orthonormal basis.
static int qr_jfixed(const cplx* X, int64_t n, int64_t m, cplx* Q, bool* ok_out, cudaStream_t s,
                     bool sliced) {
  *ok_out = false;
  Workspace ws(s);
  cplx *C, *G, *Linv, *T, *Q1;
  int* info_d;
  double* diag_d;
  CB_TRY(ws.alloc(&C, m * m));
  CB_TRY(ws.alloc(&G, m * m));
  CB_TRY(ws.alloc(&Linv, m * m));
  CB_TRY(ws.alloc(&T, m * 32));
  CB_TRY(ws.alloc(&Q1, n * m));
  CB_TRY(ws.alloc(&info_d, 1));
  CB_TRY(ws.alloc(&diag_d, m));
  std::vector<double> dg(m);
  // sliced tensor-core operands: the columns (Gram), the real-form rows of the
  // block and the conjugated rows of L^{-1} (X L^{-*})
  SlicedOp sc, sr, sl;
  double* tmp = nullptr;
  if (sliced) {
    CB_TRY(sliced_alloc(ws, sc, m, 2 * n, s));
    CB_TRY(sliced_alloc(ws, sr, 2 * n, 2 * m, s));
    CB_TRY(sliced_alloc(ws, sl, m, 2 * m, s));
    CB_TRY(ws.alloc(&tmp, 4 * n * m));
  }
  const cplx* src = X;
  StageTimer tm(s, "qr(J)");
  for (int pass = 0; pass < 2; ++pass) {
    cplx* dst = (pass == 0) ? Q1 : Q;
    if (sliced) {  // Gram of the J-fixed vectors: 2 Re(X^* X), real part of G
      CB_TRY(slice_rows(reinterpret_cast<const double*>(src), 2 * n, 0, sc, s));
      CB_CUDA(cudaMemsetAsync(G, 0, sizeof(cplx) * m * m, s));
      CB_TRY(sliced_gemm(sc, sc, 2.0, reinterpret_cast<double*>(G), 2, 2 * m, false, s));
    } else {
      CB_TRY(zgemm('C', 'N', m, m, n, mk(1, 0), src, n, src, n, mk(0, 0), C, m, s));
      CB_TRY(re_im_part(C, G, m, 0, s));  // Gram of the J-fixed vectors: 2 Re(X^* X)
    }
    tm.mark("gram");
    int info = 0;
    CB_TRY(cholesky(G, m, info_d, &info, s, true));  // the Gram is real
    tm.mark("chol");
    if (info != 0) return CHASE_BSE_OK;
    if (pass == 0) {
      CB_TRY(diag_real(G, m, diag_d, s));
      CB_CUDA(cudaMemcpyAsync(dg.data(), diag_d, sizeof(double) * m, cudaMemcpyDeviceToHost, s));
      CB_CUDA(cudaStreamSynchronize(s));
      const double mx = *std::max_element(dg.begin(), dg.end());
      const double mn = *std::min_element(dg.begin(), dg.end());
      if (!(mn > 0.0) || (mx / mn) * (mx / mn) > 1e12) return CHASE_BSE_OK;
    }
    CB_TRY(tri_inverse(G, m, Linv, T, s, true));  // the Gram is real
    tm.mark("trinv");
    if (sliced) {
      CB_TRY(slice_complex_rows(src, n, n, m, tmp, sr, s));
      CB_TRY(slice_conj_rows(Linv, m, sl, s));
      CB_TRY(sliced_gemm(sr, sl, 1.0, reinterpret_cast<double*>(dst), 1, 2 * n, false, s));
    } else {
      CB_TRY(zgemm('N', 'C', n, m, m, mk(1, 0), src, n, Linv, m, mk(0, 0), dst, n, s));
    }
    tm.mark("apply");
    src = Q1;
  }
  *ok_out = true;
  return CHASE_BSE_OK;
}

static int rayleigh_ritz_jfixed(const cplx* A, const cplx* B, int64_t n, const cplx* Qt, int64_t k, double* ritz_host,
                                cplx* Wpos, cplx* R, double* res, cudaStream_t s, const SlicedOp* ph,
                                double jthr = 2e-16) {
  if (k <= 0 || (k % 2) != 0) return CHASE_BSE_BAD_ARG;
  const int64_t n2 = 2 * n, h = k / 2;
  Workspace ws(s);
  cplx *Tt, *C, *M, *Linv, *M2, *Tmp, *G, *V, *Ypos, *Z, *rot, *scratch, *Qc, *Tc, *SHW;
  double *theta, *red, *rz;
  int *info_d, *idx_d;
  CB_TRY(ws.alloc(&Tt, n * k));
  CB_TRY(ws.alloc(&C, k * k));
  CB_TRY(ws.alloc(&M, k * k));
  CB_TRY(ws.alloc(&Linv, k * k));
  CB_TRY(ws.alloc(&M2, k * k));
  CB_TRY(ws.alloc(&Tmp, k * k));
  CB_TRY(ws.alloc(&G, k * k));
  CB_TRY(ws.alloc(&V, k * k));
  CB_TRY(ws.alloc(&Ypos, k * h));
  CB_TRY(ws.alloc(&Z, k * h));
  CB_TRY(ws.alloc(&rot, 2 * k));
  CB_TRY(ws.alloc(&scratch, k * 32));
  const bool sliced = ph != nullptr;
  SlicedOp sq, sqr, st, sqa, sta, sz, szc;
  double* tmp = nullptr;
  if (sliced) {
    CB_TRY(sliced_alloc(ws, sq, k, 2 * n, s));       // columns of Q (J-fixed top halves)
    CB_TRY(sliced_alloc(ws, sqr, k, 2 * n, s));      // the same, pairs (a, b) -> (b, -a)
    CB_TRY(sliced_alloc(ws, st, k, 2 * n, s));       // columns of T
    CB_TRY(sliced_alloc(ws, sqa, 2 * n, 2 * k, s));  // real-form rows of Q
    CB_TRY(sliced_alloc(ws, sta, 2 * n, 2 * k, s));  // real-form rows of T
    CB_TRY(sliced_alloc(ws, sz, h, 2 * k, s));       // columns of Z
    CB_TRY(sliced_alloc(ws, szc, h, 2 * k, s));      // columns of conj(Z)
    CB_TRY(ws.alloc(&tmp, 4 * (n > k ? n : k) * k));  // real-form rows of an n x k or k x k block
  } else {
    CB_TRY(ws.alloc(&Qc, n * k));
    CB_TRY(ws.alloc(&Tc, n * k));
  }
  CB_TRY(ws.alloc(&SHW, n2 * h));
  CB_TRY(ws.alloc(&theta, k));
  CB_TRY(ws.alloc(&red, 2));
  CB_TRY(ws.alloc(&rz, h));
  CB_TRY(ws.alloc(&info_d, 1));
  CB_TRY(ws.alloc(&idx_d, h));
  StageTimer tm(s, "rr(J)");
  // Algorithm 2: T = S H Q (top halves y = A x + B conj x), M = Q^* T = 2 Re(X^* Y)
  if (sliced) {
    CB_TRY(slice_rows(reinterpret_cast<const double*>(Qt), 2 * n, 0, sq, s));
    CB_TRY(sliced_gemm(*ph, sq, 1.0, reinterpret_cast<double*>(Tt), 1, 2 * n, false, s));
  } else {
    CB_TRY(hop_top_fp64(A, B, n, Qt, k, Tt, s));
  }
  tm.mark("HQ");
  // The J-fixed columns come in pairs spanning {u, J u}; the small problem is set up in
  // the basis Q U (U = pairwise [[1, 1], [-i, i]] / sqrt 2), whose pairs point along
  // (u, J u): G then starts close to diagonal, as for the general basis.
  if (sliced) {
    CB_TRY(slice_rows(reinterpret_cast<const double*>(Tt), 2 * n, 0, st, s));
    CB_CUDA(cudaMemsetAsync(Tmp, 0, sizeof(cplx) * k * k, s));
    CB_TRY(sliced_gemm(sq, st, 2.0, reinterpret_cast<double*>(Tmp), 2, 2 * k, false, s));
  } else {
    CB_TRY(zgemm('C', 'N', k, k, n, mk(1, 0), Qt, n, Tt, n, mk(0, 0), C, k, s));
    CB_TRY(re_im_part(C, Tmp, k, 0, s));
  }
  CB_TRY(pair_transform(Tmp, M, k, s));
  int info = 0;
  CB_TRY(cholesky(M, k, info_d, &info, s));  // M = L L^*
  if (info != 0) return CHASE_BSE_NOT_DEFINITE;
  CB_TRY(tri_inverse(M, k, Linv, scratch, s));
  // Q^* S Q = 2 i Im(X^* X)
  if (sliced) {  // Im(x_i^* x_j) = x_i . (Im x_j, -Re x_j) on (re, im) pairs
    CB_TRY(slice_rows(reinterpret_cast<const double*>(Qt), 2 * n, 1, sqr, s));
    CB_CUDA(cudaMemsetAsync(Tmp, 0, sizeof(cplx) * k * k, s));
    CB_TRY(sliced_gemm(sq, sqr, 2.0, reinterpret_cast<double*>(Tmp) + 1, 2, 2 * k, false, s));
  } else {
    CB_TRY(zgemm('C', 'N', k, k, n, mk(1, 0), Qt, n, Qt, n, mk(0, 0), C, k, s));
    CB_TRY(re_im_part(C, Tmp, k, 1, s));
  }
  CB_TRY(pair_transform(Tmp, M2, k, s));
  // G = L^{-1} M2 L^{-*}
  SlicedOp sl_rows, sl_b;  // real-form rows of a k x k factor, and the right operand
  if (sliced) {
    CB_TRY(sliced_alloc(ws, sl_rows, 2 * k, 2 * k, s));
    CB_TRY(sliced_alloc(ws, sl_b, k, 2 * k, s));
    CB_TRY(slice_complex_rows(Linv, k, k, k, tmp, sl_rows, s));
    CB_TRY(slice_rows(reinterpret_cast<const double*>(M2), 2 * k, 0, sl_b, s));
    CB_TRY(sliced_gemm(sl_rows, sl_b, 1.0, reinterpret_cast<double*>(Tmp), 1, 2 * k, false, s));
    CB_TRY(slice_complex_rows(Tmp, k, k, k, tmp, sl_rows, s));
    CB_TRY(slice_conj_rows(Linv, k, sl_b, s));
    CB_TRY(sliced_gemm(sl_rows, sl_b, 1.0, reinterpret_cast<double*>(G), 1, 2 * k, false, s));
  } else {
    CB_TRY(zgemm('N', 'N', k, k, k, mk(1, 0), Linv, k, M2, k, mk(0, 0), Tmp, k, s));
    CB_TRY(zgemm('N', 'C', k, k, k, mk(1, 0), Tmp, k, Linv, k, mk(0, 0), G, k, s));
  }
  CB_TRY(hermitize(G, k, s));
  tm.mark("small");
  int sweeps = 0;
  int sweeps32 = 0;
  if (sliced) CB_TRY(jacobi_eigh_mixed(G, k, V, theta, rot, red, &sweeps32, &sweeps, s, jthr));  // G y = theta y
  else CB_TRY(jacobi_eigh(G, k, V, theta, rot, red, 40, &sweeps, s, jthr));
  tm.mark("jacobi");
  std::vector<double> th(k);
  CB_CUDA(cudaMemcpyAsync(th.data(), theta, sizeof(double) * k, cudaMemcpyDeviceToHost, s));
  CB_CUDA(cudaStreamSynchronize(s));
  std::vector<int> pos(k);
  std::iota(pos.begin(), pos.end(), 0);
  std::stable_sort(pos.begin(), pos.end(), [&](int x, int y) { return th[x] > th[y]; });
  pos.resize(h);
  if (!(th[pos[h - 1]] > 0.0)) return CHASE_BSE_QR_FAILED;
  for (int64_t i = 0; i < h; ++i) ritz_host[i] = 1.0 / th[pos[i]];
  CB_CUDA(cudaMemcpyAsync(idx_d, pos.data(), sizeof(int) * h, cudaMemcpyHostToDevice, s));
  CB_CUDA(cudaMemcpyAsync(rz, ritz_host, sizeof(double) * h, cudaMemcpyHostToDevice, s));
  CB_TRY(gather_cols(Ypos, V, idx_d, k, h, s));
  // z = L^{-*} y, back to the J-fixed basis (Z = U Z');
  // W+ = Q Z+ = [X Z; conj(X) Z]; S H W+ = [Y Z; conj(Y) Z]
  if (sliced) {  // Tmp = L^{-*} Y+: rows of L^{-*} are the conjugated columns of L^{-1}
    CB_TRY(conj_transpose(Linv, k, M2, s));
    CB_TRY(slice_complex_rows(M2, k, k, k, tmp, sl_rows, s));
    SlicedOp sy;
    CB_TRY(sliced_alloc(ws, sy, h, 2 * k, s));
    CB_TRY(slice_rows(reinterpret_cast<const double*>(Ypos), 2 * k, 0, sy, s));
    CB_TRY(sliced_gemm(sl_rows, sy, 1.0, reinterpret_cast<double*>(Tmp), 1, 2 * k, false, s));
  } else {
    CB_TRY(zgemm('C', 'N', k, h, k, mk(1, 0), Linv, k, Ypos, k, mk(0, 0), Tmp, k, s));
  }
  CB_TRY(pair_apply(Tmp, Z, k, h, s));
  if (sliced) {  // conj(X) Z = conj(X conj(Z)): the conjugated halves negate the odd (imaginary) rows
    CB_TRY(slice_rows(reinterpret_cast<const double*>(Z), 2 * k, 0, sz, s));
    CB_TRY(slice_rows(reinterpret_cast<const double*>(Z), 2 * k, 2, szc, s));
    CB_TRY(slice_complex_rows(Qt, n, n, k, tmp, sqa, s));
    CB_TRY(sliced_gemm(sqa, sz, 1.0, reinterpret_cast<double*>(Wpos), 1, 2 * n2, false, s));
    CB_TRY(sliced_gemm(sqa, szc, 1.0, reinterpret_cast<double*>(Wpos + n), 1, 2 * n2, true, s));
    CB_TRY(slice_complex_rows(Tt, n, n, k, tmp, sta, s));
    CB_TRY(sliced_gemm(sta, sz, 1.0, reinterpret_cast<double*>(SHW), 1, 2 * n2, false, s));
    CB_TRY(sliced_gemm(sta, szc, 1.0, reinterpret_cast<double*>(SHW + n), 1, 2 * n2, true, s));
  } else {
    CB_TRY(conj_copy(Qc, n, Qt, n, n, k, s));
    CB_TRY(conj_copy(Tc, n, Tt, n, n, k, s));
    CB_TRY(zgemm('N', 'N', n, h, k, mk(1, 0), Qt, n, Z, k, mk(0, 0), Wpos, n2, s));
    CB_TRY(zgemm('N', 'N', n, h, k, mk(1, 0), Qc, n, Z, k, mk(0, 0), Wpos + n, n2, s));
    CB_TRY(zgemm('N', 'N', n, h, k, mk(1, 0), Tt, n, Z, k, mk(0, 0), SHW, n2, s));
    CB_TRY(zgemm('N', 'N', n, h, k, mk(1, 0), Tc, n, Z, k, mk(0, 0), SHW + n, n2, s));
  }
  CB_TRY(normalize_and_residual(Wpos, SHW, rz, n, h, R, s));
  CB_TRY(col_norms(R, n2, h, res, s));
  CB_CUDA(cudaStreamSynchronize(s));  // host vectors must outlive the copies
  tm.mark("back");
  if (verbose())
    fprintf(stderr, "[chase_bse] rr(J) k %ld jacobi %d FP32 + %d FP64 sweeps\n", (long)k, sweeps32, sweeps);
  return CHASE_BSE_OK;
}

int residuals(const cplx* A, const cplx* B, int64_t n, const cplx* W, const double* lambda, int64_t k, double* res,
              cudaStream_t s, cplx* Rout) {
  if (k == 0) return CHASE_BSE_OK;
  Workspace ws(s);
  cplx* R = Rout;
  if (!R) CB_TRY(ws.alloc(&R, 2 * n * k));
  HopArgs a{};
  a.A = A; a.B = B; a.n = n; a.W = W; a.k = k; a.out = R; a.mode = HOP_RESID; a.lambda = lambda;
  CB_TRY(hop_fp64(a, s));
  CB_TRY(col_norms(R, 2 * n, k, res, s));
  return CHASE_BSE_OK;
}

int gradient(const cplx* V, const double* w, int64_t n, int64_t nev, cplx* gA, cplx* gB, cudaStream_t s) {
  Workspace ws(s);
  cplx *Uc, *U2, *Ub, *U3;
  double* cbuf;
  const int64_t sz = n * 2 * nev;
  CB_TRY(ws.alloc(&Uc, sz));
  CB_TRY(ws.alloc(&U2, sz));
  CB_TRY(ws.alloc(&Ub, sz));
  CB_TRY(ws.alloc(&U3, sz));
  CB_TRY(ws.alloc(&cbuf, nev));
  CB_TRY(grad_prepare(V, w, n, nev, cbuf, Uc, U2, Ub, U3, s));
  // row-major gA is the column-major conj(gA) = Uc U2^T; row-major gB = gB = Ub U3^T
  if (mixed_available()) {  // FP64-accurate products on the tensor cores (sliced GEMM)
    SlicedOp sa, sb;
    double* tmp;
    CB_TRY(sliced_alloc(ws, sa, 2 * n, 4 * nev, s));
    CB_TRY(sliced_alloc(ws, sb, n, 4 * nev, s));
    CB_TRY(ws.alloc(&tmp, 8 * n * nev));
    CB_TRY(slice_complex_rows(Uc, n, n, 2 * nev, tmp, sa, s));
    CB_TRY(slice_plain_rows(U2, n, sb, s));
    CB_TRY(sliced_gemm(sa, sb, 1.0, reinterpret_cast<double*>(gA), 1, 2 * n, false, s));
    CB_TRY(slice_complex_rows(Ub, n, n, 2 * nev, tmp, sa, s));
    CB_TRY(slice_plain_rows(U3, n, sb, s));
    return sliced_gemm(sa, sb, 1.0, reinterpret_cast<double*>(gB), 1, 2 * n, false, s);
  }
  CB_TRY(zgemm('N', 'T', n, n, 2 * nev, mk(1, 0), Uc, n, U2, n, mk(0, 0), gA, n, s));
  CB_TRY(zgemm('N', 'T', n, n, 2 * nev, mk(1, 0), Ub, n, U3, n, mk(0, 0), gB, n, s));
  return CHASE_BSE_OK;
}

// -------------------------------------------------------------------- solve
namespace {
struct PhaseClock {
  cudaStream_t s;
  cudaEvent_t a, b;
  explicit PhaseClock(cudaStream_t st) : s(st) {
    cudaEventCreate(&a);
    cudaEventCreate(&b);
  }
  ~PhaseClock() {
    cudaEventDestroy(a);
    cudaEventDestroy(b);
  }
  void start() { cudaEventRecord(a, s); }
  double stop() {
    cudaEventRecord(b, s);
    cudaEventSynchronize(b);
    float ms = 0;
    cudaEventElapsedTime(&ms, a, b);
    return ms;
  }
};

}  // namespace

// Per-vector degree from the convergence rate: predicted rate per H^2 step
// rho = 1/(|t| + sqrt(t^2 - 1)), t = (lambda^2 - c)/e, replaced by the observed
// rate (r/r_prev)^(1/deg_prev) when that is slower; deg = ceil(ln(tol/r)/ln rho) + 1.
void degrees_update(const std::vector<double>& ritz, const std::vector<double>& res,
                    const std::vector<double>& prev_res, const std::vector<int>& prev_deg, double tol, double mu_ne,
                    double muN, int dmin, int dmax, std::vector<int>& degs) {
  const double a = mu_ne * mu_ne, b = muN * muN;
  const double c = 0.5 * (a + b), e = 0.5 * (b - a);
  degs.resize(ritz.size());
  for (size_t i = 0; i < ritz.size(); ++i) {
    const double t = (ritz[i] * ritz[i] - c) / e;
    const double r = res[i];
    double rho = (std::fabs(t) <= 1.0) ? 1.0 : 1.0 / (std::fabs(t) + std::sqrt(t * t - 1.0));
    if (std::isfinite(prev_res[i]) && r > 0.0 && r < prev_res[i])
      rho = std::max(rho, std::pow(r / prev_res[i], 1.0 / prev_deg[i]));
    int d;
    if (!(r > tol)) d = dmin;
    else if (rho >= 1.0) d = dmax;
    else d = (int)std::ceil(std::log(tol / r) / std::log(rho)) + 1;
    degs[i] = std::min(std::max(d, dmin), dmax);
  }
}

// One fallback Rayleigh-Ritz step of the solver on the general basis Q (2n x 2 kf): the kf
// positive Ritz pairs (ritz host, Wpos 2n x kf) and their FP64 residual vectors and norms
// (R 2n x kf, res device).  Fewer than kf Ritz values with positive real part:
// QR_FAILED.
static int rayleigh_ritz_fallback_step(const cplx* A, const cplx* B, int64_t n, const cplx* Q, int64_t kf,
                                       double* ritz, cplx* Wpos, cplx* R, double* res, cudaStream_t s) {
  const int64_t n2 = 2 * n, k = 2 * kf;
  Workspace ws(s);
  cplx* Wall;
  double* lam;
  CB_TRY(ws.alloc(&Wall, n2 * k));
  CB_TRY(ws.alloc(&lam, kf));
  std::vector<double> rz(k);
  int64_t npos = 0;
  CB_TRY(rayleigh_ritz_fallback(A, B, n, Q, k, rz.data(), Wall, &npos, s));
  if (npos < kf) return CHASE_BSE_QR_FAILED;
  for (int64_t i = 0; i < kf; ++i) ritz[i] = rz[i];
  CB_CUDA(cudaMemcpyAsync(Wpos, Wall, sizeof(cplx) * n2 * kf, cudaMemcpyDeviceToDevice, s));
  CB_CUDA(cudaMemcpyAsync(lam, ritz, sizeof(double) * kf, cudaMemcpyHostToDevice, s));
  CB_TRY(residuals(A, B, n, Wpos, lam, kf, res, s, R));
  CB_CUDA(cudaStreamSynchronize(s));
  return CHASE_BSE_OK;
}

int solve(const cplx* A, const cplx* B, int64_t n, int64_t nev, int64_t nex, int deg, double tol,
          const chase_bse_opts* opts_in, double* evals, cplx* evecs, chase_bse_stats* stats) {
  chase_bse_opts o{};
  o.size = sizeof(o);
  o.precision = CHASE_BSE_FP64;
  o.maxiter = 25;
  o.deg_min = deg;
  o.deg_max = deg;
  o.lanczos_steps = 26;
  o.lanczos_vecs = 4;
  o.gamma = 1e-3;
  o.switch_tol = 1e-8;
  o.seed = 0;
  if (opts_in) {
    if (opts_in->size != sizeof(chase_bse_opts)) return CHASE_BSE_BAD_ARG;
    o = *opts_in;
  }
  if (!A || !B || !evals || !evecs || n < 1 || nev < 1 || nex < 0 || nev + nex > n || deg < 1 || !(tol > 0) ||
      o.maxiter < 1 || o.deg_min < 1 || o.deg_max < o.deg_min || o.lanczos_steps < 2 || o.lanczos_vecs < 1 ||
      o.lanczos_vecs > 64 ||
      (o.precision != CHASE_BSE_FP64 && o.precision != CHASE_BSE_MIXED_BF16X3 &&
       o.precision != CHASE_BSE_MIXED_BF16X6 && o.precision != CHASE_BSE_MIXED_FP16X3 &&
       o.precision != CHASE_BSE_FP64_TC))
    return CHASE_BSE_BAD_ARG;
  if (o.fp64_products != 0 && o.fp64_products != 1) return CHASE_BSE_BAD_ARG;
  if (o.rr != 0 && o.rr != 1) return CHASE_BSE_BAD_ARG;
  if (o.h2 != 0 && o.h2 != 1) return CHASE_BSE_BAD_ARG;
  if (o.h2 == 1 && (o.precision == CHASE_BSE_FP64 || o.precision == CHASE_BSE_FP64_TC)) return CHASE_BSE_BAD_ARG;
  const bool fp64tc = o.precision == CHASE_BSE_FP64_TC;
  const bool mixed = o.precision != CHASE_BSE_FP64 && !fp64tc;
  // FP64-accurate products on the tensor cores: FP64_TC always, mixed unless fp64_products
  const bool sliced = fp64tc || (mixed && o.fp64_products == 0);
  // FilterScheme codes equal the mixed precision codes (unused when no column is mixed)
  const int scheme = mixed ? o.precision : (int)CHASE_BSE_MIXED_FP16X3;
  if ((mixed || fp64tc) && !mixed_available()) return CHASE_BSE_UNSUPPORTED;
  cudaStream_t s = (cudaStream_t)o.stream;
  const int64_t n2 = 2 * n, nevex = nev + nex;
  {  // inputs with a NaN or an Inf: a defined status, nothing computed
    Workspace cws(s);
    int* cnt;
    CB_TRY(cws.alloc(&cnt, 1));
    int bad = 0, c = 0;
    CB_TRY(count_nonfinite(A, n * n, cnt, &c, s));
    bad += c;
    CB_TRY(count_nonfinite(B, n * n, cnt, &c, s));
    bad += c;
    if (o.W0) {
      CB_TRY(count_nonfinite((const cplx*)o.W0, n2 * nevex, cnt, &c, s));
      bad += c;
    }
    if (o.V0) {
      CB_TRY(count_nonfinite((const cplx*)o.V0, n2 * o.lanczos_vecs, cnt, &c, s));
      bad += c;
    }
    if (bad) return CHASE_BSE_NONFINITE;
  }
  chase_bse_stats st{};
  st.size = sizeof(st);
  auto t_start = std::chrono::steady_clock::now();
  Workspace ws(s);
  cplx *W, *Ylock, *X, *Qf, *Wpos, *V0;
  double *lam_d, *res_d;
  CB_TRY(ws.alloc(&W, n2 * nevex));
  CB_TRY(ws.alloc(&Ylock, n2 * nev));
  CB_TRY(ws.alloc(&X, n2 * 2 * nevex));
  CB_TRY(ws.alloc(&Qf, n2 * 2 * nevex));
  CB_TRY(ws.alloc(&Wpos, n2 * nevex));
  CB_TRY(ws.alloc(&V0, n2 * o.lanczos_vecs));
  CB_TRY(ws.alloc(&lam_d, nevex));
  CB_TRY(ws.alloc(&res_d, nevex));
  cplx *Rall = nullptr, *Rkeep = nullptr;
  if (mixed) {
    CB_TRY(ws.alloc(&Rall, n2 * nevex));
    CB_TRY(ws.alloc(&Rkeep, n2 * nevex));
  }
  std::vector<double> ritz_keep;  // Ritz values of the columns of W (mixed correction form)
  PhaseClock clk(s);

  // Algorithm 3 start: W+ = randn(2n, nevex), lower half scaled by gamma
  if (o.W0) CB_CUDA(cudaMemcpyAsync(W, o.W0, sizeof(cplx) * n2 * nevex, cudaMemcpyDeviceToDevice, s));
  else CB_TRY(randn_complex(W, n2 * nevex, o.seed, 1, s));
  CB_TRY(scale_lower(W, n, nevex, o.gamma, s));
  if (o.V0) CB_CUDA(cudaMemcpyAsync(V0, o.V0, sizeof(cplx) * n2 * o.lanczos_vecs, cudaMemcpyDeviceToDevice, s));
  else CB_TRY(randn_complex(V0, n2 * o.lanczos_vecs, o.seed, 2, s));

  // mixed mode: the rows of H's top block row, y = A x + B conj(x), as sliced
  // tensor-core operand for the Lanczos and Rayleigh-Ritz products with H (cut
  // once per solve)
  SlicedOp ph;
  if (sliced) {
    CB_TRY(sliced_alloc(ws, ph, 2 * n, 2 * n, s));
    CB_TRY(slice_hamiltonian(A, B, n, ph, s));
  }

  // explicit-H^2 variant (not the paper's method): the blocks of H^2, formed once
  cplx *P2 = nullptr, *Q2 = nullptr;
  if (o.h2 == 1) {
    clk.start();
    CB_TRY(ws.alloc(&P2, n * n));
    CB_TRY(ws.alloc(&Q2, n * n));
    CB_TRY(form_h2(A, B, n, P2, Q2, s));
    st.ms_h2 = clk.stop();
  }

  // spectral bounds
  clk.start();
  double mu[4];
  CB_TRY(lanczos_bounds(A, B, n, V0, o.lanczos_vecs, o.lanczos_steps, nevex, mu, s, sliced ? &ph : nullptr));
  if (verbose())
    fprintf(stderr, "[chase_bse] setup wall %.2f ms\n",
            std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count());
  st.ms_lanczos = clk.stop();
  double mu1 = mu[0], mu_ne = mu[1], muN = mu[2];
  const double rhat = mu[3];
  st.lanczos_mu1 = mu[0];
  st.lanczos_mu_nevex = mu[1];
  st.lanczos_muN = mu[2];
  // mu_1 is the normalisation point p(mu_1^2) = 1 and must stay below mu_nevex
  mu1 = std::min(mu1, 0.5 * mu_ne);

  int64_t locked = 0;
  std::vector<double> lam_locked;
  std::vector<int> degs(nevex, deg), prec(nevex, mixed ? 1 : 0);
  std::vector<double> prev_res(nevex, INFINITY);
  int it = 0;
  FilterStats fs;
  int status = CHASE_BSE_OK;
  while (locked < nev && it < o.maxiter) {
    ++it;
    const auto it_start = std::chrono::steady_clock::now();
    const double ph0 = st.ms_filter + st.ms_qr + st.ms_rr + st.ms_resid;
    const int64_t kf = nevex - locked;
    // filter: W+ <- p(H^2) W+
    clk.start();
    const bool corr = mixed && !ritz_keep.empty();
    CB_TRY(filter(A, B, n, W, kf, degs.data(), prec.data(), mu1, mu_ne, muN, scheme,
                  corr ? ritz_keep.data() : nullptr, corr ? Rkeep : nullptr, s, &fs, sliced ? &ph : nullptr, P2,
                  Q2));
    st.ms_filter += clk.stop();
    // orthonormalisation: W- = K conj(W+), Q = [S Y+, S Y-, W+, W-] R^{-1}, drop the locked part;
    // J-fixed basis (top halves) unless its CholeskyQR2 breaks down
    clk.start();
    const bool force_fallback = o.rr == 1;
    bool jok = false;
    if (!force_fallback) {
      CB_TRY(build_jfixed(X, Ylock, locked, W, kf, n, s));
      CB_TRY(qr_jfixed(X, n, 2 * nevex, Qf, &jok, s, sliced));
    }
    int hh = 0;
    if (!jok) {
      CB_TRY(build_qr_input(X, Ylock, locked, W, kf, n, s));
      CB_TRY(qr(X, n2, 2 * nevex, Qf, &hh, s));
      st.householder += hh;
    }
    st.ms_qr += clk.stop();
    clk.start();
    std::vector<double> ritz(kf);
    cplx* Rvec = Rall;
    Workspace rws(s);
    if (!Rvec) CB_TRY(rws.alloc(&Rvec, n2 * kf));
    // Rayleigh-Ritz, W+ = Q Z+ and the residuals of the positive half
    // Jacobi accuracy of the small eigenproblem: the Ritz vectors need not be more
    // accurate than the subspace they come from; 1e-4 of the smallest residual of the
    // previous iteration (1e-8 before the first), down to the rounding level
    double jthr = 1e-8;
    for (int64_t i = 0; i < kf; ++i) jthr = std::min(jthr, 1e-4 * prev_res[i]);
    jthr = std::max(jthr, 2e-16);
    int rs = CHASE_BSE_NOT_DEFINITE;
    if (!force_fallback)
      rs = jok ? rayleigh_ritz_jfixed(A, B, n, Qf + 2 * locked * n, 2 * kf, ritz.data(), Wpos, Rvec, res_d, s,
                                      sliced ? &ph : nullptr, jthr)
               : rayleigh_ritz(A, B, n, Qf + 2 * locked * n2, 2 * kf, ritz.data(), Wpos, s, Rvec, res_d);
    if (rs == CHASE_BSE_NOT_DEFINITE) {
      // Q^* S H Q not positive definite (or the fallback asked for): the non-hermitian
      // fallback (Section 4.4, last paragraph) in the general basis, where the diagonal of
      // Q^* S Q is not identically zero as in the J-fixed one
      if (jok) {
        CB_TRY(build_qr_input(X, Ylock, locked, W, kf, n, s));
        CB_TRY(qr(X, n2, 2 * nevex, Qf, &hh, s));
        st.householder += hh;
      }
      const int fb = rayleigh_ritz_fallback_step(A, B, n, Qf + 2 * locked * n2, kf, ritz.data(), Wpos, Rvec, res_d, s);
      // no usable positive Ritz values either: the problem is not definite
      rs = (fb == CHASE_BSE_QR_FAILED && !force_fallback) ? CHASE_BSE_NOT_DEFINITE : fb;
      st.fallback_rr += 1;
    }
    st.ms_rr += clk.stop();
    if (rs != CHASE_BSE_OK) { status = rs; break; }
    clk.start();
    std::vector<double> res(kf);
    CB_CUDA(cudaMemcpyAsync(res.data(), res_d, sizeof(double) * kf, cudaMemcpyDeviceToHost, s));
    CB_CUDA(cudaStreamSynchronize(s));
    st.ms_resid += clk.stop();
    for (auto& r : res) r /= rhat;
    if (verbose()) {
      double mx = 0;
      for (auto r : res) mx = std::max(mx, r);
      fprintf(stderr, "[chase_bse] it %d locked %ld kf %ld res0 %.3e resmax %.3e mu %.6g %.6g %.6g hh %d\n", it,
              (long)locked, (long)kf, res[0], mx, mu1, mu_ne, muN, hh);
    }
    // lock converged positive pairs
    const int64_t want = std::min<int64_t>(nev - locked, kf);
    std::vector<int> conv, keep;
    for (int64_t i = 0; i < kf; ++i) {
      if (i < want && res[i] <= tol) conv.push_back((int)i);
      else keep.push_back((int)i);
    }
    int* idx_d;
    Workspace its(s);
    CB_TRY(its.alloc(&idx_d, kf));
    if (!conv.empty()) {
      CB_CUDA(cudaMemcpyAsync(idx_d, conv.data(), sizeof(int) * conv.size(), cudaMemcpyHostToDevice, s));
      CB_TRY(gather_cols(Ylock + locked * n2, Wpos, idx_d, n2, (int64_t)conv.size(), s));
      for (int i : conv) lam_locked.push_back(ritz[i]);
      locked += (int64_t)conv.size();
    }
    if (!keep.empty()) {
      CB_CUDA(cudaMemcpyAsync(idx_d, keep.data(), sizeof(int) * keep.size(), cudaMemcpyHostToDevice, s));
      CB_TRY(gather_cols(W, Wpos, idx_d, n2, (int64_t)keep.size(), s));
      if (mixed) {
        CB_TRY(gather_cols(Rkeep, Rall, idx_d, n2, (int64_t)keep.size(), s));
        ritz_keep.clear();
        for (int i : keep) ritz_keep.push_back(ritz[i]);
      }
    }
    CB_CUDA(cudaStreamSynchronize(s));
    if (locked >= nev || keep.empty()) break;
    // filter bounds and per-vector degrees for the next iteration
    std::vector<double> kr, kres, kprev;
    std::vector<int> kdeg;
    for (int i : keep) {
      kr.push_back(ritz[i]);
      kres.push_back(res[i]);
      kprev.push_back(prev_res[i]);
      kdeg.push_back(degs[i]);
    }
    // mu_nevex <- largest non-locked Ritz value below mu_N (larger ones are spurious).
    // The first Rayleigh-Ritz replaces the Lanczos estimate (growing by at most 2x);
    // afterwards mu_nevex never increases: the top Ritz values of the unconverged guard
    // vectors approach the spectrum from above, so a growing value is drift
    double cand = -1.0;
    for (double r : kr)
      if (r < muN) cand = std::max(cand, r);
    if (cand > 0.0) mu_ne = (it == 1) ? std::min(cand, 2.0 * mu_ne) : std::min(cand, mu_ne);
    if (ritz[0] > 0.0) mu1 = std::min(mu1, ritz[0]);
    mu1 = std::min(mu1, 0.5 * mu_ne);
    degrees_update(kr, kres, kprev, kdeg, tol, mu_ne, muN, o.deg_min, o.deg_max, degs);
    // precision flags: a tensor-core column moves to the FP64 filter only if its
    // residual is below switch_tol and stopped decreasing (the correction form
    // normally converges to FP64 accuracy on the tensor cores)
    std::vector<int> nprec(keep.size(), 0);
    if (mixed) {
      for (size_t i = 0; i < keep.size(); ++i) {
        const bool stalled = std::isfinite(kprev[i]) && kres[i] <= o.switch_tol && kres[i] >= kprev[i];
        nprec[i] = (stalled || prec[keep[i]] == 0) ? 0 : 1;
      }
    }
    prec = nprec;
    prev_res = kres;
    if (verbose()) {
      const double wall =
          std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - it_start).count();
      fprintf(stderr, "[chase_bse] it %d wall %.2f ms, timed phases %.2f ms\n", it, wall,
              st.ms_filter + st.ms_qr + st.ms_rr + st.ms_resid - ph0);
    }
  }
  st.iterations = it;
  // output: the nev smallest locked pairs in ascending order
  const int64_t nout = std::min<int64_t>(locked, nev);
  std::vector<int> order(locked);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return lam_locked[x] < lam_locked[y]; });
  if (nout > 0) {
    int* od;
    Workspace ows(s);
    CB_TRY(ows.alloc(&od, nout));
    std::vector<double> lo(nout);
    for (int64_t i = 0; i < nout; ++i) lo[i] = lam_locked[order[i]];
    CB_CUDA(cudaMemcpyAsync(od, order.data(), sizeof(int) * nout, cudaMemcpyHostToDevice, s));
    CB_TRY(gather_cols(evecs, Ylock, od, n2, nout, s));
    CB_TRY(phase_fix(evecs, n, nout, s));
    CB_CUDA(cudaMemcpyAsync(evals, lo.data(), sizeof(double) * nout, cudaMemcpyHostToDevice, s));
    // residual of the returned pairs (mixed mode: H V by the FP64-accurate tensor-core
    // product, as the rest of the iteration)
    if (sliced) {
      Workspace rws(s);
      cplx *HV, *Rr;
      CB_TRY(rws.alloc(&HV, n2 * nout));
      CB_TRY(rws.alloc(&Rr, n2 * nout));
      CB_TRY(hop_sliced(ph, evecs, n, nout, HV, s));
      CB_TRY(residual_from_hv(HV, evecs, evals, n2, nout, Rr, s));
      CB_TRY(col_norms(Rr, n2, nout, res_d, s));
    } else {
      CB_TRY(residuals(A, B, n, evecs, evals, nout, res_d, s));
    }
    std::vector<double> rr(nout);
    CB_CUDA(cudaMemcpyAsync(rr.data(), res_d, sizeof(double) * nout, cudaMemcpyDeviceToHost, s));
    CB_CUDA(cudaStreamSynchronize(s));
    for (auto r : rr) st.max_residual = std::max(st.max_residual, r / rhat);
  }
  CB_CUDA(cudaStreamSynchronize(s));
  st.converged = (int32_t)nout;
  st.mu1 = mu1;
  st.mu_nevex = mu_ne;
  st.muN = muN;
  st.rho_hat = rhat;
  st.filter_flops = fs.flops;
  st.filter_flops_fp64 = fs.flops_fp64;
  st.ms_filter_fp64 = fs.ms_fp64;
  st.ms_filter_mixed = fs.ms_mixed;
  st.filter_launches = fs.launches;
  st.ms_total = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count();
  if (stats) {
    if (stats->size != sizeof(chase_bse_stats)) return CHASE_BSE_BAD_ARG;
    *stats = st;
  }
  if (status != CHASE_BSE_OK) return status;
  return (nout < nev) ? CHASE_BSE_NOT_CONVERGED : CHASE_BSE_OK;
}

}  // namespace cb
