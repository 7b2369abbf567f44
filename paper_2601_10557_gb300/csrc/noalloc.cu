// Residual norms without any device allocation.
//
// chase_bse_residuals obtains its 2n x k scratch block (the residual vectors
// H w_j - lambda_j w_j, reduced to norms afterwards) from stream-ordered
// allocation.  Some callers cannot let a library allocate: applications whose
// memory pool already owns the whole device and forbids outside
// cudaMalloc/cudaMallocAsync, programs with a fixed device-memory budget, and
// latency-critical loops where an allocation or a free may synchronise the
// device.  For them this file keeps the scratch in a fixed array in the
// library's own device memory: it is created when the library is loaded on a
// device and held until the process exits.
#include <mutex>

#include "dense_kernels.cuh"
#include "fp64_kernels.cuh"

namespace {

// 2n * k complex128 entries at most: 8 MiB per device.
constexpr int64_t kMaxEntries = CHASE_BSE_NOALLOC_MAX_ENTRIES;
__device__ __align__(256) cb::cplx g_scratch[kMaxEntries];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
cb::cplx* g_ptr[kMaxDevices] = {};

// Device address of g_scratch on the current device, looked up once per device
// (host code only sees a host-side stand-in under the array's name).
int scratch_address(cb::cplx** out) {
  int dev = 0;
  CB_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return CHASE_BSE_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_ptr[dev]) {
    void* p = nullptr;
    CB_CUDA(cudaGetSymbolAddress(&p, g_scratch));
    g_ptr[dev] = static_cast<cb::cplx*>(p);
  }
  *out = g_ptr[dev];
  return CHASE_BSE_OK;
}

}  // namespace

extern "C" int chase_bse_residuals_noalloc(const void* A, const void* B, int64_t n, const void* W,
                                           const double* lambda, int64_t k, double* res, void* stream) {
  if (k == 0) return CHASE_BSE_OK;
  if (!A || !B || !W || !lambda || !res || n < 1 || k < 0) return CHASE_BSE_BAD_ARG;
  if (2 * n > kMaxEntries / k) return CHASE_BSE_BAD_ARG;  // 2n * k exceeds the fixed scratch
  cb::cplx* R = nullptr;
  CB_TRY(scratch_address(&R));
  cudaStream_t s = (cudaStream_t)stream;
  // every entry of the 2n x k block is written by the residual kernel, so the
  // previous call's contents need no clearing; the H product runs as one launch over
  // the whole K range (no split-K partial sums, which would need workspace)
  cb::HopArgs a{};
  a.no_split = 1;
  a.A = (const cb::cplx*)A;
  a.B = (const cb::cplx*)B;
  a.n = n;
  a.W = (const cb::cplx*)W;
  a.k = k;
  a.out = R;
  a.mode = cb::HOP_RESID;
  a.lambda = lambda;
  CB_TRY(cb::hop_fp64(a, s));
  CB_TRY(cb::col_norms(R, 2 * n, k, res, s));
  return CHASE_BSE_OK;
}
