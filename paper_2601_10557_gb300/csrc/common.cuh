// Shared device/host helpers of the ChASE-BSE library (complex128 arithmetic,
// status handling, launch helpers).
#pragma once
#include <cuda_runtime.h>
#include <cstdint>
#include <cstdio>
#include "chase_bse.h"

namespace cb {

using cplx = double2;  // (re, im), interleaved complex128

__host__ __device__ inline cplx mk(double r, double i) { return make_double2(r, i); }
__host__ __device__ inline cplx cadd(cplx a, cplx b) { return mk(a.x + b.x, a.y + b.y); }
__host__ __device__ inline cplx csub(cplx a, cplx b) { return mk(a.x - b.x, a.y - b.y); }
__host__ __device__ inline cplx cmul(cplx a, cplx b) { return mk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__host__ __device__ inline cplx cconj(cplx a) { return mk(a.x, -a.y); }
__host__ __device__ inline cplx cscale(cplx a, double s) { return mk(a.x * s, a.y * s); }
__host__ __device__ inline double cabs2(cplx a) { return a.x * a.x + a.y * a.y; }
// c += a * b with four FMAs
__device__ __forceinline__ void cfma(cplx& c, cplx a, cplx b) {
  c.x = fma(a.x, b.x, c.x);
  c.x = fma(-a.y, b.y, c.x);
  c.y = fma(a.x, b.y, c.y);
  c.y = fma(a.y, b.x, c.y);
}

// Status plumbing: every host helper returns an int status (chase_bse_status).
#define CB_CUDA(call)                                                            \
  do {                                                                           \
    cudaError_t e_ = (call);                                                     \
    if (e_ != cudaSuccess) {                                                     \
      if (cb::verbose()) fprintf(stderr, "[chase_bse] %s:%d %s -> %s\n", __FILE__, \
                                 __LINE__, #call, cudaGetErrorString(e_));       \
      return (e_ == cudaErrorMemoryAllocation) ? CHASE_BSE_OOM : CHASE_BSE_CUDA_ERROR; \
    }                                                                            \
  } while (0)
#define CB_LAUNCH()                                                              \
  do {                                                                           \
    cudaError_t e_ = cudaGetLastError();                                         \
    if (e_ != cudaSuccess) {                                                     \
      if (cb::verbose()) fprintf(stderr, "[chase_bse] %s:%d launch -> %s\n",     \
                                 __FILE__, __LINE__, cudaGetErrorString(e_));    \
      return CHASE_BSE_CUDA_ERROR;                                               \
    }                                                                            \
  } while (0)
#define CB_TRY(expr)            \
  do {                          \
    int s_ = (expr);            \
    if (s_ != CHASE_BSE_OK) return s_; \
  } while (0)

bool verbose();

// Number of kernels this library has launched (diagnostics for benchmarks).
void count_launch();
int64_t launch_count();

// Device-time record of the filter's H applications (diagnostics): kind 0 the
// tensor-core filter GEMM, kind 1 the FP64 H application, kind 2 the sliced
// FP64-accurate H application, each with its algorithmic flops.  timer_begin returns an id (-1 while the record is off) that timer_end
// closes after the launch.
int64_t timer_begin(int kind, double flops, cudaStream_t s);
void timer_end(int64_t id, cudaStream_t s);
void timer_enable(bool on);
int timer_read(int kind, double* ms, double* flops, int64_t* launches);

inline unsigned cdiv(int64_t a, int64_t b) { return (unsigned)((a + b - 1) / b); }

// Stream-ordered device allocation from the library's memory pool (one per
// device).  The pool keeps freed memory cached (release threshold: unlimited),
// so the per-iteration workspaces of a solve reuse their pages instead of
// mapping new ones; pool_trim() returns the cached memory to the driver.
cudaError_t dalloc(void** p, size_t bytes, cudaStream_t s);
template <class T>
inline cudaError_t dalloc(T** p, size_t bytes, cudaStream_t s) {
  return dalloc(reinterpret_cast<void**>(p), bytes, s);
}
void pool_trim();
// Number of device allocations the library has requested (every one goes through
// dalloc), for diagnostics and for the allocation-free entry point's tests.
int64_t alloc_count();
// Bound of the grid-barrier waits of the cooperative kernels (0: default 2 s).
uint64_t wait_limit_ns();
void set_wait_limit_ns(uint64_t ns);

// Stream-ordered workspace: every buffer is released when the owner goes out
// of scope (cudaFreeAsync on the same stream).
struct Workspace {
  cudaStream_t s;
  void* ptrs[64];
  int count = 0;
  explicit Workspace(cudaStream_t st) : s(st) {}
  ~Workspace() {
    for (int i = count - 1; i >= 0; --i) cudaFreeAsync(ptrs[i], s);
  }
  template <class T>
  int alloc(T** p, size_t elems) {
    *p = nullptr;
    if (elems == 0) elems = 1;
    if (count >= 64) return CHASE_BSE_OOM;
    void* q = nullptr;
    cudaError_t e = dalloc(&q, elems * sizeof(T), s);
    if (e != cudaSuccess) { cudaGetLastError(); return CHASE_BSE_OOM; }
    ptrs[count++] = q;
    *p = static_cast<T*>(q);
    return CHASE_BSE_OK;
  }
};

}  // namespace cb
