// Device helpers shared by the cooperative kernels (grid barrier) and the Jacobi
// eigensolvers (round-robin pairing).
#pragma once
#include <cuda_runtime.h>
#include <cstdint>

namespace cb {

// ------------------------------------------------------------ grid barrier
// For kernels launched cooperatively (all CTAs co-resident): a counter plus a
// generation word in global memory.  Every wait is bounded (2 s of
// %globaltimer by default, GridSync::limit_ns when set), after which the kernel
// records an error, and all CTAs leave at their next barrier.  Data written by other CTAs before a barrier is read
// with __ldcg (L2) after it.
struct GridSync {
  unsigned count;                // arrival word: its top bit flips once per completed barrier
  unsigned gen;                  // unused (kept zero)
  unsigned long long limit_ns;   // bound of a wait; 0: the default of 2 s
};

// Bound of the grid-barrier waits set by chase_bse_set_wait_limit (0: default).
uint64_t wait_limit_ns();

// Zero a GridSync on the stream and set its wait bound.
static inline cudaError_t gsync_init(GridSync* g, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(g, 0, sizeof(GridSync), s);
  const unsigned long long lim = (unsigned long long)wait_limit_ns();
  if (e == cudaSuccess && lim != 0)
    e = cudaMemcpyAsync(&g->limit_ns, &lim, sizeof(lim), cudaMemcpyHostToDevice, s);
  return e;
}
__device__ __forceinline__ unsigned long long gtimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// CTA 0 adds 2^31 - (gridDim.x - 1), every other CTA adds 1 (release), so the
// top bit of the word flips exactly when the last CTA arrives; the waiters poll
// it with acquire loads.  The wait is bounded: after the limit, or once another CTA
// has recorded an error, the CTA records the error and returns false.
__device__ inline bool grid_barrier(GridSync* gsync, int* err) {
  __shared__ int ok_sh;
  __syncthreads();
  if (threadIdx.x == 0) {
    ok_sh = 1;
    const unsigned inc = (blockIdx.x == 0) ? (0x80000000u - (gridDim.x - 1)) : 1u;
    unsigned old, cur;
    __threadfence();  // the CTA's writes (ordered before by __syncthreads) become visible first
    asm volatile("atom.add.release.gpu.u32 %0, [%1], %2;" : "=r"(old) : "l"(&gsync->count), "r"(inc) : "memory");
    const unsigned long long lim = gsync->limit_ns ? gsync->limit_ns : 2000000000ull;
    const unsigned long long t0 = gtimer_ns();
    unsigned it = 0;
    while (true) {
      asm volatile("ld.acquire.gpu.u32 %0, [%1];" : "=r"(cur) : "l"(&gsync->count) : "memory");
      if (((old ^ cur) & 0x80000000u) != 0) break;
      if ((++it & 7) == 0) {
        if (*(volatile int*)err) { ok_sh = 0; break; }
        if (gtimer_ns() - t0 > lim) {
          atomicExch(err, 1);
          ok_sh = 0;
          break;
        }
      }
    }
    __threadfence();
  }
  __syncthreads();
  return ok_sh != 0;
}


// Round-robin (circle) ordering of k indices (k even) over k - 1 rounds: position 0
// holds index 0, position p > 0 holds ((p - 1 + r) mod (k - 1)) + 1; slot s pairs the
// positions s and k - 1 - s.
// position of index x in round r (inverse of the pairing in jpair)
__device__ __forceinline__ int jpos(int x, int r, int k) {
  if (x == 0) return 0;
  int t = (x - 1 - r) % (k - 1);
  if (t < 0) t += k - 1;
  return t + 1;
}
__device__ __forceinline__ int jat(int pos, int r, int k) { return pos == 0 ? 0 : ((pos - 1 + r) % (k - 1)) + 1; }

__device__ __forceinline__ void jpair32(int slot, int r, int k, int& p, int& q) {
  const int a = jat(slot, r, k), b = jat(k - 1 - slot, r, k);
  p = a < b ? a : b;
  q = a < b ? b : a;
}


}  // namespace cb
