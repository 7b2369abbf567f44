// FP64-accurate sliced GEMM on tcgen05 tensor cores (see tc_dgemm.cuh).
//
// Kernel (one CTA per 128 x 32 output tile and K split, 384 threads):
//   warp 0    TMA producer: per 32-long K block, all 7 digit planes of the A tile
//             (one 3-D box of 32 x 128 x 7) and of the B tile (32 x 32 x 7), 64-byte
//             swizzle, into a 3-stage ring (70 KB per stage)
//   warp 1    allocates 512 TMEM columns; one lane issues, per 16-long K step and
//             A digit t, one MMA against the B digits u = 0 .. 6 - t stacked along N
//             (N = (7 - t) * 32), accumulating into the TMEM columns of the weight
//             groups w = t + u = t .. 6; two buffers of 7 x 32 columns alternate
//             every 128 K
//   warps 4-11 drain each finished buffer (warps 4-7 columns 0-15, warps 8-11
//             columns 16-31 of every group): the exact integer group sums of
//             weights 2^0 .. 2^-24 into one 64-bit integer per output, those of
//             2^-32 .. 2^-48 into a second one; at the end they write both to a
//             per-split partial tile
// A second kernel sums the splits in order, applies the row and column exponents
// and writes the FP64 result with arbitrary strides.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>

#include "tc_common.cuh"
#include "solver.cuh"
#include "tc_dgemm.cuh"

namespace cb {
namespace tcd {

using namespace cb::tc;

constexpr int S = SLICES;
constexpr int BM = 128, BNS = 32, BK = 32;
constexpr int A_SLICE = BM * BK * 2;                    // 8 KB
constexpr int B_SLICE = BNS * BK * 2;                   // 2 KB
constexpr int STAGE_BYTES = S * (A_SLICE + B_SLICE);    // 70 KB
constexpr int ST = 3;
constexpr int CHUNK = 4;                                // K blocks per exact partial sum (128 K)
constexpr int GCOLS = S * BNS;                          // TMEM columns per buffer
constexpr uint32_t TMEM_COLS = 512;
constexpr int THREADS = 384;
constexpr int DRAIN_WARPS = 8;
constexpr int NBAR = 2 * ST + 5;
constexpr int SMEM_BYTES = ST * STAGE_BYTES + 1024 + 256;
static_assert(2 * GCOLS <= (int)TMEM_COLS, "two accumulator buffers must fit in TMEM");
// a weight group holds at most S digit products of |d| <= 128 over CHUNK * BK terms
static_assert((double)S * 16384.0 * CHUNK * BK < 16777216.0, "group sums must stay exact in FP32");

__device__ __forceinline__ uint32_t idesc_n(int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
}
// K-major tile with 64-byte rows and 64-byte swizzle: 8-row groups 512 bytes apart.
__device__ __forceinline__ uint64_t sdesc64(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(512 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)4 << 61;  // 64-byte swizzle
  return d;
}

struct Args {
  int num_m, num_n, kb_total, kb_per_split;
  int n_fast;          // raster: the CTAs of one A tile (1) or of one B tile (0) run together
  int64_t mp;          // rows of a partial tile column (A rows_pad)
  int64_t np;          // columns per split (B rows_pad)
  long long* hi;       // [split][col][row]
  long long* lo;
  int* err;
};

__global__ void __launch_bounds__(THREADS, 1)
    sliced_gemm_kernel(const __grid_constant__ CUtensorMap ma, const __grid_constant__ CUtensorMap mb, Args g) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + ST * STAGE_BYTES);
  uint32_t full[ST], empty[ST];
#pragma unroll
  for (int s = 0; s < ST; ++s) {
    full[s] = smem_u32(bars + s);
    empty[s] = smem_u32(bars + ST + s);
  }
  const uint32_t accf[2] = {smem_u32(bars + 2 * ST), smem_u32(bars + 2 * ST + 1)};
  const uint32_t acce[2] = {smem_u32(bars + 2 * ST + 2), smem_u32(bars + 2 * ST + 3)};
  const uint32_t done = smem_u32(bars + 2 * ST + 4);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + NBAR);
  volatile int* abort_sh = reinterpret_cast<volatile int*>(tmem_slot + 1);
  int* issued_sh = reinterpret_cast<int*>(tmem_slot + 2);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  // the CTAs sharing a tile of the larger operand run together, so that it is read
  // from DRAM once and the other operand's tiles come from L2
  const int bid = blockIdx.x;
  const int mt = g.n_fast ? (bid / g.num_n) % g.num_m : bid % g.num_m;
  const int nt = g.n_fast ? bid % g.num_n : (bid / g.num_m) % g.num_n;
  const int sp = bid / (g.num_m * g.num_n);
  const int kb0 = sp * g.kb_per_split;
  const int nkb = min(g.kb_per_split, g.kb_total - kb0);

  if (threadIdx.x == 0) {
    for (int s = 0; s < ST; ++s) {
      mbar_init(full[s], 1);
      mbar_init(empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(accf[b], 1);
      mbar_init(acce[b], DRAIN_WARPS);
    }
    mbar_init(done, 1);
    *abort_sh = 0;
    *issued_sh = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const uint32_t sbase = smem_u32(smem);

  if (warp == 0 && lane == 0) {
    int issued = 0;
    for (int kb = 0; kb < nkb; ++kb) {
      const int s = kb % ST;
      const uint32_t ph = (uint32_t)(kb / ST) & 1u;
      if (kb >= ST && !mbar_wait(empty[s], ph ^ 1u, abort_sh, g.err, true)) break;
      const uint32_t st = sbase + s * STAGE_BYTES;
      mbar_expect_tx(full[s], STAGE_BYTES);
      tma_load_3d(st, &ma, (kb0 + kb) * BK, mt * BM, 0, full[s]);
      tma_load_3d(st + S * A_SLICE, &mb, (kb0 + kb) * BK, nt * BNS, 0, full[s]);
      issued = kb + 1;
    }
    *issued_sh = issued;
  } else if (warp == 1 && lane == 0) {
    const uint64_t dbase = sdesc64(sbase);
    for (int kb = 0; kb < nkb; ++kb) {
      const int grp = kb / CHUNK, b = grp & 1;
      const bool first = (kb % CHUNK) == 0;
      const bool last = (kb % CHUNK) == CHUNK - 1 || kb == nkb - 1;
      if (first && grp >= 2 && !mbar_wait(acce[b], (uint32_t)((grp >> 1) - 1) & 1u, abort_sh, g.err, true)) break;
      const int s = kb % ST;
      const uint32_t ph = (uint32_t)(kb / ST) & 1u;
      if (!mbar_wait(full[s], ph, abort_sh, g.err, true)) break;
      tc_fence_after();
      const uint32_t st = sbase + s * STAGE_BYTES;
      const uint32_t buf = tmem + (uint32_t)(b * GCOLS);
#pragma unroll
      for (int kk = 0; kk < BK / 16; ++kk) {
        // sdesc64 is linear in the address here (its 14-bit start field holds address / 16
        // of a ring below 256 KB and cannot carry): a hoisted base plus constants
        const uint64_t sd = dbase + (uint64_t)((uint32_t)(st - sbase) >> 4);
        const uint64_t bd = sd + (uint64_t)((S * A_SLICE + kk * 32) >> 4);
#pragma unroll
        for (int t = 0; t < S; ++t) {
          const uint64_t ad = sd + (uint64_t)((t * A_SLICE + kk * 32) >> 4);
          const uint32_t acc = (first && kk == 0 && t == 0) ? 0u : 1u;
          mma_bf16(buf + (uint32_t)(t * BNS), ad, bd, idesc_n((S - t) * BNS), acc);
        }
      }
      mma_commit(empty[s]);
      if (last) mma_commit(accf[b]);
    }
    mma_commit(done);
  } else if (warp >= 4) {
    // TMEM lanes 32 (warp % 4) .. +31 are the rows; half selects columns 0-15 or 16-31
    const int q = warp & 3, half = (warp - 4) >> 2;
    const uint32_t lane_base = (uint32_t)(q * 32) << 16;
    constexpr int NC = BNS / 2;
    long long hi[NC], lo[NC];
#pragma unroll
    for (int i = 0; i < NC; ++i) {
      hi[i] = 0;
      lo[i] = 0;
    }
    bool ok = true;
    const int ngrp = (nkb + CHUNK - 1) / CHUNK;
    for (int grp = 0; grp < ngrp; ++grp) {
      const int b = grp & 1;
      const bool w = mbar_wait(accf[b], (uint32_t)(grp >> 1) & 1u, abort_sh, g.err, true);
      if (!__all_sync(0xffffffffu, w)) {
        ok = false;
        break;
      }
      tc_fence_after();
      const uint32_t col = tmem + lane_base + (uint32_t)(b * GCOLS + half * NC);
      uint32_t r0[NC], r1[NC], r2[NC];
      // group sums g_w are integers below 2^24 (exact in FP32)
      // hi += (g0 2^8 + g1) 2^16 + g2 2^8 + g3       (each bracket below 2^31)
      tmem_ld16_nowait(col, r0);
      tmem_ld16_nowait(col + 32, r1);
      tmem_wait_ld();
#pragma unroll
      for (int i = 0; i < NC; ++i) {
        const int v = __float2int_rn(__uint_as_float(r0[i])) * 256 + __float2int_rn(__uint_as_float(r1[i]));
        hi[i] += (long long)v * 65536;
      }
      tmem_ld16_nowait(col + 64, r0);
      tmem_ld16_nowait(col + 96, r1);
      tmem_wait_ld();
#pragma unroll
      for (int i = 0; i < NC; ++i) {
        const int v = __float2int_rn(__uint_as_float(r0[i])) * 256 + __float2int_rn(__uint_as_float(r1[i]));
        hi[i] += (long long)v;
      }
      // lo += g4 2^16 + g5 2^8 + g6
      tmem_ld16_nowait(col + 128, r0);
      tmem_ld16_nowait(col + 160, r1);
      tmem_ld16_nowait(col + 192, r2);
      tmem_wait_ld();
#pragma unroll
      for (int i = 0; i < NC; ++i) {
        lo[i] += (long long)__float2int_rn(__uint_as_float(r0[i])) * 65536 +
                 (long long)__float2int_rn(__uint_as_float(r1[i])) * 256 +
                 (long long)__float2int_rn(__uint_as_float(r2[i]));
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(acce[b]);
    }
    if (ok && !*abort_sh) {
      const int64_t row = (int64_t)mt * BM + q * 32 + lane;  // < mp: rows are padded to whole tiles
      const int64_t base = ((int64_t)sp * g.np + (int64_t)nt * BNS + half * NC) * g.mp + row;
#pragma unroll
      for (int i = 0; i < NC; ++i) {
        g.hi[base + (int64_t)i * g.mp] = hi[i];
        g.lo[base + (int64_t)i * g.mp] = lo[i];
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (threadIdx.x == 0 && *abort_sh) {
    const int issued = *issued_sh;
    for (int kb = max(0, issued - ST); kb < issued; ++kb)
      mbar_wait(full[kb % ST], (uint32_t)(kb / ST) & 1u, abort_sh, g.err, false);
  }
  if (warp == 1) {
    if (lane == 0) mbar_wait(done, 0, abort_sh, g.err, false);
    __syncwarp();
  }
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
  }
}

__global__ void sliced_finalize_kernel(const long long* hi, const long long* lo, int splits, int64_t mp, int64_t np,
                                       const int* ea, const int* eb, int64_t M, int64_t N, double alpha,
                                       double* out, int64_t rs, int64_t cs, int neg_odd) {
  const int64_t total = M * N;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = idx % M, c = idx / M;
    long long h = 0, l = 0;
    for (int sp = 0; sp < splits; ++sp) {
      const int64_t o = ((int64_t)sp * np + c) * mp + r;
      h += hi[o];
      l += lo[o];
    }
    // exact when |h|, |l| < 2^53; one rounding for the sum
    const double v = fma((double)l, 0x1p-48, (double)h * 0x1p-24);
    double y = alpha * ldexp(v, ea[r] + eb[c] - 14);
    if (neg_odd && (r & 1)) y = -y;
    out[r * rs + c * cs] = y;
  }
}

// ---------------------------------------------------------------- slicing
// One warp per row: exponent e with |x| < 2^e on the row, then the digits
// d_t = rint(r_t), r_0 = x 2^(7-e), r_{t+1} = (r_t - d_t) 2^8.
// Balanced base-256 digits of s = x 2^(7 - e) (|x| <= 2^e), in integer arithmetic:
// N = round(x 2^(55 - e)) from the exponent and mantissa bits (|N| < 2^55, rounded half
// away from zero), then d_6 .. d_1 the balanced low bytes of N (in [-128, 127]) and d_0
// what is left (|d_0| <= 128): s = sum_t d_t 2^(-8t) up to 2^-49.
__device__ __forceinline__ void int_digits(double x, int e, int* d) {
  const long long b = __double_as_longlong(x);
  const int ef = (int)((b >> 52) & 0x7ff);
  long long mant = b & 0xfffffffffffffLL;
  int ex = ef;
  if (ef == 0) ex = 1;
  else mant |= 1LL << 52;
  const int sh = ex - 1020 - e;  // N = mant 2^sh; sh <= 2 for every |x| <= 2^e
  long long N = 0;
  if (sh >= 0) N = mant << sh;
  else if (sh > -63) N = (mant + (1LL << (-sh - 1))) >> (-sh);
  if (b < 0) N = -N;
#pragma unroll
  for (int t = S - 1; t >= 1; --t) {
    const int dt = (int)((N + 128) & 255) - 128;
    d[t] = dt;
    N = (N - dt) >> 8;
  }
  d[0] = (int)N;
}
// frexp exponent of the largest |x| of a row from the magnitudes' bit patterns
// (non-negative doubles order like their bits): 0 for a zero row.
__device__ __forceinline__ int row_exponent(unsigned long long mbits) {
  if (mbits == 0) return 0;
  const int ef = (int)(mbits >> 52);
  if (ef) return ef - 1022;
  return (64 - __clzll((long long)mbits)) - 1074;  // subnormal
}
template <class Src>
__global__ void slice_kernel(Src src, int64_t rows, int64_t K, int64_t kpad, int64_t plane, __nv_bfloat16* planes,
                             int* exps) {
  const int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (r >= rows) return;
  unsigned long long m = 0;
  for (int64_t p = lane; 2 * p < K; p += 32) {
    const double2 v = src.pair(r, p);
    const unsigned long long a0 = (unsigned long long)__double_as_longlong(v.x) & 0x7fffffffffffffffull;
    const unsigned long long a1 = (unsigned long long)__double_as_longlong(v.y) & 0x7fffffffffffffffull;
    m = max(m, max(a0, a1));
  }
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  const int e = row_exponent(m);
  __nv_bfloat16* row = planes + r * kpad;
  for (int64_t p = lane; 2 * p < kpad; p += 32) {
    double2 v = make_double2(0.0, 0.0);
    if (2 * p < K) v = src.pair(r, p);
    int d0[S], d1[S];
    int_digits(v.x, e, d0);
    int_digits(v.y, e, d1);
#pragma unroll
    for (int t = 0; t < S; ++t)
      *reinterpret_cast<__nv_bfloat162*>(row + t * plane + 2 * p) =
          __halves2bfloat162(__int2bfloat16_rn(d0[t]), __int2bfloat16_rn(d1[t]));
  }
  if (lane == 0) exps[r] = e;
}

struct RowsSrc {  // row r at p + r * ld, pairs transformed by mode
  const double* p;
  int64_t ld;
  int mode;
  __device__ double2 pair(int64_t r, int64_t q) const {
    const double2 v = *reinterpret_cast<const double2*>(p + r * ld + 2 * q);
    if (mode == 1) return make_double2(v.y, -v.x);
    if (mode == 2) return make_double2(v.x, -v.y);
    return v;
  }
};
struct RowsSrcUnaligned {  // same, for an odd ld or offset
  const double* p;
  int64_t ld;
  int mode;
  __device__ double2 pair(int64_t r, int64_t q) const {
    const double a = p[r * ld + 2 * q], b = p[r * ld + 2 * q + 1];
    if (mode == 1) return make_double2(b, -a);
    if (mode == 2) return make_double2(a, -b);
    return make_double2(a, b);
  }
};
struct HamSrc {  // rows of P': y = A x + B conj(x) in (re, im) interleaved form
  const cplx* A;
  const cplx* B;
  int64_t n;
  __device__ double2 pair(int64_t r, int64_t l) const {
    const int64_t i = r >> 1;
    const cplx a = A[i * n + l], b = B[i * n + l];
    if ((r & 1) == 0) return make_double2(a.x + b.x, b.y - a.y);  // Re y: (Re x, Im x) coefficients
    return make_double2(a.y + b.y, a.x - b.x);                    // Im y
  }
};

// The blocks of H^2 as C = [A | -B] R, R = [[A, B], [conj B, conj A]], computed as
// C^T = R^T [A | -B]^T so that the result lands row-major: the A operand holds the
// real-form rows of the columns j0 + r/2 of R's left (part 0: P2) or right (part 1: Q2)
// block column, the B operand the rows of [A | -B] as (re, im) pairs.
struct H2ColsSrc {
  const cplx* A;
  const cplx* B;
  int64_t n, j0;
  int part;
  __device__ double2 pair(int64_t r, int64_t l) const {
    const int64_t j = j0 + (r >> 1);
    cplx v;
    if (l < n) v = part == 0 ? A[l * n + j] : B[l * n + j];
    else v = cconj(part == 0 ? B[(l - n) * n + j] : A[(l - n) * n + j]);
    // row 2j: (Re, -Im); row 2j + 1: (Im, Re) -> (Re, Im) of sum_l R_lj w_l for w pairs (Re, Im)
    return (r & 1) == 0 ? make_double2(v.x, -v.y) : make_double2(v.y, v.x);
  }
};
struct H2RowsSrc {  // row i of [A | -B] as (re, im) pairs
  const cplx* A;
  const cplx* B;
  int64_t n;
  __device__ double2 pair(int64_t i, int64_t l) const {
    if (l < n) {
      const cplx v = A[i * n + l];
      return make_double2(v.x, v.y);
    }
    const cplx v = B[i * n + (l - n)];
    return make_double2(-v.x, -v.y);
  }
};

struct ComplexRowsSrc {  // row r of the complex column-major M, optionally conjugated
  const cplx* M;
  int64_t ld;
  double sign;  // -1: conjugate
  __device__ double2 pair(int64_t r, int64_t l) const {
    const cplx v = M[r + l * ld];
    return make_double2(v.x, sign * v.y);
  }
};

// out (2n x 2m, row-major): rows 2i, 2i+1 of the real form of row i of X.
__global__ void complex_rows_kernel(const cplx* X, int64_t ldx, int64_t n, int64_t m, double* out) {
  __shared__ cplx t[32][33];
  const int64_t i0 = (int64_t)blockIdx.x * 32, l0 = (int64_t)blockIdx.y * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
  for (int j = ty; j < 32; j += 8) {
    const int64_t i = i0 + tx, l = l0 + j;
    t[j][tx] = (i < n && l < m) ? X[i + l * ldx] : mk(0, 0);
  }
  __syncthreads();
  for (int j = ty; j < 32; j += 8) {
    const int64_t i = i0 + j, l = l0 + tx;
    if (i < n && l < m) {
      const cplx x = t[tx][j];
      double* r0 = out + (2 * i) * (2 * m) + 2 * l;
      double* r1 = r0 + 2 * m;
      r0[0] = x.x;
      r0[1] = -x.y;
      r1[0] = x.y;
      r1[1] = x.x;
    }
  }
}

// Z (n x 2k, column-major) from W (2n x k): the J-fixed halves of w_j = [x; y],
// a_j = (x + conj(y))/2 and c_j = i (x - conj(y))/2, so that w = [a; conj(a)] - i [c; conj(c)].
__global__ void jsplit_kernel(const cplx* W, int64_t n, int64_t k, cplx* Z) {
  const int64_t total = n * k;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = idx % n, j = idx / n;
    const cplx x = W[j * 2 * n + i], y = W[j * 2 * n + n + i];
    const cplx a = mk(0.5 * (x.x + y.x), 0.5 * (x.y - y.y));
    const cplx d = mk(0.5 * (x.x - y.x), 0.5 * (x.y + y.y));  // (x - conj(y)) / 2
    Z[(2 * j) * n + i] = a;
    Z[(2 * j + 1) * n + i] = mk(-d.y, d.x);                  // i d
  }
}
// H w_j from T = [P'a_j, P'c_j] (y = A z + B conj(z) of the J-fixed halves):
// top = P'a - i P'c, bottom = -conj(P'a) + i conj(P'c).
__global__ void jcombine_kernel(const cplx* T, int64_t n, int64_t k, cplx* out) {
  const int64_t total = n * k;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = idx % n, j = idx / n;
    const cplx ta = T[(2 * j) * n + i], tc = T[(2 * j + 1) * n + i];
    out[j * 2 * n + i] = mk(ta.x + tc.y, ta.y - tc.x);       // ta - i tc
    out[j * 2 * n + n + i] = mk(-ta.x + tc.y, ta.y + tc.x);  // -conj(ta) + i conj(tc)
  }
}

static unsigned gsz(int64_t total) {
  const int64_t b = (total + 255) / 256;
  return (unsigned)std::min<int64_t>(std::max<int64_t>(b, 1), 16384);
}

static int make_map3(CUtensorMap* m, const void* base, int64_t kpad, int64_t rows_pad, int box_rows) {
  auto fn = encode_fn();
  if (!fn) return CHASE_BSE_UNSUPPORTED;
  const cuuint64_t dims[3] = {(cuuint64_t)kpad, (cuuint64_t)rows_pad, (cuuint64_t)S};
  const cuuint64_t strides[2] = {(cuuint64_t)kpad * 2, (cuuint64_t)(rows_pad * kpad * 2)};
  const cuuint32_t box[3] = {(cuuint32_t)BK, (cuuint32_t)box_rows, (cuuint32_t)S};
  const cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(base), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? CHASE_BSE_OK : CHASE_BSE_CUDA_ERROR;
}

template <class Src>
static int run_slice(const Src& src, SlicedOp& op, cudaStream_t s) {
  const int64_t warps = op.rows;
  slice_kernel<Src><<<(unsigned)((warps * 32 + 255) / 256), 256, 0, s>>>(src, op.rows, op.K, op.kpad,
                                                                          op.rows_pad * op.kpad, op.planes, op.exps);
  count_launch();
  CB_LAUNCH();
  return CHASE_BSE_OK;
}

}  // namespace tcd

int sliced_alloc(Workspace& ws, SlicedOp& op, int64_t rows, int64_t K, cudaStream_t s) {
  using namespace tcd;
  if (rows <= 0 || K <= 0 || (K % 2) != 0) return CHASE_BSE_BAD_ARG;
  op.rows = rows;
  op.K = K;
  op.rows_pad = ((rows + BM - 1) / BM) * BM;
  op.kpad = ((K + BK - 1) / BK) * BK;
  const int64_t elems = (int64_t)S * op.rows_pad * op.kpad;
  CB_TRY(ws.alloc(&op.planes, elems));
  CB_TRY(ws.alloc(&op.exps, op.rows_pad));
  // rows beyond `rows` stay zero (and their exponent 0)
  if (op.rows_pad > rows) {
    for (int t = 0; t < S; ++t)
      CB_CUDA(cudaMemsetAsync(op.planes + (int64_t)t * op.rows_pad * op.kpad + rows * op.kpad, 0,
                              sizeof(__nv_bfloat16) * (op.rows_pad - rows) * op.kpad, s));
    CB_CUDA(cudaMemsetAsync(op.exps + rows, 0, sizeof(int) * (op.rows_pad - rows), s));
  }
  CB_TRY(make_map3(&op.map_a, op.planes, op.kpad, op.rows_pad, BM));
  CB_TRY(make_map3(&op.map_b, op.planes, op.kpad, op.rows_pad, BNS));
  return CHASE_BSE_OK;
}

int slice_rows(const double* src, int64_t ld, int mode, SlicedOp& op, cudaStream_t s) {
  if ((reinterpret_cast<uintptr_t>(src) % 16) == 0 && (ld % 2) == 0)
    return tcd::run_slice(tcd::RowsSrc{src, ld, mode}, op, s);
  return tcd::run_slice(tcd::RowsSrcUnaligned{src, ld, mode}, op, s);
}

int slice_complex_rows(const cplx* X, int64_t ldx, int64_t n, int64_t m, double* tmp, SlicedOp& op,
                       cudaStream_t s) {
  if (op.rows != 2 * n || op.K != 2 * m) return CHASE_BSE_BAD_ARG;
  dim3 grid((unsigned)((n + 31) / 32), (unsigned)((m + 31) / 32));
  tcd::complex_rows_kernel<<<grid, dim3(32, 8), 0, s>>>(X, ldx, n, m, tmp);
  count_launch();
  CB_LAUNCH();
  return slice_rows(tmp, 2 * m, 0, op, s);
}

int slice_conj_rows(const cplx* M, int64_t ld, SlicedOp& op, cudaStream_t s) {
  return tcd::run_slice(tcd::ComplexRowsSrc{M, ld, -1.0}, op, s);
}

int slice_plain_rows(const cplx* M, int64_t ld, SlicedOp& op, cudaStream_t s) {
  return tcd::run_slice(tcd::ComplexRowsSrc{M, ld, 1.0}, op, s);
}

int hop_sliced(const SlicedOp& ph, const cplx* W, int64_t n, int64_t k, cplx* out, cudaStream_t s) {
  if (k == 0) return CHASE_BSE_OK;
  if (ph.rows != 2 * n || ph.K != 2 * n) return CHASE_BSE_BAD_ARG;
  Workspace ws(s);
  cplx *Z, *T;
  CB_TRY(ws.alloc(&Z, n * 2 * k));
  CB_TRY(ws.alloc(&T, n * 2 * k));
  SlicedOp sz;
  CB_TRY(sliced_alloc(ws, sz, 2 * k, 2 * n, s));
  const int64_t tid = timer_begin(2, 32.0 * (double)n * (double)n * (double)k, s);
  tcd::jsplit_kernel<<<tcd::gsz(n * k), 256, 0, s>>>(W, n, k, Z);
  count_launch();
  CB_LAUNCH();
  CB_TRY(slice_rows(reinterpret_cast<const double*>(Z), 2 * n, 0, sz, s));
  CB_TRY(sliced_gemm(ph, sz, 1.0, reinterpret_cast<double*>(T), 1, 2 * n, false, s));
  tcd::jcombine_kernel<<<tcd::gsz(n * k), 256, 0, s>>>(T, n, k, out);
  timer_end(tid, s);
  count_launch();
  CB_LAUNCH();
  return CHASE_BSE_OK;
}

int form_h2(const cplx* A, const cplx* B, int64_t n, cplx* P2, cplx* Q2, cudaStream_t s) {
  Workspace ws(s);
  SlicedOp rows;  // [A | -B]: n rows of 2n complex entries
  CB_TRY(sliced_alloc(ws, rows, n, 4 * n, s));
  CB_TRY(tcd::run_slice(tcd::H2RowsSrc{A, B, n}, rows, s));
  // columns of R in chunks: the A operand of a chunk of cj columns holds 7 digit planes of
  // 2 cj x 4n BF16 values (about 8 GB at most)
  int64_t cj = std::max<int64_t>(64, (int64_t)(8.0e9 / (112.0 * (double)n)) / 64 * 64);
  cj = std::min(cj, n);
  for (int part = 0; part < 2; ++part) {
    cplx* out = part == 0 ? P2 : Q2;
    for (int64_t j0 = 0; j0 < n; j0 += cj) {
      const int64_t m = std::min(cj, n - j0);
      Workspace cws(s);
      SlicedOp cols;
      CB_TRY(sliced_alloc(cws, cols, 2 * m, 4 * n, s));
      CB_TRY(tcd::run_slice(tcd::H2ColsSrc{A, B, n, j0, part}, cols, s));
      // C^T[2(j - j0) + t][i] -> (Re, Im) of C_ij at double 2 (i n + j) + t
      CB_TRY(sliced_gemm(cols, rows, 1.0, reinterpret_cast<double*>(out + j0), 1, 2 * n, false, s));
    }
  }
  return CHASE_BSE_OK;
}

int slice_hamiltonian(const cplx* A, const cplx* B, int64_t n, SlicedOp& op, cudaStream_t s) {
  if (op.rows != 2 * n || op.K != 2 * n) return CHASE_BSE_BAD_ARG;
  return tcd::run_slice(tcd::HamSrc{A, B, n}, op, s);
}

int sliced_gemm(const SlicedOp& a, const SlicedOp& b, double alpha, double* out, int64_t rs, int64_t cs,
                bool neg_odd, cudaStream_t s) {
  using namespace tcd;
  if (a.K != b.K || a.kpad != b.kpad) return CHASE_BSE_BAD_ARG;
  static bool attr = false;
  if (!attr) {
    CB_CUDA(cudaFuncSetAttribute(sliced_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES));
    attr = true;
  }
  const int num_m = (int)(a.rows_pad / BM);
  const int num_n = (int)((b.rows + BNS - 1) / BNS);
  const int kb_total = (int)(a.kpad / BK);
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  // split K until about two CTAs per SM, keeping whole 128-long chunks per split
  const int64_t tiles = (int64_t)num_m * num_n;
  const int max_split = std::max(1, kb_total / CHUNK);
  int splits = (int)std::min<int64_t>(max_split, std::max<int64_t>(1, (2 * sms + tiles - 1) / tiles));
  int kb_per = (kb_total + splits - 1) / splits;
  kb_per = ((kb_per + CHUNK - 1) / CHUNK) * CHUNK;
  splits = (kb_total + kb_per - 1) / kb_per;
  Workspace ws(s);
  const int64_t np = (int64_t)num_n * BNS, mp = a.rows_pad;
  Args g{};
  g.num_m = num_m;
  g.num_n = num_n;
  g.n_fast = a.rows_pad >= b.rows_pad ? 1 : 0;
  g.kb_total = kb_total;
  g.kb_per_split = kb_per;
  g.mp = mp;
  g.np = np;
  CB_TRY(ws.alloc(&g.hi, (size_t)splits * np * mp));
  CB_TRY(ws.alloc(&g.lo, (size_t)splits * np * mp));
  CB_TRY(ws.alloc(&g.err, 1));
  CB_CUDA(cudaMemsetAsync(g.err, 0, sizeof(int), s));
  sliced_gemm_kernel<<<(unsigned)(tiles * splits), THREADS, SMEM_BYTES, s>>>(a.map_a, b.map_b, g);
  count_launch();
  CB_LAUNCH();
  sliced_finalize_kernel<<<gsz(a.rows * b.rows), 256, 0, s>>>(g.hi, g.lo, splits, mp, np, a.exps, b.exps, a.rows,
                                                              b.rows, alpha, out, rs, cs, neg_odd ? 1 : 0);
  count_launch();
  CB_LAUNCH();
  int herr = 0;
  CB_CUDA(cudaMemcpyAsync(&herr, g.err, sizeof(int), cudaMemcpyDeviceToHost, s));
  CB_CUDA(cudaStreamSynchronize(s));
  return herr ? CHASE_BSE_DEVICE_TIMEOUT : CHASE_BSE_OK;
}

}  // namespace cb
