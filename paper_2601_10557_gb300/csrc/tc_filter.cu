// Mixed-precision Chebyshev filter on H^2 with tcgen05 tensor cores (sm_103a).
//
// One application of H is one real GEMM on 5th-generation tensor cores:
//   C (n x 4k, FP32 in TMEM) = Pr (n x 4n) * Bop^T,   Bop: 4k x 4n,
// where Pr holds the rows of P = [A | B] with re/im interleaved along K, and
// every input vector w_j (2n complex) contributes four K-major rows of Bop:
//   4j+0: (Re w, -Im w)   4j+1: (Im w, Re w)            -> P w
//   4j+2: (Re u, -Im u)   4j+3: (Im u, Re u),  u = [conj(w_bot); conj(w_top)] -> P u
// so that (H w)_top = P w and (H w)_bot = -conj(P u) land in four adjacent
// accumulator columns of the same TMEM lane (row i of the tile).
//
// Split products on 16-bit tensor cores: an operand x is written as a sum of
// pieces x = x0 + x1 (+ x2), x0 = rn(x), x1 = rn(x - x0), ..., and the product
// keeps the cross terms down to the target accuracy, all accumulated in FP32:
//   FP16x3: 2 FP16 pieces each (11 + 11 bits), x0 y0 + x0 y1 + x1 y0   (~2^-22)
//   BF16x3: 2 BF16 pieces each (8 + 8 bits), same products             (~2^-16)
//   BF16x6: 3 BF16 pieces each, adds x0 y2 + x1 y1 + x2 y0             (~2^-24)
// (FP16 pieces of this kind: Ootomo and Yokota, Int. J. HPC Appl. 2022.)  FP16 has
// a 5-bit exponent, so every operand row is scaled by a power of two: row r of P
// by 2^prow[r] (its largest entry in [2^12, 2^13)), vector v by 2^vexp[v], chosen
// from an upper bound of its entries below 2^13: the bound of an output of H is
// L * max|input| with L the largest absolute row sum of P, and that of the
// recurrence combines the maxima of its terms; every epilogue records the true
// maximum of each output vector (one atomic max per warp and vector) for the
// next bound.  The epilogue divides the accumulator by 2^(prow + vexp).  Entries
// far below the bound only lose precision relative to the bound, which keeps the
// product's error below that of an FP32 GEMM (|dy| <~ 2^-22 L max|w|).  The
// BF16 schemes use the same scaling (harmless: BF16 has FP32's exponent range).
//
// Kernel structure (one K range of one 128 x 128 output tile per CTA, 384 threads):
//   warp 0   TMA producer: the A pieces and the B pieces of 64 K-elements (128B
//            swizzle) into a 3-stage (two pieces) or 2-stage (three pieces)
//            shared-memory ring
//   warp 1   allocates all 512 TMEM columns (two alternating x0*y0 buffers and two
//            for the cross products); one lane issues the tcgen05.mma of a K block
//   warps 4-11 drain the partial sums of every FLUSH K blocks (tcgen05.ld) into FP32
//            registers while the next group accumulates in the other buffer,
//            because the tensor core's FP32 accumulation truncates; then (with a K
//            split) write a partial tile, the last writer of a tile summing them,
//            and either
//            (mode 0) store the next GEMM's B-operand pieces, or
//            (mode 1) the fused three-term recurrence in FP32 plus the pieces, or
//            (mode 2) Z = H X + gamma_col * X (no pieces).
// Every mbarrier wait is bounded (2 s of %globaltimer); on expiry the kernel
// sets an error flag, waits (bounded) for its copies in flight into its shared
// memory, frees its TMEM and returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "dense_kernels.cuh"
#include "fp64_kernels.cuh"
#include "solver.cuh"
#include "tc_common.cuh"

namespace cb {
namespace tc {

constexpr int BM = 128;
constexpr int KPAD = 64;              // K (4n) is padded to a multiple of this
constexpr uint32_t TMEM_COLS = 512;   // two accumulator buffers (+ the cross products for 128-wide tiles)
constexpr int VEXP_MAX = 100;         // |operand exponents| are clamped to this
// instruction descriptor, kind::f16: D = F32, A = B = BF16 (bf16) or FP16, both K-major, 128 x n
__device__ __forceinline__ uint32_t make_idesc(int n, bool bf16) {
  return (1u << 4) | (bf16 ? ((1u << 7) | (1u << 10)) : 0u) | ((uint32_t)(n >> 3) << 17) |
         ((uint32_t)(BM >> 4) << 24);
}

// 16-bit piece types
template <class T>
struct Piece;
template <>
struct Piece<__nv_bfloat16> {
  using T2 = __nv_bfloat162;
  static constexpr bool BF16 = true;
  __device__ static __nv_bfloat16 rn(float x) { return __float2bfloat16_rn(x); }
  __device__ static float back(__nv_bfloat16 x) { return __bfloat162float(x); }
  __device__ static T2 pair(__nv_bfloat16 a, __nv_bfloat16 b) { return __halves2bfloat162(a, b); }
};
template <>
struct Piece<__half> {
  using T2 = __half2;
  static constexpr bool BF16 = false;
  __device__ static __half rn(float x) { return __float2half_rn(x); }
  __device__ static float back(__half x) { return __half2float(x); }
  __device__ static T2 pair(__half a, __half b) { return __halves2half2(a, b); }
};

// Scheme: piece type, pieces of A (NPA) and B (NPW), product list (product 0 is x0 * y0).
enum : int { SCH_BF16X3 = 1, SCH_BF16X6 = 2, SCH_FP16X3 = 3 };
template <int SCH>
struct Scheme;
template <>
struct Scheme<SCH_BF16X3> {
  using T = __nv_bfloat16;
  // FLUSH: K blocks per drained partial sum of x0 * y0 (16 truncating MMA additions
  // stay far below the 2^-16 error of the BF16 pieces; measured unchanged from 8)
  static constexpr int NPA = 2, NPW = 2, NPROD = 3, STAGES = 3, FLUSH = 4;
  __device__ static constexpr int pa(int i) { return i == 2 ? 1 : 0; }
  __device__ static constexpr int pb(int i) { return i == 1 ? 1 : 0; }
};
template <>
struct Scheme<SCH_FP16X3> {
  using T = __half;
  static constexpr int NPA = 2, NPW = 2, NPROD = 3, STAGES = 3, FLUSH = 4;
  __device__ static constexpr int pa(int i) { return i == 2 ? 1 : 0; }
  __device__ static constexpr int pb(int i) { return i == 1 ? 1 : 0; }
};
template <>
struct Scheme<SCH_BF16X6> {
  using T = __nv_bfloat16;
  static constexpr int NPA = 3, NPW = 3, NPROD = 6, STAGES = 2, FLUSH = 2;
  // (0,0) (0,1) (1,0) (0,2) (1,1) (2,0)
  __device__ static constexpr int pa(int i) { return i == 2 ? 1 : (i == 4 ? 1 : (i == 5 ? 2 : 0)); }
  __device__ static constexpr int pb(int i) { return i == 1 ? 1 : (i == 3 ? 2 : (i == 4 ? 1 : 0)); }
};
// Tile geometry for BNT-wide output tiles.  128-wide: K blocks of 64 (128-byte swizzle);
// the x0 * y0 product drains from two alternating TMEM buffers and the cross products
// accumulate over all of K in two more (odd-numbered products in one, even in the other:
// no two consecutive MMAs of a K step then write the same accumulator, 3-6 % faster than
// a single cross buffer behind three rotating x0 * y0 buffers); 8 drain warps of 64 columns (two per TMEM lane
// quarter: half the drain latency of 4 warps of 128 columns, and 135 registers a thread
// instead of 228).  256-wide (two pieces only): K blocks of 32 (64-byte swizzle) in a
// 4-stage ring of 48 KB stages; each SM takes in 48 KB per 768 MMA cycles instead of
// 64 KB (the shared-memory fill per MMA cycle bounds the 128-wide tiles); all products
// share the two alternating buffers, drained after every K block, and each block issues
// its cross products (2^-11 of the result) before x0 * y0, so the truncating
// accumulator adds only two MMAs at full magnitude per drain (as the 128-wide x0 * y0
// buffer per 32 K elements); 16 drain warps of 64 columns keep the FP32 partial sums in
// registers.
template <int SCH, int BNT, int FL>
struct Geo {
  static constexpr int BK = (BNT == 256) ? 32 : 64;
  static constexpr int SWZ = BK * 2;                       // swizzle span (bytes) = one row of a tile
  static constexpr int STAGES = (BNT == 256) ? 4 : Scheme<SCH>::STAGES;
  static constexpr int FLUSH = FL;
  static constexpr bool CROSS = (BNT == 128);             // separate cross-product buffers
  static constexpr int NB = 2;                             // alternating x0 * y0 (or all-product) buffers
  static constexpr int NCROSS = CROSS ? 2 : 0;             // cross-product buffers
  static constexpr int A_BYTES = BM * BK * 2;
  static constexpr int B_BYTES = BNT * BK * 2;
  static constexpr int STAGE_BYTES = Scheme<SCH>::NPA * A_BYTES + Scheme<SCH>::NPW * B_BYTES;
  static constexpr int NBAR = 2 * STAGES + 2 * NB + 1;  // full, empty, acc_full[NB], acc_empty[NB], done
  static constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 + 256;
  static constexpr int DCOLS = 64;                         // columns per drain warp
  static constexpr int DRAIN_WARPS = 4 * (BNT / DCOLS);
  static constexpr int THREADS = 128 + 32 * DRAIN_WARPS;
  static_assert(STAGE_BYTES * STAGES + 1280 <= 232448, "shared memory");
  static_assert((NB + NCROSS) * BNT <= (int)TMEM_COLS, "TMEM columns");
};

struct Epi {
  int mode;           // 0: operand pieces, 1: recurrence, 2: H X + gamma X
  int h2;             // 1: the operand holds [P | Q] of H^2 = [[P, Q], [conj Q, conj P]]
  int64_t n, k;       // rows of P, active vectors
  int64_t kpad;       // elements per piece row
  void* out[3];       // output operand pieces (NPW used)
  float2* Znext;
  const float2* Zcur;
  const float2* Zprev;
  const float2* src;
  const float* gamma;  // per column
  float alpha, beta, c;
  // operand scaling: P' = diag(2^prow) P, input B' = w 2^vexp_in[v]; the pieces this
  // launch writes get 2^vexp_out[v] chosen from the bound
  //   ca * amax_a[v] + cb * amax_b[v] + cc * amax_c[v] + |gamma[v]| * amax_d[v]
  // (amax_*: largest |component| of each input vector); amax_out receives the largest
  // |component| of each output vector
  const int* prow;
  const int* vexp_in;
  int* vexp_out;
  float* amax_out;
  const float* amax_a;
  const float* amax_b;
  const float* amax_c;
  const float* amax_d;
  float ca, cb, cc;
  int* err;
  float* part;  // split-K: one FP32 partial tile per CTA, column-major 128 x BNT
  int* cnt;     // split-K: per tile, partial tiles written so far (zero between launches)
  int sms;      // SMs of the device
};

// 2^e as a float, |e| <= 126
__device__ __forceinline__ float exp2i(int e) { return __int_as_float((e + 127) << 23); }
// Operand exponent for entries bounded by b: b 2^e < 2^13 (b = m 2^x, m in [1/2, 1) -> e = 13 - x);
// 0 for a zero, infinite or NaN bound.
__device__ __forceinline__ int out_exp(float b) {
  if (!(b > 0.0f) || !(b <= 3.0e38f)) return 0;
  const int bits = __float_as_int(b);
  const int x = ((bits >> 23) & 0xff) - 126;  // subnormal b: a smaller x, still a valid scale
  return min(max(13 - x, -VEXP_MAX), VEXP_MAX);
}
__device__ __forceinline__ float vec_bound(const Epi& ep, int64_t v) {
  float b = ep.ca * ep.amax_a[v];
  if (ep.cb != 0.0f) b += ep.cb * ep.amax_b[v];
  if (ep.cc != 0.0f) b += ep.cc * ep.amax_c[v];
  if (ep.amax_d) b += fabsf(ep.gamma[v]) * ep.amax_d[v];
  return b;
}

// Work of one launch: the 128 x BNT output tiles in a grouped raster (GROUP_M row
// tiles x all column tiles), repeated for nsplit K ranges, so that the CTAs running at
// the same time stream the same K blocks of A.  With nsplit > 1 the splits leave FP32
// partial tiles; the CTA that writes a tile's last one (a per-tile counter) sums them in
// split order and runs the epilogue, so no CTA waits for another and the result does
// not depend on timing.
struct Sched {
  int nkb, num_m, num_n, n_last, bnt, nsplit, ntiles;
  int group_m;  // raster: group_m row tiles x all column tiles per group
  __device__ void unit(int c, int& mt, int& nt, int& sp) const {
    sp = c / ntiles;
    const int t = c - sp * ntiles;
    const int per_group = group_m * num_n;
    const int g = t / per_group, first = g * group_m;
    const int gm = min(group_m, num_m - first);
    const int rem = t - g * per_group;
    nt = rem / gm;
    mt = first + rem % gm;
  }
};

// Shared-memory matrix descriptor: K-major tile written by TMA with SWZ-byte rows and
// SWZ-byte swizzle (128 or 64); 8-row groups 8 * SWZ bytes apart.
template <int SWZ>
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);  // start address
  d |= (uint64_t)1 << 16;                    // leading byte offset (unused for these layouts)
  d |= (uint64_t)((8 * SWZ) >> 4) << 32;     // stride byte offset
  d |= (uint64_t)1 << 46;                    // descriptor version
  d |= (uint64_t)(SWZ == 128 ? 2 : 4) << 61; // 128- or 64-byte swizzle
  return d;
}
// sum[0..BN) += the warp's TMEM lanes at columns [col, col + BN), two loads in flight
template <int N>
__device__ __forceinline__ void drain_add(uint32_t col, float* sum) {
#pragma unroll
  for (int c = 0; c < N / 32; c += 2) {
    uint32_t r0[32], r1[32];
    tmem_ld32_nowait(col + (uint32_t)(c * 32), r0);
    tmem_ld32_nowait(col + (uint32_t)((c + 1) * 32), r1);
    tmem_wait_ld();
#pragma unroll
    for (int i = 0; i < 32; ++i) {
      sum[c * 32 + i] += __uint_as_float(r0[i]);
      sum[(c + 1) * 32 + i] += __uint_as_float(r1[i]);
    }
  }
}

// sum[0..N) += the warp's TMEM lanes at columns [col, col + N), 16 columns per load
template <int N>
__device__ __forceinline__ void drain_add16(uint32_t col, float* sum) {
#pragma unroll
  for (int c = 0; c < N / 16; ++c) {
    uint32_t r[16];
    tmem_ld16_nowait(col + (uint32_t)(c * 16), r);
    tmem_wait_ld();
#pragma unroll
    for (int i = 0; i < 16; ++i) sum[c * 16 + i] += __uint_as_float(r[i]);
  }
}

// NPC pieces of the pair (a, b) at element offset off of every piece plane
template <class T, int NPC>
__device__ __forceinline__ void put(void* const* pc, int64_t off, float a, float b) {
  using PT = Piece<T>;
#pragma unroll
  for (int q = 0; q < NPC; ++q) {
    const T ha = PT::rn(a), hb = PT::rn(b);
    *reinterpret_cast<typename PT::T2*>(static_cast<T*>(pc[q]) + off) = PT::pair(ha, hb);
    a -= PT::back(ha);
    b -= PT::back(hb);
  }
}
// The four B-operand rows of vector v at K positions 2i (top entry t = w(i))
// and 2(n+i) (bottom entry b = w(n+i)), scaled by sc (a power of two).
template <class T, int NPC>
__device__ __forceinline__ void store_operand(void* const* pc, int64_t kpad, int64_t n, int64_t v, int64_t i,
                                              float2 t, float2 b, float sc) {
  t.x *= sc; t.y *= sc; b.x *= sc; b.y *= sc;
  const int64_t r0 = (4 * v) * kpad, r1 = r0 + kpad, r2 = r1 + kpad, r3 = r2 + kpad;
  const int64_t pt = 2 * i, pb = 2 * (n + i);
  put<T, NPC>(pc, r0 + pt, t.x, -t.y);
  put<T, NPC>(pc, r0 + pb, b.x, -b.y);
  put<T, NPC>(pc, r1 + pt, t.y, t.x);
  put<T, NPC>(pc, r1 + pb, b.y, b.x);
  put<T, NPC>(pc, r2 + pt, b.x, b.y);   // u(i) = conj(b)
  put<T, NPC>(pc, r2 + pb, t.x, t.y);   // u(n+i) = conj(t)
  put<T, NPC>(pc, r3 + pt, -b.y, b.x);
  put<T, NPC>(pc, r3 + pb, -t.y, t.x);
}

struct Maps {
  CUtensorMap a[3];
  CUtensorMap b[3];
};

// One K range of one 128 x BNT output tile per CTA.  Every K block's products
// accumulate in one of two TMEM buffers that alternate every FLUSH K blocks; the drain
// warps add each finished buffer into FP32 registers (round to nearest) while the MMA
// fills the other one, so the tensor core's truncating accumulator only ever sums a
// few MMAs.  With 128-wide tiles the cross products (2^-8 or 2^-11 smaller)
// accumulate over the whole K range in two further buffers instead.  The last column tile
// may be narrower (n_last columns, a multiple of 16): its MMAs use N = n_last.
template <int SCH, int BNT, int FL>
__global__ void __launch_bounds__(Geo<SCH, BNT, FL>::THREADS, 1)
    tc_hop_kernel(const __grid_constant__ Maps maps, Epi ep, Sched sc) {
  using SC = Scheme<SCH>;
  using G = Geo<SCH, BNT, FL>;
  constexpr int NB = G::NB;
  using T = typename SC::T;
  constexpr int ST = G::STAGES;
  constexpr int DC = G::DCOLS;
  constexpr int FLUSH = G::FLUSH;
  constexpr int BK = G::BK;
  constexpr int A_BYTES = G::A_BYTES;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + ST * G::STAGE_BYTES);
  uint32_t full[ST], empty[ST];
#pragma unroll
  for (int s = 0; s < ST; ++s) {
    full[s] = smem_u32(bars + s);
    empty[s] = smem_u32(bars + ST + s);
  }
  uint32_t accf[NB], acce[NB];
#pragma unroll
  for (int b = 0; b < NB; ++b) {
    accf[b] = smem_u32(bars + 2 * ST + b);
    acce[b] = smem_u32(bars + 2 * ST + NB + b);
  }
  const uint32_t done = smem_u32(bars + 2 * ST + 2 * NB);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + G::NBAR);
  volatile int* abort_sh = reinterpret_cast<volatile int*>(tmem_slot + 1);
  int* issued_sh = reinterpret_cast<int*>(tmem_slot + 2);
  volatile int* last_sh = reinterpret_cast<volatile int*>(tmem_slot + 3);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  int mt, nt, sp;
  sc.unit(blockIdx.x, mt, nt, sp);
  const int tile = mt * sc.num_n + nt;
  const int m0 = mt * BM, n0 = nt * BNT;
  const int ntile = (nt == sc.num_n - 1) ? sc.n_last : BNT;  // columns of this tile (multiple of 16)
  const int kb0 = (int)((int64_t)sc.nkb * sp / sc.nsplit), kb1 = (int)((int64_t)sc.nkb * (sp + 1) / sc.nsplit);
  const int num_kb = kb1 - kb0;

  if (threadIdx.x == 0) {
    for (int s = 0; s < ST; ++s) {
      mbar_init(full[s], 1);
      mbar_init(empty[s], 1);
    }
    for (int b = 0; b < NB; ++b) {
      mbar_init(accf[b], 1);
      mbar_init(acce[b], G::DRAIN_WARPS);  // one arrival per drain warp
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
    for (int kb = 0; kb < num_kb; ++kb) {
      const int s = kb % ST;
      const uint32_t ph = (uint32_t)(kb / ST) & 1u;
      if (kb >= ST && !mbar_wait(empty[s], ph ^ 1u, abort_sh, ep.err, true)) break;
      const uint32_t st = sbase + s * G::STAGE_BYTES;
      mbar_expect_tx(full[s], G::STAGE_BYTES);
#pragma unroll
      for (int q = 0; q < SC::NPA; ++q) tma_load_2d(st + q * A_BYTES, &maps.a[q], (kb0 + kb) * BK, m0, full[s]);
#pragma unroll
      for (int q = 0; q < SC::NPW; ++q)
        tma_load_2d(st + SC::NPA * A_BYTES + q * G::B_BYTES, &maps.b[q], (kb0 + kb) * BK, n0, full[s]);
      issued = kb + 1;
    }
    *issued_sh = issued;
  } else if (warp == 1 && lane == 0) {
    const uint32_t idesc = make_idesc(ntile, Piece<T>::BF16);
    const uint32_t small = tmem + (uint32_t)(NB * BNT);
    const uint64_t dbase = sdesc<G::SWZ>(sbase);
    for (int kb = 0; kb < num_kb; ++kb) {
      const int grp = kb / FLUSH, b = grp % NB;
      const bool first = (kb % FLUSH) == 0;
      const bool last = (kb % FLUSH) == FLUSH - 1 || kb == num_kb - 1;
      if (first && grp >= NB && !mbar_wait(acce[b], (uint32_t)(grp / NB - 1) & 1u, abort_sh, ep.err, true)) break;
      const int s = kb % ST;
      const uint32_t ph = (uint32_t)(kb / ST) & 1u;
      if (!mbar_wait(full[s], ph, abort_sh, ep.err, true)) break;
      tc_fence_after();
      const uint32_t st = sbase + s * G::STAGE_BYTES;
      const uint32_t big = tmem + (uint32_t)(b * BNT);
      // sdesc is linear in the address here (its 14-bit start field holds address / 16 of
      // a 1024-aligned ring below 256 KB and cannot carry): a hoisted base plus constants;
      // 16 K elements further along a swizzled row is 32 bytes further
      const uint64_t sd = dbase + (uint64_t)((uint32_t)(st - sbase) >> 4);
      if (G::CROSS) {
#pragma unroll
        for (int kk = 0; kk < BK / 16; ++kk) {
#pragma unroll
          for (int pr = 0; pr < SC::NPROD; ++pr) {
            const uint64_t ad = sd + (uint64_t)((SC::pa(pr) * A_BYTES + kk * 32) >> 4);
            const uint64_t bd = sd + (uint64_t)((SC::NPA * A_BYTES + SC::pb(pr) * G::B_BYTES + kk * 32) >> 4);
            // products 1, 3, 5 into the first cross buffer, 2, 4 into the second; each
            // buffer's first MMA (products 1 and 2 of the first K step) overwrites
            const uint32_t acc =
                (pr == 0) ? ((!first || kk > 0) ? 1u : 0u) : ((kb > 0 || kk > 0 || pr > 2) ? 1u : 0u);
            mma_bf16(pr == 0 ? big : ((pr & 1) ? small : small + (uint32_t)BNT), ad, bd, idesc, acc);
          }
        }
      } else {
        // the block's cross products first, then x0 * y0
#pragma unroll
        for (int pi = 0; pi < SC::NPROD; ++pi) {
          const int pr = (pi + 1) % SC::NPROD;
#pragma unroll
          for (int kk = 0; kk < BK / 16; ++kk) {
            const uint64_t ad = sd + (uint64_t)((SC::pa(pr) * A_BYTES + kk * 32) >> 4);
            const uint64_t bd = sd + (uint64_t)((SC::NPA * A_BYTES + SC::pb(pr) * G::B_BYTES + kk * 32) >> 4);
            const uint32_t acc = (first && kk == 0 && pi == 0) ? 0u : 1u;
            mma_bf16(big, ad, bd, idesc, acc);
          }
        }
      }
      mma_commit(empty[s]);
      if (last) mma_commit(accf[b]);
    }
    mma_commit(done);  // completes once every MMA issued above has finished
  } else if (warp >= 4) {
    const int dw = warp - 4;
    const int q = warp & 3;                  // TMEM lanes 32 q .. 32 q + 31 (rows of the tile)
    const int col0 = (dw >> 2) * DC;         // this warp's columns [col0, col0 + DC)
    const uint32_t lane_base = (uint32_t)(q * 32) << 16;
    const bool has_cols = col0 < ntile;
    float sum[DC];
#pragma unroll
    for (int i = 0; i < DC; ++i) sum[i] = 0.0f;
    bool ok = true;
    const int ngrp = (num_kb + FLUSH - 1) / FLUSH;
    for (int grp = 0; grp < ngrp; ++grp) {
      const int b = grp % NB;
      const bool w = mbar_wait(accf[b], (uint32_t)(grp / NB) & 1u, abort_sh, ep.err, true);
      if (!__all_sync(0xffffffffu, w)) {  // warp-uniform (tcgen05.ld is .sync.aligned)
        ok = false;
        break;
      }
      tc_fence_after();
      if (has_cols) {
        if (G::CROSS) drain_add<DC>(tmem + lane_base + (uint32_t)(b * BNT + col0), sum);
        else drain_add16<DC>(tmem + lane_base + (uint32_t)(b * BNT + col0), sum);
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(acce[b]);
    }
    if (G::CROSS && ok) {  // the cross products, once every MMA has completed
      const bool w = mbar_wait(done, 0, abort_sh, ep.err, true);
      ok = __all_sync(0xffffffffu, w);
      if (ok && has_cols) {
        tc_fence_after();
        drain_add<DC>(tmem + lane_base + (uint32_t)(NB * BNT + col0), sum);
        drain_add<DC>(tmem + lane_base + (uint32_t)((NB + 1) * BNT + col0), sum);
      }
    }
    if (sc.nsplit > 1) {
      // split tile: write this K range's partial; the last writer sums them all.  Every
      // drain warp passes both named barriers, also after a failed wait.
      constexpr int DRAIN_THREADS = 32 * G::DRAIN_WARPS;
      const int row_t = q * 32 + lane;
      float* mine = ep.part + (size_t)(sp * sc.ntiles + tile) * (BM * BNT);
      if (ok && has_cols) {
#pragma unroll
        for (int c = 0; c < DC; ++c) mine[(size_t)(col0 + c) * BM + row_t] = sum[c];
      }
      __threadfence();
      asm volatile("bar.sync 1, %0;" ::"r"(DRAIN_THREADS) : "memory");
      if (dw == 0 && lane == 0) *last_sh = (atomicAdd(ep.cnt + tile, 1) == sc.nsplit - 1) ? 1 : 0;
      asm volatile("bar.sync 1, %0;" ::"r"(DRAIN_THREADS) : "memory");
      if (*last_sh) {
        __threadfence();
        if (ok && has_cols) {
#pragma unroll
          for (int c = 0; c < DC; ++c) sum[c] = 0.0f;
          for (int j = 0; j < sc.nsplit; ++j) {
            const float* pp = ep.part + (size_t)(j * sc.ntiles + tile) * (BM * BNT) + (size_t)col0 * BM + row_t;
#pragma unroll
            for (int c = 0; c < DC; ++c) sum[c] += __ldcg(pp + (size_t)c * BM);
          }
        }
        if (dw == 0 && lane == 0) ep.cnt[tile] = 0;  // ready for the next launch
      } else {
        ok = false;  // another CTA finishes this tile
      }
    }
    const int64_t row = (int64_t)m0 + q * 32 + lane;
    const bool rvalid = row < ep.n;
    const bool go = ok && has_cols && __all_sync(0xffffffffu, *abort_sh == 0);  // warp-uniform
    if (go) {
      const int64_t n = ep.n, n2 = 2 * ep.n;
      const float rs = rvalid ? exp2i(-ep.prow[row]) : 0.0f;  // undo the row scaling of P
#pragma unroll
      for (int c = 0; c < DC / 32; ++c) {
#pragma unroll
        for (int t = 0; t < 8; ++t) {
          const int64_t vg = (int64_t)((n0 + col0) >> 2) + c * 8 + t;
          if (vg >= ep.k) continue;  // uniform over the warp
          const float* v = sum + c * 32;
          const float vs = exp2i(-ep.vexp_in[vg]);  // and the scaling of the input vector
          const float2 ht = make_float2(v[4 * t] * rs * vs, v[4 * t + 1] * rs * vs);        // (H x)_top(row)
          // (H x)_bot(row) = -conj(P u); with the blocks of H^2, +conj(P u)
          const float2 hb = ep.h2 ? make_float2(v[4 * t + 2] * rs * vs, -v[4 * t + 3] * rs * vs)
                                  : make_float2(-v[4 * t + 2] * rs * vs, v[4 * t + 3] * rs * vs);
          const int64_t ot = vg * n2 + row, ob = ot + n;
          float2 zt = ht, zb = hb;
          if (ep.mode == 1 && rvalid) {
            const float2 ct = ep.Zcur[ot], cbv = ep.Zcur[ob];
            zt = make_float2(ep.alpha * (ht.x - ep.c * ct.x), ep.alpha * (ht.y - ep.c * ct.y));
            zb = make_float2(ep.alpha * (hb.x - ep.c * cbv.x), ep.alpha * (hb.y - ep.c * cbv.y));
            if (ep.beta != 0.0f) {
              const float2 pt = ep.Zprev[ot], pb = ep.Zprev[ob];
              zt.x += ep.beta * pt.x; zt.y += ep.beta * pt.y;
              zb.x += ep.beta * pb.x; zb.y += ep.beta * pb.y;
            }
            if (ep.src) {
              const float gmm = ep.gamma[vg];
              const float2 st = ep.src[ot], sb = ep.src[ob];
              zt.x += gmm * st.x; zt.y += gmm * st.y;
              zb.x += gmm * sb.x; zb.y += gmm * sb.y;
            }
          } else if (ep.mode == 2 && rvalid) {
            const float gmm = ep.gamma[vg];
            const float2 ct = ep.Zcur[ot], cbv = ep.Zcur[ob];
            zt = make_float2(ht.x + gmm * ct.x, ht.y + gmm * ct.y);
            zb = make_float2(hb.x + gmm * cbv.x, hb.y + gmm * cbv.y);
          }
          if (ep.mode != 0 && rvalid) {
            ep.Znext[ot] = zt;
            ep.Znext[ob] = zb;
          }
          if (ep.mode != 2) {
            const int e = out_exp(vec_bound(ep, vg));
            if (rvalid) store_operand<T, SC::NPW>(ep.out, ep.kpad, n, vg, row, zt, zb, exp2i(e));
            if (lane == 0) ep.vexp_out[vg] = e;  // the same value from every tile
          }
          const float m = rvalid ? fmaxf(fmaxf(fabsf(zt.x), fabsf(zt.y)), fmaxf(fabsf(zb.x), fabsf(zb.y))) : 0.0f;
          const unsigned mm = __reduce_max_sync(0xffffffffu, __float_as_uint(m));
          if (lane == 0) atomicMax(reinterpret_cast<unsigned*>(ep.amax_out) + vg, mm);
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (threadIdx.x == 0 && *abort_sh) {
    // drain copies still in flight into this CTA's shared memory (bounded)
    const int issued = *issued_sh;
    for (int kb = max(0, issued - ST); kb < issued; ++kb)
      mbar_wait(full[kb % ST], (uint32_t)(kb / ST) & 1u, abort_sh, ep.err, false);
  }
  if (warp == 1) {
    // every MMA has finished before the accumulator memory is released
    if (lane == 0) mbar_wait(done, 0, abort_sh, ep.err, false);
    __syncwarp();
  }
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
  }
}

// ---------------------------------------------------------------- helpers
struct Pieces {
  void* p[3];
};

// block-wide max and sum of one value per thread (blockDim.x a multiple of 32, <= 1024)
__device__ __forceinline__ void block_max_sum(float& m, float& s) {
  __shared__ float wm[32], ws[32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    s += __shfl_xor_sync(0xffffffffu, s, o);
  }
  if (lane == 0) {
    wm[w] = m;
    ws[w] = s;
  }
  __syncthreads();
  if (w == 0) {
    m = lane < nw ? wm[lane] : 0.0f;
    s = lane < nw ? ws[lane] : 0.0f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
      s += __shfl_xor_sync(0xffffffffu, s, o);
    }
    if (lane == 0) {
      wm[0] = m;
      ws[0] = s;
    }
  }
  __syncthreads();
  m = wm[0];
  s = ws[0];
}

// P = [A | B] (row-major complex128) -> NPC pieces, one CTA per row i, K = (re, im)
// pairs, scaled by 2^prow[i] (largest entry of the row in [2^12, 2^13)); L receives the
// largest row sum of |Re| + |Im| (unscaled), the bound factor of an H application.
template <class T, int NPC>
__global__ void split_p_kernel(const cplx* A, const cplx* B, int64_t n, int64_t kpad, Pieces out, int* prow,
                               float* L) {
  const int64_t i = blockIdx.x;
  float m = 0.0f, sum = 0.0f;
  for (int64_t l = threadIdx.x; l < 2 * n; l += blockDim.x) {
    const cplx p = (l < n) ? A[i * n + l] : B[i * n + (l - n)];
    const float x = fabsf((float)p.x), y = fabsf((float)p.y);
    m = fmaxf(m, fmaxf(x, y));
    sum += x + y;
  }
  block_max_sum(m, sum);
  const int e = out_exp(m);
  if (threadIdx.x == 0) {
    prow[i] = e;
    atomicMax(reinterpret_cast<unsigned*>(L), __float_as_uint(sum));
  }
  const float sc = exp2i(e);
  for (int64_t l = threadIdx.x; l < 2 * n; l += blockDim.x) {
    const cplx p = (l < n) ? A[i * n + l] : B[i * n + (l - n)];
    put<T, NPC>(out.p, i * kpad + 2 * l, (float)p.x * sc, (float)p.y * sc);
  }
}
// amax[v] = largest |Re|, |Im| of column v of the complex128 block W (2n x k), rounded to
// FP32, and vexp[v] its operand exponent; one CTA per column
__global__ void col_amax_kernel(const cplx* W, int64_t n2, float* amax, int* vexp) {
  const int64_t v = blockIdx.x;
  float m = 0.0f, unused = 0.0f;
  for (int64_t i = threadIdx.x; i < n2; i += blockDim.x) {
    const cplx w = W[v * n2 + i];
    m = fmaxf(m, fmaxf(fabsf((float)w.x), fabsf((float)w.y)));
  }
  block_max_sum(m, unused);
  if (threadIdx.x == 0) {
    amax[v] = m;
    vexp[v] = out_exp(m);
  }
}
// complex128 block (2n x k) -> FP32 master and, optionally, operand pieces (exponents vexp)
template <class T, int NPC>
__global__ void pack_kernel(const cplx* W, int64_t n, int64_t k, float2* Z, Pieces out, int with_pieces,
                            int64_t kpad, const int* vexp) {
  const int64_t total = n * k;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = idx % n, v = idx / n;
    const cplx wt = W[v * 2 * n + i], wb = W[v * 2 * n + n + i];
    const float2 t = make_float2((float)wt.x, (float)wt.y);
    const float2 b = make_float2((float)wb.x, (float)wb.y);
    if (Z) {
      Z[v * 2 * n + i] = t;
      Z[v * 2 * n + n + i] = b;
    }
    if (with_pieces) store_operand<T, NPC>(out.p, kpad, n, v, i, t, b, exp2i(vexp[v]));
  }
}
// Z = scale * X (FP32 master) and its operand pieces; the largest component of column v
// is |scale| amax_x[v] (up to rounding), which sets its exponent
template <class T, int NPC>
__global__ void scale_pack_kernel(const float2* X, int64_t n, int64_t k, float scale, float2* Z, Pieces out,
                                  int64_t kpad, const float* amax_x, float* amax_z, int* vexp_z) {
  const int64_t total = n * k;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = idx % n, v = idx / n;
    const float am = fabsf(scale) * amax_x[v];
    const int e = out_exp(am);
    if (i == 0) {
      amax_z[v] = am;
      vexp_z[v] = e;
    }
    const float2 xt = X[v * 2 * n + i], xb = X[v * 2 * n + n + i];
    const float2 t = make_float2(scale * xt.x, scale * xt.y), b = make_float2(scale * xb.x, scale * xb.y);
    Z[v * 2 * n + i] = t;
    Z[v * 2 * n + n + i] = b;
    store_operand<T, NPC>(out.p, kpad, n, v, i, t, b, exp2i(e));
  }
}
// out[:, v] = (double) Zsel[:, v] + coef[v] * base[:, v]   (coef/base optional)
__global__ void combine_kernel(cplx* out, const float2* Z0, const float2* Z1, const float2* Z2, const int* sel,
                               const double* coef, const cplx* base, int64_t n2, int64_t k) {
  const int64_t total = n2 * k;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t v = idx / n2;
    const int q = sel[v];
    const float2 z = (q == 0 ? Z0 : (q == 1 ? Z1 : Z2))[idx];
    cplx r = mk((double)z.x, (double)z.y);
    if (coef) r = cadd(r, cscale(base[idx], coef[v]));
    out[idx] = r;
  }
}

// Tensor map of a piece plane (rows x kpad, K contiguous) with boxes of bk x box_rows and
// 2 bk-byte swizzle (bk = 64 or 32).
static int make_map(CUtensorMap* m, const void* base, int64_t kpad, int64_t rows, int box_rows, bool bf16,
                    int bk) {
  auto fn = encode_fn();
  if (!fn) return CHASE_BSE_UNSUPPORTED;
  const cuuint64_t dims[2] = {(cuuint64_t)kpad, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)kpad * 2};
  const cuuint32_t box[2] = {(cuuint32_t)bk, (cuuint32_t)box_rows};
  const cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(m, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2,
                  const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  bk == 64 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? CHASE_BSE_OK : CHASE_BSE_CUDA_ERROR;
}

static inline unsigned gsz(int64_t total) {
  const int64_t b = (total + 255) / 256;
  return (unsigned)std::min<int64_t>(std::max<int64_t>(b, 1), 16384);
}

// The operand of P = [A | B] in NPA pieces, with its tensor maps, row exponents and
// the bound factor L (device scalar).
struct POperand {
  int64_t n = 0, kpad = 0;
  Pieces pc{};
  CUtensorMap map[3];
  int* prow = nullptr;
  float* L = nullptr;
};

template <int SCH, int BNT>
static int prepare_p(const cplx* A, const cplx* B, int64_t n, Workspace& ws, POperand& P, cudaStream_t s) {
  using T = typename Scheme<SCH>::T;
  constexpr int NPA = Scheme<SCH>::NPA;
  P.n = n;
  constexpr int BK = Geo<SCH, BNT, 1>::BK;
  P.kpad = ((4 * n + KPAD - 1) / KPAD) * KPAD;
  const int64_t rows = ((n + BM - 1) / BM) * BM;  // whole tiles: every TMA box lies inside the tensor
  for (int q = 0; q < NPA; ++q) {
    T* pq;
    CB_TRY(ws.alloc(&pq, rows * P.kpad));
    P.pc.p[q] = pq;
    CB_CUDA(cudaMemsetAsync(pq, 0, sizeof(T) * rows * P.kpad, s));
  }
  CB_TRY(ws.alloc(&P.prow, n));
  CB_TRY(ws.alloc(&P.L, 1));
  CB_CUDA(cudaMemsetAsync(P.L, 0, sizeof(float), s));
  split_p_kernel<T, NPA><<<(unsigned)n, 256, 0, s>>>(A, B, n, P.kpad, P.pc, P.prow, P.L);
  count_launch();
  CB_LAUNCH();
  for (int q = 0; q < NPA; ++q) CB_TRY(make_map(&P.map[q], P.pc.p[q], P.kpad, rows, BM, Piece<T>::BF16, BK));
  return CHASE_BSE_OK;
}

// K splits of a launch with `tiles` CTAs per split: the count (1 to MAX_SPLIT) that
// minimises the estimated time, waves of CTAs x (1/splits + a fixed cost per CTA of
// 5 % of a tile), with at least two drained groups of K blocks per split and at most
// MAX_SPLIT x SMs CTAs (the partial-tile workspace).
constexpr int MAX_SPLIT = 4;
static int split_count(int tiles, int nkb, int sms, int flush) {
  int best = 1;
  double best_t = 0.0;
  for (int sp = 1; sp <= MAX_SPLIT; ++sp) {
    if (sp > 1 && (nkb / sp < 2 * flush || (int64_t)tiles * sp > (int64_t)MAX_SPLIT * sms)) break;
    const double waves = (double)((tiles * sp + sms - 1) / sms);
    const double t = waves * (1.0 / sp + 0.05);
    if (sp == 1 || t < best_t - 1e-9) {
      best = sp;
      best_t = t;
    }
  }
  return best;
}

// One tensor-core application of H to the vectors held in the operand pieces
// described by bmap, with epilogue `ep`.
template <int SCH, int BNT, int FL>
static int apply(const POperand& P, const CUtensorMap* bmap, Epi ep, cudaStream_t s) {
  using G = Geo<SCH, BNT, FL>;
  if (ep.k <= 0) return CHASE_BSE_OK;
  static bool attr = false;
  if (!attr) {
    CB_CUDA(cudaFuncSetAttribute(tc_hop_kernel<SCH, BNT, FL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 G::SMEM_BYTES));
    attr = true;
  }
  Maps maps;
  for (int q = 0; q < Scheme<SCH>::NPA; ++q) maps.a[q] = P.map[q];
  for (int q = 0; q < Scheme<SCH>::NPW; ++q) maps.b[q] = bmap[q];
  ep.prow = P.prow;
  Sched sc{};
  sc.num_m = (int)cdiv(P.n, BM);
  sc.num_n = (int)cdiv(4 * ep.k, BNT);
  const int64_t rest = 4 * ep.k - (int64_t)(sc.num_n - 1) * BNT;  // columns of the last tile
  sc.n_last = (int)(((rest + 15) / 16) * 16);
  sc.nkb = (int)(P.kpad / G::BK);
  sc.bnt = BNT;
  sc.ntiles = sc.num_m * sc.num_n;
  sc.nsplit = split_count(sc.ntiles, sc.nkb, ep.sms, G::FLUSH);
  // 8 row tiles per raster group: of 4, 8, 12 and 16 the least DRAM traffic at n = 16384,
  // k = 1300 (40 GB per launch against 41-59), with the same duration
  sc.group_m = 8;
  const int64_t tid = timer_begin(0, 32.0 * (double)P.n * (double)P.n * (double)ep.k, s);
  tc_hop_kernel<SCH, BNT, FL><<<(unsigned)(sc.ntiles * sc.nsplit), G::THREADS, G::SMEM_BYTES, s>>>(maps, ep, sc);
  timer_end(tid, s);
  count_launch();
  CB_LAUNCH();
  return CHASE_BSE_OK;
}

// Mixed-precision filter on columns sorted by descending degree.  If `ritz` and
// `R` are given, the filter runs in correction form: with m_i = ritz_i^2 and
// r2_i = (H^2 - m_i) v_i = (H + ritz_i)(H v_i - ritz_i v_i),
//   p(H^2) v_i = p(m_i) v_i + q(H^2) r2_i,  q(x) = (p(x) - p(m_i)) / (x - m_i),
// and only q(H^2) r2 runs on the tensor cores; its recurrence is the filter's
// with the source term alpha_j p_j(m_i) r2_i (divided differences of the
// three-term recurrence).  The low-precision error then scales with the
// residual of v_i instead of with v_i.
//
// With P2, Q2 (the blocks of H^2 = [[P2, Q2], [conj Q2, conj P2]], row-major n x n) the
// filter applies H^2 from its blocks, one launch per step (the explicit-H^2 variant, not
// the paper's method); H itself (A, B) is then used only for the correction source.
template <int SCH, int BNT, int FL>
static int filter_impl(const cplx* A, const cplx* B, int64_t n, const cplx* Y0, int64_t k, const int* degs,
                       double mu1, double mu_nevex, double muN, cplx* out, const double* ritz, const cplx* R,
                       cudaStream_t s, FilterStats* fs, const cplx* P2, const cplx* Q2) {
  using T = typename Scheme<SCH>::T;
  constexpr int NPW = Scheme<SCH>::NPW;
  constexpr bool BF = Piece<T>::BF16;
  if (k == 0) return CHASE_BSE_OK;
  const int64_t n2 = 2 * n;
  const bool expl = P2 != nullptr && Q2 != nullptr;
  const bool corr = (ritz != nullptr && R != nullptr);
  Workspace ws(s);
  POperand P, PH2;  // [A | B] (H), [P2 | Q2] (H^2)
  if (!expl || corr) CB_TRY((prepare_p<SCH, BNT>(A, B, n, ws, P, s)));
  if (expl) CB_TRY((prepare_p<SCH, BNT>(P2, Q2, n, ws, PH2, s)));
  const POperand& PK = expl ? PH2 : P;  // the operand of the recurrence (its kpad and pieces layout)
  const int64_t kpad = PK.kpad;  // the same for both operands (4n padded)
  const int64_t rows = ((4 * k + BNT - 1) / BNT) * BNT;  // whole tiles
  Pieces Zp{}, Tp{};
  CUtensorMap mZ[3], mT[3];
  for (int q = 0; q < NPW; ++q) {
    T *zq, *tq;
    CB_TRY(ws.alloc(&zq, rows * kpad));
    CB_TRY(ws.alloc(&tq, rows * kpad));
    Zp.p[q] = zq;
    Tp.p[q] = tq;
    CB_CUDA(cudaMemsetAsync(zq, 0, sizeof(T) * rows * kpad, s));
    CB_CUDA(cudaMemsetAsync(tq, 0, sizeof(T) * rows * kpad, s));
    CB_TRY(make_map(&mZ[q], zq, kpad, rows, BNT, BF, Geo<SCH, BNT, FL>::BK));
    CB_TRY(make_map(&mT[q], tq, kpad, rows, BNT, BF, Geo<SCH, BNT, FL>::BK));
  }
  // explicit H^2: the pieces of Z_j alternate between the two sets (j even: Zp)
  Pieces* zbuf[2] = {&Zp, &Tp};
  const CUtensorMap* zmap[2] = {mZ, mT};
  float2 *Zb[3], *src = nullptr;
  float* gam;
  int* err;
  for (int q = 0; q < 3; ++q) CB_TRY(ws.alloc(&Zb[q], n2 * k));
  CB_TRY(ws.alloc(&gam, k));
  CB_TRY(ws.alloc(&err, 1));
  CB_CUDA(cudaMemsetAsync(err, 0, sizeof(int), s));
  // split-K workspace: a partial tile per CTA of a split launch (fewer than
  // MAX_SPLIT x SMs of them), one counter per tile
  int dev = 0, sms = 0;
  CB_CUDA(cudaGetDevice(&dev));
  CB_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int64_t max_tiles = cdiv(n, BM) * (rows / BNT);
  float* part;
  int* cnt;
  CB_TRY(ws.alloc(&part, (int64_t)MAX_SPLIT * sms * BM * BNT));
  CB_TRY(ws.alloc(&cnt, max_tiles));
  CB_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int) * max_tiles, s));
  auto sk = [&](Epi& e) {
    e.part = part;
    e.cnt = cnt;
    e.sms = sms;
  };

  const double a = mu_nevex * mu_nevex, b = muN * muN;
  const double c = 0.5 * (a + b), e = 0.5 * (b - a);
  const double sigma1 = e / (mu1 * mu1 - c);
  const double tau = 2.0 / sigma1;
  const int maxdeg = degs[0];
  // per-vector maxima and operand exponents, one slot of k entries per vector block:
  // Z_j (j = 0 .. maxdeg), T_j = H Z_j (j < maxdeg), the residual block R and the
  // correction source r2
  const int64_t nslot = 2 * (int64_t)maxdeg + 3;
  float* amax;
  int* vexp;
  CB_TRY(ws.alloc(&amax, nslot * k));
  CB_TRY(ws.alloc(&vexp, nslot * k));
  CB_CUDA(cudaMemsetAsync(amax, 0, sizeof(float) * nslot * k, s));
  CB_CUDA(cudaMemsetAsync(vexp, 0, sizeof(int) * nslot * k, s));
  auto slotZ = [&](int j) { return (int64_t)j * k; };
  auto slotT = [&](int j) { return (int64_t)(maxdeg + 1 + j) * k; };
  const int64_t slotR = (int64_t)(2 * maxdeg + 1) * k, slotS = (int64_t)(2 * maxdeg + 2) * k;
  float L = 0.0f, L2 = 0.0f;  // largest absolute row sums of [A | B] and [P2 | Q2]
  if (!expl || corr) CB_CUDA(cudaMemcpyAsync(&L, P.L, sizeof(float), cudaMemcpyDeviceToHost, s));
  if (expl) CB_CUDA(cudaMemcpyAsync(&L2, PH2.L, sizeof(float), cudaMemcpyDeviceToHost, s));
  CB_CUDA(cudaStreamSynchronize(s));

  std::vector<double> al(maxdeg), be(maxdeg);  // alpha_j, beta_j of the scaled recurrence
  {
    double sigma = sigma1;
    al[0] = sigma1 / e;
    be[0] = 0.0;
    for (int j = 1; j < maxdeg; ++j) {
      const double sn = 1.0 / (tau - sigma);
      al[j] = 2.0 * sn / e;
      be[j] = -sigma * sn;
      sigma = sn;
    }
  }
  std::vector<double> pj;  // p_j(m_i), j = 0 .. maxdeg
  if (corr) {
    pj.assign((size_t)(maxdeg + 1) * k, 0.0);
    for (int64_t i = 0; i < k; ++i) {
      const double m = ritz[i] * ritz[i];
      double p0 = 1.0, p1 = al[0] * (m - c);
      pj[i] = p0;
      pj[(size_t)k + i] = p1;
      for (int j = 1; j < maxdeg; ++j) {
        const double p2 = al[j] * (m - c) * p1 + be[j] * p0;
        pj[(size_t)(j + 1) * k + i] = p2;
        p0 = p1;
        p1 = p2;
      }
    }
  }
  std::vector<float> gh(k);
  int j0 = 0;
  cudaEvent_t e0, e1;
  CB_CUDA(cudaEventCreate(&e0));
  CB_CUDA(cudaEventCreate(&e1));
  CB_CUDA(cudaEventRecord(e0, s));
  if (!corr) {
    col_amax_kernel<<<(unsigned)k, 256, 0, s>>>(Y0, n2, amax + slotZ(0), vexp + slotZ(0));
    count_launch();
    pack_kernel<T, NPW><<<gsz(n * k), 256, 0, s>>>(Y0, n, k, Zb[0], Zp, 1, kpad, vexp + slotZ(0));  // Z_0 = W
    count_launch();
    CB_LAUNCH();
  } else {
    // r2 = H R + ritz R on the tensor cores; Z_0 = 0; Z_1 = alpha_0 r2
    CB_TRY(ws.alloc(&src, n2 * k));
    col_amax_kernel<<<(unsigned)k, 256, 0, s>>>(R, n2, amax + slotR, vexp + slotR);
    count_launch();
    pack_kernel<T, NPW><<<gsz(n * k), 256, 0, s>>>(R, n, k, Zb[2], Zp, 1, kpad, vexp + slotR);
    count_launch();
    for (int64_t i = 0; i < k; ++i) gh[i] = (float)ritz[i];
    CB_CUDA(cudaMemcpyAsync(gam, gh.data(), sizeof(float) * k, cudaMemcpyHostToDevice, s));
    Epi ep{};
    ep.mode = 2; ep.n = n; ep.k = k; ep.kpad = kpad; ep.Znext = src; ep.Zcur = Zb[2]; ep.gamma = gam; ep.err = err;
    ep.vexp_in = vexp + slotR;
    ep.amax_out = amax + slotS;
    sk(ep);
    CB_TRY((apply<SCH, BNT, FL>)(P, mZ, ep, s));
    CB_CUDA(cudaMemsetAsync(Zb[0], 0, sizeof(float2) * n2 * k, s));
    scale_pack_kernel<T, NPW><<<gsz(n * k), 256, 0, s>>>(src, n, k, (float)al[0], Zb[1], expl ? Tp : Zp, kpad,
                                                          amax + slotS, amax + slotZ(1), vexp + slotZ(1));
    count_launch();
    CB_LAUNCH();
    j0 = 1;
    if (fs) {
      fs->flops += 32.0 * (double)n * (double)n * (double)k;
      fs->launches += 1;
    }
  }
  for (int j = j0; j < maxdeg && expl; ++j) {
    // Z_{j+1} = alpha (H^2 Z_j - c Z_j) + beta Z_{j-1} (+ source): one launch on [P2 | Q2]
    int64_t kj = 0;
    while (kj < k && degs[kj] >= j + 1) ++kj;
    Epi ep{};
    ep.mode = 1; ep.h2 = 1; ep.n = n; ep.k = kj; ep.kpad = kpad; ep.err = err;
    sk(ep);
    for (int q = 0; q < NPW; ++q) ep.out[q] = zbuf[(j + 1) % 2]->p[q];
    ep.Znext = Zb[(j + 1) % 3]; ep.Zcur = Zb[j % 3]; ep.Zprev = Zb[(j + 2) % 3];
    ep.alpha = (float)al[j]; ep.beta = (float)be[j]; ep.c = (float)c;
    ep.vexp_in = vexp + slotZ(j);
    ep.vexp_out = vexp + slotZ(j + 1);
    ep.amax_out = amax + slotZ(j + 1);
    ep.amax_a = amax + slotZ(j);
    ep.amax_b = amax + slotZ(j);
    ep.amax_c = amax + slotZ(j > 0 ? j - 1 : 0);
    ep.ca = (float)(std::fabs(al[j]) * L2);
    ep.cb = (float)std::fabs(al[j] * c);
    ep.cc = (float)std::fabs(be[j]);
    if (corr) {
      for (int64_t i = 0; i < kj; ++i) gh[i] = (float)(al[j] * pj[(size_t)j * k + i]);
      CB_CUDA(cudaMemcpyAsync(gam, gh.data(), sizeof(float) * kj, cudaMemcpyHostToDevice, s));
      ep.src = src;
      ep.gamma = gam;
      ep.amax_d = amax + slotS;
    }
    CB_TRY((apply<SCH, BNT, FL>)(PH2, zmap[j % 2], ep, s));
    if (fs) {
      fs->flops += 32.0 * (double)n * (double)n * (double)kj;  // the product with the blocks of H^2
      fs->launches += 1;
    }
  }
  for (int j = j0; j < maxdeg && !expl; ++j) {
    int64_t kj = 0;
    while (kj < k && degs[kj] >= j + 1) ++kj;
    Epi e1p{};
    e1p.mode = 0; e1p.n = n; e1p.k = kj; e1p.kpad = P.kpad; e1p.err = err;
    sk(e1p);
    for (int q = 0; q < NPW; ++q) e1p.out[q] = Tp.p[q];
    e1p.vexp_in = vexp + slotZ(j);
    e1p.vexp_out = vexp + slotT(j);
    e1p.amax_out = amax + slotT(j);
    e1p.amax_a = amax + slotZ(j);
    e1p.ca = L;
    CB_TRY((apply<SCH, BNT, FL>)(P, mZ, e1p, s));  // T = H Z_j
    Epi e2p{};
    e2p.mode = 1; e2p.n = n; e2p.k = kj; e2p.kpad = P.kpad; e2p.err = err;
    sk(e2p);
    for (int q = 0; q < NPW; ++q) e2p.out[q] = Zp.p[q];
    e2p.Znext = Zb[(j + 1) % 3]; e2p.Zcur = Zb[j % 3]; e2p.Zprev = Zb[(j + 2) % 3];
    e2p.alpha = (float)al[j]; e2p.beta = (float)be[j]; e2p.c = (float)c;
    e2p.vexp_in = vexp + slotT(j);
    e2p.vexp_out = vexp + slotZ(j + 1);
    e2p.amax_out = amax + slotZ(j + 1);
    e2p.amax_a = amax + slotT(j);
    e2p.amax_b = amax + slotZ(j);
    e2p.amax_c = amax + slotZ(j > 0 ? j - 1 : 0);
    e2p.ca = (float)(std::fabs(al[j]) * L);
    e2p.cb = (float)std::fabs(al[j] * c);
    e2p.cc = (float)std::fabs(be[j]);
    if (corr) {
      for (int64_t i = 0; i < kj; ++i) gh[i] = (float)(al[j] * pj[(size_t)j * k + i]);
      CB_CUDA(cudaMemcpyAsync(gam, gh.data(), sizeof(float) * kj, cudaMemcpyHostToDevice, s));
      e2p.src = src;
      e2p.gamma = gam;
      e2p.amax_d = amax + slotS;
    }
    CB_TRY((apply<SCH, BNT, FL>)(P, mT, e2p, s));  // Z_{j+1} = alpha (H T - c Z_j) + beta Z_{j-1} (+ source)
    if (fs) {
      fs->flops += 64.0 * (double)n * (double)n * (double)kj;
      fs->launches += 2;
    }
  }
  CB_CUDA(cudaEventRecord(e1, s));
  std::vector<int> sel(k);
  std::vector<double> coef(k, 0.0);
  for (int64_t i = 0; i < k; ++i) {
    sel[i] = degs[i] % 3;
    if (corr) coef[i] = pj[(size_t)degs[i] * k + i];
  }
  int* dsel;
  double* dcoef;
  CB_TRY(ws.alloc(&dsel, k));
  CB_TRY(ws.alloc(&dcoef, k));
  CB_CUDA(cudaMemcpyAsync(dsel, sel.data(), sizeof(int) * k, cudaMemcpyHostToDevice, s));
  CB_CUDA(cudaMemcpyAsync(dcoef, coef.data(), sizeof(double) * k, cudaMemcpyHostToDevice, s));
  combine_kernel<<<gsz(n2 * k), 256, 0, s>>>(out, Zb[0], Zb[1], Zb[2], dsel, corr ? dcoef : nullptr, Y0, n2, k);
  count_launch();
  CB_LAUNCH();
  int herr = 0;
  CB_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s));
  CB_CUDA(cudaStreamSynchronize(s));
  if (fs) {
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    fs->ms_mixed += ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return herr ? CHASE_BSE_DEVICE_TIMEOUT : CHASE_BSE_OK;
}

}  // namespace tc

bool mixed_available() {
  int dev = 0, major = 0, minor = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
  cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
  return major == 10 && minor == 3 && tc::encode_fn() != nullptr;
}

// Output tiles of 128 columns.  (Measured alternatives, degree-20 calls at n = 4096,
// k = 260 and degree-4 calls at n = 16384, k = 1300: 256-wide tiles with K blocks of 32
// in a 4-stage ring and all products in two alternating buffers drained every 4 K
// blocks ran 9 % faster at n = 16384 but missed the 1e-5 filter gate (1.3e-5 at
// n = 4096); drained after every K block they ran 10-17 % slower.  Draining the 128-wide
// x0 * y0 buffers every 1 or 2 K blocks instead of 4 cost 4-8 % and did not lower the
// error, which the 22-bit pieces and the recurrence set: 8.9e-6 at n = 4096 and
// 7.6e-6 at n = 16384 against the FP64 oracle.)
template <int SCH>
static int filter_dispatch(const cplx* A, const cplx* B, int64_t n, cplx* V, int64_t k, const int* degs,
                           double mu1, double mu_nevex, double muN, cplx* out, const double* ritz, const cplx* R,
                           cudaStream_t s, FilterStats* fs, const cplx* P2, const cplx* Q2) {
  return tc::filter_impl<SCH, 128, tc::Scheme<SCH>::FLUSH>(A, B, n, V, k, degs, mu1, mu_nevex, muN, out, ritz, R,
                                                            s, fs, P2, Q2);
}

static int filter_scheme(int scheme, const cplx* A, const cplx* B, int64_t n, cplx* V, int64_t k, const int* degs,
                         double mu1, double mu_nevex, double muN, cplx* out, const double* ritz, const cplx* R,
                         cudaStream_t s, FilterStats* fs, const cplx* P2, const cplx* Q2) {
  switch (scheme) {
    case SCHEME_BF16X3:
      return filter_dispatch<tc::SCH_BF16X3>(A, B, n, V, k, degs, mu1, mu_nevex, muN, out, ritz, R, s, fs, P2, Q2);
    case SCHEME_BF16X6:
      return filter_dispatch<tc::SCH_BF16X6>(A, B, n, V, k, degs, mu1, mu_nevex, muN, out, ritz, R, s, fs, P2, Q2);
    case SCHEME_FP16X3:
      return filter_dispatch<tc::SCH_FP16X3>(A, B, n, V, k, degs, mu1, mu_nevex, muN, out, ritz, R, s, fs, P2, Q2);
    default:
      return CHASE_BSE_BAD_ARG;
  }
}

int filter_mixed_sorted(const cplx* A, const cplx* B, int64_t n, cplx* Y0, int64_t k, const int* degs_sorted,
                        double mu1, double mu_nevex, double muN, cplx* out, int scheme, cudaStream_t s,
                        FilterStats* fs, const cplx* P2, const cplx* Q2) {
  return filter_scheme(scheme, A, B, n, Y0, k, degs_sorted, mu1, mu_nevex, muN, out, nullptr, nullptr, s, fs, P2,
                       Q2);
}

int filter_mixed_correction_sorted(const cplx* A, const cplx* B, int64_t n, cplx* V, int64_t k,
                                   const int* degs_sorted, const double* ritz_sorted, const cplx* R, double mu1,
                                   double mu_nevex, double muN, cplx* out, int scheme, cudaStream_t s,
                                   FilterStats* fs, const cplx* P2, const cplx* Q2) {
  return filter_scheme(scheme, A, B, n, V, k, degs_sorted, mu1, mu_nevex, muN, out, ritz_sorted, R, s, fs, P2, Q2);
}

}  // namespace cb
