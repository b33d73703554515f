// FP64 GEMM emulated on the BF16 tensor cores (tcgen05, TMA, TMEM accumulators).
//
// Used for the block-GCR products of Sec. 3.5 (Grams Q^T Z and updates X + P C),
// which must stay FP64-accurate while GB300's FP64 units run at a small fraction of
// its tensor rate.
//
// Slicing.  Row i of A (column j of B) is scaled by 2^-e_i (2^-f_j) so that its
// entries lie in (-1, 1); the 56 leading bits of |a| * 2^-e_i are cut into S = 8
// digits of 7 bits, a = 2^(e_i-7) * sum_s a''_s with a''_s = +-digit_s * 2^(-7s).
// Every a''_s is exact in BF16.  The product of two scaled slices is
// a''_s b''_t = digit_s digit_t 2^(-7(s+t)), so for a fixed d = s + t all terms share
// the scale 2^(-7d) and
//     sum_k A(i,k) B(k,j) = 2^(e_i+f_j-14) sum_{s+t<=7} sum_k a''_s b''_t
// (pairs with s + t > 7 and the bits below the 56th are dropped: relative error
// about 2^-53 per term, the FP64 level).
//
// Accumulation.  The diagonals d = 0..5 each get their own FP32 TMEM accumulator;
// it holds integers times 2^(-7d) below 2^24 as long as (d+1) * 127^2 * R < 2^24,
// i.e. for R = 160 k-rows, after which the flush warps add it exactly into an int64
// fixed-point sum (units 2^-35) with integer instructions only.  The diagonals
// d = 6, 7 (15 pairs, terms below 2^-42 of the leading ones) share one FP32
// accumulator that is never flushed; its rounding stays far below the FP64 level
// for the chunk lengths used (at most 96 flush groups, which also bounds the int64
// sum below 2^63).
//
// Kernel structure (one 128 x 64 output tile per CTA, one CTA per SM):
//   warp 0: TMA producer (4-D tensor maps over the pre-sliced operands, 2 stages),
//   warp 1: MMA issuer (36 tcgen05.mma per 16 k-rows),
//   warps 2..9: flush and epilogue (TMEM lanes = output rows; two warps per lane
//   quadrant, 32 columns each).
// TMEM: 6 exact + 1 merged accumulators x 64 columns = 448 of 512 columns.
// Every mbarrier wait is bounded; a timeout sets an error flag and every role
// leaves its loop, waits (bounded) for its own asynchronous work and frees TMEM.
#include "common.cuh"
#include "tcgen05.cuh"

#include <cuda.h>
#include <cuda_bf16.h>
#include <algorithm>
#include <cstdint>
#include <mutex>

namespace {

constexpr int OZ_S = 8;              // slices per operand
constexpr int OZ_BI = 128;           // output rows per CTA (MMA M)
constexpr int OZ_BJ = 64;            // output columns per CTA (MMA N)
constexpr int OZ_BK = 32;            // k rows per pipeline stage (2 MMAs of K = 16)
constexpr int OZ_G = 5;              // stages per flush group: 160 k rows
constexpr int OZ_NEXACT = 6;         // diagonals with exact accumulators
constexpr int OZ_MAX_GROUPS = 96;    // flush groups per chunk (int64 fixed-point range)
constexpr int OZ_STAGES = 2;
constexpr int OZ_A_STAGE = OZ_S * OZ_BI * OZ_BK * 2;   // 64 KB
constexpr int OZ_B_STAGE = OZ_S * OZ_BJ * OZ_BK * 2;   // 32 KB
constexpr int OZ_STAGE = OZ_A_STAGE + OZ_B_STAGE;
constexpr int OZ_SMEM = OZ_STAGES * OZ_STAGE + 1024;  // + alignment slack
constexpr int OZ_THREADS = 320;      // producer warp, MMA warp, 8 flush warps
constexpr int OZ_WAIT_LIMIT = 1 << 20;
constexpr int OZ_RG = 32;             // rows per TMA row group: 32 x 8 BF16 = 512 contiguous bytes
__host__ __device__ constexpr int64_t oz_rows(int64_t R) { return (R + OZ_RG - 1) / OZ_RG * OZ_RG; }

static_assert(OZ_SMEM <= 227 * 1024, "stage ring exceeds shared memory");
static_assert((OZ_NEXACT + 1) * OZ_BJ <= 512, "accumulators exceed TMEM");
static_assert(OZ_BJ == 64, "two flush warps of 32 columns per lane quadrant");
static_assert(OZ_NEXACT * 127 * 127 * OZ_G * OZ_BK < (1 << 24), "exact accumulators overflow FP32 integers");
static_assert(OZ_NEXACT == 6, "fixed-point units 2^-35 assume diagonals 0..5");

using tc::smem_u32;
using tc::smem_desc;
using tc::mma_commit;
using tc::mbar_try;
using tc::tmem_ld32;

// kind::f16 instruction descriptor: D f32, A/B bf16, both K-major, N = OZ_BJ, M = 128
constexpr uint32_t OZ_IDESC = tc::bf16_idesc(OZ_BI, OZ_BJ);

__device__ __forceinline__ void mma_bf16(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t acc) {
  tc::mma_bf16(tmem, ad, bd, OZ_IDESC, acc);
}

// Bounded wait.  Gives up when another role has aborted or after OZ_WAIT_LIMIT tries
// (then it raises the abort flag and the error flag itself).
__device__ __forceinline__ bool oz_wait(uint32_t bar, uint32_t parity, volatile int* abort_flag, int* err) {
  for (int it = 0; it < OZ_WAIT_LIMIT; ++it) {
    if (mbar_try(bar, parity)) return true;
    if (*abort_flag) return false;
  }
  *abort_flag = 1;
  atomicExch(err, 1);
  return false;
}

// Wait that ignores the abort flag (own asynchronous work before TMEM is freed); bounded.
__device__ __forceinline__ void oz_drain(uint32_t bar, uint32_t parity, int* err) {
  for (int it = 0; it < OZ_WAIT_LIMIT; ++it)
    if (mbar_try(bar, parity)) return;
  atomicExch(err, 1);
}

__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                            uint32_t bar) {
  asm volatile("cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
               " [%0], [%1, {%2, %3, %4, %5}], [%6];"
               :: "r"(dst), "l"((uint64_t)map), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(bar) : "memory");
}

// 56-bit fixed-point magnitude of x * 2^-e (|x| < 2^e) as hi (24 bits) / lo (32 bits)
__device__ __forceinline__ void oz_fixed(double x, int e, uint32_t& hi, uint32_t& lo, uint32_t& neg) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  neg = (uint32_t)(b >> 63);
  int ex = (int)((b >> 52) & 0x7FF);
  unsigned long long m = b & 0xFFFFFFFFFFFFFull;
  if (ex) m |= 1ull << 52; else ex = 1;                 // subnormals: no implicit bit
  const int sh = ex - 1019 - e;                          // F = m 2^sh; sh <= 3 since |x| < 2^e
  unsigned long long F;
  if (sh >= 0) F = m << min(sh, 3);
  else F = (sh > -64) ? (((m >> (-sh - 1)) + 1ull) >> 1) : 0ull;   // to nearest (ties away): unbiased
  // (no overflow: F < 2^56 needs rounding only when sh < 0, where F <= 2^53)
  hi = (uint32_t)(F >> 32);
  lo = (uint32_t)F;
}

// digit s (7 bits, most significant first) of the 56-bit magnitude
__device__ __forceinline__ uint32_t oz_digit(uint32_t hi, uint32_t lo, int s) {
  switch (s) {
    case 0: return (hi >> 17) & 127u;
    case 1: return (hi >> 10) & 127u;
    case 2: return (hi >> 3) & 127u;
    case 3: return ((hi & 7u) << 4) | (lo >> 28);
    case 4: return (lo >> 21) & 127u;
    case 5: return (lo >> 14) & 127u;
    case 6: return (lo >> 7) & 127u;
    default: return lo & 127u;
  }
}

// BF16 bits of +-digit * 2^(-7s) (exact: at most 7 significant bits, normal exponent)
__device__ __forceinline__ uint32_t oz_bf16(uint32_t dg, int s, uint32_t neg) {
  const float f = __uint_as_float(0x4B000000u | dg) - 8388608.0f;   // = dg exactly
  uint32_t u = __float_as_uint(f);
  u = dg ? (u - ((uint32_t)(7 * s) << 23)) : 0u;
  return (u >> 16) | (neg << 15);
}

// FP32 value v = n * 2^(-7d) with |n| < 2^24 (d <= 5) as int64 in units of 2^-35 (exact):
// v * 2^35 = mant * 2^(e - 115) = (mant << 35) >> (150 - e)
__device__ __forceinline__ long long oz_fix35(uint32_t u) {
  const uint32_t e = (u >> 23) & 0xFFu;
  const unsigned long long m = (unsigned long long)((u & 0x7FFFFFu) | 0x800000u) << 35;
  const uint32_t sh = min(150u - min(e, 150u), 63u);
  const long long r = e ? (long long)(m >> sh) : 0ll;
  return (u >> 31) ? -r : r;
}

// Max-magnitude exponent (x < 2^e) of rows i: max over k of |X[i*si + k*sk]|.
__global__ void k_oz_exp(const double* __restrict__ X, int64_t si, int64_t sk, int n, int64_t K, int* __restrict__ e) {
  const int i = blockIdx.x;
  if (i >= n) return;
  double mx = 0.0;
  for (int64_t k = threadIdx.x; k < K; k += blockDim.x) mx = fmax(mx, fabs(X[i * si + k * sk]));
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  __shared__ double r[32];
  if ((threadIdx.x & 31) == 0) r[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x + 31) / 32; ++w) mx = fmax(mx, r[w]);
    int ex = -1060;
    if (mx > 0) frexp(mx, &ex);
    e[i] = ex;
  }
}

// Max-magnitude exponents of the n rows of a row-major n x K block: a warp takes four
// consecutive rows at a time, their loads all issued before the four reductions.
__global__ void __launch_bounds__(256) k_oz_exp_rows(const double* __restrict__ X, int64_t n, int K, int* __restrict__ e) {
  constexpr int RPW = 4;
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i0 = (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * RPW; i0 < n; i0 += nw * RPW) {
    double mx[RPW];
#pragma unroll
    for (int r = 0; r < RPW; ++r) mx[r] = 0.0;
    for (int k = lane; k < K; k += 32)
#pragma unroll
      for (int r = 0; r < RPW; ++r)
        if (i0 + r < n) mx[r] = fmax(mx[r], fabs(X[(i0 + r) * K + k]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
      for (int r = 0; r < RPW; ++r) mx[r] = fmax(mx[r], __shfl_xor_sync(0xffffffffu, mx[r], o));
    double v = mx[0];
#pragma unroll
    for (int r = 1; r < RPW; ++r) if (lane == r) v = mx[r];
    if (lane < RPW && i0 + lane < n) {
      int ex = -1060;
      if (v > 0) frexp(v, &ex);
      e[i0 + lane] = ex;
    }
  }
}

// Column exponents of a row-major L x m block (e preset to -1060). The 256 threads of a
// block cover a window of w = min(m, 256) columns on 256 / w rows at a time, so that
// consecutive threads read consecutive entries; each block takes a contiguous range of
// rows, reduces its maxima in shared memory and merges them into e by atomicMax.
__global__ void __launch_bounds__(256) k_oz_exp_cols(const double* __restrict__ A, int64_t L, int m, int* __restrict__ e) {
  __shared__ int sx[256];
  const int w = min(m, 256), rpi = 256 / w;                 // window width, rows per step
  const int tid = threadIdx.x, jr = tid / w, jc = tid % w;
  const int64_t rows = (L + gridDim.x - 1) / gridDim.x;
  const int64_t r0 = (int64_t)blockIdx.x * rows, r1 = min(L, r0 + rows);
  for (int c0 = 0; c0 < m; c0 += w) {
    const int j = c0 + jc;
    const bool act = jr < rpi && j < m;
    double mx = 0.0;
    if (act)
      for (int64_t r = r0 + jr; r < r1; r += rpi) mx = fmax(mx, fabs(A[r * m + j]));
    int ex = -1060;
    if (mx > 0) frexp(mx, &ex);
    if (tid < w) sx[tid] = -1060;
    __syncthreads();
    if (act) atomicMax(&sx[jc], ex);
    __syncthreads();
    if (tid < w && c0 + tid < m) atomicMax(&e[c0 + tid], sx[tid]);
    __syncthreads();
  }
}

__global__ void k_fill_int(int* __restrict__ p, int n, int v) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) p[i] = v;
}

// Slices of X(r, k) = X[r*sr + k*sk] (R rows, K columns, row exponents e) into
// dst[s][kg][r] (16 bytes = 8 consecutive k each), kg < Kg = ceil(K / 8); the tail of
// the last group is zero.  One thread per (r, kg): consecutive threads take consecutive
// rows, so the 16-byte stores of each slice are contiguous.
__global__ void k_oz_slice(const double* __restrict__ X, int64_t R, int64_t K, int64_t sr, int64_t sk,
                           const int* __restrict__ e, uint4* __restrict__ dst, int64_t Kg) {
  const int64_t Rp = oz_rows(R);                 // row stride of the slices; rows [R, Rp) are zero
  const int64_t total = Rp * Kg;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = t % Rp, kg = t / Rp;
    if (r >= R) {
#pragma unroll
      for (int s = 0; s < OZ_S; ++s) dst[((int64_t)s * Kg + kg) * Rp + r] = make_uint4(0u, 0u, 0u, 0u);
      continue;
    }
    const int er = e[r];
    uint32_t hi[8], lo[8], ng[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int64_t k = kg * 8 + q;
      const double x = (k < K) ? X[r * sr + k * sk] : 0.0;
      oz_fixed(x, er, hi[q], lo[q], ng[q]);
    }
#pragma unroll
    for (int s = 0; s < OZ_S; ++s) {
      uint32_t w[4];
#pragma unroll
      for (int q = 0; q < 4; ++q)
        w[q] = oz_bf16(oz_digit(hi[2 * q], lo[2 * q], s), s, ng[2 * q]) |
               (oz_bf16(oz_digit(hi[2 * q + 1], lo[2 * q + 1], s), s, ng[2 * q + 1]) << 16);
      dst[((int64_t)s * Kg + kg) * Rp + r] = make_uint4(w[0], w[1], w[2], w[3]);
    }
  }
}

struct OzMma {
  int Mi, Nj;                 // output rows (A slices) and columns (B slices)
  int64_t nsteps;             // k steps of 32 rows in total
  int64_t chunk_steps;        // steps per blockIdx.z chunk
  const int* ea; const int* eb;
  double* out; int64_t soi, soj;
  const double* init;         // update mode: out = (init ? init : out) + alpha * AB
  double alpha;
  int partial;                // 1: out is a [chunks][Mi][Nj] partial buffer
  int upper;                  // 1 (A^T A): only tiles meeting the upper triangle j >= i are needed
  int* err;
};

__global__ void __launch_bounds__(OZ_THREADS, 1)
k_oz_mma(const __grid_constant__ CUtensorMap ta, const __grid_constant__ CUtensorMap tb, OzMma p) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  __shared__ __align__(8) uint64_t bar_full[OZ_STAGES], bar_empty[OZ_STAGES];
  __shared__ __align__(8) uint64_t bar_accfull, bar_accempty, bar_done;
  __shared__ uint32_t tmem_slot;
  __shared__ volatile int abort_flag;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int j0 = blockIdx.x * OZ_BJ, i0 = blockIdx.y * OZ_BI;
  if (p.upper && j0 + OZ_BJ - 1 < i0) return;        // tile strictly below the diagonal: not read
  const int64_t s_beg = (int64_t)blockIdx.z * p.chunk_steps;
  const int64_t n = max((int64_t)0, min(p.nsteps, s_beg + p.chunk_steps) - s_beg);

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" :: "r"(smem_u32(&tmem_slot)), "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 32) {
    for (int st = 0; st < OZ_STAGES; ++st) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_u32(&bar_full[st])), "r"(1));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_u32(&bar_empty[st])), "r"(1));
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_u32(&bar_accfull)), "r"(1));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_u32(&bar_accempty)), "r"(256));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_u32(&bar_done)), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;");
    abort_flag = 0;
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_slot;

  if (warp == 0) {
    // ---------------- TMA producer ----------------
    if (lane == 0 && n > 0) {
      int64_t issued = 0;
      for (int64_t q = 0; q < n; ++q) {
        const int st = (int)(q & 1);
        if (q >= OZ_STAGES && !oz_wait(smem_u32(&bar_empty[st]), (uint32_t)(((q >> 1) - 1) & 1), &abort_flag, p.err)) break;
        const uint32_t fb = smem_u32(&bar_full[st]);
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(fb), "r"(OZ_STAGE) : "memory");
        const uint32_t sa = smem_u32(smem + st * OZ_STAGE);
        const int kg = (int)((s_beg + q) * (OZ_BK / 8));
        tma_load_4d(sa, &ta, 0, i0 / OZ_RG, kg, 0, fb);
        tma_load_4d(sa + OZ_A_STAGE, &tb, 0, j0 / OZ_RG, kg, 0, fb);
        issued = q + 1;
      }
      // the last loads issued must land before the CTA exits
      for (int64_t q = (issued > OZ_STAGES ? issued - OZ_STAGES : 0); q < issued; ++q)
        oz_drain(smem_u32(&bar_full[q & 1]), (uint32_t)((q >> 1) & 1), p.err);
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    if (lane == 0 && n > 0) {
      bool merged_first = true;
      for (int64_t q = 0; q < n; ++q) {
        const int st = (int)(q & 1);
        if (!oz_wait(smem_u32(&bar_full[st]), (uint32_t)((q >> 1) & 1), &abort_flag, p.err)) break;
        asm volatile("tcgen05.fence::after_thread_sync;");
        const uint32_t sa = smem_u32(smem + st * OZ_STAGE);
        const uint32_t sb = sa + OZ_A_STAGE;
        // diagonals 6, 7 into the shared accumulator (no flush needed)
#pragma unroll 1
        for (int h = 0; h < 2; ++h)
#pragma unroll 1
          for (int s = 0; s < OZ_S; ++s)
#pragma unroll 1
            for (int t = (s < OZ_NEXACT ? OZ_NEXACT - s : 0); s + t < OZ_S; ++t) {
              const uint64_t ad = smem_desc(sa + s * (OZ_BI * OZ_BK * 2) + h * (2 * OZ_BI * 16), 16 * OZ_BI, 128);
              const uint64_t bd = smem_desc(sb + t * (OZ_BJ * OZ_BK * 2) + h * (2 * OZ_BJ * 16), 16 * OZ_BJ, 128);
              mma_bf16(tmem + (uint32_t)(OZ_NEXACT * OZ_BJ), ad, bd, merged_first ? 0u : 1u);
              merged_first = false;
            }
        const bool group_start = (q % OZ_G) == 0;
        if (group_start && q > 0) {
          if (!oz_wait(smem_u32(&bar_accempty), (uint32_t)((q / OZ_G - 1) & 1), &abort_flag, p.err)) break;
          asm volatile("tcgen05.fence::after_thread_sync;");
        }
        // diagonals 0..5: one exact accumulator each, restarted after every flush
#pragma unroll 1
        for (int h = 0; h < 2; ++h)
#pragma unroll 1
          for (int s = 0; s < OZ_NEXACT; ++s)
#pragma unroll 1
            for (int t = 0; s + t < OZ_NEXACT; ++t) {
              const uint64_t ad = smem_desc(sa + s * (OZ_BI * OZ_BK * 2) + h * (2 * OZ_BI * 16), 16 * OZ_BI, 128);
              const uint64_t bd = smem_desc(sb + t * (OZ_BJ * OZ_BK * 2) + h * (2 * OZ_BJ * 16), 16 * OZ_BJ, 128);
              const uint32_t accf = (group_start && h == 0 && s == 0) ? 0u : 1u;
              mma_bf16(tmem + (uint32_t)((s + t) * OZ_BJ), ad, bd, accf);
            }
        mma_commit(smem_u32(&bar_empty[st]));
        if ((q % OZ_G) == OZ_G - 1 || q == n - 1) mma_commit(smem_u32(&bar_accfull));
      }
      mma_commit(smem_u32(&bar_done));
      oz_drain(smem_u32(&bar_done), 0u, p.err);
    }
  } else {
    // ---------------- flush and epilogue (warps 2..9) ----------------
    const int quad = warp & 3;                         // TMEM lanes 32*quad .. 32*quad+31
    const int cbase = ((warp - 2) >> 2) * 32;          // this warp's 32 output columns
    const int row = quad * 32 + lane;
    const int my_i = i0 + row;
    const uint32_t tlane = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)cbase;
    long long V[32];
#pragma unroll
    for (int c = 0; c < 32; ++c) V[c] = 0;
    const int64_t ngroups = (n + OZ_G - 1) / OZ_G;
    bool ok = true;
    for (int64_t g = 0; g < ngroups; ++g) {
      if (!oz_wait(smem_u32(&bar_accfull), (uint32_t)(g & 1), &abort_flag, p.err)) { ok = false; break; }
      asm volatile("tcgen05.fence::after_thread_sync;");
#pragma unroll 1
      for (int d = 0; d < OZ_NEXACT; ++d) {
        uint32_t r[32];
        tmem_ld32(tlane + (uint32_t)(d * OZ_BJ), r);
#pragma unroll
        for (int q = 0; q < 32; ++q) V[q] += oz_fix35(r[q]);
      }
      asm volatile("tcgen05.fence::before_thread_sync;");
      asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" :: "r"(smem_u32(&bar_accempty)) : "memory");
    }
    if (ok && n > 0) {
      const int ei = (my_i < p.Mi) ? p.ea[my_i] : 0;
      {
        uint32_t r[32];
        tmem_ld32(tlane + (uint32_t)(OZ_NEXACT * OZ_BJ), r);
#pragma unroll
        for (int q = 0; q < 32; ++q) {
          const int j = j0 + cbase + q;
          if (my_i < p.Mi && j < p.Nj) {
            const double sum = (double)V[q] * 0x1p-35 + (double)__uint_as_float(r[q]);
            const double v = ldexp(sum, ei + p.eb[j] - 14);
            if (p.partial) {
              p.out[((int64_t)blockIdx.z * p.Mi + my_i) * p.Nj + j] = v;
            } else {
              double* o = p.out + (int64_t)my_i * p.soi + (int64_t)j * p.soj;
              const double base = p.init ? p.init[(int64_t)my_i * p.soi + (int64_t)j * p.soj] : *o;
              *o = base + p.alpha * v;
            }
          }
        }
      }
    } else if (n == 0 && p.partial && my_i < p.Mi) {
      for (int q = 0; q < 32 && j0 + cbase + q < p.Nj; ++q)
        p.out[((int64_t)blockIdx.z * p.Mi + my_i) * p.Nj + j0 + cbase + q] = 0.0;
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
  }
  __syncthreads();
  if (warp == 0) {
    __syncwarp();
    asm volatile("tcgen05.fence::after_thread_sync;");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(512));
  }
}

// One warp per entry of G: lane l adds the chunks l, l + 32, ... in order, then the lanes'
// sums are added by a butterfly (every lane ends with the same value; a fixed order, so the
// result is the same from run to run)
__global__ void __launch_bounds__(256) k_oz_reduce(int Mi, int Nj, int nch, const double* __restrict__ part,
                                                   double* __restrict__ G, double scale, int sym) {
  const int lane = threadIdx.x & 31;
  const int64_t e = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (e >= (int64_t)Mi * Nj) return;                       // uniform per warp
  const int i = (int)(e / Nj), j = (int)(e % Nj);
  // A^T A: only the upper triangle was computed; the lower one mirrors it (exactly symmetric)
  const int a = (sym && i > j) ? j : i, b = (sym && i > j) ? i : j;
  double s = 0.0;
  for (int c = lane; c < nch; c += 32) s += part[((int64_t)c * Mi + a) * Nj + b];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) G[e] = scale * s;
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn lookup_encode() {
  void* f = nullptr;
  cudaDriverEntryPointQueryResult q;
  if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
      q == cudaDriverEntryPointSuccess)
    return (EncodeTiledFn)f;
  return nullptr;
}

EncodeTiledFn encode_fn() {
  static const EncodeTiledFn fn = lookup_encode();    // thread-safe one-time initialisation
  return fn;
}

// 4-D map over slices stored as [S][Kg][R][8 bf16]: dims (8, R, Kg, S), box (8, rows, 4, S).
int slice_map(CUtensorMap* map, const void* base, int64_t R, int64_t Kg, int box_rows) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return HF_ERR_CUDA;
  if (((uintptr_t)base & 15) != 0) return HF_ERR_ARG;
  // [S][Kg][Rp][8] BF16 seen as (8 * 32, Rp / 32, Kg, S): the inner dimension is a group of
  // 32 rows (512 contiguous bytes); the shared-memory image, [S][4][box_rows][8], is that
  // of a box with an 8-element inner dimension
  const int64_t Rp = oz_rows(R);
  const cuuint64_t dims[4] = {(cuuint64_t)(8 * OZ_RG), (cuuint64_t)(Rp / OZ_RG), (cuuint64_t)Kg, (cuuint64_t)OZ_S};
  const cuuint64_t strides[3] = {(cuuint64_t)OZ_RG * 16, (cuuint64_t)Rp * 16, (cuuint64_t)Kg * Rp * 16};
  const cuuint32_t box[4] = {(cuuint32_t)(8 * OZ_RG), (cuuint32_t)(box_rows / OZ_RG), (cuuint32_t)(OZ_BK / 8),
                             (cuuint32_t)OZ_S};
  const cuuint32_t es[4] = {1, 1, 1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void*>(base), dims, strides, box, es,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? HF_OK : HF_ERR_CUDA;
}

bool oz_attr_done = false;
std::mutex oz_attr_mu;

int oz_setup() {
  std::lock_guard<std::mutex> lk(oz_attr_mu);
  if (!oz_attr_done) {
    HF_CUDA_TRY(cudaFuncSetAttribute(k_oz_mma, cudaFuncAttributeMaxDynamicSharedMemorySize, OZ_SMEM));
    oz_attr_done = true;
  }
  return HF_OK;
}

unsigned slice_grid(int64_t items) {
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>((items + 255) / 256, 152 * 16));
}

}  // namespace

// Bytes of slice storage for an operand with R rows and K columns.
size_t hf_oz_slice_bytes(int64_t R, int64_t K) { return (size_t)OZ_S * (size_t)((K + 7) / 8) * (size_t)oz_rows(R) * 16; }

// Number of split-K chunks hf_oz_gram uses (sizes its partial-sum scratch).
int64_t hf_oz_gram_chunks(int64_t L, int ma, int mb) {
  const int tiles = ((ma + OZ_BI - 1) / OZ_BI) * ((mb + OZ_BJ - 1) / OZ_BJ);
  const int64_t nsteps = ((L + 7) / 8 + OZ_BK / 8 - 1) / (OZ_BK / 8);
  int64_t nch = std::max<int64_t>(1, (3 * 152) / tiles);
  nch = std::max<int64_t>(nch, (nsteps + OZ_MAX_GROUPS * OZ_G - 1) / (OZ_MAX_GROUPS * OZ_G));
  const int64_t chunk_steps = (nsteps + nch - 1) / nch;
  return (nsteps + chunk_steps - 1) / chunk_steps;
}

// G = scale * A^T B for row-major L x ma (A) and L x mb (B) blocks.
int hf_oz_gram(hf_ctx* c, int64_t L, int ma, int mb, const double* A, const double* B, double* G, double scale,
               double* scratch, size_t scratch_bytes, void* slices, size_t slice_bytes, int* iscratch, int* err) {
  cudaStream_t s = hf_stream(c);
  int rc;
  if ((rc = oz_setup())) return rc;
  if (L <= 0 || ma <= 0 || mb <= 0) return HF_ERR_ARG;
  const bool same = (A == B && ma == mb);
  const int64_t Kg = (L + 7) / 8;
  const size_t sa_bytes = hf_oz_slice_bytes(ma, L), sb_bytes = same ? 0 : hf_oz_slice_bytes(mb, L);
  if (sa_bytes + sb_bytes > slice_bytes) return HF_ERR_ARG;
  uint4* SA = (uint4*)slices;
  uint4* SB = same ? SA : (uint4*)((unsigned char*)slices + sa_bytes);
  int* ea = iscratch;
  int* eb = same ? ea : iscratch + ma;
  const int ne = same ? ma : ma + mb;
  HF_LAUNCH(c, HF_PROF_TC_PREP, k_fill_int<<<(ne + 255) / 256, 256, 0, s>>>(ea, ne, -1060));
  const unsigned gx = (unsigned)std::min<int64_t>((L + 255) / 256, 1216);
  HF_LAUNCH(c, HF_PROF_TC_PREP, k_oz_exp_cols<<<gx, 256, 0, s>>>(A, L, ma, ea));
  HF_LAUNCH(c, HF_PROF_TC_PREP, k_oz_slice<<<slice_grid(oz_rows(ma) * Kg), 256, 0, s>>>(A, ma, L, 1, ma, ea, SA, Kg));
  if (!same) {
    HF_LAUNCH(c, HF_PROF_TC_PREP, k_oz_exp_cols<<<gx, 256, 0, s>>>(B, L, mb, eb));
    HF_LAUNCH(c, HF_PROF_TC_PREP, k_oz_slice<<<slice_grid(oz_rows(mb) * Kg), 256, 0, s>>>(B, mb, L, 1, mb, eb, SB, Kg));
  }
  CUtensorMap ta, tb;
  if ((rc = slice_map(&ta, SA, ma, Kg, OZ_BI))) return rc;
  if ((rc = slice_map(&tb, SB, mb, Kg, OZ_BJ))) return rc;
  const int64_t nsteps = (Kg + OZ_BK / 8 - 1) / (OZ_BK / 8);
  const int64_t nch = hf_oz_gram_chunks(L, ma, mb);
  const int64_t chunk_steps = (nsteps + nch - 1) / nch;
  if ((size_t)nch * ma * mb * 8 > scratch_bytes) return HF_ERR_ARG;
  OzMma a;
  a.Mi = ma; a.Nj = mb; a.nsteps = nsteps; a.chunk_steps = chunk_steps;
  a.ea = ea; a.eb = eb;
  a.out = scratch; a.soi = 0; a.soj = 0; a.init = nullptr; a.alpha = 1.0; a.partial = 1; a.err = err;
  a.upper = same ? 1 : 0;
  dim3 grid((mb + OZ_BJ - 1) / OZ_BJ, (ma + OZ_BI - 1) / OZ_BI, (unsigned)nch);
  HF_LAUNCH(c, HF_PROF_GRAM, k_oz_mma<<<grid, OZ_THREADS, OZ_SMEM, s>>>(ta, tb, a));
  HF_LAUNCH(c, HF_PROF_TC_PREP, k_oz_reduce<<<(unsigned)(((int64_t)ma * mb * 32 + 255) / 256), 256, 0, s>>>(ma, mb, (int)nch, scratch, G, scale,
                                                                               same ? 1 : 0));
  HF_CUDA_TRY(cudaGetLastError());
  return HF_OK;
}

// Y = (Yinit ? Yinit : Y) + sgn * A C for row-major L x m (A, Y) and m x m (C).
int hf_oz_update(hf_ctx* c, int64_t L, int m, const double* A, const double* C, double* Y, const double* Yinit,
                 double sgn, void* slices, size_t slice_bytes, int* iscratch, int* err) {
  cudaStream_t s = hf_stream(c);
  int rc;
  if ((rc = oz_setup())) return rc;
  if (L <= 0 || m <= 0) return HF_ERR_ARG;
  const int64_t Kg = (m + 7) / 8;
  const size_t sa_bytes = hf_oz_slice_bytes(L, m), sb_bytes = hf_oz_slice_bytes(m, m);
  if (sa_bytes + sb_bytes > slice_bytes) return HF_ERR_ARG;
  uint4* SA = (uint4*)slices;
  uint4* SB = (uint4*)((unsigned char*)slices + sa_bytes);
  int* ea = iscratch;                      // L row exponents of A
  int* eb = iscratch + L;                  // m column exponents of C
  HF_LAUNCH(c, HF_PROF_TC_PREP, k_oz_exp_rows<<<(unsigned)std::min<int64_t>((L + 7) / 8, 4864), 256, 0, s>>>(A, L, m, ea));
  HF_LAUNCH(c, HF_PROF_TC_PREP, k_oz_exp<<<m, 32, 0, s>>>(C, 1, m, m, m, eb));
  HF_LAUNCH(c, HF_PROF_TC_PREP, k_oz_slice<<<slice_grid(oz_rows(L) * Kg), 256, 0, s>>>(A, L, m, m, 1, ea, SA, Kg));
  HF_LAUNCH(c, HF_PROF_TC_PREP, k_oz_slice<<<slice_grid(oz_rows(m) * Kg), 256, 0, s>>>(C, m, m, 1, m, eb, SB, Kg));
  CUtensorMap ta, tb;
  if ((rc = slice_map(&ta, SA, L, Kg, OZ_BI))) return rc;
  if ((rc = slice_map(&tb, SB, m, Kg, OZ_BJ))) return rc;
  const int64_t nsteps = (Kg + OZ_BK / 8 - 1) / (OZ_BK / 8);
  if (nsteps > (int64_t)OZ_MAX_GROUPS * OZ_G) return HF_ERR_ARG;   // m > 15360: no split-K here
  OzMma a;
  a.Mi = (int)L; a.Nj = m; a.nsteps = nsteps; a.chunk_steps = nsteps;
  a.ea = ea; a.eb = eb;
  a.out = Y; a.soi = m; a.soj = 1; a.init = Yinit; a.alpha = sgn; a.partial = 0; a.err = err;
  a.upper = 0;
  dim3 grid((m + OZ_BJ - 1) / OZ_BJ, (unsigned)((L + OZ_BI - 1) / OZ_BI), 1);
  HF_LAUNCH(c, HF_PROF_BLOCK_UPDATE, k_oz_mma<<<grid, OZ_THREADS, OZ_SMEM, s>>>(ta, tb, a));
  HF_CUDA_TRY(cudaGetLastError());
  return HF_OK;
}
