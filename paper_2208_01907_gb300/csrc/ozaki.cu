// FP64 GEMM emulated on the BF16 tensor cores (tcgen05, TMEM accumulators).
//
// Used for the block-GCR products of Sec. 3.5 (Grams Q^T Z and updates X + P C),
// which must stay FP64-accurate.  Each row i of A (resp. column j of B) is scaled
// by 2^-e_i so that its entries lie in (-1, 1) and cut into S = 8 slices of 7-bit
// signed integers: a = 2^e_i * sum_s a_s 2^(-7(s+1)) + r, |r| < 2^(e_i - 56).
// Every slice is exact in BF16.  The product is
//     sum_k A(i,k) B(k,j) = 2^(e_i+f_j) sum_d 2^(-7(d+2)) sum_{s+t=d} sum_k a_s b_t,
// keeping the 36 slice pairs with s + t <= 7.  The inner sums are integers; one
// FP32 TMEM accumulator per diagonal d holds at most 8 pairs x 128 k-rows x 127^2
// < 2^24 before it is flushed into FP64 registers, so every partial sum is exact
// and the result carries the slicing error only (2^-56 relative to the row and
// column maxima, per term).
//
// Tile: 128 rows (i) x 64 columns (j) per CTA of 128 threads; 8 accumulators x 64
// TMEM columns = all 512 columns of the SM; K staged 32 rows at a time; split-K over
// blockIdx.z for the long Gram reductions.
#include "common.cuh"

#include <cuda_bf16.h>
#include <algorithm>
#include <cstdint>

namespace {

constexpr int OZ_S = 8;            // slices
constexpr int OZ_BI = 128;         // output rows per CTA (MMA M)
constexpr int OZ_BJ = 64;          // output columns per CTA (MMA N)
constexpr int OZ_BK = 32;          // k rows staged per step (2 MMAs of K = 16)
constexpr int OZ_FLUSH = 4;        // steps per flush: 128 k-rows
constexpr int OZ_A_SLICE = OZ_BI * OZ_BK * 2;   // bytes of one A slice tile (8 KB)
constexpr int OZ_B_SLICE = OZ_BJ * OZ_BK * 2;   // bytes of one B slice tile (4 KB)
constexpr int OZ_SMEM = 120 * 1024;   // > half of the SM: one CTA (one 512-column TMEM owner) per SM

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// K-major, no-swizzle canonical layout: core matrices of 8 rows x 16 bytes; core (g, kk)
// of a rows x 32 tile at ((kk * rows/8) + g) * 128.  Descriptor: LBO = K-adjacent core
// stride, SBO = row-group stride (checked on GB300 against a host reference).
__device__ __forceinline__ int tile_off(int r, int k, int rows) {
  return (((k >> 3) * (rows >> 3)) + (r >> 3)) * 128 + (r & 7) * 16 + (k & 7) * 2;
}

__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;                         // descriptor version of the sm_100 family
  return d;                                      // base offset 0, no swizzle
}

// kind::f16 instruction descriptor: D f32, A/B bf16, both K-major, N = 64, M = 128
constexpr uint32_t OZ_IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(OZ_BJ >> 3) << 17) |
                              ((uint32_t)(OZ_BI >> 4) << 24);

__device__ __forceinline__ void mma_bf16(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t acc) {
  asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
               " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
               :: "r"(tmem), "l"(ad), "l"(bd), "r"(OZ_IDESC), "r"(acc));
}

// bounded wait for an mbarrier phase; returns 0 on timeout
__device__ __forceinline__ int mbar_wait(uint32_t addr, uint32_t phase) {
  uint32_t done = 0;
  for (int it = 0; it < (1 << 24) && !done; ++it) {
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                 " selp.u32 %0, 1, 0, p;\n}\n" : "=r"(done) : "r"(addr), "r"(phase));
  }
  return (int)done;
}

struct OzArgs {
  const double* A; int64_t sai, sak;       // A(i, k) = A[i * sai + k * sak]
  const double* B; int64_t sbk, sbj;       // B(k, j) = B[k * sbk + j * sbj]
  int Mi, Nj;
  int64_t K, kchunk;                       // K split into chunks of kchunk (multiple of 128)
  const int* ea; const int* eb;            // scaling exponents per i and per j
  double* out; int64_t soi, soj;           // output
  const double* init;                      // update mode: out = (init ? init : out) + alpha * AB
  double alpha;
  int partial;                             // 1: out is a [kchunks][Mi][Nj] partial buffer
  int* err;                                // timeout flag
};

// Max-magnitude exponent of rows (dir 0: over k of A(i,k) = A[i*si + k*sk]) into e[i].
__global__ void k_oz_exp(const double* __restrict__ A, int64_t si, int64_t sk, int n, int64_t K, int* __restrict__ e) {
  const int i = blockIdx.x;
  if (i >= n) return;
  double mx = 0.0;
  for (int64_t k = threadIdx.x; k < K; k += blockDim.x) mx = fmax(mx, fabs(A[i * si + k * sk]));
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  __shared__ double r[32];
  if ((threadIdx.x & 31) == 0) r[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x + 31) / 32; ++w) mx = fmax(mx, r[w]);
    int ex = -1060;
    if (mx > 0) frexp(mx, &ex);                  // mx < 2^ex
    e[i] = ex;
  }
}

// column-wise exponents of a row-major L x m block, L large: per-block maxima, then atomicMax
__global__ void k_oz_exp_cols(const double* __restrict__ A, int64_t L, int m, int* __restrict__ e) {
  const int j = blockIdx.y * blockDim.x + threadIdx.x;
  if (j >= m) return;
  const int64_t rows = (L + gridDim.x - 1) / gridDim.x;
  const int64_t r0 = (int64_t)blockIdx.x * rows, r1 = min(L, r0 + rows);
  double mx = 0.0;
  for (int64_t r = r0; r < r1; ++r) mx = fmax(mx, fabs(A[r * m + j]));
  int ex = -1060;
  if (mx > 0) frexp(mx, &ex);
  atomicMax(&e[j], ex);
}

__global__ void k_fill_int(int* __restrict__ p, int n, int v) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) p[i] = v;
}

__device__ __forceinline__ void slice_store(double v, unsigned char* base, int stride_bytes, int off) {
  // v in (-1, 1): 8 slices of 7-bit signed integers, exact in bf16
#pragma unroll
  for (int s = 0; s < OZ_S; ++s) {
    v *= 128.0;
    double a = trunc(v);
    v -= a;
    *(__nv_bfloat16*)(base + s * stride_bytes + off) = __float2bfloat16_rn((float)a);
  }
}

__global__ void __launch_bounds__(128, 1) k_oz_gemm(OzArgs p) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char* sA = smem;                                  // OZ_S slices of 128 x 32
  unsigned char* sB = smem + OZ_S * OZ_A_SLICE;              // OZ_S slices of 64 x 32
  __shared__ uint32_t tmem_slot;
  __shared__ __align__(8) uint64_t mbar;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int i0 = blockIdx.x * OZ_BI, j0 = blockIdx.y * OZ_BJ;
  const int64_t kbeg = (int64_t)blockIdx.z * p.kchunk;
  const int64_t kend = min(p.K, kbeg + p.kchunk);
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" :: "r"(smem_u32(&tmem_slot)), "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_u32(&mbar)), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_slot;
  // per-thread scaling of the staged entries
  const int my_i = i0 + tid;                                  // output row owned in the epilogue
  double acc[OZ_BJ];
#pragma unroll
  for (int q = 0; q < OZ_BJ; ++q) acc[q] = 0.0;
  uint32_t phase = 0;
  int steps_in_flush = 0;
  bool any = false;
  const bool a_i_fast = (p.sai == 1);
  const bool b_j_fast = (p.sbj == 1);
  for (int64_t k0 = kbeg; k0 < kend; k0 += OZ_BK) {
    // ---- stage A (rows i0.., k0..k0+32) and B (k0.., cols j0..) as bf16 slices ----
    for (int e = tid; e < OZ_BI * OZ_BK; e += 128) {
      int ii, kk;
      if (a_i_fast) { ii = e % OZ_BI; kk = e / OZ_BI; } else { kk = e % OZ_BK; ii = e / OZ_BK; }
      const int i = i0 + ii;
      const int64_t k = k0 + kk;
      double v = 0.0;
      if (i < p.Mi && k < kend) v = ldexp(p.A[(int64_t)i * p.sai + k * p.sak], -p.ea[i]);
      slice_store(v, sA, OZ_A_SLICE, tile_off(ii, kk, OZ_BI));
    }
    for (int e = tid; e < OZ_BJ * OZ_BK; e += 128) {
      int jj, kk;
      if (b_j_fast) { jj = e % OZ_BJ; kk = e / OZ_BJ; } else { kk = e % OZ_BK; jj = e / OZ_BK; }
      const int j = j0 + jj;
      const int64_t k = k0 + kk;
      double v = 0.0;
      if (j < p.Nj && k < kend) v = ldexp(p.B[k * p.sbk + (int64_t)j * p.sbj], -p.eb[j]);
      slice_store(v, sB, OZ_B_SLICE, tile_off(jj, kk, OZ_BJ));
    }
    asm volatile("fence.proxy.async.shared::cta;");
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (tid == 0) {
      for (int s = 0; s < OZ_S; ++s)
        for (int t = 0; s + t < OZ_S; ++t) {
          const int d = s + t;
          for (int h = 0; h < 2; ++h) {                      // two K = 16 halves of the 32-row step
            uint64_t ad = smem_desc(smem_u32(sA + s * OZ_A_SLICE) + h * 4096, 2048, 128);
            uint64_t bd = smem_desc(smem_u32(sB + t * OZ_B_SLICE) + h * 2048, 1024, 128);
            // the first product into an accumulator after a flush overwrites it
            const uint32_t accf = (steps_in_flush > 0 || h > 0 || s > 0) ? 1u : 0u;
            mma_bf16(tmem + (uint32_t)(d * OZ_BJ), ad, bd, accf);
          }
        }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" :: "r"(smem_u32(&mbar)));
    }
    if (!mbar_wait(smem_u32(&mbar), phase)) { if (tid == 0) atomicExch(p.err, 1); }
    phase ^= 1u;
    any = true;
    ++steps_in_flush;
    const bool last = (k0 + OZ_BK >= kend);
    if (steps_in_flush == OZ_FLUSH || last) {
      asm volatile("tcgen05.fence::after_thread_sync;");
      // accumulator d: exact integers; scale 2^-7(d+2) and add in FP64
#pragma unroll
      for (int d = 0; d < OZ_S; ++d) {
        const double w = ldexp(1.0, -7 * (d + 2));
#pragma unroll
        for (int c0 = 0; c0 < OZ_BJ; c0 += 32) {
          uint32_t r[32];
          const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(d * OZ_BJ + c0);
          asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 "
                       "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                       "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                       : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                         "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
                         "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]),
                         "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]),
                         "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                       : "r"(taddr));
          asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
          for (int q = 0; q < 32; ++q) acc[c0 + q] += (double)__uint_as_float(r[q]) * w;
        }
      }
      steps_in_flush = 0;
      asm volatile("tcgen05.fence::before_thread_sync;");
    }
    __syncthreads();     // smem slices and TMEM may be reused by the next step
  }
  // ---- epilogue: row my_i, columns j0 .. j0+63 ----
  if (any && my_i < p.Mi) {
    const int ei = p.ea[my_i];
#pragma unroll
    for (int q = 0; q < OZ_BJ; ++q) {
      const int j = j0 + q;
      if (j >= p.Nj) continue;
      const double v = ldexp(acc[q], ei + p.eb[j]);
      if (p.partial) {
        p.out[((int64_t)blockIdx.z * p.Mi + my_i) * p.Nj + j] = v;
      } else {
        double* o = p.out + (int64_t)my_i * p.soi + (int64_t)j * p.soj;
        const double base = p.init ? p.init[(int64_t)my_i * p.soi + (int64_t)j * p.soj] : *o;
        *o = base + p.alpha * v;
      }
    }
  } else if (!any && my_i < p.Mi && p.partial) {
    for (int q = 0; q < OZ_BJ && j0 + q < p.Nj; ++q) p.out[((int64_t)blockIdx.z * p.Mi + my_i) * p.Nj + j0 + q] = 0.0;
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(512));
}

__global__ void k_oz_reduce(int Mi, int Nj, int nch, const double* __restrict__ part, double* __restrict__ G,
                            double scale, int sym) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= Mi * Nj) return;
  int i = e / Nj, j = e % Nj;
  double s = 0.0;
  for (int c = 0; c < nch; ++c) s += part[((int64_t)c * Mi + i) * Nj + j];
  if (sym) {   // A^T A: average the two triangles so the result is exactly symmetric
    double s2 = 0.0;
    for (int c = 0; c < nch; ++c) s2 += part[((int64_t)c * Mi + j) * Nj + i];
    s = 0.5 * (s + s2);
  }
  G[e] = scale * s;
}

}  // namespace

static bool oz_attr_done = false;

// G = scale * A^T B for row-major L x ma (A) and L x mb (B) blocks.
int hf_oz_gram(hf_ctx* c, int64_t L, int ma, int mb, const double* A, const double* B, double* G, double scale,
               double* scratch, size_t scratch_bytes, int* iscratch, int* err) {
  cudaStream_t s = hf_stream(c);
  if (!oz_attr_done) {
    HF_CUDA_TRY(cudaFuncSetAttribute(k_oz_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, OZ_SMEM));
    oz_attr_done = true;
  }
  int* ea = iscratch;
  int* eb = iscratch + ma;
  HF_LAUNCH(c, HF_PROF_GRAM, k_fill_int<<<(ma + mb + 255) / 256, 256, 0, s>>>(ea, ma + mb, -1060));
  const unsigned gx = (unsigned)std::min<int64_t>(std::max<int64_t>(1, L / 1024), 512);
  HF_LAUNCH(c, HF_PROF_GRAM, k_oz_exp_cols<<<dim3(gx, (ma + 127) / 128), 128, 0, s>>>(A, L, ma, ea));
  HF_LAUNCH(c, HF_PROF_GRAM, k_oz_exp_cols<<<dim3(gx, (mb + 127) / 128), 128, 0, s>>>(B, L, mb, eb));
  // split-K so that the grid covers the GPU about twice
  const int tiles = ((ma + OZ_BI - 1) / OZ_BI) * ((mb + OZ_BJ - 1) / OZ_BJ);
  int64_t nch = std::max<int64_t>(1, (2 * 152 + tiles - 1) / tiles);
  int64_t kchunk = (L + nch - 1) / nch;
  kchunk = (kchunk + 127) / 128 * 128;
  nch = (L + kchunk - 1) / kchunk;
  if ((size_t)nch * ma * mb * 8 > scratch_bytes) return HF_ERR_ARG;
  OzArgs a;
  a.A = A; a.sai = 1; a.sak = ma;
  a.B = B; a.sbk = mb; a.sbj = 1;
  a.Mi = ma; a.Nj = mb; a.K = L; a.kchunk = kchunk;
  a.ea = ea; a.eb = eb;
  a.out = scratch; a.soi = 0; a.soj = 0; a.init = nullptr; a.alpha = 1.0; a.partial = 1; a.err = err;
  dim3 grid((ma + OZ_BI - 1) / OZ_BI, (mb + OZ_BJ - 1) / OZ_BJ, (unsigned)nch);
  HF_LAUNCH(c, HF_PROF_GRAM, k_oz_gemm<<<grid, 128, OZ_SMEM, s>>>(a));
  const int sym = (A == B && ma == mb) ? 1 : 0;
  HF_LAUNCH(c, HF_PROF_GRAM, k_oz_reduce<<<(ma * mb + 255) / 256, 256, 0, s>>>(ma, mb, (int)nch, scratch, G, scale, sym));
  HF_CUDA_TRY(cudaGetLastError());
  return HF_OK;
}

// Y = (Yinit ? Yinit : Y) + sgn * A C for row-major L x m (A, Y) and m x m (C).
int hf_oz_update(hf_ctx* c, int64_t L, int m, const double* A, const double* C, double* Y, const double* Yinit,
                 double sgn, int* iscratch, int* err) {
  cudaStream_t s = hf_stream(c);
  if (!oz_attr_done) {
    HF_CUDA_TRY(cudaFuncSetAttribute(k_oz_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, OZ_SMEM));
    oz_attr_done = true;
  }
  int* ea = iscratch;                      // L row exponents of A
  int* eb = iscratch + L;                  // m column exponents of C
  HF_LAUNCH(c, HF_PROF_BLOCK_UPDATE, k_oz_exp<<<(unsigned)L, 32, 0, s>>>(A, m, 1, (int)L, m, ea));
  HF_LAUNCH(c, HF_PROF_BLOCK_UPDATE, k_oz_exp<<<m, 32, 0, s>>>(C, 1, m, m, m, eb));
  OzArgs a;
  a.A = A; a.sai = m; a.sak = 1;
  a.B = C; a.sbk = m; a.sbj = 1;
  a.Mi = (int)L; a.Nj = m; a.K = m; a.kchunk = ((int64_t)m + 127) / 128 * 128;
  a.ea = ea; a.eb = eb;
  a.out = Y; a.soi = m; a.soj = 1; a.init = Yinit; a.alpha = sgn; a.partial = 0; a.err = err;
  dim3 grid((unsigned)((L + OZ_BI - 1) / OZ_BI), (m + OZ_BJ - 1) / OZ_BJ, 1);
  HF_LAUNCH(c, HF_PROF_BLOCK_UPDATE, k_oz_gemm<<<grid, 128, OZ_SMEM, s>>>(a));
  HF_CUDA_TRY(cudaGetLastError());
  return HF_OK;
}
