// Alg. 1 steps 2-5 and Alg. 2 on the GPU:
//  - the lower-precision solve Q^-1 (Sec. 3.1-3.2) as a multifrontal forward /
//    backward substitution over the fronts of the factorization,
//  - block GCR ("Algorithm 5", Sec. 3.5) in FP64 with SpMM by K11,
//  - S22 = K22 - K21 X12 (Alg. 1 step 4), Bunch-Kaufman LDL^T of S22 with kernel
//    detection (Alg. 1 step 5), and the block substitution of Alg. 2.
// Vectors are row-major L x m blocks (the m right-hand sides of a row contiguous),
// indexed by original unknown; rows of Lambda_2 are kept at zero in K11 blocks.
#include "common.cuh"

#include <cooperative_groups.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <mutex>
#include <vector>

namespace {

constexpr int SB = 32;       // column block of the triangular solves

// ---------------------------------------------------------------------------
// Multifrontal triangular solves with the stored factor, level by level.
// Forward (levels bottom-up): V_t rows [0, n) start from b, the other rows from 0,
// the children's update rows are added (maps in pivoted order), then
// V = L11^-1 V over the K11 columns [0, ksolve), blocked by SB columns: a diagonal
// triangular solve and a GEMM update of every row below.  Pivot rows leave
// y_i / d_i (the D^-1 step) in Y; rows of Lambda_2 leave their value unscaled.
// Backward (levels top-down): rows [ks, f) take the solution of later unknowns from
// X, then x = L11^-T (y - L21^T x2) blocked from the bottom.
// ---------------------------------------------------------------------------
constexpr int TS = 64;       // row tile / diagonal block of the triangular solves
constexpr int TR = 64;       // right-hand-side tile
constexpr int TKK = 16;      // k chunk of the GEMM updates

// Start of a forward sweep level: row i of front t's vectors is its own right-hand side (or
// 0), plus the contribution row of child 0 mapped to it, plus that of child 1, in that order
// (one gather through the reverse maps gmap instead of a write and two scatter-adds)
template <typename TV>
__global__ void k_fwd_gather(const NodeDesc* __restrict__ nd, const NodeState* __restrict__ st, int t0,
                             const int32_t* __restrict__ rowid, const int32_t* __restrict__ gmap, int64_t rows,
                             TV* __restrict__ vec, const TV* __restrict__ B, int m, int vs) {
  const int t = t0 + blockIdx.y;
  const NodeDesc d = nd[t];
  const int f = st[t].f;
  const int nown = d.cand_all ? 0 : d.n;
  TV* V = vec + d.row_off * vs;
  const int32_t* rid = rowid + d.row_off;
  const int32_t* g0 = gmap + d.row_off;
  const int32_t* g1 = gmap + rows + d.row_off;
  const TV* U0 = nullptr;
  const TV* U1 = nullptr;
  if (d.child0 >= 0) U0 = vec + (nd[d.child0].row_off + st[d.child0].k) * vs;
  if (d.child1 >= 0) U1 = vec + (nd[d.child1].row_off + st[d.child1].k) * vs;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < (int64_t)f * m; e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / m), c = (int)(e - (int64_t)i * m);
    TV v = (i < nown) ? B[(int64_t)rid[i] * m + c] : TV(0);
    const int a0 = U0 ? g0[i] : -1, a1 = U1 ? g1[i] : -1;
    if (a0 >= 0) v += U0[(int64_t)a0 * vs + c];
    if (a1 >= 0) v += U1[(int64_t)a1 * vs + c];
    V[(int64_t)i * vs + c] = v;
  }
}

// pivot rows -> Y (scaled by 1/d for the K11 pivots); moved / unfactorized rows unscaled
template <typename TF, typename TV>
__global__ void k_fwd_store(const NodeDesc* __restrict__ nd, const NodeState* __restrict__ st, int t0,
                           const TF* __restrict__ arena, const int32_t* __restrict__ rowid,
                           const TV* __restrict__ vec, TV* __restrict__ Y, int m, int vs) {
  const int t = t0 + blockIdx.y;
  const NodeDesc d = nd[t];
  const NodeState S = st[t];
  const int hi = d.cand_all ? S.f : S.k;
  const TF* F = arena + d.front_off;
  const TV* V = vec + d.row_off * vs;
  const int32_t* rid = rowid + d.row_off;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < (int64_t)hi * m; e += (int64_t)gridDim.x * blockDim.x) {
    int i = (int)(e / m), c = (int)(e - (int64_t)i * m);
    TV v = V[(int64_t)i * vs + c];
    if (i < S.ksolve) v = v / (TV)F[i + (int64_t)i * d.ld];
    Y[(int64_t)rid[i] * m + c] = v;
  }
}

template <typename TV>
__global__ void k_bwd_init(const NodeDesc* __restrict__ nd, const NodeState* __restrict__ st, int t0,
                           const int32_t* __restrict__ rowid, TV* __restrict__ vec, const TV* __restrict__ Y,
                           const TV* __restrict__ X, int m, int vs) {
  const int t = t0 + blockIdx.y;
  const NodeDesc d = nd[t];
  const NodeState S = st[t];
  if (S.ksolve == 0) return;
  TV* V = vec + d.row_off * vs;
  const int32_t* rid = rowid + d.row_off;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < (int64_t)S.f * m; e += (int64_t)gridDim.x * blockDim.x) {
    int i = (int)(e / m), c = (int)(e - (int64_t)i * m);
    V[(int64_t)i * vs + c] = (i < S.ksolve) ? Y[(int64_t)rid[i] * m + c] : X[(int64_t)rid[i] * m + c];
  }
}

template <typename TV>
__global__ void k_bwd_store(const NodeDesc* __restrict__ nd, const NodeState* __restrict__ st, int t0,
                            const int32_t* __restrict__ rowid, const TV* __restrict__ vec, TV* __restrict__ X, int m,
                            int vs) {
  const int t = t0 + blockIdx.y;
  const NodeDesc d = nd[t];
  const int ks = st[t].ksolve;
  const TV* V = vec + d.row_off * vs;
  const int32_t* rid = rowid + d.row_off;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < (int64_t)ks * m; e += (int64_t)gridDim.x * blockDim.x) {
    int i = (int)(e / m), c = (int)(e - (int64_t)i * m);
    X[(int64_t)rid[i] * m + c] = V[(int64_t)i * vs + c];
  }
}

// Diagonal block solve of block step b: forward (unit L, columns [b*TS, ...)) or
// backward (unit L^T, blocks counted from ksolve down), for a tile of DR right-hand
// sides.  The block of L and the right-hand sides are staged in shared memory; the
// block is processed in sub-blocks of DSB rows: a sub-block is solved by one thread
// per right-hand side in registers, then the rows after it (before it, backward) are
// updated by all threads.
template <typename TV> struct DiagRhs { static constexpr int value = sizeof(TV) == 8 ? 16 : 64; };  // rhs per CTA
constexpr int DSB = 16;      // sub-block rows
constexpr int DTH = 256;     // threads

// Unit-triangular solve of a jb x jb diagonal block (forward: L, backward: L^T) for the
// NR right-hand sides staged in Vs; sub-blocks of DSB rows are solved by one thread per
// right-hand side in registers, the rows after (before) them updated by all NTH threads.
template <typename TV, bool FWD, int NR, int NTH, int LS, int VS>
__device__ __forceinline__ void diag_solve(const TV (*Ls)[LS], TV (*Vs)[VS], int jb, int tid) {
  constexpr int DR = NR;
  const int nsb = (jb + DSB - 1) / DSB;
  for (int sbi = 0; sbi < nsb; ++sbi) {
    const int s = FWD ? sbi : nsb - 1 - sbi;             // sub-block index
    const int r0 = s * DSB, r1 = min(jb, r0 + DSB);
    if (tid < DR) {
      TV x[DSB];
#pragma unroll
      for (int i = 0; i < DSB; ++i) x[i] = (r0 + i < r1) ? Vs[r0 + i][tid] : TV(0);
      if (FWD) {
#pragma unroll
        for (int i = 1; i < DSB; ++i)
#pragma unroll
          for (int q = 0; q < i; ++q) x[i] -= Ls[r0 + i][r0 + q] * x[q];
      } else {
#pragma unroll
        for (int i = DSB - 2; i >= 0; --i)
#pragma unroll
          for (int q = i + 1; q < DSB; ++q) x[i] -= Ls[r0 + q][r0 + i] * x[q];
      }
#pragma unroll
      for (int i = 0; i < DSB; ++i)
        if (r0 + i < r1) Vs[r0 + i][tid] = x[i];
    }
    __syncthreads();
    // rows after (forward) / before (backward) the sub-block
    const int u0 = FWD ? r1 : 0, u1 = FWD ? jb : r0;
    for (int e = tid; e < (u1 - u0) * DR; e += NTH) {
      const int r = u0 + e / DR, c = e % DR;
      TV acc = Vs[r][c];
      if (FWD) {
#pragma unroll
        for (int q = 0; q < DSB; ++q)
          if (r0 + q < r1) acc -= Ls[r][r0 + q] * Vs[r0 + q][c];
      } else {
#pragma unroll
        for (int q = 0; q < DSB; ++q)
          if (r0 + q < r1) acc -= Ls[r0 + q][r] * Vs[r0 + q][c];
      }
      Vs[r][c] = acc;
    }
    __syncthreads();
  }
}

template <typename TF, typename TV, bool FWD>
__global__ void __launch_bounds__(DTH) k_trsm_diag(const NodeDesc* __restrict__ nd, const NodeState* __restrict__ st,
                                                  int t0, const TF* __restrict__ arena, TV* __restrict__ vec, int m,
                                                  int b) {
  constexpr int DR = DiagRhs<TV>::value;
  __shared__ TV Ls[TS][TS + 1];
  __shared__ TV Vs[TS][DR + 1];
  const int t = t0 + blockIdx.y;
  const NodeDesc d = nd[t];
  const int ks = st[t].ksolve;
  int j0, jb;
  if (FWD) { j0 = b * TS; if (j0 >= ks) return; jb = min(TS, ks - j0); }
  else { int j1 = ks - b * TS; if (j1 <= 0) return; j0 = max(0, j1 - TS); jb = j1 - j0; }
  const TF* F = arena + d.front_off;
  const int64_t ld = d.ld;
  const int tid = threadIdx.x;
  const int c0 = blockIdx.x * DR;
  for (int e = tid; e < TS * TS; e += DTH) {
    const int r = e % TS, c = e / TS;                     // r fastest: contiguous in column c of F
    Ls[r][c] = (r < jb && c < jb && r > c) ? (TV)F[(j0 + r) + (int64_t)(j0 + c) * ld] : TV(0);
  }
  TV* V = vec + (d.row_off + j0) * m;
  for (int e = tid; e < TS * DR; e += DTH) {
    const int r = e / DR, c = e % DR;
    Vs[r][c] = (r < jb && c0 + c < m) ? V[(int64_t)r * m + c0 + c] : TV(0);
  }
  __syncthreads();
  diag_solve<TV, FWD, DR, DTH>(Ls, Vs, jb, tid);
  for (int e = tid; e < jb * DR; e += DTH) {
    const int r = e / DR, c = e % DR;
    if (c0 + c < m) V[(int64_t)r * m + c0 + c] = Vs[r][c];
  }
}

// GEMM update C -= A B on the front vectors of a level.
//  MODE 0 (forward, block step b):  rows [j0+jb, f),  A(i,q) = L(i, j0+q),  B = V rows [j0, j0+jb)
//  MODE 1 (backward, block step b): rows [0, j0),     A(i,q) = L(j0+q, i),  B = V rows [j0, j1)
//  MODE 2 (backward start):         rows [0, ks),     A(i,q) = L(ks+q, i),  B = V rows [ks, f)
// CTA tile SGR rows x SGC right-hand sides, 128 threads with 8 x 8 outputs each; the k
// chunks are double-buffered (the next chunk is loaded into registers while the
// current one is multiplied from shared memory).
constexpr int SGR = 128;      // rows per CTA
constexpr int SGC = 64;       // right-hand sides per CTA
constexpr int SGTH = 128;     // threads
template <typename TV> struct GemmK { static constexpr int value = sizeof(TV) == 8 ? 8 : 16; };

// With SOLVE (MODE 0 / 1), the CTAs of the row tile that holds the next diagonal block
// (forward: rows [j0+jb, ...), the first tile; backward: rows [.., j0), the first tile,
// tiles counted from the top) also solve that block after their update, so that the next
// block step needs no separate diagonal-solve launch.
template <typename TF, typename TV, int MODE, bool SOLVE>
__global__ void __launch_bounds__(SGTH) k_gemm_upd(const NodeDesc* __restrict__ nd, const NodeState* __restrict__ st,
                                                  int t0, const TF* __restrict__ arena, TV* __restrict__ vec, int m, int b) {
  constexpr int GK = GemmK<TV>::value;
  constexpr int AL = GK * SGR / SGTH;          // A elements per thread per chunk
  constexpr int BL = GK * SGC / SGTH;          // B elements per thread per chunk
  const int t = t0 + blockIdx.z;
  const NodeDesc d = nd[t];
  const int ks = st[t].ksolve, f = st[t].f;
  int r_lo, r_hi, k_lo, k_hi;
  if (MODE == 0) { int j0 = b * TS; if (j0 >= ks) return; int jb = min(TS, ks - j0); r_lo = j0 + jb; r_hi = f; k_lo = j0; k_hi = j0 + jb; }
  else if (MODE == 1) { int j1 = ks - b * TS; if (j1 <= 0) return; int j0 = max(0, j1 - TS); r_lo = 0; r_hi = j0; k_lo = j0; k_hi = j1; }
  else { r_lo = 0; r_hi = ks; k_lo = ks; k_hi = f; }
  // row tile: forward / start from the first row, backward block steps from the last
  const int r0 = MODE == 1 ? r_hi - (int)(blockIdx.x + 1) * SGR : r_lo + (int)blockIdx.x * SGR;
  const int c0 = blockIdx.y * SGC;
  if (r0 >= r_hi || r0 + SGR <= r_lo || c0 >= m || k_hi <= k_lo) return;
  const TF* F = arena + d.front_off;
  const int64_t ld = d.ld;
  TV* V = vec + d.row_off * m;
  __shared__ __align__(16) TV As[2][GK][SGR + 4];
  __shared__ __align__(16) TV Bs[2][GK][SGC + 4];
  __shared__ TV Ls[SOLVE ? TS : 1][SOLVE ? TS + 1 : 1];   // next diagonal block (SOLVE)
  const int tid = threadIdx.x;
  const int tx = tid & 7, ty = tid >> 3;     // 8 rhs groups x 16 row groups
  TV pa[AL], pb[BL];
  auto load = [&](int kc) {
#pragma unroll
    for (int u = 0; u < AL; ++u) {
      int kk, rr;
      if (MODE == 0) { const int e = tid + u * SGTH; kk = e / SGR; rr = e % SGR; }   // rows contiguous in column q
      else { rr = tid; kk = u; }                                                 // k contiguous in column i
      const int q = kc + kk, i = r0 + rr;
      TV a = TV(0);
      if (q < k_hi && i < r_hi && i >= r_lo) a = (TV)(MODE == 0 ? F[i + (int64_t)q * ld] : F[q + (int64_t)i * ld]);
      pa[u] = a;
    }
#pragma unroll
    for (int u = 0; u < BL; ++u) {
      const int e = tid + u * SGTH;
      const int kk = e / SGC, cc = e % SGC;
      const int q = kc + kk, c = c0 + cc;
      pb[u] = (q < k_hi && c < m) ? V[(int64_t)q * m + c] : TV(0);
    }
  };
  auto store = [&](int buf) {
#pragma unroll
    for (int u = 0; u < AL; ++u) {
      int kk, rr;
      if (MODE == 0) { const int e = tid + u * SGTH; kk = e / SGR; rr = e % SGR; }
      else { rr = tid; kk = u; }
      As[buf][kk][rr] = pa[u];
    }
#pragma unroll
    for (int u = 0; u < BL; ++u) {
      const int e = tid + u * SGTH;
      Bs[buf][e / SGC][e % SGC] = pb[u];
    }
  };
  TV acc[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = TV(0);
  load(k_lo);
  store(0);
  __syncthreads();
  int buf = 0;
  for (int kc = k_lo; kc < k_hi; kc += GK) {
    const bool more = kc + GK < k_hi;
    if (more) load(kc + GK);
#pragma unroll
    for (int kk = 0; kk < GK; ++kk) {
      TV av[8], bv[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) av[i] = As[buf][kk][ty * 8 + i];
#pragma unroll
      for (int j = 0; j < 8; ++j) bv[j] = Bs[buf][kk][tx * 8 + j];
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] += av[i] * bv[j];
    }
    if (more) store(buf ^ 1);
    __syncthreads();
    buf ^= 1;
  }
  // next diagonal block held by this tile (SOLVE): rows [nb0, nb0 + njb)
  int nb0 = 0, njb = 0;
  if (SOLVE && blockIdx.x == 0) {
    if (MODE == 0 && r_lo < ks) { nb0 = r_lo; njb = min(TS, ks - r_lo); }
    if (MODE == 1 && r_hi > 0) { njb = min(TS, r_hi); nb0 = r_hi - njb; }
  }
  static_assert(!SOLVE || (SGR + 4) * 2 * GK >= TS * (SGC + 1), "block staging reuses As");
  TV (*Vs)[SGC + 1] = (TV (*)[SGC + 1])&As[0][0][0];
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int r = r0 + ty * 8 + i;
    if (r >= r_hi || r < r_lo) continue;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int c = c0 + tx * 8 + j;
      if (c >= m) continue;
      const TV v = V[(int64_t)r * m + c] - acc[i][j];
      if (SOLVE && njb > 0 && r >= nb0 && r < nb0 + njb) Vs[r - nb0][tx * 8 + j] = v;
      else V[(int64_t)r * m + c] = v;
    }
  }
  if (SOLVE && njb > 0) {                   // uniform across the CTA
    for (int e = tid; e < TS * TS; e += SGTH) {
      const int r = e % TS, c = e / TS;
      Ls[r][c] = (r < njb && c < njb && r > c) ? (TV)F[(nb0 + r) + (int64_t)(nb0 + c) * ld] : TV(0);
    }
    __syncthreads();
    diag_solve<TV, MODE == 0, SGC, SGTH>(Ls, Vs, njb, tid);
    for (int e = tid; e < njb * SGC; e += SGTH) {
      const int r = e / SGC, c = e % SGC;
      if (c0 + c < m) V[(int64_t)(nb0 + r) * m + c0 + c] = Vs[r][c];
    }
  }
}

// ---------------------------------------------------------------------------
// Dataflow sweep of one level (FP32 factor and vectors): one launch per level instead
// of a launch per diagonal block.
//
// Work item = (front t, block, 64-column tile C).  Forward: triangle block R (rows
// [64R, 64R+64) of [0, ks)) takes y_R = L_RR^-1 (v_R - sum_{b<R} L_Rb y_b); a
// contribution block j (rows [ks + 64j, ...) of [ks, f)) takes v -= sum_b L_jb y_b.
// Backward: triangle block R takes x_R = L_RR^-T (v_R - sum_{r>=ks} L_rR^T x_r -
// sum_{b>R} L_bR^T x_b).  The updates accumulate in registers over the whole k range,
// so no row is re-read between block steps; a triangle block publishes its columns
// tile with a flag once solved, and an item waits for the flag of every block it reads.
//
// Persistent CTAs take items by ticket (an atomic counter).  Items are listed so that
// an item only waits for items of lower tickets (forward: blocks by ascending R, then
// the contribution blocks; backward: descending R).  A ticket is held by a running CTA,
// so the lowest unfinished item always has its inputs and the level cannot deadlock,
// whatever the number of resident CTAs.  Every wait is bounded: on timeout the CTA sets
// the abort word, and every later wait of the launch gives up at once.
// ---------------------------------------------------------------------------
constexpr int DF_R = 64;       // rows per item (= TS, the diagonal block)
constexpr int DF_C = 64;       // right-hand sides per item
constexpr int DF_TH = 128;     // threads: 8 row groups x 16 column groups, 8 x 4 outputs each
constexpr int DF_K = 16;       // k chunk of the register double buffer
constexpr int DF_SPIN = 1 << 22;
static_assert(DF_R == TS, "the triangle blocks are the diagonal blocks of the solve");

__device__ __forceinline__ int df_ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void df_st_release(int* p, int v) {
  asm volatile("st.release.gpu.global.b32 [%0], %1;" :: "l"(p), "r"(v) : "memory");
}

// Thread 0 waits for *flag != 0 (at most `spin` polls); false (uniform) on timeout or abort.
__device__ __forceinline__ bool df_wait(const int* flag, int* abort_word, int* s_ok, int spin) {
  if (threadIdx.x == 0) {
    int ok = 0;
    for (int it = 0; it < spin; ++it) {
      if (df_ld_acquire(flag)) { ok = 1; break; }
      if (*(volatile int*)abort_word) break;
      __nanosleep(32);
    }
    if (!ok) atomicExch(abort_word, 1);
    *s_ok = ok;
  }
  __syncthreads();
  return *s_ok != 0;
}

// After block `from` is known to be ready: the end of the run of blocks that are
// ready as well (ascending from+1, from+2, ... below `lim`, or descending from-1, ...
// above `lim`), looking at up to DF_TH flags at once.  Uniform; one barrier.
__device__ __forceinline__ int df_ready_run(const int* fl, int gt, int from, int lim, bool up, int* s_e) {
  const int tid = threadIdx.x;
  if (tid == 0) *s_e = up ? min(lim, from + 1 + DF_TH) : max(lim, from - 1 - DF_TH);
  __syncthreads();
  const int b = up ? from + 1 + tid : from - 1 - tid;
  if (up ? b < lim : b > lim) {
    if (!df_ld_acquire(fl + (int64_t)b * gt)) {
      if (up) atomicMin(s_e, b);
      else atomicMax(s_e, b);
    }
  }
  __syncthreads();
  const int e = *s_e;
  __syncthreads();
  return e;   // up: blocks [from, e) ready; down: blocks (e, from] ready
}

// cp.async (global -> shared, no registers): 4-byte copies for the factor (read-only in
// the sweeps), 16-byte L2-only copies for the vectors (written by other CTAs of the launch)
__device__ __forceinline__ uint32_t df_smem(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void df_cp4(void* dst, const void* src, bool pred) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" :: "r"(df_smem(dst)), "l"(src), "r"(pred ? 4 : 0) : "memory");
}
__device__ __forceinline__ void df_cp16(void* dst, const void* src, bool pred) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" :: "r"(df_smem(dst)), "l"(src), "r"(pred ? 16 : 0) : "memory");
}
__device__ __forceinline__ void df_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N> __device__ __forceinline__ void df_wait_copies() { asm volatile("cp.async.wait_group %0;" :: "n"(N) : "memory"); }

constexpr int DF_ST = 4;       // cp.async pipeline stages (three chunks in flight)
// shared memory of a sweep CTA (dynamic: above the 48 KB of static shared memory): the GEMM
// stages, which the block being solved reuses, then the staged diagonal-block inverse
struct DfGemm { float A[DF_ST][DF_K][DF_R + 4]; float B[DF_ST][DF_K][DF_C + 4]; };
constexpr size_t DF_UB = sizeof(DfGemm) > sizeof(float) * DF_R * (DF_C + 1) ? sizeof(DfGemm)
                                                                              : sizeof(float) * DF_R * (DF_C + 1);
constexpr size_t DF_SMEM = DF_UB + sizeof(float) * TS * (TS + 1);
static_assert(DF_UB % 16 == 0, "the inverse follows the stages 16-byte aligned");

// vs: row stride of the per-front vectors (m rounded up to 4, so that rows are 16-byte aligned)
template <bool FWD>
__global__ void __launch_bounds__(DF_TH, 4) k_sweep_df(const NodeDesc* __restrict__ nd, const NodeState* __restrict__ st,
                                                   const float* __restrict__ arena, float* vec, int m, int vs, int gt,
                                                   const int2* __restrict__ items, int nitems,
                                                   const int* __restrict__ blockbase, int* flags, int* counter,
                                                   int* abort_word, int spin, const float* __restrict__ dinv) {
  constexpr int APT = DF_K * DF_R / DF_TH;       // 4-byte A copies per thread per chunk
  constexpr int BPT = DF_K * DF_C / 4 / DF_TH;   // 16-byte B copies per thread per chunk
  constexpr int VS = DF_C + 1;
  extern __shared__ __align__(16) unsigned char dsm[];  // DF_SMEM bytes
  __shared__ int s_ticket, s_ok, s_e;
  DfGemm& G = *reinterpret_cast<DfGemm*>(dsm);          // GEMM stages, then the block being solved
  float (*Vs)[VS] = reinterpret_cast<float (*)[VS]>(dsm);
  float (*Ls)[TS + 1] = reinterpret_cast<float (*)[TS + 1]>(dsm + DF_UB);
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int64_t total = (int64_t)nitems * gt;
  int next = 0;
  if (tid == 0) next = atomicAdd(counter, 1);
  for (;;) {
    if (tid == 0) s_ticket = next;
    __syncthreads();
    const int ticket = s_ticket;
    if (ticket >= total) return;
    if (tid == 0) next = atomicAdd(counter, 1);          // the next item's ticket, taken early
    const int2 it = items[ticket / gt];
    const int C = ticket - (ticket / gt) * gt;
    const int t = it.x, code = it.y;
    const NodeDesc d = nd[t];
    const int ks = st[t].ksolve, f = st[t].f;
    const int nblk = (ks + DF_R - 1) / DF_R;
    const int64_t ld = d.ld;
    const float* F = arena + d.front_off;
    float* V = vec + d.row_off * vs;
    const int c0 = C * DF_C;
    const bool tri = code >= 0;
    const int r0 = tri ? code * DF_R : ks + (-1 - code) * DF_R;
    const int nr = min(DF_R, (tri ? ks : f) - r0);
    int* fl = flags + (int64_t)blockbase[t] * gt + C;     // flag of block b: fl[b * gt]
    // a triangle block stages the inverse of its unit lower diagonal block (made once per
    // factorization by k_diag_inverse) before it waits
    if (tri) {
      const float* Di = dinv + ((int64_t)blockbase[t] + code) * (TS * TS);
      for (int e = tid; e < TS * TS; e += DF_TH) Ls[e / TS][e % TS] = Di[e];
    }
    // blocked summation: acc holds the products of at most DF_R consecutive k, then is
    // added into tot (the error of a long FP32 dot product grows with its length; this
    // keeps it at that of the per-block updates).  An item starts tot at -v (its own rows of
    // the vectors, which no other item of the launch writes), so that the loads are made
    // before the waits, all at once, and not after the last one: a triangle item then solves
    // for -tot = v_R - (the blocks' products), a contribution item stores -tot.
    float acc[8][4], tot[8][4];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int r = ty * 8 + i;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int c = c0 + tx * 4 + j;
        acc[i][j] = 0.f;
        tot[i][j] = (r < nr && c < m) ? -__ldcg(V + (int64_t)(r0 + r) * vs + c) : 0.f;
      }
    }
    // acc += A(rows of the item, k in [k_lo, k_hi)) * V(k rows, tile columns); k_lo is a
    // multiple of DF_R or the start of the ancestors' rows.  The chunks of DF_K rows run
    // upward, or downward with `down`; acc goes into tot at every boundary of DF_R rows, so
    // tot sums the blocks in ascending (descending) order however the range was split
    auto gemm_range = [&](int k_lo, int k_hi, bool down) {
      const int nch = (k_hi - k_lo + DF_K - 1) / DF_K;
      auto kc_of = [&](int ch) { return k_lo + (down ? nch - 1 - ch : ch) * DF_K; };
      auto issue = [&](int ch) {
        const int kc = kc_of(ch), stg = ch % DF_ST;
#pragma unroll
        for (int u = 0; u < APT; ++u) {
          const int e = tid + u * DF_TH;
          int kk, rr;
          if (FWD) { kk = e / DF_R; rr = e % DF_R; }    // rows contiguous in column q
          else { rr = e / DF_K; kk = e % DF_K; }        // k contiguous in column r0 + rr
          const int q = kc + kk;
          const bool ok = q < k_hi && rr < nr;
          const float* src = ok ? (FWD ? F + (r0 + rr) + (int64_t)q * ld : F + q + (int64_t)(r0 + rr) * ld) : F;
          df_cp4(&G.A[stg][kk][rr], src, ok);
        }
#pragma unroll
        for (int u = 0; u < BPT; ++u) {
          const int e = tid + u * DF_TH;
          const int kk = e / (DF_C / 4), c4 = e % (DF_C / 4);
          const int q = kc + kk, c = c0 + 4 * c4;
          const bool ok = q < k_hi && c < vs;
          df_cp16(&G.B[stg][kk][4 * c4], ok ? V + (int64_t)q * vs + c : V, ok);
        }
      };
#pragma unroll
      for (int ch = 0; ch < DF_ST - 1; ++ch) {
        if (ch < nch) issue(ch);
        df_commit();
      }
      for (int ch = 0; ch < nch; ++ch) {
        df_wait_copies<DF_ST - 2>();                     // chunk ch has landed (this thread's copies)
        __syncthreads();                                 // ... everyone's; stage of ch-1 is free
        if (ch + DF_ST - 1 < nch) issue(ch + DF_ST - 1);
        df_commit();
        const int stg = ch % DF_ST;
#pragma unroll
        for (int kk = 0; kk < DF_K; ++kk) {
          const float4 a0 = *reinterpret_cast<const float4*>(&G.A[stg][kk][ty * 8]);
          const float4 a1 = *reinterpret_cast<const float4*>(&G.A[stg][kk][ty * 8 + 4]);
          const float4 b = *reinterpret_cast<const float4*>(&G.B[stg][kk][tx * 4]);
          const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
          const float bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
          for (int i = 0; i < 8; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] += av[i] * bv[j];
        }
        if (ch == nch - 1 || (down ? (kc_of(ch) - k_lo) % DF_R == 0 : ((ch + 1) * DF_K) % DF_R == 0)) {
#pragma unroll
          for (int i = 0; i < 8; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) { tot[i][j] += acc[i][j]; acc[i][j] = 0.f; }
        }
      }
      __syncthreads();                                   // stages free for the next range / Vs
    };
    // the blocks an item reads are taken in runs: wait for the next one, then extend the
    // run over the blocks already published, and multiply the run as one k range
    bool ok = true;
    if (FWD) {
      const int bend = tri ? code : nblk;                 // blocks [0, bend) feed this item
      for (int b = 0; b < bend && ok;) {
        {
          // the factor block this item multiplies once block b is published, into L2 while
          // it waits (columns 64b.. of rows r0..r0+nr: two 128-byte lines per column)
          const int q = b * DF_R + (tid >> 1), rr = (tid & 1) * 32;
          if (q < ks && rr < nr) asm volatile("prefetch.global.L2 [%0];" :: "l"(F + (r0 + rr) + (int64_t)q * ld));
        }
        ok = df_wait(fl + (int64_t)b * gt, abort_word, &s_ok, spin);
        if (!ok) break;
        // the last block the item reads ends the run (no flags to look at)
        const int e = b + 1 == bend ? bend : df_ready_run(fl, gt, b, bend, true, &s_e);
        gemm_range(b * DF_R, min(ks, e * DF_R), false);
        b = e;
      }
    } else {
      if (f > ks) gemm_range(ks, f, false);               // solved rows of the ancestors
      for (int b = nblk - 1; b > code && ok;) {
        {
          // the factor block L(64b.., r0..)^T this item multiplies once block b is published
          // (rows 64b.. of columns r0..r0+nr: two 128-byte lines per column)
          const int rr = tid >> 1, q = b * DF_R + (tid & 1) * 32;
          if (rr < nr && q < ks) asm volatile("prefetch.global.L2 [%0];" :: "l"(F + q + (int64_t)(r0 + rr) * ld));
        }
        ok = df_wait(fl + (int64_t)b * gt, abort_word, &s_ok, spin);
        if (!ok) break;
        const int e = b - 1 == code ? code : df_ready_run(fl, gt, b, code, false, &s_e);
        // the run downward: the partial sums go into tot in descending block order whatever
        // runs the blocks were published in (deterministic)
        gemm_range((e + 1) * DF_R, min(ks, (b + 1) * DF_R), true);
        b = e;
      }
    }
    if (!ok) return;                                      // uniform: s_ok after a barrier
    if (!tri) {                                           // contribution rows: v - the products
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int r = ty * 8 + i;
        if (r >= nr) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int c = c0 + tx * 4 + j;
          if (c < m) V[(int64_t)(r0 + r) * vs + c] = -tot[i][j];
        }
      }
      __syncthreads();
      continue;
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int r = ty * 8 + i;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int cc = tx * 4 + j, c = c0 + cc;
        Vs[r][cc] = (r < nr && c < m) ? -tot[i][j] : 0.f;
      }
    }
    __syncthreads();
    // y = L_RR^-1 v (forward) or x = L_RR^-T v (backward) as one product with the staged
    // inverse, in place of the row-by-row substitution: the triangle ends the chain of the
    // front's blocks, and a product has no dependency from row to row.  A thread's eight
    // rows are four from the top (4ty..) and four from the bottom (60-4ty..), so that each
    // warp does the same share of the triangle (row r takes q <= r forward, q >= r backward);
    // the loop bounds are the warp's, and terms past a row's own bound multiply the stored
    // zeros of the inverse.
    {
      float o[8][4];
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) o[i][j] = 0.f;
      const int w = tid >> 5;                            // rows 8w.. and 56-8w.. (ty = 2w, 2w+1)
      auto term = [&](int q, bool top, bool bot) {
        float b[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) b[j] = Vs[q][tx * 4 + j];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          if (i < 4 ? !top : !bot) continue;
          const int r = i < 4 ? ty * 4 + i : 60 - ty * 4 + (i - 4);
          const float a = FWD ? Ls[r][q] : Ls[q][r];
#pragma unroll
          for (int j = 0; j < 4; ++j) o[i][j] += a * b[j];
        }
      };
      if (FWD) {
        const int qa = min(nr, 8 * w + 8), qb = min(nr, TS - 8 * w);
        int q = 0;
        for (; q < qa; ++q) term(q, true, true);
        for (; q < qb; ++q) term(q, false, true);
      } else {
        const int qa = min(nr, TS - 8 - 8 * w);
        int q = 8 * w;
        for (; q < qa; ++q) term(q, true, false);
        for (; q < nr; ++q) term(q, true, true);
      }
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int r = i < 4 ? ty * 4 + i : 60 - ty * 4 + (i - 4);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int c = c0 + tx * 4 + j;
          if (r < nr && c < m) V[(int64_t)(r0 + r) * vs + c] = o[i][j];
        }
      }
    }
    // the block barrier orders every thread's stores before thread 0's release store
    // (cumulative at gpu scope), which publishes the block to the acquiring readers
    __syncthreads();
    if (tid == 0) df_st_release(fl + (int64_t)code * gt, 1);
  }
}

// Inverse of the unit lower triangular 64 x 64 diagonal block of a triangle item (R of front
// t, rows [64R, 64R + nr) of the solved columns), for the dataflow sweeps: column j of
// L_RR^-1 by forward substitution on e_j (thread j), x_i = -sum_{j <= q < i} L_iq x_q in
// ascending q, zero outside the nr x nr block; stored row-major at the block's index.
__global__ void __launch_bounds__(TS) k_diag_inverse(const NodeDesc* __restrict__ nd, const NodeState* __restrict__ st,
                                                     const float* __restrict__ arena, const int2* __restrict__ items,
                                                     const int* __restrict__ blockbase, float* __restrict__ dinv) {
  const int2 itm = items[blockIdx.x];
  if (itm.y < 0) return;                               // contribution block
  const int t = itm.x, R = itm.y, j = threadIdx.x;
  const NodeDesc d = nd[t];
  const int r0 = R * TS, nr = min(TS, st[t].ksolve - r0);
  const float* F = arena + d.front_off;
  const int64_t ld = d.ld;
  __shared__ float Ls[TS][TS + 1];
  __shared__ float Xs[TS][TS + 1];
  for (int e = j; e < TS * TS; e += TS) {
    const int r = e % TS, cc = e / TS;
    Ls[r][cc] = (r < nr && cc < nr && r > cc) ? F[(r0 + r) + (int64_t)(r0 + cc) * ld] : 0.f;
  }
  __syncthreads();
  for (int i = 0; i < TS; ++i) {
    float v = i == j ? 1.f : 0.f;
    for (int q = j; q < i; ++q) v -= Ls[i][q] * Xs[q][j];
    Xs[i][j] = (i < nr && j < nr) ? v : 0.f;
  }
  __syncthreads();
  float* D = dinv + ((int64_t)blockbase[t] + R) * (TS * TS);
  for (int e = j; e < TS * TS; e += TS) D[e] = Xs[e / TS][e % TS];
}

// r (FP64) -> lower precision with Lambda_2 rows zeroed (the cast of Sec. 3.1)
template <typename TV>
__global__ void k_cast_in(int64_t n, int m, const double* __restrict__ R, const int32_t* __restrict__ lam2pos,
                          TV* __restrict__ out) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * m) return;
  int64_t i = e / m;
  out[e] = (lam2pos && lam2pos[i] >= 0) ? TV(0) : (TV)R[e];
}

template <typename TV>
__global__ void k_cast_out(int64_t n, int m, const TV* __restrict__ Xl, const int32_t* __restrict__ lam2pos,
                           double* __restrict__ W) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * m) return;
  int64_t i = e / m;
  W[e] = (lam2pos && lam2pos[i] >= 0) ? 0.0 : (double)Xl[e];
}

// set X rows of Lambda_2 from x2 (M x m) or to zero
template <typename TV>
__global__ void k_set_lam2(int M, int m, const int32_t* __restrict__ lam2, const double* __restrict__ x2,
                           TV* __restrict__ X) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= M * m) return;
  int i = e / m, c = e - i * m;
  X[(int64_t)lam2[i] * m + c] = x2 ? (TV)x2[e] : TV(0);
}

template <typename TV>
__global__ void k_get_lam2(int M, int m, const int32_t* __restrict__ lam2, const TV* __restrict__ Y,
                           double* __restrict__ y2) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= M * m) return;
  int i = e / m, c = e - i * m;
  y2[e] = (double)Y[(int64_t)lam2[i] * m + c];
}

// ---------------------------------------------------------------------------
// SpMM Z = K11 W (FP64, Sec. 3.5): one warp per row, lanes over the rhs
// ---------------------------------------------------------------------------
__global__ void k_spmm(int64_t L, int m, const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                       const double* __restrict__ val, const int32_t* __restrict__ lam2pos,
                       const double* __restrict__ W, double* __restrict__ Z) {
  int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (row >= L) return;
  const bool skip = lam2pos[row] >= 0;
  for (int c0 = 0; c0 < m; c0 += 32) {
    int c = c0 + lane;
    double acc = 0.0;
    if (!skip) {
      for (int64_t e = rowptr[row]; e < rowptr[row + 1]; ++e) {
        int j = col[e];
        if (c < m) acc += val[e] * W[(int64_t)j * m + c];
      }
    }
    if (c < m) Z[row * m + c] = acc;
  }
}

// zero the columns of a row-major L x m block whose mask entry is set (deflation)
__global__ void k_zero_cols(int64_t L, int m, const int* __restrict__ mask, double* __restrict__ R) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= L * m) return;
  if (mask[e % m]) R[e] = 0.0;
}

// R = B - Z (elementwise)
__global__ void k_sub(int64_t n, const double* __restrict__ B, const double* __restrict__ Z, double* __restrict__ R) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < n) R[e] = B[e] - Z[e];
}

// ---------------------------------------------------------------------------
// Block Gram G = A^T B (A: L x ma, B: L x mb, row-major), two-stage deterministic
// ---------------------------------------------------------------------------
constexpr int GR = 32;     // rows per tile
constexpr int GO = 32;     // output block edge

__global__ void k_gram_partial(int64_t L, int ma, int mb, const double* __restrict__ A, const double* __restrict__ B,
                               double* __restrict__ part, int nchunks, int sym) {
  __shared__ double As[GR][GO + 1];
  __shared__ double Bs[GR][GO + 1];
  const int ob = blockIdx.y;                       // output block
  const int nbb = (mb + GO - 1) / GO;
  const int a0 = (ob / nbb) * GO, b0 = (ob % nbb) * GO;
  if (sym && a0 > b0) return;                      // A^T A: lower blocks mirror the upper ones
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // 32 x 8 threads
  double acc[4] = {0, 0, 0, 0};
  const int64_t rows_per = (L + nchunks - 1) / nchunks;
  const int64_t r_begin = (int64_t)blockIdx.x * rows_per, r_end = min(L, r_begin + rows_per);
  for (int64_t r0 = r_begin; r0 < r_end; r0 += GR) {
    for (int e = threadIdx.x; e < GR * GO; e += blockDim.x) {
      int rr = e / GO, cc = e % GO;
      int64_t r = r0 + rr;
      As[rr][cc] = (r < r_end && a0 + cc < ma) ? A[r * ma + a0 + cc] : 0.0;
      Bs[rr][cc] = (r < r_end && b0 + cc < mb) ? B[r * mb + b0 + cc] : 0.0;
    }
    __syncthreads();
#pragma unroll 4
    for (int rr = 0; rr < GR; ++rr) {
      double bv = Bs[rr][tx];
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[q] += As[rr][ty + 8 * q] * bv;
    }
    __syncthreads();
  }
  double* P = part + ((int64_t)blockIdx.y * gridDim.x + blockIdx.x) * GO * GO;
#pragma unroll
  for (int q = 0; q < 4; ++q) P[(ty + 8 * q) * GO + tx] = acc[q];
}

// Column sums of squares of a row-major L x m block: per row-chunk partials (pass 1),
// then a fixed-order reduction (pass 2), so the result does not depend on scheduling.
// Column sums of squares of a row-major L x m block over one chunk of rows per block: the
// CSQ_TH threads cover a window of w = min(m, CSQ_TH) columns on CSQ_TH / w rows at a time
// (consecutive threads read consecutive entries, and many rows are in flight); the row
// lanes' partial sums are added in lane order (deterministic).
constexpr int CSQ_TH = 512;
__global__ void __launch_bounds__(CSQ_TH) k_colsq_partial(int64_t L, int m, const double* __restrict__ A,
                                                         double* __restrict__ part) {
  __shared__ double sp[CSQ_TH];
  const int w = min(m, CSQ_TH), rpi = CSQ_TH / w;
  const int tid = threadIdx.x, jr = tid / w, jc = tid % w;
  const int64_t rows = (L + gridDim.x - 1) / gridDim.x;
  const int64_t r0 = (int64_t)blockIdx.x * rows, r1 = min(L, r0 + rows);
  for (int c0 = 0; c0 < m; c0 += w) {
    const int j = c0 + jc;
    double s = 0.0;
    if (jr < rpi && j < m)
      for (int64_t r = r0 + jr; r < r1; r += rpi) { const double v = A[r * m + j]; s += v * v; }
    sp[tid] = s;
    __syncthreads();
    if (tid < w && c0 + tid < m) {
      double t = 0.0;
      for (int q = 0; q < rpi; ++q) t += sp[q * w + tid];
      part[(int64_t)blockIdx.x * m + c0 + tid] = t;
    }
    __syncthreads();
  }
}

__global__ void k_colsq_reduce(int m, int nchunks, const double* __restrict__ part, double* __restrict__ out) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= m) return;
  double s = 0.0;
  for (int c = 0; c < nchunks; ++c) s += part[(int64_t)c * m + j];
  out[j] = s;
}

__global__ void k_gram_reduce(int ma, int mb, int nchunks, const double* __restrict__ part, double* __restrict__ G,
                              double scale, int sym) {
  const int nbb = (mb + GO - 1) / GO;
  const int nob = ((ma + GO - 1) / GO) * nbb;
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nob * GO * GO) return;
  int ob = e / (GO * GO), w = e % (GO * GO);
  int ab = ob / nbb, bb = ob % nbb;
  if (sym && ab > bb) return;
  int a = ab * GO + w / GO, b = bb * GO + w % GO;
  if (a >= ma || b >= mb) return;
  double s = 0.0;
  const double* P = part + (int64_t)ob * nchunks * GO * GO + w;
  for (int c = 0; c < nchunks; ++c) s += P[(int64_t)c * GO * GO];
  G[a * mb + b] = scale * s;
  if (sym && ab < bb) G[b * mb + a] = scale * s;
}

// ---------------------------------------------------------------------------
// Small SPD matrices of block GCR: M = Q^T Q = R^T R by a right-looking Cholesky in
// one CTA (in place, upper triangle R); a pivot below 1e-13 of its own diagonal marks a
// dependent direction, which is dropped (its row of R is zero and its coefficients are 0).
// Solves R^T R C = Y run one warp per column of Y with warp-shuffle dot products.
// ---------------------------------------------------------------------------
// ---------------------------------------------------------------------------
// Cholesky M = R^T R of the small SPD Gram (upper R, row-major), dropping directions whose
// pivot fell below 1e-13 of the original diagonal (reading R8), and the two triangular
// solves C = R^-1 R^-T Y; blocked by CB rows and spread over all SMs: cooperative kernels with grid-wide barriers between
// the phases of a block step (GB300 runs about two FP64 FMAs per clock per SM, so the
// O(m^3) FP64 work of one SM took milliseconds at m ~ 400).
// ---------------------------------------------------------------------------
constexpr int CB = 32;

__global__ void __launch_bounds__(256) k_chol_coop(int m, double* __restrict__ A, int* __restrict__ drop) {
  namespace cg = cooperative_groups;
  cg::grid_group grid = cg::this_grid();
  __shared__ double s_rjj;
  __shared__ int s_drop;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int gtid = blockIdx.x * nt + tid, gnt = gridDim.x * nt;
  double* dref = (double*)(drop + 2 * ((m + 1) / 2) + 2);
  for (int j = gtid; j < m; j += gnt) dref[j] = A[j * m + j];
  grid.sync();
  for (int jb = 0; jb < m; jb += CB) {
    const int je = min(m, jb + CB);
    // 1. the diagonal block, right-looking inside the block (block 0)
    if (blockIdx.x == 0) {
      for (int j = jb; j < je; ++j) {
        if (tid == 0) {
          const double sj = A[j * m + j];
          const double ref = dref[j];
          const int dz = !(sj > 1e-13 * ref) || !(ref > 0);
          drop[j] = dz;
          s_drop = dz;
          s_rjj = dz ? 0.0 : sqrt(sj);
          A[j * m + j] = s_rjj;
        }
        __syncthreads();
        const double rjj = s_rjj;
        const int dz = s_drop;
        for (int l = j + 1 + tid; l < je; l += nt) A[j * m + l] = dz ? 0.0 : A[j * m + l] / rjj;
        __syncthreads();
        if (!dz) {
          const int n2 = je - j - 1;
          for (int e = tid; e < n2 * n2; e += nt) {
            const int a = j + 1 + e / n2, b = j + 1 + e % n2;
            if (b >= a) A[a * m + b] -= A[j * m + a] * A[j * m + b];
          }
        }
        __syncthreads();
      }
    }
    grid.sync();
    // 2. rows [jb, je) right of the block: forward substitution with the block, per column
    for (int l = je + gtid; l < m; l += gnt) {
      double x[CB];
#pragma unroll
      for (int u = 0; u < CB; ++u) {
        const int j = jb + u;
        if (j < je) {
          double v = A[j * m + l];
#pragma unroll
          for (int w = 0; w < u; ++w) v -= A[(jb + w) * m + j] * x[w];
          x[u] = drop[j] ? 0.0 : v / A[j * m + j];
          A[j * m + l] = x[u];
        }
      }
    }
    grid.sync();
    // 3. trailing update of the upper triangle [je, m)^2
    const int n2 = m - je;
    for (int64_t e = gtid; e < (int64_t)n2 * n2; e += gnt) {
      const int a = je + (int)(e / n2), b = je + (int)(e % n2);
      if (b < a) continue;
      double acc = 0.0;
      for (int k = jb; k < je; ++k) acc += A[k * m + a] * A[k * m + b];
      A[a * m + b] -= acc;
    }
    grid.sync();
  }
}

// C = R^-1 R^-T Y (dropped directions give zero rows), m x ny row-major, blocked by CB
// rows.  The right-hand sides are independent: block b solves the columns [b cpb, (b+1) cpb)
// alone (block barriers only); per element the operations and their order are those of the
// blocked substitution (diagonal block solved in registers, then the rows below (above)
// updated by the CB-term dot product of the block).
__global__ void __launch_bounds__(256) k_chol_solve_cols(int m, int ny, int cpb, const double* __restrict__ R,
                                                       const int* __restrict__ drop, const double* __restrict__ Y,
                                                       double* __restrict__ C) {
  const int c0 = blockIdx.x * cpb, c1 = min(ny, c0 + cpb);
  const int nc = c1 - c0;
  if (nc <= 0) return;
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int e = tid; e < m * nc; e += nt) {
    const int64_t x = (int64_t)(e / nc) * ny + c0 + e % nc;
    C[x] = Y[x];
  }
  __syncthreads();
  // forward: R^T z = y
  for (int jb = 0; jb < m; jb += CB) {
    const int je = min(m, jb + CB);
    if (tid < nc) {
      const int c = c0 + tid;
      double x[CB];
#pragma unroll
      for (int u = 0; u < CB; ++u) {
        const int j = jb + u;
        if (j < je) {
          double v = C[(int64_t)j * ny + c];
#pragma unroll
          for (int w = 0; w < u; ++w) v -= R[(jb + w) * m + j] * x[w];
          x[u] = drop[j] ? 0.0 : v / R[j * m + j];
          C[(int64_t)j * ny + c] = x[u];
        }
      }
    }
    __syncthreads();
    const int nr = m - je;
    for (int e = tid; e < nr * nc; e += nt) {
      const int i = je + e / nc, c = c0 + e % nc;
      double acc = 0.0;
      for (int k = jb; k < je; ++k) acc += R[k * m + i] * C[(int64_t)k * ny + c];
      C[(int64_t)i * ny + c] -= acc;
    }
    __syncthreads();
  }
  // backward: R x = z, blocks from the bottom
  for (int je = m; je > 0; je -= CB) {
    const int jb = max(0, je - CB);
    if (tid < nc) {
      const int c = c0 + tid;
      double x[CB];
#pragma unroll
      for (int u = CB - 1; u >= 0; --u) {
        const int j = jb + u;
        if (j < je) {
          double v = C[(int64_t)j * ny + c];
#pragma unroll
          for (int w = u + 1; w < CB; ++w)
            if (jb + w < je) v -= R[j * m + jb + w] * x[w];
          x[u] = drop[j] ? 0.0 : v / R[j * m + j];
          C[(int64_t)j * ny + c] = x[u];
        }
      }
    }
    __syncthreads();
    for (int e = tid; e < jb * nc; e += nt) {
      const int i = e / nc, c = c0 + e % nc;
      double acc = 0.0;
      for (int k = jb; k < je; ++k) acc += R[i * m + k] * C[(int64_t)k * ny + c];
      C[(int64_t)i * ny + c] -= acc;
    }
    __syncthreads();
  }
}

// Y(+)= sgn * A C  (A: L x m, C: m x m); when Yinit is given Y = Yinit + sgn * A C
__global__ void k_block_axpy(int64_t L, int m, const double* __restrict__ A, const double* __restrict__ Cm,
                             double* __restrict__ Y, const double* __restrict__ Yinit, double sgn, int use_smem) {
  extern __shared__ double Csm[];
  const double* Cs = Cm;
  if (use_smem) {
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) Csm[e] = Cm[e];
    __syncthreads();
    Cs = Csm;
  }
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= L * m) return;
  int64_t i = e / m;
  int c = (int)(e - i * m);
  double s = 0.0;
  const double* a = A + i * m;
  for (int k = 0; k < m; ++k) s += a[k] * Cs[k * m + c];
  Y[e] = (Yinit ? Yinit[e] : Y[e]) + sgn * s;
}

// ---------------------------------------------------------------------------
// K12 block (Alg. 1 step 2): B[j, c] = K[j, lam2[c]] for j in Lambda_1 (K symmetric)
// ---------------------------------------------------------------------------
__global__ void k_extract_k12(int M, const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                              const double* __restrict__ val, const int32_t* __restrict__ lam2,
                              const int32_t* __restrict__ lam2pos, double* __restrict__ B) {
  int c = blockIdx.x;
  int g = lam2[c];
  for (int64_t e = rowptr[g] + threadIdx.x; e < rowptr[g + 1]; e += blockDim.x) {
    int j = col[e];
    if (lam2pos[j] < 0) B[(int64_t)j * M + c] = val[e];
  }
}

// S = K22 - K21 X   (S: M x m; X: L x m row-major). One warp per Lambda_2 row.
// mode 0: S = K22 - K21 X;  mode 1: S = Bbase(Lambda_2 rows) - K21 X;  mode 2: S = -K21 X
__global__ void k_schur_rows(int M, int m, const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                             const double* __restrict__ val, const int32_t* __restrict__ lam2,
                             const int32_t* __restrict__ lam2pos, const double* __restrict__ X,
                             const double* __restrict__ Bbase, int64_t ldb, double* __restrict__ S, int mode) {
  int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (i >= M) return;
  int g = lam2[i];
  for (int c0 = 0; c0 < m; c0 += 32) {
    int c = c0 + lane;
    double acc = 0.0;
    if (c < m) {
      if (mode == 1) acc = Bbase[(int64_t)g * ldb + c];
      for (int64_t e = rowptr[g]; e < rowptr[g + 1]; ++e) {
        int j = col[e];
        int p = lam2pos[j];
        if (p < 0) acc -= val[e] * X[(int64_t)j * m + c];
        else if (mode == 0 && p == c) acc += val[e];
      }
      S[i * m + c] = acc;
    }
  }
}

__global__ void k_symmetrize(int M, double* __restrict__ S) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= M * M) return;
  int i = e / M, j = e % M;
  if (j <= i) return;
  double v = 0.5 * (S[i * M + j] + S[j * M + i]);
  S[i * M + j] = v;
  S[j * M + i] = v;
}

// ---------------------------------------------------------------------------
// LDL^T of S22 (FP64) with complete symmetric (Bunch-Parlett) pivoting, 1x1 / 2x2
// blocks, alpha = (1+sqrt 17)/8 (reading R11), then kernel detection (R10).
// One CTA; A is the full symmetric working copy (M x M row-major).
// ---------------------------------------------------------------------------
__device__ void block_argmax(double& v, long long& key, double* rv, long long* rk) {
  // maximum of v; ties go to the smaller key
  for (int o = 16; o > 0; o >>= 1) {
    double ov = __shfl_xor_sync(0xffffffffu, v, o);
    long long ok = __shfl_xor_sync(0xffffffffu, key, o);
    if (ov > v || (ov == v && ok < key)) { v = ov; key = ok; }
  }
  if ((threadIdx.x & 31) == 0) { rv[threadIdx.x >> 5] = v; rk[threadIdx.x >> 5] = key; }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x + 31) / 32; ++w)
      if (rv[w] > v || (rv[w] == v && rk[w] < key)) { v = rv[w]; key = rk[w]; }
    rv[0] = v; rk[0] = key;
  }
  __syncthreads();
  v = rv[0]; key = rk[0];
  __syncthreads();
}

__device__ void bp_swap(double* A, double* Lf, int* perm, int M, int a, int b) {
  if (a == b) return;
  for (int j = threadIdx.x; j < M; j += blockDim.x) { double t = A[a * M + j]; A[a * M + j] = A[b * M + j]; A[b * M + j] = t; }
  __syncthreads();
  for (int i = threadIdx.x; i < M; i += blockDim.x) { double t = A[i * M + a]; A[i * M + a] = A[i * M + b]; A[i * M + b] = t; }
  for (int j = threadIdx.x; j < a; j += blockDim.x) { double t = Lf[a * M + j]; Lf[a * M + j] = Lf[b * M + j]; Lf[b * M + j] = t; }
  if (threadIdx.x == 0) { int t = perm[a]; perm[a] = perm[b]; perm[b] = t; }
  __syncthreads();
}

// Kernel detection after the S22 LDL^T (reading R10): magnitudes per 1x1 pivot / 2x2
// eigenvalue, sorted; the kernel is the tail after the largest ratio gap >= kernel_gap
// whose entries are below max(kernel_eps * scale, noise); one thread.
__device__ void bp_kernel_rule(int M, const int* __restrict__ blk, const double* __restrict__ dval,
                               int* __restrict__ nullp, double kernel_eps, double kernel_gap,
                               const int32_t* __restrict__ lam2, const int64_t* __restrict__ diagpos,
                               const double* __restrict__ kval, double noise, int* __restrict__ kdim_out,
                               double* __restrict__ mags_work) {
  double ref = 0.0;                // max |K_ii| over Lambda_2: the unit reference
  for (int i = 0; i < M; ++i) ref = fmax(ref, fabs(kval[diagpos[lam2[i]]]));
  double* mg = mags_work;          // M magnitudes, then M sorted copies
  for (int i = 0; i < M;) {
    if (blk[i] == 1) { mg[i] = fabs(dval[2 * i]); ++i; }
    else {
      double a = dval[2 * i], b = dval[2 * i + 1], c = dval[2 * (i + 1)];
      double mean = 0.5 * (a + c), rad = sqrt(0.25 * (a - c) * (a - c) + b * b);
      mg[i] = fabs(mean + rad); mg[i + 1] = fabs(mean - rad);
      i += 2;
    }
  }
  double* s = mg + M;
  for (int i = 0; i < M; ++i) s[i] = mg[i];
  for (int i = 1; i < M; ++i) {               // insertion sort, descending
    double v = s[i]; int j = i - 1;
    while (j >= 0 && s[j] < v) { s[j + 1] = s[j]; --j; }
    s[j + 1] = v;
  }
  int dim = 0;
  if (M > 0) {
    const double scale = fmax(s[0], ref);
    const double thr = fmax(kernel_eps * scale, noise);
    if (scale == 0.0 || s[0] <= thr) dim = M;
    else {
      double best = 0.0;
      for (int i = 1; i < M; ++i) {
        if (s[i] > thr) continue;
        double ratio = (s[i] == 0.0) ? INFINITY : s[i - 1] / s[i];
        if (ratio >= kernel_gap && ratio > best) { best = ratio; dim = M - i; }
      }
    }
  }
  *kdim_out = dim;
  // mark the `dim` smallest magnitudes as null pivots (ties: later position first)
  for (int cnt = 0; cnt < dim; ++cnt) {
    int bi = -1; double bv = INFINITY;
    for (int i = 0; i < M; ++i)
      if (!nullp[i] && (mg[i] < bv || (mg[i] == bv && i > bi))) { bv = mg[i]; bi = i; }
    if (bi >= 0) nullp[bi] = 1;
  }
}

// The same rule with all threads of one CTA and shared-memory scratch (3 M doubles):
// magnitudes in parallel, a stable descending sort by ranks (rank of i = number of
// magnitudes larger, or equal at a smaller position), and the `dim` last entries of that
// order marked null -- the same positions the one-thread loop picks (smallest
// magnitudes, ties to the later position).
__device__ void bp_kernel_rule_block(int M, const int* __restrict__ blk, const double* __restrict__ dval,
                                     int* __restrict__ nullp, double kernel_eps, double kernel_gap,
                                     const int32_t* __restrict__ lam2, const int64_t* __restrict__ diagpos,
                                     const double* __restrict__ kval, double noise, int* __restrict__ kdim_out,
                                     double* __restrict__ scratch) {
  __shared__ double red[32];
  __shared__ int s_dim;
  double* mg = scratch;                 // M: magnitude per position
  double* srt = scratch + M;            // M: descending order
  int* rk = (int*)(scratch + 2 * M);    // M: rank of each position
  const int tid = threadIdx.x, nt = blockDim.x;
  double ref = 0.0;                     // max |K_ii| over Lambda_2: the unit reference
  for (int i = tid; i < M; i += nt) ref = fmax(ref, fabs(kval[diagpos[lam2[i]]]));
  for (int o = 16; o > 0; o >>= 1) ref = fmax(ref, __shfl_xor_sync(0xffffffffu, ref, o));
  if ((tid & 31) == 0) red[tid >> 5] = ref;
  for (int i = tid; i < M; i += nt) {
    if (blk[i] == 1) {
      mg[i] = fabs(dval[2 * i]);
    } else if (blk[i] == 2) {
      const double a = dval[2 * i], b = dval[2 * i + 1], c = dval[2 * (i + 1)];
      const double mean = 0.5 * (a + c), rad = sqrt(0.25 * (a - c) * (a - c) + b * b);
      mg[i] = fabs(mean + rad);
      mg[i + 1] = fabs(mean - rad);
    }
  }
  __syncthreads();
  if (tid == 0) for (int w = 1; w < (nt + 31) / 32; ++w) ref = fmax(ref, red[w]);
  for (int i = tid; i < M; i += nt) {
    const double v = mg[i];
    int r = 0;
    for (int j = 0; j < M; ++j) r += (mg[j] > v || (mg[j] == v && j < i)) ? 1 : 0;
    rk[i] = r;
    srt[r] = v;
  }
  __syncthreads();
  if (tid == 0) {
    int dim = 0;
    if (M > 0) {
      const double scale = fmax(srt[0], ref);
      const double thr = fmax(kernel_eps * scale, noise);
      if (scale == 0.0 || srt[0] <= thr) dim = M;
      else {
        double best = 0.0;
        for (int i = 1; i < M; ++i) {
          if (srt[i] > thr) continue;
          const double ratio = (srt[i] == 0.0) ? INFINITY : srt[i - 1] / srt[i];
          if (ratio >= kernel_gap && ratio > best) { best = ratio; dim = M - i; }
        }
      }
    }
    *kdim_out = dim;
    s_dim = dim;
  }
  __syncthreads();
  for (int i = tid; i < M; i += nt) nullp[i] = rk[i] >= M - s_dim ? 1 : 0;
}

__global__ void k_bunch_parlett(int M, double* __restrict__ A, double* __restrict__ Lf, int* __restrict__ perm,
                                int* __restrict__ blk, double* __restrict__ dval, int* __restrict__ nullp,
                                double kernel_eps, double kernel_gap, const int32_t* __restrict__ lam2,
                                const int64_t* __restrict__ diagpos, const double* __restrict__ kval,
                                double noise, int* __restrict__ kdim_out, double* __restrict__ mags_work) {
  __shared__ double rv[32];
  __shared__ long long rk[32];
  const int tid = threadIdx.x, nt = blockDim.x;
  const double alpha = (1.0 + sqrt(17.0)) / 8.0;
  for (int e = tid; e < M * M; e += nt) Lf[e] = ((e / M) == (e % M)) ? 1.0 : 0.0;
  for (int i = tid; i < M; i += nt) { perm[i] = i; blk[i] = 0; dval[2 * i] = 0; dval[2 * i + 1] = 0; nullp[i] = 0; }
  __syncthreads();
  int k = 0;
  while (k < M) {
    // mu0 = max |a_ii| (ties: smaller i); mu1 = max_{i>j} |a_ij| (ties: smaller j, then i)
    double mu0 = -1.0;
    long long i0 = 0x7fffffffffffffffLL;
    for (int i = k + tid; i < M; i += nt) {
      double v = fabs(A[i * M + i]);
      if (v > mu0 || (v == mu0 && i < i0)) { mu0 = v; i0 = i; }
    }
    block_argmax(mu0, i0, rv, rk);
    double mu1 = -1.0;
    long long key1 = 0x7fffffffffffffffLL;
    const int n2 = M - k;
    for (long long e = tid; e < (long long)n2 * n2; e += nt) {
      int j = k + (int)(e / n2), i = k + (int)(e % n2);
      if (i <= j) continue;
      double v = fabs(A[i * M + j]);
      long long kk = (long long)j * M + i;
      if (v > mu1 || (v == mu1 && kk < key1)) { mu1 = v; key1 = kk; }
    }
    block_argmax(mu1, key1, rv, rk);
    if (mu1 < 0) mu1 = 0.0;
    if (mu0 == 0.0 && mu1 == 0.0) {                 // the rest is exactly zero: zero 1x1 pivots
      if (tid == 0) { blk[k] = 1; dval[2 * k] = 0.0; }
      __syncthreads();
      k += 1;
      continue;
    }
    if (mu0 >= alpha * mu1) {
      bp_swap(A, Lf, perm, M, k, (int)i0);
      const double dk = A[k * M + k];
      if (tid == 0) { blk[k] = 1; dval[2 * k] = dk; }
      for (int i = k + 1 + tid; i < M; i += nt) Lf[i * M + k] = A[i * M + k] / dk;
      __syncthreads();
      const int m2 = M - k - 1;
      for (int e = tid; e < m2 * m2; e += nt) {
        int i = k + 1 + e / m2, j = k + 1 + e % m2;
        A[i * M + j] -= Lf[i * M + k] * A[j * M + k];
      }
      __syncthreads();
      k += 1;
    } else {
      const int bj = (int)(key1 / M), bi = (int)(key1 % M);
      bp_swap(A, Lf, perm, M, k, bj);
      bp_swap(A, Lf, perm, M, k + 1, bi);
      const double a = A[k * M + k], b = A[(k + 1) * M + k], c = A[(k + 1) * M + k + 1];
      const double det = a * c - b * b;
      if (tid == 0) { blk[k] = 2; blk[k + 1] = 0; dval[2 * k] = a; dval[2 * k + 1] = b; dval[2 * (k + 1)] = c; }
      for (int i = k + 2 + tid; i < M; i += nt) {
        double x0 = A[i * M + k], x1 = A[i * M + k + 1];
        Lf[i * M + k] = (x0 * c - x1 * b) / det;
        Lf[i * M + k + 1] = (x1 * a - x0 * b) / det;
      }
      __syncthreads();
      const int m2 = M - k - 2;
      for (int e = tid; e < m2 * m2; e += nt) {
        int i = k + 2 + e / m2, j = k + 2 + e % m2;
        A[i * M + j] -= Lf[i * M + k] * A[j * M + k] + Lf[i * M + k + 1] * A[j * M + k + 1];
      }
      __syncthreads();
      k += 2;
    }
  }
  if (tid == 0)
    bp_kernel_rule(M, blk, dval, nullp, kernel_eps, kernel_gap, lam2, diagpos, kval, noise, kdim_out, mags_work);
}

// ---------------------------------------------------------------------------
// The same Bunch-Parlett LDL^T (complete pivoting, alpha = (1+sqrt 17)/8, the same tie
// rules and the same physical row/column swaps, so the same pivot order), spread over all
// SMs: a cooperative kernel with grid-wide barriers between the phases of a pivot step.
// The two maxima use the bit patterns of |a| as integer keys (non-negative FP64 values
// order like their bit patterns; NaN is never chosen, as with the FP64 comparisons), so
// the O(M^2) search per step runs on the integer units instead of the FP64 pipe.
// ---------------------------------------------------------------------------
struct BpPart {
  long long v0, i0, v1, j1;      // max |a_ii| key and i; max |a_ij| (i > j) key and j*M+i
};

__device__ __forceinline__ long long abs_key(double x) {
  const long long b = __double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFLL;
  return b > 0x7FF0000000000000LL ? -1LL : b;
}

__device__ __forceinline__ void bp_better(long long& v, long long& k, long long ov, long long ok) {
  if (ov > v || (ov == v && ok < k)) { v = ov; k = ok; }
}

constexpr int BP_THREADS = 256;
constexpr int BP_MAX_M = 2048;   // Lf columns of a step staged in shared memory (2 x M doubles)

__global__ void __launch_bounds__(BP_THREADS) k_bp_coop(int M, double* __restrict__ A, double* __restrict__ Lf,
                                                        int* __restrict__ perm, int* __restrict__ blk,
                                                        double* __restrict__ dval, int* __restrict__ nullp,
                                                        double kernel_eps, double kernel_gap,
                                                        const int32_t* __restrict__ lam2,
                                                        const int64_t* __restrict__ diagpos,
                                                        const double* __restrict__ kval, double noise,
                                                        int* __restrict__ kdim_out, double* __restrict__ mags_work,
                                                        BpPart* __restrict__ parts) {
  namespace cg = cooperative_groups;
  cg::grid_group grid = cg::this_grid();
  extern __shared__ double lcol[];                 // 3 x M: the new Lf column(s) of the step; rule scratch
  __shared__ long long w0[BP_THREADS / 32], wi0[BP_THREADS / 32], w1[BP_THREADS / 32], wj1[BP_THREADS / 32];
  __shared__ int s_act, s_a, s_b;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int gtid = blockIdx.x * nt + tid, gnt = gridDim.x * nt;
  const double alpha = (1.0 + sqrt(17.0)) / 8.0;
  for (int64_t e = gtid; e < (int64_t)M * M; e += gnt) Lf[e] = ((e / M) == (e % M)) ? 1.0 : 0.0;
  for (int i = gtid; i < M; i += gnt) { perm[i] = i; blk[i] = 0; dval[2 * i] = 0; dval[2 * i + 1] = 0; nullp[i] = 0; }
  grid.sync();
  // the symmetric swap of positions a < b (rows, then columns, as one set of disjoint pair
  // exchanges), the rows of Lf left of a, and perm
  auto swap_pos = [&](int a, int b) {
    if (a == b) return;
    const int np = 2 * M + a;
    for (int e = gtid; e < np; e += gnt) {
      int64_t x, y;
      if (e < M) {                                 // row pairs (a, j) <-> (b, j), j not in {a, b}
        const int j = e;
        if (j == a || j == b) continue;
        x = (int64_t)a * M + j; y = (int64_t)b * M + j;
      } else if (e < 2 * M) {                      // column pairs (i, a) <-> (i, b)
        const int i = e - M;
        if (i == a || i == b) {
          if (i != a) continue;                    // the 2 x 2 corner once: (a,a)<->(b,b), (a,b)<->(b,a)
          double t = A[(int64_t)a * M + a]; A[(int64_t)a * M + a] = A[(int64_t)b * M + b]; A[(int64_t)b * M + b] = t;
          t = A[(int64_t)a * M + b]; A[(int64_t)a * M + b] = A[(int64_t)b * M + a]; A[(int64_t)b * M + a] = t;
          continue;
        }
        x = (int64_t)i * M + a; y = (int64_t)i * M + b;
      } else {                                     // Lf rows left of a
        const int j = e - 2 * M;
        const double t = Lf[(int64_t)a * M + j]; Lf[(int64_t)a * M + j] = Lf[(int64_t)b * M + j]; Lf[(int64_t)b * M + j] = t;
        continue;
      }
      const double t = A[x]; A[x] = A[y]; A[y] = t;
    }
    if (gtid == 0) { const int t = perm[a]; perm[a] = perm[b]; perm[b] = t; }
  };
  int k = 0, it = 0;
  while (k < M) {
    BpPart* pp = parts + (it & 1) * gridDim.x;
    // 1. the two maxima, per block
    long long v0 = -1, i0 = 0x7fffffffffffffffLL, v1 = -1, j1 = 0x7fffffffffffffffLL;
    for (int i = k + gtid; i < M; i += gnt) bp_better(v0, i0, abs_key(A[(int64_t)i * M + i]), i);
    const int n2 = M - k;
    for (int e = gtid; e < n2 * n2; e += gnt) {                   // n2^2 < 2^31 for M <= BP_MAX_M
      const int j = k + e / n2, i = k + e % n2;
      if (i <= j) continue;
      bp_better(v1, j1, abs_key(A[(int64_t)i * M + j]), (long long)j * M + i);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      bp_better(v0, i0, __shfl_xor_sync(0xffffffffu, v0, o), __shfl_xor_sync(0xffffffffu, i0, o));
      bp_better(v1, j1, __shfl_xor_sync(0xffffffffu, v1, o), __shfl_xor_sync(0xffffffffu, j1, o));
    }
    if ((tid & 31) == 0) { w0[tid >> 5] = v0; wi0[tid >> 5] = i0; w1[tid >> 5] = v1; wj1[tid >> 5] = j1; }
    __syncthreads();
    if (tid == 0) {
      for (int w = 1; w < nt / 32; ++w) { bp_better(v0, i0, w0[w], wi0[w]); bp_better(v1, j1, w1[w], wj1[w]); }
      pp[blockIdx.x] = BpPart{v0, i0, v1, j1};
    }
    grid.sync();
    // 2. the decision, the same in every block
    if (tid == 0) {
      long long g0 = -1, gi = 0x7fffffffffffffffLL, g1 = -1, gj = 0x7fffffffffffffffLL;
      for (int b = 0; b < (int)gridDim.x; ++b) { bp_better(g0, gi, pp[b].v0, pp[b].i0); bp_better(g1, gj, pp[b].v1, pp[b].j1); }
      const double mu0 = g0 < 0 ? -1.0 : __longlong_as_double(g0);
      double mu1 = g1 < 0 ? -1.0 : __longlong_as_double(g1);
      if (mu1 < 0) mu1 = 0.0;
      int act;
      if (mu0 == 0.0 && mu1 == 0.0) act = 0;            // the rest is exactly zero: zero 1x1 pivots
      else if (mu0 >= alpha * mu1) act = 1;
      else act = 2;
      s_act = act;
      s_a = act == 1 ? (int)gi : (int)(gj / M);
      s_b = act == 2 ? (int)(gj % M) : 0;
    }
    __syncthreads();
    const int act = s_act;
    if (act == 0) {
      if (gtid == 0) { blk[k] = 1; dval[2 * k] = 0.0; }
      k += 1; ++it;
      continue;
    }
    if (act == 1) {
      swap_pos(k, s_a);
      grid.sync();
      const double dk = A[(int64_t)k * M + k];
      if (gtid == 0) { blk[k] = 1; dval[2 * k] = dk; }
      for (int i = k + 1 + tid; i < M; i += nt) {
        const double l = A[(int64_t)i * M + k] / dk;
        lcol[i] = l;
        if (blockIdx.x == 0) Lf[(int64_t)i * M + k] = l;
      }
      __syncthreads();
      const int m2 = M - k - 1;
      for (int e = gtid; e < m2 * m2; e += gnt) {
        const int i = k + 1 + e / m2, j = k + 1 + e % m2;
        A[(int64_t)i * M + j] -= lcol[i] * A[(int64_t)j * M + k];
      }
      grid.sync();
      k += 1; ++it;
    } else {
      swap_pos(k, s_a);
      grid.sync();
      swap_pos(k + 1, s_b);
      grid.sync();
      const double a = A[(int64_t)k * M + k], b = A[(int64_t)(k + 1) * M + k], cc = A[(int64_t)(k + 1) * M + k + 1];
      const double det = a * cc - b * b;
      if (gtid == 0) { blk[k] = 2; blk[k + 1] = 0; dval[2 * k] = a; dval[2 * k + 1] = b; dval[2 * (k + 1)] = cc; }
      for (int i = k + 2 + tid; i < M; i += nt) {
        const double x0 = A[(int64_t)i * M + k], x1 = A[(int64_t)i * M + k + 1];
        const double l0 = (x0 * cc - x1 * b) / det, l1 = (x1 * a - x0 * b) / det;
        lcol[i] = l0;
        lcol[M + i] = l1;
        if (blockIdx.x == 0) { Lf[(int64_t)i * M + k] = l0; Lf[(int64_t)i * M + k + 1] = l1; }
      }
      __syncthreads();
      const int m2 = M - k - 2;
      for (int e = gtid; e < m2 * m2; e += gnt) {
        const int i = k + 2 + e / m2, j = k + 2 + e % m2;
        A[(int64_t)i * M + j] -= lcol[i] * A[(int64_t)j * M + k] + lcol[M + i] * A[(int64_t)j * M + k + 1];
      }
      grid.sync();
      k += 2; ++it;
    }
  }
  grid.sync();
  if (blockIdx.x == 0)
    bp_kernel_rule_block(M, blk, dval, nullp, kernel_eps, kernel_gap, lam2, diagpos, kval, noise, kdim_out, lcol);
  (void)mags_work;
}

// Null vectors of S22 from its LDL^T (one CTA): for every null pivot direction v (e_i for
// a 1x1 null pivot, the eigenvector of the null eigenvalue of a 2x2 block), y = Lf^-T v
// and n2 = P y, so that S22 n2 = P Lf D v = 0 up to the null pivot.  N2: M x kdim,
// column-major; w: M doubles of work.
__global__ void k_s22_nullvecs(int M, const double* __restrict__ Lf, const int* __restrict__ perm,
                               const int* __restrict__ blk, const double* __restrict__ dval,
                               const int* __restrict__ nullp, int kdim, double* __restrict__ N2,
                               double* __restrict__ w) {
  const int tid = threadIdx.x, nt = blockDim.x;
  __shared__ int s_pos;
  int d = 0;
  for (int i = 0; i < M && d < kdim; ++i) {
    if (!nullp[i]) continue;
    // v: the null direction at position i (within its pivot block)
    for (int e = tid; e < M; e += nt) w[e] = 0.0;
    __syncthreads();
    if (tid == 0) {
      const int start = (blk[i] == 0) ? i - 1 : i;   // second row of a 2x2 belongs to the block at i-1
      if (blk[start] == 1) {
        w[i] = 1.0;
      } else {
        const double a = dval[2 * start], b = dval[2 * start + 1], cc = dval[2 * (start + 1)];
        const double mean = 0.5 * (a + cc), rad = sqrt(0.25 * (a - cc) * (a - cc) + b * b);
        const int q = i - start;                       // eigenvalue mean + rad (q = 0) or mean - rad
        const double ev = q == 0 ? mean + rad : mean - rad;
        double vx = b, vy = ev - a;
        if (fabs(vx) + fabs(vy) < 1e-300) { vx = ev - cc; vy = b; }
        if (fabs(vx) + fabs(vy) < 1e-300) { vx = (q == 0) ? 1.0 : 0.0; vy = (q == 0) ? 0.0 : 1.0; }
        const double nr = sqrt(vx * vx + vy * vy);
        w[start] = vx / nr;
        w[start + 1] = vy / nr;
      }
      s_pos = d;
    }
    __syncthreads();
    // y = Lf^-T w, from the last row up (Lf unit lower, row-major)
    for (int j = M - 1; j >= 0; --j) {
      const double yj = w[j];
      __syncthreads();
      for (int r = tid; r < j; r += nt) w[r] -= Lf[(int64_t)j * M + r] * yj;
      __syncthreads();
    }
    for (int r = tid; r < M; r += nt) N2[(int64_t)s_pos * M + perm[r]] = w[r];
    __syncthreads();
    ++d;
  }
}

// Kernel basis of K-bar: column c = Q [-X12 n2_c ; n2_c] in original unknowns
// (X12: L x M row-major, zero on Lambda_2 rows; basis: L x kdim column-major, ld ldb).
__global__ void k_kernel_basis(int64_t L, int M, int kdim, const double* __restrict__ X12,
                               const double* __restrict__ N2, const int32_t* __restrict__ lam2pos,
                               const double* __restrict__ q, double* __restrict__ basis, int64_t ldb) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int c = blockIdx.y;
  if (r >= L || c >= kdim) return;
  const double* n2 = N2 + (int64_t)c * M;
  double x;
  const int p = lam2pos[r];
  if (p >= 0) {
    x = n2[p];
  } else {
    double acc = 0.0;
    for (int j = 0; j < M; ++j) acc += X12[r * M + j] * n2[j];
    x = -acc;
  }
  basis[(int64_t)c * ldb + r] = q[r] * x;
}

// ---------------------------------------------------------------------------
// The same Bunch-Parlett LDL^T with S22 resident in the distributed shared memory of a
// thread-block cluster: CTA r holds the rows [r R, (r+1) R) (FP64, row stride M).  Per
// pivot step two cluster barriers: (1) after every CTA pushed its two maxima (integer keys
// of |a|, the same tie rules); (2) after the moved rows were sent to their new owners and
// every CTA pushed, for its rows, the entries of the pivot column(s) before the
// permutation.  Each CTA then permutes its own rows and columns and updates them with the
// pivot column exactly as the one-CTA kernel does (same operations per element).
// ---------------------------------------------------------------------------
constexpr int BPC_THREADS = 512;
constexpr int BPC_CMAX = 16;
constexpr size_t BPC_SMEM = 200 * 1024;
constexpr int BPC_RMAX = 128;                        // rows per CTA

__global__ void __launch_bounds__(BPC_THREADS, 1)
k_bp_cluster(int M, int R, const double* __restrict__ S22, double* __restrict__ Lf, int* __restrict__ perm,
             int* __restrict__ blk, double* __restrict__ dval, int* __restrict__ nullp, double kernel_eps,
             double kernel_gap, const int32_t* __restrict__ lam2, const int64_t* __restrict__ diagpos,
             const double* __restrict__ kval, double noise, int* __restrict__ kdim_out,
             double* __restrict__ mags_work) {
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  extern __shared__ __align__(16) double bpc[];
  const int C = (int)cl.num_blocks(), rank = (int)cl.block_rank();
  const int tid = threadIdx.x, nt = blockDim.x;
  double* Arow = bpc;                               // R x M: own rows
  double* rowbuf = Arow + (size_t)R * M;            // 4 x M: incoming rows for own moved positions
  double* colbuf = rowbuf + 4 * (size_t)M;          // 2 x M: old pivot columns, by old row index
  double* newcol = colbuf + 2 * (size_t)M;          // 2 x M: new pivot columns, by new row index
  long long* slots = (long long*)(newcol + 2 * (size_t)M);   // [2][BPC_CMAX][4]
  __shared__ double ltmp[2 * BPC_RMAX];             // multipliers of the own rows
  __shared__ long long w0[BPC_THREADS / 32], wi0[BPC_THREADS / 32], w1[BPC_THREADS / 32], wj1[BPC_THREADS / 32];
  __shared__ int s_act, s_np, s_pos[4], s_src[4], s_colsrc[2];
  const int p0 = rank * R, p1 = min(M, p0 + R);
  auto owner = [&](int pos) { return pos / R; };
  const double alpha = (1.0 + sqrt(17.0)) / 8.0;
  for (int64_t e = tid; e < (int64_t)(p1 - p0) * M; e += nt) Arow[e] = S22[(int64_t)p0 * M + e];
  for (int64_t e = tid; e < (int64_t)(p1 - p0) * M; e += nt) {
    const int r = p0 + (int)(e / M), c = (int)(e % M);
    Lf[(int64_t)r * M + c] = (r == c) ? 1.0 : 0.0;
  }
  for (int i = p0 + tid; i < p1; i += nt) { perm[i] = i; blk[i] = 0; dval[2 * i] = 0; dval[2 * i + 1] = 0; nullp[i] = 0; }
  cl.sync();
  int k = 0, it = 0;
  while (k < M) {
    long long* sl = slots + (it & 1) * BPC_CMAX * 4;
    // 1. own maxima: max |a_ii| (i >= k, ties: smaller i); max |a_ij|, i > j >= k (ties: smaller j*M+i)
    long long v0 = -1, i0 = 0x7fffffffffffffffLL, v1 = -1, j1 = 0x7fffffffffffffffLL;
    for (int i = max(k, p0) + tid; i < p1; i += nt) bp_better(v0, i0, abs_key(Arow[(int64_t)(i - p0) * M + i]), i);
    {
      const int warp = tid >> 5, lane = tid & 31, nw = nt >> 5;   // warps over rows, lanes over columns
      for (int i = max(k, p0) + warp; i < p1; i += nw) {
        const double* row = Arow + (size_t)(i - p0) * M;
        for (int j = k + lane; j < i; j += 32) bp_better(v1, j1, abs_key(row[j]), (long long)j * M + i);
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      bp_better(v0, i0, __shfl_xor_sync(0xffffffffu, v0, o), __shfl_xor_sync(0xffffffffu, i0, o));
      bp_better(v1, j1, __shfl_xor_sync(0xffffffffu, v1, o), __shfl_xor_sync(0xffffffffu, j1, o));
    }
    if ((tid & 31) == 0) { w0[tid >> 5] = v0; wi0[tid >> 5] = i0; w1[tid >> 5] = v1; wj1[tid >> 5] = j1; }
    __syncthreads();
    if (tid == 0) {
      for (int w = 1; w < nt / 32; ++w) { bp_better(v0, i0, w0[w], wi0[w]); bp_better(v1, j1, w1[w], wj1[w]); }
      w0[0] = v0; wi0[0] = i0; w1[0] = v1; wj1[0] = j1;
    }
    __syncthreads();
    if (tid < C) {
      long long* d = cl.map_shared_rank(sl, tid) + rank * 4;
      d[0] = w0[0]; d[1] = wi0[0]; d[2] = w1[0]; d[3] = wj1[0];
    }
    cl.sync();                                                      // barrier 1
    // 2. the decision (identical in every CTA) and the position permutation sigma
    if (tid == 0) {
      long long g0 = -1, gi = 0x7fffffffffffffffLL, g1 = -1, gj = 0x7fffffffffffffffLL;
      for (int b = 0; b < C; ++b) { bp_better(g0, gi, sl[b * 4 + 0], sl[b * 4 + 1]); bp_better(g1, gj, sl[b * 4 + 2], sl[b * 4 + 3]); }
      const double mu0 = g0 < 0 ? -1.0 : __longlong_as_double(g0);
      double mu1 = g1 < 0 ? -1.0 : __longlong_as_double(g1);
      if (mu1 < 0) mu1 = 0.0;
      int act;
      if (mu0 == 0.0 && mu1 == 0.0) act = 0;
      else if (mu0 >= alpha * mu1) act = 1;
      else act = 2;
      s_act = act;
      // affected positions and their sources: content at pos[x] after the step = old content at src[x]
      int pos[4], src[4], np = 0;
      auto addp = [&](int p) { for (int x = 0; x < np; ++x) if (pos[x] == p) return; pos[np] = p; src[np] = p; ++np; };
      auto swp = [&](int a, int b) {                  // content exchange of positions a and b
        int xa = -1, xb = -1;
        for (int x = 0; x < np; ++x) { if (pos[x] == a) xa = x; if (pos[x] == b) xb = x; }
        const int t = src[xa]; src[xa] = src[xb]; src[xb] = t;
      };
      if (act == 1) { const int a = (int)gi; addp(k); addp(a); swp(k, a); }
      if (act == 2) {
        const int bj = (int)(gj / M), bi = (int)(gj % M);
        addp(k); addp(bj); addp(k + 1); addp(bi);
        swp(k, bj);
        swp(k + 1, bi);
      }
      s_np = act == 0 ? 0 : np;
      for (int x = 0; x < np; ++x) { s_pos[x] = pos[x]; s_src[x] = src[x]; }
      int ck = k, ck1 = k + 1;
      for (int x = 0; x < np; ++x) { if (pos[x] == k) ck = src[x]; if (pos[x] == k + 1) ck1 = src[x]; }
      s_colsrc[0] = ck;
      s_colsrc[1] = ck1;
    }
    __syncthreads();
    const int act = s_act, np = s_np;
    if (act == 0) {
      if (rank == 0 && tid == 0) { blk[k] = 1; dval[2 * k] = 0.0; }
      k += 1; ++it;
      continue;
    }
    const int ncol = act;                                           // pivot columns: 1 or 2
    // 3. pushes: moved rows to their new owners, old pivot columns (own rows) to everyone
    for (int x = 0; x < np; ++x) {
      const int pd = s_pos[x], ps = s_src[x];
      if (pd == ps || owner(ps) != rank) continue;
      double* dst = cl.map_shared_rank(rowbuf, owner(pd)) + (size_t)x * M;
      const double* srcrow = Arow + (size_t)(ps - p0) * M;
      for (int c = tid; c < M; c += nt) dst[c] = srcrow[c];
    }
    for (int e = tid; e < C * ncol * (p1 - p0); e += nt) {
      const int r = e / (ncol * (p1 - p0)), rem = e % (ncol * (p1 - p0));
      const int cidx = rem / (p1 - p0), i = p0 + rem % (p1 - p0);
      cl.map_shared_rank(colbuf, r)[(size_t)cidx * M + i] = Arow[(size_t)(i - p0) * M + s_colsrc[cidx]];
    }
    cl.sync();                                                      // barrier 2
    // 4. permute own rows (moved rows from rowbuf) and the affected columns of all own rows
    for (int x = 0; x < np; ++x) {
      const int pd = s_pos[x], ps = s_src[x];
      if (pd == ps || owner(pd) != rank) continue;
      double* drow = Arow + (size_t)(pd - p0) * M;
      for (int c = tid; c < M; c += nt) drow[c] = rowbuf[(size_t)x * M + c];
    }
    __syncthreads();
    for (int i = p0 + tid; i < p1; i += nt) {
      double* row = Arow + (size_t)(i - p0) * M;
      double tmp[4];
      for (int x = 0; x < np; ++x) tmp[x] = row[s_src[x]];
      for (int x = 0; x < np; ++x) row[s_pos[x]] = tmp[x];
    }
    // the new pivot column(s) for every row j: new A[j][k(+1)] = old A[sigma(j)][sigma(k(+1))]
    auto src_of = [&](int j) { for (int x = 0; x < np; ++x) if (s_pos[x] == j) return s_src[x]; return j; };
    __syncthreads();
    if (rank == 0) {
      // Lf rows of the moved positions, columns < k (the eliminated part)
      for (int x = 0; x < np; ++x) {
        if (s_pos[x] == s_src[x]) continue;
        for (int c = tid; c < k; c += nt) rowbuf[(size_t)x * M + c] = Lf[(int64_t)s_src[x] * M + c];
      }
      __syncthreads();
      for (int x = 0; x < np; ++x) {
        if (s_pos[x] == s_src[x]) continue;
        for (int c = tid; c < k; c += nt) Lf[(int64_t)s_pos[x] * M + c] = rowbuf[(size_t)x * M + c];
      }
      if (tid == 0) {
        int pv[4];
        for (int x = 0; x < np; ++x) pv[x] = perm[s_src[x]];
        for (int x = 0; x < np; ++x) perm[s_pos[x]] = pv[x];
      }
    }
    // the new pivot column(s) in old-row order -> new-row order (sigma applied once)
    for (int j = tid; j < M; j += nt) {
      const int sj = src_of(j);
      newcol[j] = colbuf[sj];
      if (act == 2) newcol[M + j] = colbuf[M + sj];
    }
    __syncthreads();
    const int ib = max(k + act, p0);                               // first own row updated
    if (act == 1) {
      const double dk = newcol[k];
      if (rank == 0 && tid == 0) { blk[k] = 1; dval[2 * k] = dk; }
      for (int i = ib + tid; i < p1; i += nt) {
        const double l = Arow[(size_t)(i - p0) * M + k] / dk;
        ltmp[i - p0] = l;
        Lf[(int64_t)i * M + k] = l;
      }
      __syncthreads();
      for (int i = ib + (tid >> 5); i < p1; i += nt >> 5) {
        double* row = Arow + (size_t)(i - p0) * M;
        const double l = ltmp[i - p0];
        for (int j = k + 1 + (tid & 31); j < M; j += 32) row[j] -= l * newcol[j];
      }
      k += 1;
    } else {
      const double a = newcol[k], b = newcol[k + 1], cc = newcol[M + k + 1];
      const double det = a * cc - b * b;
      if (rank == 0 && tid == 0) { blk[k] = 2; blk[k + 1] = 0; dval[2 * k] = a; dval[2 * k + 1] = b; dval[2 * (k + 1)] = cc; }
      for (int i = ib + tid; i < p1; i += nt) {
        const double* row = Arow + (size_t)(i - p0) * M;
        const double x0 = row[k], x1 = row[k + 1];
        const double l0 = (x0 * cc - x1 * b) / det, l1 = (x1 * a - x0 * b) / det;
        ltmp[i - p0] = l0;
        ltmp[BPC_RMAX + i - p0] = l1;
        Lf[(int64_t)i * M + k] = l0;
        Lf[(int64_t)i * M + k + 1] = l1;
      }
      __syncthreads();
      for (int i = ib + (tid >> 5); i < p1; i += nt >> 5) {
        double* row = Arow + (size_t)(i - p0) * M;
        const double l0 = ltmp[i - p0], l1 = ltmp[BPC_RMAX + i - p0];
        for (int j = k + 2 + (tid & 31); j < M; j += 32) row[j] -= l0 * newcol[j] + l1 * newcol[M + j];
      }
      k += 2;
    }
    ++it;
    __syncthreads();
  }
  cl.sync();
  if (rank == 0)
    bp_kernel_rule_block(M, blk, dval, nullp, kernel_eps, kernel_gap, lam2, diagpos, kval, noise, kdim_out, rowbuf);
  (void)mags_work;
}

constexpr size_t BKS_SMEM_MAX = 200 * 1024;  // largest shared work vector of k_bk_solve

// x = S22^+ y with null pivots treated as zero; y, x: M x m row-major.  One CTA per
// right-hand side; the work vector z sits in shared memory (zg == nullptr) or, when
// M doubles do not fit there, in the column c of the global M x m buffer zg.  The
// substitutions are column-oriented (one barrier per column, the updates of the
// other rows in parallel).
__global__ void __launch_bounds__(256) k_bk_solve(int M, int m, const double* __restrict__ Lf,
                                                const int* __restrict__ perm, const int* __restrict__ blk,
                                                const double* __restrict__ dval, const int* __restrict__ nullp,
                                                const double* __restrict__ y, double* __restrict__ x,
                                                double* zg) {
  extern __shared__ double zs[];
  const int c = blockIdx.x, tid = threadIdx.x, nt = blockDim.x;
  if (c >= m) return;
  double* z = zg ? zg + (int64_t)c * M : zs;
  for (int i = tid; i < M; i += nt) z[i] = y[(int64_t)perm[i] * m + c];
  __syncthreads();
  // Lf z' = z (unit lower): z_i -= Lf_ij z_j for j = 0, 1, ... in order
  for (int j = 0; j < M; ++j) {
    const double zj = z[j];
    for (int i = j + 1 + tid; i < M; i += nt) z[i] -= Lf[(int64_t)i * M + j] * zj;
    __syncthreads();
  }
  // D^+ (1x1: divide unless null; 2x2: eigen-decomposition, null eigenvalues dropped)
  for (int i = tid; i < M; i += nt) {
    if (blk[i] == 1) {
      const double dd = dval[2 * i];
      z[i] = (nullp[i] || dd == 0.0) ? 0.0 : z[i] / dd;
    } else if (blk[i] == 2) {
      const double a = dval[2 * i], b = dval[2 * i + 1], cc = dval[2 * (i + 1)];
      const double mean = 0.5 * (a + cc), rad = sqrt(0.25 * (a - cc) * (a - cc) + b * b);
      const double ev[2] = {mean + rad, mean - rad};
      double v[2][2];
      for (int q = 0; q < 2; ++q) {
        double vx = b, vy = ev[q] - a;
        if (fabs(vx) + fabs(vy) < 1e-300) { vx = ev[q] - cc; vy = b; }
        if (fabs(vx) + fabs(vy) < 1e-300) { vx = (q == 0) ? 1.0 : 0.0; vy = (q == 0) ? 0.0 : 1.0; }
        const double nr = sqrt(vx * vx + vy * vy);
        v[q][0] = vx / nr; v[q][1] = vy / nr;
      }
      const double z0 = z[i], z1 = z[i + 1];
      double o0 = 0.0, o1 = 0.0;
      for (int q = 0; q < 2; ++q) {
        if (nullp[i + q] || ev[q] == 0.0) continue;
        const double pr = (v[q][0] * z0 + v[q][1] * z1) / ev[q];
        o0 += v[q][0] * pr; o1 += v[q][1] * pr;
      }
      z[i] = o0;
      z[i + 1] = o1;
    }
  }
  __syncthreads();
  // Lf^T z'' = z' (from the last row up)
  for (int j = M - 1; j >= 0; --j) {
    const double zj = z[j];
    for (int i = tid; i < j; i += nt) z[i] -= Lf[(int64_t)j * M + i] * zj;
    __syncthreads();
  }
  for (int i = tid; i < M; i += nt) x[(int64_t)perm[i] * m + c] = z[i];
}

// x1 = y1 - X12 x2 on Lambda_1 rows; Lambda_2 rows = x2
__global__ void k_backsub_x1(int64_t L, int M, int m, const double* __restrict__ X12, const double* __restrict__ x2,
                             const int32_t* __restrict__ lam2pos, double* __restrict__ Y) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= L * m) return;
  int64_t i = e / m;
  int c = (int)(e - i * m);
  int p = lam2pos[i];
  if (p >= 0) { Y[e] = x2[p * m + c]; return; }
  double s = Y[e];
  for (int k = 0; k < M; ++k) s -= X12[i * M + k] * x2[k * m + c];
  Y[e] = s;
}

// user column-major b (ldb) -> internal row-major Q b ;  and back: x_user = Q x
__global__ void k_scale_in(int64_t L, int m, const double* __restrict__ b, int64_t ldb, const double* __restrict__ q,
                           double* __restrict__ out) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= L * m) return;
  int64_t i = e / m;
  int c = (int)(e - i * m);
  out[e] = q[i] * b[i + c * ldb];
}

__global__ void k_scale_out(int64_t L, int m, const double* __restrict__ xin, const double* __restrict__ q,
                            double* __restrict__ x, int64_t ldx) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= L * m) return;
  int64_t i = e % L;
  int c = (int)(e / L);
  x[i + c * ldx] = q[i] * xin[i * m + c];
}

__global__ void k_zero_lam2_rows(int M, int m, const int32_t* __restrict__ lam2, double* __restrict__ V) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= M * m) return;
  V[(int64_t)lam2[e / m] * m + (e % m)] = 0.0;
}

inline unsigned nblk(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

}  // namespace

int hf_oz_gram(hf_ctx* c, int64_t L, int ma, int mb, const double* A, const double* B, double* G, double scale,
               double* scratch, size_t scratch_bytes, void* slices, size_t slice_bytes, int* iscratch, int* err);
int hf_oz_update(hf_ctx* c, int64_t L, int m, const double* A, const double* C, double* Y, const double* Yinit,
                 double sgn, void* slices, size_t slice_bytes, int* iscratch, int* err);
size_t hf_oz_slice_bytes(int64_t R, int64_t K);
int64_t hf_oz_gram_chunks(int64_t L, int ma, int mb);

static int* oz_err(hf_ctx* c) { return (int*)c->d_flags.p + FLAG_COUNT + 10; }

static int oz_iscratch(hf_ctx* c, size_t n, int** p) {
  int rc = hf_ensure(c->d_ozint, n * 4 + 256);
  *p = (int*)c->d_ozint.p;
  return rc;
}

// ============================================================================
// Host drivers
// ============================================================================
struct Work {
  // Krylov workspace carved from ctx->d_work
  double *X, *R, *W, *Z, *B;
  double* P[64];
  double* Qv[64];
  double* Ms[64];
  int slots;
};

// The per-front vectors (row_elems x m), then the flags and tickets of the dataflow
// sweeps: [forward tickets | forward flags | backward tickets | backward flags], one
// ticket counter per level and one flag per (diagonal block, column tile).
static size_t sweep_vec_bytes(const hf_ctx* c, int m, size_t esz) {
  const size_t vs = (size_t)(m + 3) / 4 * 4;      // the dataflow sweeps pad the rows to 16 bytes
  return ((size_t)c->row_elems * vs * esz + 255) / 256 * 256;
}
static int sweep_tickets(const hf_ctx* c) { return (2 * (c->m + 1) + 63) / 64 * 64 / 2 + 32; }
static size_t sweep_half_ints(const hf_ctx* c, int m) {
  const size_t gt = (size_t)((m + DF_C - 1) / DF_C);
  return ((size_t)sweep_tickets(c) + (size_t)c->sw_blocks * gt + 63) / 64 * 64;
}
static size_t sweep_sync_bytes(const hf_ctx* c, int m) { return 2 * sweep_half_ints(c, m) * sizeof(int); }
static int* sweep_err(hf_ctx* c) { return (int*)c->d_flags.p + FLAG_COUNT + 11; }
// polls of a dataflow wait before it gives up (hf_opts.spin_limit, 0 = built in)
static int sweep_spin(const hf_ctx* c) { return c->opts.spin_limit > 0 ? c->opts.spin_limit : DF_SPIN; }

// Synchronises the stream; HF_ERR_TIMEOUT once a wait of a dataflow sweep has given up
// (the word stays set until the next factorization: the solves of this factor are void).
static int sweep_status(hf_ctx* c) {
  int h = 0;
  cudaStream_t s = hf_stream(c);
  HF_CUDA_TRY(cudaMemcpyAsync(&h, sweep_err(c), sizeof(int), cudaMemcpyDeviceToHost, s));
  HF_CUDA_TRY(cudaStreamSynchronize(s));
  return h ? HF_ERR_TIMEOUT : HF_OK;
}

static int ensure_vec(hf_ctx* c, int m, size_t esz) {
  size_t need = sweep_vec_bytes(c, m, esz) + sweep_sync_bytes(c, m) + 64;
  return hf_ensure(c->d_vec, need);
}

int hf_sweep_plan(hf_ctx* c) {
  const int nlev = c->m + 1;
  const int nt = (int)c->state_host.size();
  std::vector<int32_t> bb(nt + 1, 0);
  int blocks = 0;
  auto nblk = [&](int t) { return (c->state_host[t].ksolve + DF_R - 1) / DF_R; };
  for (int t = 0; t < nt; ++t) { bb[t] = blocks; blocks += nblk(t); }
  std::vector<int32_t> it;   // pairs (front, code)
  c->sw_fwd_start.assign(nlev, 0); c->sw_fwd_cnt.assign(nlev, 0);
  c->sw_bwd_start.assign(nlev, 0); c->sw_bwd_cnt.assign(nlev, 0);
  for (int lev = 0; lev < nlev; ++lev) {
    const int t0 = c->level_start[lev], cnt = c->level_count[lev];
    int maxb = 0;
    for (int t = t0; t < t0 + cnt; ++t) maxb = std::max(maxb, nblk(t));
    // forward: triangle blocks by ascending R, then the contribution blocks
    c->sw_fwd_start[lev] = (int)(it.size() / 2);
    for (int R = 0; R < maxb; ++R)
      for (int t = t0; t < t0 + cnt; ++t)
        if (nblk(t) > R) { it.push_back(t); it.push_back(R); }
    for (int t = t0; t < t0 + cnt; ++t) {
      if (nblk(t) == 0) continue;
      const int ncb = (c->state_host[t].f - c->state_host[t].ksolve + DF_R - 1) / DF_R;
      for (int j = 0; j < ncb; ++j) { it.push_back(t); it.push_back(-1 - j); }
    }
    c->sw_fwd_cnt[lev] = (int)(it.size() / 2) - c->sw_fwd_start[lev];
    // backward: triangle blocks by descending R
    c->sw_bwd_start[lev] = (int)(it.size() / 2);
    for (int R = maxb - 1; R >= 0; --R)
      for (int t = t0; t < t0 + cnt; ++t)
        if (nblk(t) > R) { it.push_back(t); it.push_back(R); }
    c->sw_bwd_cnt[lev] = (int)(it.size() / 2) - c->sw_bwd_start[lev];
  }
  c->sw_blocks = blocks;
  const size_t ib = it.size() * sizeof(int32_t), bbytes = bb.size() * sizeof(int32_t);
  int rc;
  if ((rc = hf_ensure(c->d_swplan, ib + bbytes + 256))) return rc;
  cudaStream_t s = hf_stream(c);
  if (ib) HF_CUDA_TRY(cudaMemcpyAsync(c->d_swplan.p, it.data(), ib, cudaMemcpyHostToDevice, s));
  HF_CUDA_TRY(cudaMemcpyAsync((char*)c->d_swplan.p + ib, bb.data(), bbytes, cudaMemcpyHostToDevice, s));
  HF_CUDA_TRY(cudaStreamSynchronize(s));   // the host vectors go out of scope
  return HF_OK;
}

// first diagonal block of every front (after the item pairs in d_swplan)
static const int* sweep_bbase(const hf_ctx* c) {
  size_t pairs = 0;
  if (!c->sw_bwd_start.empty()) pairs = (size_t)c->sw_bwd_start.back() + c->sw_bwd_cnt.back();
  return (const int*)((const char*)c->d_swplan.p + pairs * 2 * sizeof(int32_t));
}

// The inverses of every diagonal block of the FP32 factor, for the dataflow sweeps (one CTA
// per triangle item of the forward lists; called after hf_sweep_plan)
int hf_diag_inverses(hf_ctx* c) {
  if (c->prec == HF_PREC_FP64) return HF_OK;           // the FP64 factor uses the per-block sweeps
  int rc;
  if ((rc = hf_ensure(c->d_dinv, (size_t)std::max(1, c->sw_blocks) * TS * TS * sizeof(float) + 64))) return rc;
  cudaStream_t s = hf_stream(c);
  const int2* items = (const int2*)c->d_swplan.p;
  for (int lev = 0; lev <= c->m; ++lev) {
    const int ni = c->sw_fwd_cnt[lev];
    if (ni > 0)
      HF_LAUNCH(c, HF_PROF_DIAG_INV, k_diag_inverse<<<ni, TS, 0, s>>>((const NodeDesc*)c->d_nodes.p,
                                                                   (const NodeState*)c->d_state.p,
                                                                   (const float*)c->d_front.p,
                                                                   items + c->sw_fwd_start[lev], sweep_bbase(c),
                                                                   (float*)c->d_dinv.p));
  }
  HF_CUDA_TRY(cudaGetLastError());
  return HF_OK;
}

// CTAs of a dataflow sweep launch: all resident at once is not required, only useful
static int sweep_grid(bool fwd) {
  static std::mutex mu;
  static int per[2] = {0, 0}, sms = 0;
  std::lock_guard<std::mutex> lk(mu);
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    // errors show at the launch (cudaGetLastError after it)
    cudaFuncSetAttribute(k_sweep_df<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)DF_SMEM);
    cudaFuncSetAttribute(k_sweep_df<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)DF_SMEM);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per[0], k_sweep_df<false>, DF_TH, DF_SMEM);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per[1], k_sweep_df<true>, DF_TH, DF_SMEM);
    sms = std::max(sms, 1);
  }
  return sms * std::max(1, per[fwd ? 1 : 0]);
}

// HF_LEVEL_TIMES=1: device time of every level of the sweeps (diagnostic)
struct SweepTimer {
  cudaStream_t s;
  const char* name;
  int m;
  bool on;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  SweepTimer(cudaStream_t st, const char* nm, int mm) : s(st), name(nm), m(mm) {
    const char* v = std::getenv("HF_LEVEL_TIMES");
    on = v && v[0] == '1';
    if (on) { cudaEventCreate(&e0); cudaEventCreate(&e1); }
  }
  ~SweepTimer() { if (on) { cudaEventDestroy(e0); cudaEventDestroy(e1); } }
  void begin() { if (on) cudaEventRecord(e0, s); }
  void end(int lev, int cnt, int maxf, int maxks) {
    if (!on) return;
    float ms = 0;
    cudaEventRecord(e1, s);
    cudaEventSynchronize(e1);
    cudaEventElapsedTime(&ms, e0, e1);
    std::fprintf(stderr, "sweep %s m %d level %d: fronts %d max f %d max ks %d: %.3f ms\n", name, m, lev, cnt, maxf,
                 maxks, ms);
  }
};

// Largest front order, solved columns and contribution block of a level (host state)
struct LevelDims {
  int maxf = 0, maxks = 0, maxcb = 0;
};

static LevelDims level_dims(const hf_ctx* c, int lev) {
  LevelDims L;
  const int t0 = c->level_start[lev], cnt = c->level_count[lev];
  for (int t = t0; t < t0 + cnt; ++t) {
    const NodeState& S = c->state_host[t];
    L.maxf = std::max(L.maxf, S.f);
    L.maxks = std::max(L.maxks, S.ksolve);
    for (int ch : {c->nodes[t].child0, c->nodes[t].child1})
      if (ch >= 0) L.maxcb = std::max(L.maxcb, c->state_host[ch].f - c->state_host[ch].k);
  }
  return L;
}

static void sweep_work(hf_ctx* c, int cls, int m, size_t esz) {
  double ent = 0;
  for (const NodeState& S : c->state_host) ent += (double)S.f * S.ksolve - 0.5 * (double)S.ksolve * (S.ksolve + 1);
  c->work_flops[cls] += 2.0 * ent * m;
  c->work_bytes[cls] += ent * esz;
}

// HF_SWEEP_BLOCKED=1: the sweeps launch one GEMM per diagonal block (the form before
// the dataflow levels; diagnostic comparison)
static bool sweep_blocked() {
  const char* v = std::getenv("HF_SWEEP_BLOCKED");
  return v && v[0] == '1';
}

template <typename TF, typename TV>
static void fwd_sweep(hf_ctx* c, int m, const TV* Bin, TV* Ytmp, TV* vec) {
  cudaStream_t s = hf_stream(c);
  sweep_work(c, HF_PROF_TRSV_FWD, m, sizeof(TF));
  const NodeDesc* nd = (const NodeDesc*)c->d_nodes.p;
  const NodeState* st = (const NodeState*)c->d_state.p;
  const TF* arena = (const TF*)c->d_front.p;
  const int32_t* rowid = (const int32_t*)c->d_rowid.p;
  const int32_t* cbmap = (const int32_t*)c->d_cbmap.p;
  const unsigned gt = (unsigned)((m + SGC - 1) / SGC);
  constexpr bool DF = sizeof(TF) == 4 && sizeof(TV) == 4;   // dataflow levels (FP32 factor)
  static_assert(SGC == DF_C, "column tiles of both sweep forms");
  const bool use_df = DF && !sweep_blocked();
  const int vs = use_df ? (m + 3) / 4 * 4 : m;     // row stride of the per-front vectors
  const int2* items = (const int2*)c->d_swplan.p;
  const int* bbase = sweep_bbase(c);
  int* sync = (int*)((char*)vec + sweep_vec_bytes(c, m, sizeof(TV)));     // forward half
  if (use_df) (void)cudaMemsetAsync(sync, 0, sweep_half_ints(c, m) * sizeof(int), s);   // errors: cudaGetLastError
  int* flags = sync + sweep_tickets(c);
  SweepTimer tm(s, "fwd", m);
  for (int lev = c->m; lev >= 0; --lev) {
    const int t0 = c->level_start[lev], cnt = c->level_count[lev];
    const LevelDims D = level_dims(c, lev);
    tm.begin();
    const unsigned ex = (unsigned)std::min<int64_t>(std::max<int64_t>(1, (int64_t)D.maxf * m / 1024), 512);
    HF_LAUNCH(c, HF_PROF_SWEEP_IO, k_fwd_gather<TV><<<dim3(ex, cnt), 256, 0, s>>>(nd, st, t0, rowid,
                                                                                (const int32_t*)c->d_gmap.p,
                                                                                c->row_elems, vec, Bin, m, vs));
    (void)cbmap;
    if constexpr (DF) if (use_df) {
      const int ni = c->sw_fwd_cnt[lev];
      if (ni > 0) {
        const int g = (int)std::min<int64_t>((int64_t)ni * gt, sweep_grid(true));
        HF_LAUNCH(c, HF_PROF_TRSV_FWD, k_sweep_df<true><<<g, DF_TH, DF_SMEM, s>>>(nd, st, arena, vec, m, vs, (int)gt, items + c->sw_fwd_start[lev], ni,
                                                                          bbase, flags, sync + lev, sweep_err(c), sweep_spin(c),
                                                                          (const float*)c->d_dinv.p));
      }
      HF_LAUNCH(c, HF_PROF_SWEEP_IO, k_fwd_store<TF, TV><<<dim3(ex, cnt), 256, 0, s>>>(nd, st, t0, arena, rowid, vec, Ytmp, m, vs));
      tm.end(lev, cnt, D.maxf, D.maxks);
      continue;
    }
    const int nbk = (D.maxks + TS - 1) / TS;
    constexpr bool fused = sizeof(TV) == 4;          // next diagonal block solved inside the GEMM
    for (int b = 0; b < nbk; ++b) {
      if (b == 0 || !fused)
        HF_LAUNCH(c, HF_PROF_TRSV_FWD, k_trsm_diag<TF, TV, true><<<dim3((m + DiagRhs<TV>::value - 1) / DiagRhs<TV>::value, cnt), DTH, 0, s>>>(nd, st, t0, arena, vec, m, b));
      const unsigned rx = (unsigned)((D.maxf - b * TS + SGR - 1) / SGR);
      if (rx > 0)
        HF_LAUNCH(c, HF_PROF_TRSV_FWD, k_gemm_upd<TF, TV, 0, fused><<<dim3(rx, gt, cnt), SGTH, 0, s>>>(nd, st, t0, arena, vec, m, b));
    }
    HF_LAUNCH(c, HF_PROF_SWEEP_IO, k_fwd_store<TF, TV><<<dim3(ex, cnt), 256, 0, s>>>(nd, st, t0, arena, rowid, vec, Ytmp, m, vs));
    tm.end(lev, cnt, D.maxf, D.maxks);
  }
}

template <typename TF, typename TV>
static void bwd_sweep(hf_ctx* c, int m, const TV* Ytmp, TV* Xout, TV* vec) {
  cudaStream_t s = hf_stream(c);
  sweep_work(c, HF_PROF_TRSV_BWD, m, sizeof(TF));
  const NodeDesc* nd = (const NodeDesc*)c->d_nodes.p;
  const NodeState* st = (const NodeState*)c->d_state.p;
  const TF* arena = (const TF*)c->d_front.p;
  const int32_t* rowid = (const int32_t*)c->d_rowid.p;
  const unsigned gt = (unsigned)((m + SGC - 1) / SGC);
  constexpr bool DF = sizeof(TF) == 4 && sizeof(TV) == 4;   // dataflow levels (FP32 factor)
  const bool use_df = DF && !sweep_blocked();
  const int vs = use_df ? (m + 3) / 4 * 4 : m;     // row stride of the per-front vectors
  const int2* items = (const int2*)c->d_swplan.p;
  const int* bbase = sweep_bbase(c);
  int* sync = (int*)((char*)vec + sweep_vec_bytes(c, m, sizeof(TV))) + sweep_half_ints(c, m);   // backward half
  if (use_df) (void)cudaMemsetAsync(sync, 0, sweep_half_ints(c, m) * sizeof(int), s);   // errors: cudaGetLastError
  int* flags = sync + sweep_tickets(c);
  SweepTimer tm(s, "bwd", m);
  for (int lev = 0; lev <= c->m; ++lev) {
    const int t0 = c->level_start[lev], cnt = c->level_count[lev];
    const LevelDims D = level_dims(c, lev);
    if (D.maxks == 0) continue;
    tm.begin();
    const unsigned ex = (unsigned)std::min<int64_t>(std::max<int64_t>(1, (int64_t)D.maxf * m / 1024), 512);
    HF_LAUNCH(c, HF_PROF_SWEEP_IO, k_bwd_init<TV><<<dim3(ex, cnt), 256, 0, s>>>(nd, st, t0, rowid, vec, Ytmp, Xout, m, vs));
    if constexpr (DF) if (use_df) {
      const int ni = c->sw_bwd_cnt[lev];
      if (ni > 0) {
        const int g = (int)std::min<int64_t>((int64_t)ni * gt, sweep_grid(false));
        HF_LAUNCH(c, HF_PROF_TRSV_BWD, k_sweep_df<false><<<g, DF_TH, DF_SMEM, s>>>(nd, st, arena, vec, m, vs, (int)gt, items + c->sw_bwd_start[lev], ni,
                                                                           bbase, flags, sync + lev, sweep_err(c), sweep_spin(c),
                                                                          (const float*)c->d_dinv.p));
      }
      HF_LAUNCH(c, HF_PROF_SWEEP_IO, k_bwd_store<TV><<<dim3(ex, cnt), 256, 0, s>>>(nd, st, t0, rowid, vec, Xout, m, vs));
      tm.end(lev, cnt, D.maxf, D.maxks);
      continue;
    }
    HF_LAUNCH(c, HF_PROF_TRSV_BWD, k_gemm_upd<TF, TV, 2, false><<<dim3((D.maxks + SGR - 1) / SGR, gt, cnt), SGTH, 0, s>>>(nd, st, t0, arena, vec, m, 0));
    const int nbk = (D.maxks + TS - 1) / TS;
    constexpr bool fused = sizeof(TV) == 4;          // next diagonal block solved inside the GEMM
    for (int b = 0; b < nbk; ++b) {
      if (b == 0 || !fused)
        HF_LAUNCH(c, HF_PROF_TRSV_BWD, k_trsm_diag<TF, TV, false><<<dim3((m + DiagRhs<TV>::value - 1) / DiagRhs<TV>::value, cnt), DTH, 0, s>>>(nd, st, t0, arena, vec, m, b));
      const unsigned rx = (unsigned)((D.maxks - (b + 1) * TS + SGR - 1) / SGR);
      if ((int)rx > 0)
        HF_LAUNCH(c, HF_PROF_TRSV_BWD, k_gemm_upd<TF, TV, 1, fused><<<dim3(rx, gt, cnt), SGTH, 0, s>>>(nd, st, t0, arena, vec, m, b));
    }
    HF_LAUNCH(c, HF_PROF_SWEEP_IO, k_bwd_store<TV><<<dim3(ex, cnt), 256, 0, s>>>(nd, st, t0, rowid, vec, Xout, m, vs));
    tm.end(lev, cnt, D.maxf, D.maxks);
  }
}

// Apply the triangular solves with the front factor (TF) in vector precision TV.
//  full = false: K11 preconditioner (Lambda_2 rows are zero in and out)
//  full = true : forward sweep only; y2 = the Lambda_2 rows, for the S22 solve
template <typename TF, typename TV>
static int tri_solve(hf_ctx* c, int m, const TV* Bin, TV* Ytmp, TV* Xout, const double* x2_dev, bool full,
                     double* y2_dev, void* vecbuf = nullptr) {
  cudaStream_t s = hf_stream(c);
  TV* vec = (TV*)(vecbuf ? vecbuf : c->d_vec.p);
  fwd_sweep<TF, TV>(c, m, Bin, Ytmp, vec);
  HF_CUDA_TRY(cudaGetLastError());
  const int M = (int)c->M;
  if (M) {
    if (full) {
      HF_LAUNCH(c, HF_PROF_VECTOR, k_get_lam2<TV><<<nblk((int64_t)M * m, 256), 256, 0, s>>>(M, m, (const int32_t*)c->d_lam2.p, Ytmp, y2_dev));
      return 1;   // caller solves S22 and calls tri_solve_back
    }
    HF_LAUNCH(c, HF_PROF_VECTOR, k_set_lam2<TV><<<nblk((int64_t)M * m, 256), 256, 0, s>>>(M, m, (const int32_t*)c->d_lam2.p, nullptr, Xout));
  }
  bwd_sweep<TF, TV>(c, m, Ytmp, Xout, vec);
  HF_CUDA_TRY(cudaGetLastError());
  (void)x2_dev;
  return HF_OK;
}

template <typename TF, typename TV>
static int tri_solve_back(hf_ctx* c, int m, TV* Ytmp, TV* Xout, const double* x2_dev) {
  cudaStream_t s = hf_stream(c);
  const int M = (int)c->M;
  if (M) HF_LAUNCH(c, HF_PROF_VECTOR, k_set_lam2<TV><<<nblk((int64_t)M * m, 256), 256, 0, s>>>(M, m, (const int32_t*)c->d_lam2.p, x2_dev, Xout));
  bwd_sweep<TF, TV>(c, m, Ytmp, Xout, (TV*)c->d_vec.p);
  HF_CUDA_TRY(cudaGetLastError());
  return HF_OK;
}

// Gram G = scale * A^T B
static int gram(hf_ctx* c, int64_t L, int ma, int mb, const double* A, const double* B, double* G, double scale) {
  const int sym = (A == B && ma == mb) ? 1 : 0;
  if (c->opts.fp64_gemm == 0) {
    // FP64-accurate product on the tensor cores (all 2 L ma mb multiply-adds are done)
    c->work_flops[HF_PROF_GRAM] += 2.0 * (double)L * ma * mb;
    c->work_bytes[HF_PROF_GRAM] += 8.0 * (double)L * (ma + mb);
    const size_t nch = (size_t)hf_oz_gram_chunks(L, ma, mb);
    int rc = hf_ensure(c->d_small, std::max(nch * (size_t)ma * mb * 8 + 64, (size_t)(1 << 20)));
    if (rc) return rc;
    int* is = nullptr;
    if ((rc = oz_iscratch(c, (size_t)ma + mb + 64, &is))) return rc;
    const size_t sl = hf_oz_slice_bytes(ma, L) + (A == B && ma == mb ? 0 : hf_oz_slice_bytes(mb, L));
    if ((rc = hf_ensure(c->d_ozslice, sl + 256))) return rc;
    return hf_oz_gram(c, L, ma, mb, A, B, G, scale, (double*)c->d_small.p, c->d_small.bytes, c->d_ozslice.p,
                      c->d_ozslice.bytes, is, oz_err(c));
  }
  c->work_flops[HF_PROF_GRAM] += 2.0 * (double)L * ma * mb * (sym ? 0.5 : 1.0);
  c->work_bytes[HF_PROF_GRAM] += 8.0 * (double)L * (sym ? ma : ma + mb);
  cudaStream_t s = hf_stream(c);
  const int nob = ((ma + GO - 1) / GO) * ((mb + GO - 1) / GO);
  int nchunks = (int)std::min<int64_t>(std::max<int64_t>(1, L / 256), 304);
  size_t need = (size_t)nob * nchunks * GO * GO * 8 + 64;
  int rc = hf_ensure(c->d_small, std::max(need, (size_t)(1 << 20)));
  if (rc) return rc;
  HF_LAUNCH(c, HF_PROF_GRAM, k_gram_partial<<<dim3(nchunks, nob), 256, 0, s>>>(L, ma, mb, A, B, (double*)c->d_small.p, nchunks, sym));
  HF_LAUNCH(c, HF_PROF_GRAM, k_gram_reduce<<<nblk((int64_t)nob * GO * GO, 256), 256, 0, s>>>(ma, mb, nchunks, (const double*)c->d_small.p, G, scale, sym));
  HF_CUDA_TRY(cudaGetLastError());
  return HF_OK;
}

// K11-preconditioner application W = Q^-1 R (FP32 factor) or exact (FP64 factor)
// W = Q^-1 R on caller-provided scratch: tmp32 (3 L m floats, or L m doubles for the FP64
// factor) and vecbuf (the per-front vectors: row_elems m entries of the factor's type)
static int precond_on(hf_ctx* c, int m, const double* R, double* W, void* tmp32, void* vecbuf) {
  cudaStream_t s = hf_stream(c);
  const int64_t L = c->L;
  const int32_t* l2p = (const int32_t*)c->d_lam2pos.p;
  if (c->prec == HF_PREC_FP64) {
    double* y = (double*)tmp32;
    HF_CUDA_TRY(cudaMemcpyAsync(W, R, L * m * 8, cudaMemcpyDeviceToDevice, s));
    HF_LAUNCH(c, HF_PROF_VECTOR, k_zero_lam2_rows<<<nblk(c->M * m, 256), 256, 0, s>>>((int)c->M, m, (const int32_t*)c->d_lam2.p, W));
    return tri_solve<double, double>(c, m, W, y, W, nullptr, false, nullptr, vecbuf);
  }
  float* b32 = (float*)tmp32;
  float* y32 = b32 + L * m;
  float* x32 = y32 + L * m;
  int rc;
  HF_LAUNCH(c, HF_PROF_VECTOR, k_cast_in<float><<<nblk(L * m, 256), 256, 0, s>>>(L, m, R, l2p, b32));
  if ((rc = tri_solve<float, float>(c, m, b32, y32, x32, nullptr, false, nullptr, vecbuf))) return rc;
  HF_LAUNCH(c, HF_PROF_VECTOR, k_cast_out<float><<<nblk(L * m, 256), 256, 0, s>>>(L, m, x32, l2p, W));
  HF_CUDA_TRY(cudaGetLastError());
  return HF_OK;
}

static int precond(hf_ctx* c, int m, const double* R, double* W, void* tmp32) {
  int rc;
  if ((rc = ensure_vec(c, m, c->prec == HF_PREC_FP64 ? 8 : 4))) return rc;
  return precond_on(c, m, R, W, tmp32, c->d_vec.p);
}

static void spmm(hf_ctx* c, int m, const double* W, double* Z) {
  cudaStream_t s = hf_stream(c);
  c->work_flops[HF_PROF_SPMM] += 2.0 * (double)c->nnz * m;
  c->work_bytes[HF_PROF_SPMM] += 12.0 * (double)c->nnz + 16.0 * (double)c->L * m + 8.0 * (double)c->L;
  HF_LAUNCH(c, HF_PROF_SPMM, k_spmm<<<nblk(c->L * 32, 256), 256, 0, s>>>(c->L, m, (const int64_t*)c->d_rowptr.p, (const int32_t*)c->d_col.p,
                                              (const double*)c->d_kval.p, (const int32_t*)c->d_lam2pos.p, W, Z));
}

// Block GCR for K11 X = B (Sec. 3.5, readings R7/R8).  B, X: L x m row-major, Lambda_2 rows 0.
// Grid of the cooperative kernels: every block must be resident at once
static int coop_grid(hf_ctx* c) {
  static std::mutex mu;
  static int blocks = 0;
  std::lock_guard<std::mutex> lk(mu);
  if (!blocks) {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int p1 = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&p1, k_chol_coop, 256, 0);
    per = p1;
    blocks = std::max(1, sms * std::min(per, 1));
  }
  (void)c;
  return blocks;
}

static int block_gcr(hf_ctx* c, int m, const double* B, double* X, int* iters, double* relres,
                     std::vector<double>* hist_out = nullptr) {
  cudaStream_t s = hf_stream(c);
  const int64_t L = c->L;
  const int maxit = std::max(1, c->opts.gcr_maxit);
  const size_t blk = (size_t)L * m;
  // workspace: R, W, Z, tmp(3 x L x m floats or 1 x L x m doubles); the history blocks
  // P_i, Q_i are allocated when an iteration first needs them (kept for later calls)
  const size_t tmp_doubles = (blk * 3 + 1) / 2 + blk;
  size_t need = (blk * 3 + tmp_doubles) * 8 + 1024;
  int rc;
  if ((rc = hf_ensure(c->d_work, need))) return rc;
  double* base = (double*)c->d_work.p;
  double* R = base;
  double* W = R + blk;
  double* Z = W + blk;
  double* tmp = Z + blk;
  auto ensure_hist = [&](int i) -> int {           // P_i and Q_i
    if ((int)c->d_hist.size() < 2 * i + 2) c->d_hist.resize(2 * i + 2);
    int r = hf_ensure(c->d_hist[2 * i], blk * 8 + 256);
    if (!r) r = hf_ensure(c->d_hist[2 * i + 1], blk * 8 + 256);
    return r;
  };
  auto Pm = [&](int i) { return (double*)c->d_hist[2 * i].p; };
  auto Qm = [&](int i) { return (double*)c->d_hist[2 * i + 1].p; };
  // small matrices in pinned / device memory
  const size_t mm = (size_t)m * m;
  std::vector<double> hnorm(m), bnorm(m);
  DevBuf& sm = c->d_gsmall;
  size_t small_need = ((size_t)(maxit + 2) * mm * 2 + 6 * mm + 4 * (size_t)m + 64) * 8 +
                      (size_t)(maxit + 2) * (4 * ((size_t)m + 1) + 8) * 4 + 4096;
  if ((rc = hf_ensure(sm, small_need))) return rc;
  double* Mstore = (double*)sm.p;                 // (maxit+1) Gram matrices M_n
  double* Gm = Mstore + (size_t)(maxit + 1) * mm;
  double* Cm = Gm + mm;
  double* wk = Cm + mm;                           // small solve work (m*m + m)
  double* diag = wk + mm + m + 8;                 // m x m scratch for norms
  int* dmask = (int*)(diag + mm);                 // converged-column mask (m ints)
  const size_t meven = (size_t)(m + 1) / 2 * 2;
  const size_t dstride = 4 * meven + 8;           // per M_n: m drop flags, then m doubles (8-byte aligned)
  int* dropv = dmask + meven + 8;
  std::vector<int> hmask(m, 0);
  std::vector<double> hist_res;
  const unsigned nb = nblk((int64_t)blk, 256);
  const int use_smem = mm * 8 <= 48 * 1024;
  const size_t axpy_smem = use_smem ? mm * 8 : 0;
  const double axpy_flops = 2.0 * (double)L * m * m, axpy_bytes = 8.0 * (double)L * m * 3;
  int* ozis = nullptr;
  if (c->opts.fp64_gemm == 0) {
    if ((rc = oz_iscratch(c, (size_t)L + m + 64, &ozis))) return rc;
    const size_t sl = std::max(hf_oz_slice_bytes(L, m) + hf_oz_slice_bytes(m, m), 2 * hf_oz_slice_bytes(m, L));
    if ((rc = hf_ensure(c->d_ozslice, sl + 256))) return rc;
    HF_CUDA_TRY(cudaMemsetAsync(oz_err(c), 0, sizeof(int), s));
  }
  // Y = (Yinit ? Yinit : Y) + sgn * A C, FP64-accurate
  auto block_update = [&](const double* A, const double* Cmat, double* Y, const double* Yinit, double sgn) -> int {
    c->work_flops[HF_PROF_BLOCK_UPDATE] += axpy_flops;
    c->work_bytes[HF_PROF_BLOCK_UPDATE] += axpy_bytes;
    if (c->opts.fp64_gemm == 0)
      return hf_oz_update(c, L, m, A, Cmat, Y, Yinit, sgn, c->d_ozslice.p, c->d_ozslice.bytes, ozis, oz_err(c));
    HF_LAUNCH(c, HF_PROF_BLOCK_UPDATE, k_block_axpy<<<nb, 256, axpy_smem, s>>>(L, m, A, Cmat, Y, Yinit, sgn, use_smem));
    return HF_OK;
  };

  // column 2-norms; row-chunk partials in the small scratch buffer
  const int ncs = (int)std::max<int64_t>(1, std::min<int64_t>(L / 1024, 152));
  auto colnorms = [&](const double* A, std::vector<double>& out) -> int {
    c->work_flops[HF_PROF_VECTOR] += 2.0 * (double)L * m;
    c->work_bytes[HF_PROF_VECTOR] += 8.0 * (double)L * m;
    int r = hf_ensure(c->d_small, std::max((size_t)ncs * m * 8 + 64, (size_t)(1 << 20)));
    if (r) return r;
    double* part = (double*)c->d_small.p;
    HF_LAUNCH(c, HF_PROF_VECTOR, k_colsq_partial<<<ncs, CSQ_TH, 0, s>>>(L, m, A, part));
    HF_LAUNCH(c, HF_PROF_VECTOR, k_colsq_reduce<<<(m + 127) / 128, 128, 0, s>>>(m, ncs, part, diag));
    HF_CUDA_TRY(cudaGetLastError());
    std::vector<double> g(m);
    HF_CUDA_TRY(cudaMemcpyAsync(g.data(), diag, (size_t)m * 8, cudaMemcpyDeviceToHost, s));
    HF_CUDA_TRY(cudaStreamSynchronize(s));
    for (int i = 0; i < m; ++i) out[i] = std::sqrt(std::max(0.0, g[i]));
    return HF_OK;
  };
  if ((rc = colnorms(B, bnorm))) return rc;
  for (auto& v : bnorm) if (v == 0) v = 1.0;
  const char* ve = std::getenv("HF_VERBOSE");
  const bool verbose = ve && ve[0] == '1';
  // X0 = Q^-1 B, R0 = B - K11 X0, W0 = Q^-1 R0, P0 = W0, Q0 = K11 P0
  if ((rc = precond(c, m, B, X, tmp))) return rc;
  spmm(c, m, X, Z);
  HF_LAUNCH(c, HF_PROF_VECTOR, k_sub<<<nb, 256, 0, s>>>((int64_t)blk, B, Z, R));
  if (hist_out) {                                   // max_k |r0_k| / |b_k| of the start
    if ((rc = colnorms(R, hnorm))) return rc;
    double r0 = 0;
    for (int i = 0; i < m; ++i) r0 = std::max(r0, hnorm[i] / bnorm[i]);
    hist_out->assign(1, r0);
  }
  if ((rc = ensure_hist(0))) return rc;
  if ((rc = precond(c, m, R, Pm(0), tmp))) return rc;
  spmm(c, m, Pm(0), Qm(0));
  int it = 0;
  double res = 0;
  bool conv = false;
  const int cgrid = coop_grid(c);
  auto msolve = [&](int q, const double* Y, double* C) -> int {
    const double* Rq = Mstore + (size_t)q * mm;
    const int* dq = dropv + (size_t)q * dstride;
    // one block per few right-hand sides: about one block per SM
    const int cpb = std::max(1, (m + cgrid - 1) / cgrid);
    const unsigned nbk = (unsigned)((m + cpb - 1) / cpb);
    HF_LAUNCH(c, HF_PROF_VECTOR, k_chol_solve_cols<<<nbk, 256, 0, s>>>(m, m, cpb, Rq, dq, Y, C));
    return HF_OK;
  };
  for (int n = 0; n < maxit; ++n) {
    double* Mn = Mstore + (size_t)n * mm;
    if ((rc = gram(c, L, m, m, Qm(n), Qm(n), Mn, 1.0))) return rc;
    {                                                                                       // M_n = R^T R
      int mm_ = m;
      int* dn = dropv + (size_t)n * dstride;
      void* args[] = {&mm_, (void*)&Mn, (void*)&dn};
      HF_LAUNCH(c, HF_PROF_VECTOR, HF_CUDA_TRY(cudaLaunchCooperativeKernel((const void*)k_chol_coop, cgrid, 256, args, 0, s)));
    }
    if ((rc = gram(c, L, m, m, Qm(n), R, Gm, 1.0))) return rc;
    if ((rc = msolve(n, Gm, Cm))) return rc;
    if ((rc = block_update(Pm(n), Cm, X, nullptr, 1.0))) return rc;
    if ((rc = block_update(Qm(n), Cm, R, nullptr, -1.0))) return rc;
    HF_CUDA_TRY(cudaGetLastError());
    it = n + 1;
    if ((rc = colnorms(R, hnorm))) return rc;
    res = 0;
    for (int i = 0; i < m; ++i) res = std::max(res, hnorm[i] / bnorm[i]);
    if (verbose) {
      std::vector<double> rr(m);
      for (int i = 0; i < m; ++i) rr[i] = hnorm[i] / bnorm[i];
      std::sort(rr.rbegin(), rr.rend());
      const int above = (int)std::count_if(rr.begin(), rr.end(), [&](double v) { return v > c->opts.gcr_tol; });
      std::fprintf(stderr, "[hf] block GCR m=%d iter %d max |r|/|b| = %.3e (columns above tol %d; next %.3e %.3e)\n", m, it,
                   res, above, m > 1 ? rr[1] : 0.0, m > 2 ? rr[2] : 0.0);
    }
    hist_res.push_back(res);
    if (hist_out) hist_out->push_back(res);
    if (!(res > c->opts.gcr_tol)) { conv = true; break; }
    if (n + 1 >= maxit) break;
    // stagnation: less than a 2x reduction over three iterations
    const size_t h = hist_res.size();
    if (h >= 4 && hist_res[h - 1] > 0.5 * hist_res[h - 4]) {
      conv = res <= 100.0 * c->opts.gcr_tol;
      break;
    }
    // deflation: converged columns stop contributing search directions
    bool any = false;
    for (int i = 0; i < m; ++i) {
      int mk = !(hnorm[i] / bnorm[i] > c->opts.gcr_tol);
      any |= (mk != hmask[i]);
      hmask[i] = mk;
    }
    if (any) HF_CUDA_TRY(cudaMemcpyAsync(dmask, hmask.data(), m * sizeof(int), cudaMemcpyHostToDevice, s));
    if (std::count(hmask.begin(), hmask.end(), 1) > 0)
      HF_LAUNCH(c, HF_PROF_VECTOR, k_zero_cols<<<nb, 256, 0, s>>>(L, m, dmask, R));
    if ((rc = precond(c, m, R, W, tmp))) return rc;
    spmm(c, m, W, Z);
    if ((rc = ensure_hist(n + 1))) return rc;
    double* Pn = Pm(n + 1);
    double* Qn = Qm(n + 1);
    // Q_{n+1} = K11 P_{n+1} (reading R14): by the recurrence of Sec. 3.4, Z + sum_q Q_q C_q,
    // while its n+1 products of m x m blocks (on the tensor cores) cost less than one FP64
    // SpMM, i.e. while (n+1) m <= 2 nnz / L; otherwise by the SpMM
    const bool recur = (double)(n + 1) * m <= 2.0 * (double)c->nnz / (double)L;
    for (int q = 0; q <= n; ++q) {
      if ((rc = gram(c, L, m, m, Qm(q), Z, Gm, -1.0))) return rc;      // B_qn = -Q_q^T Z
      if ((rc = msolve(q, Gm, Cm))) return rc;
      if ((rc = block_update(Pm(q), Cm, Pn, q == 0 ? W : nullptr, 1.0))) return rc;
      if (recur && (rc = block_update(Qm(q), Cm, Qn, q == 0 ? Z : nullptr, 1.0))) return rc;
    }
    if (!recur) spmm(c, m, Pn, Qn);
    HF_CUDA_TRY(cudaGetLastError());
  }
  *iters = it;
  *relres = res;
  if (c->opts.fp64_gemm == 0) {
    int h = 0;
    HF_CUDA_TRY(cudaMemcpyAsync(&h, oz_err(c), sizeof(int), cudaMemcpyDeviceToHost, s));
    HF_CUDA_TRY(cudaStreamSynchronize(s));
    if (h) return HF_ERR_TIMEOUT;     // a tensor-core wait gave up: the products are not valid
  }
  if ((rc = sweep_status(c))) return rc;   // a sweep wait gave up: the preconditioner is void
  return conv ? HF_OK : HF_ERR_NOT_CONVERGED;
}

// Block GCR as hf_schur and hf_solve run it: with the emulated FP64 products, whose error
// is normwise (relative to the largest entries of each column), an iteration on vectors
// whose entries span many orders of magnitude can stagnate above the tolerance; it is then
// run again from the start with the native FP64 products (c->gcr_restarts counts these).
static int block_gcr_robust(hf_ctx* c, int m, const double* B, double* X, int* iters, double* relres) {
  int rc = block_gcr(c, m, B, X, iters, relres);
  if (c->opts.fp64_gemm != 0 || (rc != HF_OK && rc != HF_ERR_NOT_CONVERGED) || !(*relres > c->opts.gcr_tol))
    return rc;
  const int it0 = *iters;
  c->opts.fp64_gemm = 1;
  rc = block_gcr(c, m, B, X, iters, relres);
  c->opts.fp64_gemm = 0;
  *iters += it0;
  c->gcr_restarts++;
  return rc;
}

static int bk_factor(hf_ctx* c) {
  cudaStream_t s = hf_stream(c);
  const int M = (int)c->M;
  int rc;
  if ((rc = hf_ensure(c->d_bk_lf, (size_t)M * M * 8 * 2 + 64))) return rc;
  if ((rc = hf_ensure(c->d_bk_perm, (size_t)M * 4 + 64))) return rc;
  if ((rc = hf_ensure(c->d_bk_blk, (size_t)M * 4 + 64))) return rc;
  if ((rc = hf_ensure(c->d_bk_dval, (size_t)M * 16 + 64 + (size_t)M * 16))) return rc;
  if ((rc = hf_ensure(c->d_bk_null, (size_t)M * 4 + 64))) return rc;
  c->path_ldlt = 0;
  if (M == 0) { c->kernel_dim = 0; return HF_OK; }
  double* A = (double*)c->d_bk_lf.p + (size_t)M * M;     // working copy after Lf
  HF_CUDA_TRY(cudaMemcpyAsync(A, c->d_s22.p, (size_t)M * M * 8, cudaMemcpyDeviceToDevice, s));
  int* kd = (int*)((int*)c->d_flags.p + FLAG_COUNT + 8);
  double* mags = (double*)c->d_bk_dval.p + 2 * M;
  // S22 in the distributed shared memory of one cluster when it fits, else over all SMs
  static std::mutex bpc_mu;
  static int bpc_cmax = -1;
  {
    std::lock_guard<std::mutex> lk(bpc_mu);
    if (bpc_cmax < 0) {
      bpc_cmax = 0;
      if (cudaFuncSetAttribute(k_bp_cluster, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)BPC_SMEM) == cudaSuccess &&
          cudaFuncSetAttribute(k_bp_cluster, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess) {
        for (int cs = BPC_CMAX; cs >= 2; cs /= 2) {
          cudaLaunchConfig_t q = {};
          q.gridDim = dim3(cs); q.blockDim = dim3(BPC_THREADS); q.dynamicSmemBytes = BPC_SMEM;
          cudaLaunchAttribute at[1];
          at[0].id = cudaLaunchAttributeClusterDimension;
          at[0].val.clusterDim.x = cs; at[0].val.clusterDim.y = 1; at[0].val.clusterDim.z = 1;
          q.attrs = at; q.numAttrs = 1;
          int ncl = 0;
          if (cudaOccupancyMaxActiveClusters(&ncl, k_bp_cluster, &q) == cudaSuccess && ncl > 0) { bpc_cmax = cs; break; }
        }
      }
      (void)cudaGetLastError();
    }
  }
  const int bpc_C = bpc_cmax;
  const int bpc_R = bpc_C > 0 ? (M + bpc_C - 1) / bpc_C : 0;
  const size_t bpc_bytes = ((size_t)bpc_R * M + 8 * (size_t)M) * 8 + 2 * BPC_CMAX * 4 * 8 + 64;
  if (bpc_C > 0 && bpc_R <= BPC_RMAX && bpc_bytes <= BPC_SMEM) {
    c->path_ldlt = 1;
    cudaLaunchConfig_t lc = {};
    lc.gridDim = dim3(bpc_C); lc.blockDim = dim3(BPC_THREADS); lc.dynamicSmemBytes = bpc_bytes; lc.stream = s;
    cudaLaunchAttribute la[1];
    la[0].id = cudaLaunchAttributeClusterDimension;
    la[0].val.clusterDim.x = bpc_C; la[0].val.clusterDim.y = 1; la[0].val.clusterDim.z = 1;
    lc.attrs = la; lc.numAttrs = 1;
    HF_LAUNCH(c, HF_PROF_DENSE_LDLT, HF_CUDA_TRY(cudaLaunchKernelEx(&lc, k_bp_cluster, M, bpc_R, (const double*)A,
                                                                    (double*)c->d_bk_lf.p, (int*)c->d_bk_perm.p,
                                                                    (int*)c->d_bk_blk.p, (double*)c->d_bk_dval.p,
                                                                    (int*)c->d_bk_null.p, c->opts.kernel_eps,
                                                                    c->opts.kernel_gap, (const int32_t*)c->d_lam2.p,
                                                                    (const int64_t*)c->d_diagpos.p,
                                                                    (const double*)c->d_kval.p, c->s22_noise, kd, mags)));
  } else if (M <= BP_MAX_M) {
    c->path_ldlt = 2;
    // over all SMs (cooperative); partial maxima of two steps in flight per block
    static std::mutex bp_mu;
    static int bp_blocks = 0;
    {
      std::lock_guard<std::mutex> lk(bp_mu);
      if (!bp_blocks) {
        int dev = 0, sms = 0, per = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        HF_CUDA_TRY(cudaFuncSetAttribute(k_bp_coop, cudaFuncAttributeMaxDynamicSharedMemorySize, 3 * BP_MAX_M * 8));
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_bp_coop, BP_THREADS, 3 * BP_MAX_M * 8);
        bp_blocks = std::max(1, sms * std::min(std::max(per, 1), 1));
      }
    }
    if ((rc = hf_ensure(c->d_bpart, (size_t)2 * bp_blocks * sizeof(BpPart) + 64))) return rc;
    double* Lf = (double*)c->d_bk_lf.p;
    int* pm = (int*)c->d_bk_perm.p;
    int* bk = (int*)c->d_bk_blk.p;
    double* dv = (double*)c->d_bk_dval.p;
    int* nl = (int*)c->d_bk_null.p;
    double keps = c->opts.kernel_eps, kgap = c->opts.kernel_gap, noise = c->s22_noise;
    const int32_t* l2 = (const int32_t*)c->d_lam2.p;
    const int64_t* dp = (const int64_t*)c->d_diagpos.p;
    const double* kv = (const double*)c->d_kval.p;
    BpPart* parts = (BpPart*)c->d_bpart.p;
    int Mi = M;
    void* args[] = {&Mi, (void*)&A, (void*)&Lf, (void*)&pm, (void*)&bk, (void*)&dv, (void*)&nl, &keps, &kgap,
                    (void*)&l2, (void*)&dp, (void*)&kv, &noise, (void*)&kd, (void*)&mags, (void*)&parts};
    HF_LAUNCH(c, HF_PROF_DENSE_LDLT, HF_CUDA_TRY(cudaLaunchCooperativeKernel((const void*)k_bp_coop, bp_blocks, BP_THREADS,
                                                                             args, 3 * (size_t)M * 8, s)));
  } else {
    c->path_ldlt = 3;
    HF_LAUNCH(c, HF_PROF_DENSE_LDLT, k_bunch_parlett<<<1, 512, 0, s>>>(M, A, (double*)c->d_bk_lf.p, (int*)c->d_bk_perm.p, (int*)c->d_bk_blk.p,
                                      (double*)c->d_bk_dval.p, (int*)c->d_bk_null.p, c->opts.kernel_eps,
                                      c->opts.kernel_gap, (const int32_t*)c->d_lam2.p, (const int64_t*)c->d_diagpos.p,
                                      (const double*)c->d_kval.p, c->s22_noise, kd, mags));
  }
  HF_CUDA_TRY(cudaGetLastError());
  int h = 0;
  HF_CUDA_TRY(cudaMemcpyAsync(&h, kd, 4, cudaMemcpyDeviceToHost, s));
  HF_CUDA_TRY(cudaStreamSynchronize(s));
  c->kernel_dim = h;
  return HF_OK;
}

int hf_s22_from_factor(hf_ctx* c);

int hf_schur_impl(hf_ctx* c) {
  if (!c) return HF_ERR_ARG;
  if (!c->factored) return HF_ERR_STATE;
  cudaStream_t s = hf_stream(c);
  const int M = (int)c->M;
  const int64_t L = c->L;
  int rc = HF_OK, grc = HF_OK;
  c->gcr_iters = 0;
  c->gcr_relres = 0;
  if ((rc = hf_ensure(c->d_x12, (size_t)L * std::max(M, 1) * 8 + 64))) return rc;
  if ((rc = hf_ensure(c->d_s22, (size_t)M * M * 8 + 64))) return rc;
  if (M > 0) {
    if (c->prec == HF_PREC_MIXED) {
      // B = K12 (Alg. 1 step 2), X12 by block GCR (step 3), S22 = K22 - K21 X12 (step 4)
      double* X12 = (double*)c->d_x12.p;
      if ((rc = hf_ensure(c->d_k12, (size_t)L * M * 8 + 64))) return rc;
      double* B = (double*)c->d_k12.p;
      HF_CUDA_TRY(cudaMemsetAsync(B, 0, (size_t)L * M * 8, s));
      HF_LAUNCH(c, HF_PROF_SCHUR, k_extract_k12<<<M, 128, 0, s>>>(M, (const int64_t*)c->d_rowptr.p, (const int32_t*)c->d_col.p,
                                      (const double*)c->d_kval.p, (const int32_t*)c->d_lam2.p,
                                      (const int32_t*)c->d_lam2pos.p, B));
      c->gcr_restarts = 0;
      grc = block_gcr_robust(c, M, B, X12, &c->gcr_iters, &c->gcr_relres);
      if (grc && grc != HF_ERR_NOT_CONVERGED) return grc;
      // error estimate of S22 for the kernel rule: E = K21 Q^-1 (K12 - K11 X12)
      {
        const size_t blk = (size_t)L * M;
        double* Rt = (double*)c->d_work.p;
        double* Wt = Rt + blk;
        double* Zt = Wt + blk;
        double* tmp = Zt + blk;
        spmm(c, M, X12, Zt);
        HF_LAUNCH(c, HF_PROF_VECTOR, k_sub<<<nblk((int64_t)blk, 256), 256, 0, s>>>((int64_t)blk, B, Zt, Rt));
        if ((rc = precond(c, M, Rt, Wt, tmp))) return rc;
        double* E = (double*)c->d_gsmall.p;
        HF_LAUNCH(c, HF_PROF_SCHUR, k_schur_rows<<<nblk((int64_t)M * 32, 256), 256, 0, s>>>(M, M, (const int64_t*)c->d_rowptr.p,
                                                            (const int32_t*)c->d_col.p, (const double*)c->d_kval.p,
                                                            (const int32_t*)c->d_lam2.p, (const int32_t*)c->d_lam2pos.p,
                                                            Wt, nullptr, 0, E, 2));
        std::vector<double> hE((size_t)M * M);
        HF_CUDA_TRY(cudaMemcpyAsync(hE.data(), E, hE.size() * 8, cudaMemcpyDeviceToHost, s));
        HF_CUDA_TRY(cudaStreamSynchronize(s));
        double mx = 0;
        for (double v : hE) mx = std::max(mx, std::fabs(v));
        c->s22_noise = 100.0 * mx;
      }
      HF_LAUNCH(c, HF_PROF_SCHUR, k_schur_rows<<<nblk((int64_t)M * 32, 256), 256, 0, s>>>(M, M, (const int64_t*)c->d_rowptr.p,
                                                          (const int32_t*)c->d_col.p, (const double*)c->d_kval.p,
                                                          (const int32_t*)c->d_lam2.p, (const int32_t*)c->d_lam2pos.p,
                                                          X12, nullptr, 0, (double*)c->d_s22.p, 0));
      HF_LAUNCH(c, HF_PROF_SCHUR, k_symmetrize<<<nblk((int64_t)M * M, 256), 256, 0, s>>>(M, (double*)c->d_s22.p));
      HF_CUDA_TRY(cudaGetLastError());
    } else {
      if ((rc = hf_s22_from_factor(c))) return rc;
      // S22 from the factor: its error is the unit roundoff of the factor's precision
      c->s22_noise = 100.0 * (c->prec == HF_PREC_FP64 ? 1.1102230246251565e-16 : 5.9604644775390625e-08);
    }
  }
  if ((rc = bk_factor(c))) return rc;
  c->schured = true;
  return grc;
}

int hf_solve_impl(hf_ctx* c, int nrhs, const double* b, int64_t ldb, double* x, int64_t ldx) {
  if (!c || nrhs < 1 || !b || !x || ldb < c->L || ldx < c->L) return HF_ERR_ARG;
  if (!c->schured) return HF_ERR_STATE;
  cudaStream_t s = hf_stream(c);
  const int64_t L = c->L;
  const int M = (int)c->M;
  const int m = nrhs;
  const size_t blk = (size_t)L * m;
  int rc;
  size_t need = (blk * 4 + (size_t)M * m * 3 + 64) * 8;
  if ((rc = hf_ensure(c->d_solve, need))) return rc;
  double* bi = (double*)c->d_solve.p;
  double* y = bi + blk;
  double* y1 = y + blk;
  double* scratch = y1 + blk;
  double* y2 = scratch + blk;
  double* x2 = y2 + (size_t)M * m;
  double* zt = x2 + (size_t)M * m;  // work vectors of the S22 solve when they do not fit in shared memory
  // right-hand sides enter as J Q b (Q b without row signs): K x = J Q b with xbar = Q x
  const double* qrow = (const double*)(c->has_rsign ? c->d_qrow.p : c->d_q.p);
  HF_LAUNCH(c, HF_PROF_SCALE, k_scale_in<<<nblk((int64_t)blk, 256), 256, 0, s>>>(L, m, b, ldb, qrow, bi));
  int grc = HF_OK;
  auto s22_solve = [&]() {
    if (M == 0) return;
    const size_t zbytes = (size_t)M * 8;
    const bool in_smem = zbytes <= BKS_SMEM_MAX;
    if (in_smem && zbytes > 48 * 1024) {
      const cudaError_t e = cudaFuncSetAttribute(k_bk_solve, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)BKS_SMEM_MAX);
      if (e != cudaSuccess) { grc = HF_ERR_CUDA; return; }
    }
    HF_LAUNCH(c, HF_PROF_DENSE_LDLT, k_bk_solve<<<m, 256, in_smem ? zbytes : 0, s>>>(M, m, (const double*)c->d_bk_lf.p, (const int*)c->d_bk_perm.p,
                                 (const int*)c->d_bk_blk.p, (const double*)c->d_bk_dval.p,
                                 (const int*)c->d_bk_null.p, y2, x2, in_smem ? nullptr : zt));
  };
  if (c->prec == HF_PREC_MIXED) {
    // Alg. 2: y1 by block GCR on K11, y2 = b2 - K21 y1, S22 x2 = y2, x1 = y1 - X12 x2
    HF_CUDA_TRY(cudaMemcpyAsync(y, bi, blk * 8, cudaMemcpyDeviceToDevice, s));
    if (M) HF_LAUNCH(c, HF_PROF_VECTOR, k_zero_lam2_rows<<<nblk((int64_t)M * m, 256), 256, 0, s>>>(M, m, (const int32_t*)c->d_lam2.p, y));
    grc = block_gcr_robust(c, m, y, y1, &c->solve_iters, &c->solve_relres);
    if (grc && grc != HF_ERR_NOT_CONVERGED) return grc;
    if (M) {
      HF_LAUNCH(c, HF_PROF_SCHUR, k_schur_rows<<<nblk((int64_t)M * 32, 256), 256, 0, s>>>(M, m, (const int64_t*)c->d_rowptr.p,
                                                          (const int32_t*)c->d_col.p, (const double*)c->d_kval.p,
                                                          (const int32_t*)c->d_lam2.p, (const int32_t*)c->d_lam2pos.p,
                                                          y1, bi, m, y2, 1));
      s22_solve();
      HF_LAUNCH(c, HF_PROF_SCHUR, k_backsub_x1<<<nblk((int64_t)blk, 256), 256, 0, s>>>(L, M, m, (const double*)c->d_x12.p, x2,
                                                            (const int32_t*)c->d_lam2pos.p, y1));
    }
    HF_LAUNCH(c, HF_PROF_SCALE, k_scale_out<<<nblk((int64_t)blk, 256), 256, 0, s>>>(L, m, y1, (const double*)c->d_q.p, x, ldx));
  } else if (c->prec == HF_PREC_FP64) {
    // block substitution with the stored FP64 factor (Eq. 1): forward, S22 solve, backward
    if ((rc = ensure_vec(c, m, 8))) return rc;
    rc = tri_solve<double, double>(c, m, bi, y, y1, nullptr, M > 0, y2);
    if (rc != HF_OK && rc != 1) return rc;
    if (M) {
      s22_solve();
      if ((rc = tri_solve_back<double, double>(c, m, y, y1, x2))) return rc;
    }
    HF_LAUNCH(c, HF_PROF_SCALE, k_scale_out<<<nblk((int64_t)blk, 256), 256, 0, s>>>(L, m, y1, (const double*)c->d_q.p, x, ldx));
  } else {
    // FP32 form: the same substitution with the FP32 factor (S22 solved in FP64)
    if ((rc = ensure_vec(c, m, 4))) return rc;
    float* b32 = (float*)scratch;
    float* y32 = (float*)y;
    float* x32 = y32 + blk;
    HF_LAUNCH(c, HF_PROF_VECTOR, k_cast_in<float><<<nblk((int64_t)blk, 256), 256, 0, s>>>(L, m, bi, nullptr, b32));
    rc = tri_solve<float, float>(c, m, b32, y32, x32, nullptr, M > 0, y2);
    if (rc != HF_OK && rc != 1) return rc;
    if (M) {
      s22_solve();
      if ((rc = tri_solve_back<float, float>(c, m, y32, x32, x2))) return rc;
    }
    HF_LAUNCH(c, HF_PROF_VECTOR, k_cast_out<float><<<nblk((int64_t)blk, 256), 256, 0, s>>>(L, m, x32, nullptr, y1));
    HF_LAUNCH(c, HF_PROF_SCALE, k_scale_out<<<nblk((int64_t)blk, 256), 256, 0, s>>>(L, m, y1, (const double*)c->d_q.p, x, ldx));
  }
  HF_CUDA_TRY(cudaGetLastError());
  if ((rc = sweep_status(c))) return rc;
  return grc;
}

// The dense products of the block GCR on their own (public entry points): the same
// calls as inside the iteration, on a context that may not have been factorized.
static int products_prepare(hf_ctx* c) {
  const bool fresh = c->d_flags.p == nullptr;
  int rc;
  if ((rc = hf_ensure(c->d_flags, FLAG_COUNT * sizeof(int) + 64))) return rc;
  cudaStream_t s = hf_stream(c);
  if (fresh) HF_CUDA_TRY(cudaMemsetAsync(c->d_flags.p, 0, FLAG_COUNT * sizeof(int) + 64, s));
  HF_CUDA_TRY(cudaMemsetAsync(oz_err(c), 0, sizeof(int), s));
  return HF_OK;
}

static int products_status(hf_ctx* c) {
  int h = 0;
  cudaStream_t s = hf_stream(c);
  HF_CUDA_TRY(cudaGetLastError());
  HF_CUDA_TRY(cudaMemcpyAsync(&h, oz_err(c), sizeof(int), cudaMemcpyDeviceToHost, s));
  HF_CUDA_TRY(cudaStreamSynchronize(s));
  return h ? HF_ERR_TIMEOUT : HF_OK;
}

int hf_gram_fp64_impl(hf_ctx* c, int64_t L, int ma, int mb, const double* A, const double* B, double* G, double scale) {
  if (L < 1 || ma < 1 || mb < 1 || !A || !B || !G) return HF_ERR_ARG;
  int rc;
  if ((rc = products_prepare(c))) return rc;
  if ((rc = gram(c, L, ma, mb, A, B, G, scale))) return rc;
  return products_status(c);
}

int hf_update_fp64_impl(hf_ctx* c, int64_t L, int m, const double* A, const double* C, double* Y, const double* Yinit,
                        double sgn) {
  if (L < 1 || m < 1 || !A || !C || !Y || Y == A || Y == C) return HF_ERR_ARG;
  int rc;
  if ((rc = products_prepare(c))) return rc;
  cudaStream_t s = hf_stream(c);
  c->work_flops[HF_PROF_BLOCK_UPDATE] += 2.0 * (double)L * m * m;
  c->work_bytes[HF_PROF_BLOCK_UPDATE] += 8.0 * (double)L * m * 3;
  if (c->opts.fp64_gemm == 0) {
    int* is = nullptr;
    if ((rc = oz_iscratch(c, (size_t)L + m + 64, &is))) return rc;
    if ((rc = hf_ensure(c->d_ozslice, hf_oz_slice_bytes(L, m) + hf_oz_slice_bytes(m, m) + 256))) return rc;
    if ((rc = hf_oz_update(c, L, m, A, C, Y, Yinit, sgn, c->d_ozslice.p, c->d_ozslice.bytes, is, oz_err(c)))) return rc;
  } else {
    const size_t mm = (size_t)m * m;
    const int use_smem = mm * 8 <= 48 * 1024;
    HF_LAUNCH(c, HF_PROF_BLOCK_UPDATE, k_block_axpy<<<nblk(L * m, 256), 256, use_smem ? mm * 8 : 0, s>>>(L, m, A, C, Y, Yinit, sgn, use_smem));
  }
  return products_status(c);
}

__global__ void k_addto(int64_t n, const double* __restrict__ W, double* __restrict__ X) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < n) X[e] += W[e];
}

// max_k |A_k| / bnorm_k over the m columns of a row-major L x m block (device reduction)
static int max_col_ratio(hf_ctx* c, int m, const double* A, const std::vector<double>& bnorm, double* out,
                         std::vector<double>* norms = nullptr) {
  cudaStream_t s = hf_stream(c);
  const int64_t L = c->L;
  const int ncs = (int)std::max<int64_t>(1, std::min<int64_t>(L / 1024, 152));
  int rc;
  if ((rc = hf_ensure(c->d_small, std::max(((size_t)ncs + 1) * m * 8 + 64, (size_t)(1 << 20))))) return rc;
  double* part = (double*)c->d_small.p;
  double* sq = part + (size_t)ncs * m;
  HF_LAUNCH(c, HF_PROF_VECTOR, k_colsq_partial<<<ncs, CSQ_TH, 0, s>>>(L, m, A, part));
  HF_LAUNCH(c, HF_PROF_VECTOR, k_colsq_reduce<<<(m + 127) / 128, 128, 0, s>>>(m, ncs, part, sq));
  std::vector<double> g(m);
  HF_CUDA_TRY(cudaMemcpyAsync(g.data(), sq, (size_t)m * 8, cudaMemcpyDeviceToHost, s));
  HF_CUDA_TRY(cudaStreamSynchronize(s));
  double r = 0;
  for (int i = 0; i < m; ++i) {
    const double v = std::sqrt(std::max(0.0, g[i]));
    if (norms) (*norms)[i] = v;
    r = std::max(r, bnorm.empty() ? v : v / bnorm[i]);
  }
  *out = r;
  return HF_OK;
}

// The three iterations on K11 X = B that the paper compares (Sec. 3.3-3.5, Fig. 2), each
// preconditioned by the lower-precision factor Q: block GCR on all columns (Alg. 5),
// GCR one column at a time (Alg. 4: block GCR with one column), and iterative
// refinement (Alg. 3: x0 = Q^-1 b, then x += Q^-1 (b - K11 x)).  hist[n] = max over the
// columns of |r_n| / |b| after n steps (for Alg. 4 the worst column at each step).
int hf_k11_iterate_impl(hf_ctx* c, int method, int m, const double* B, double* X, int maxit, double* hist,
                        int* iters) {
  if (!c->factored) return HF_ERR_STATE;
  if (m < 1 || !B || !X || maxit < 1 || method < 0 || method > 2) return HF_ERR_ARG;
  cudaStream_t s = hf_stream(c);
  const int64_t L = c->L;
  const size_t blk = (size_t)L * m;
  std::vector<double> h;
  int it = 0, rc = HF_OK;
  if (method == 0) {
    const int save = c->opts.gcr_maxit;
    c->opts.gcr_maxit = maxit;
    double rr = 0;
    rc = block_gcr(c, m, B, X, &it, &rr, &h);
    c->opts.gcr_maxit = save;
  } else if (method == 1) {
    int r2;
    if ((r2 = hf_ensure(c->d_solve, (size_t)L * 2 * 8 + 256))) return r2;
    double* bj = (double*)c->d_solve.p;
    double* xj = bj + L;
    const int save = c->opts.gcr_maxit;
    c->opts.gcr_maxit = maxit;
    std::vector<std::vector<double>> hs(m);
    for (int j = 0; j < m && (rc == HF_OK || rc == HF_ERR_NOT_CONVERGED); ++j) {
      HF_CUDA_TRY(cudaMemcpy2DAsync(bj, 8, B + j, (size_t)m * 8, 8, L, cudaMemcpyDeviceToDevice, s));
      int itj = 0;
      double rr = 0;
      const int rj = block_gcr(c, 1, bj, xj, &itj, &rr, &hs[j]);
      if (rj != HF_OK && rj != HF_ERR_NOT_CONVERGED) { rc = rj; break; }
      if (rj == HF_ERR_NOT_CONVERGED) rc = rj;
      HF_CUDA_TRY(cudaMemcpy2DAsync(X + j, (size_t)m * 8, xj, 8, 8, L, cudaMemcpyDeviceToDevice, s));
      it = std::max(it, itj);
    }
    c->opts.gcr_maxit = save;
    size_t len = 0;
    for (const auto& v : hs) len = std::max(len, v.size());
    h.assign(len, 0.0);
    for (size_t k = 0; k < len; ++k)
      for (const auto& v : hs)
        if (!v.empty()) h[k] = std::max(h[k], v[std::min(k, v.size() - 1)]);
  } else {
    // iterative refinement, Alg. 3
    int r2;
    const size_t tmp_doubles = (blk * 3 + 1) / 2 + blk;
    if ((r2 = hf_ensure(c->d_solve, (blk * 2 + tmp_doubles) * 8 + 1024))) return r2;
    double* R = (double*)c->d_solve.p;
    double* W = R + blk;
    double* tmp = W + blk;
    std::vector<double> bnorm(m), none;
    double dummy = 0;
    if ((r2 = max_col_ratio(c, m, B, none, &dummy, &bnorm))) return r2;
    for (auto& v : bnorm) if (v == 0) v = 1.0;
    if ((r2 = precond(c, m, B, X, tmp))) return r2;                      // steps 1-2
    const unsigned nb = nblk((int64_t)blk, 256);
    rc = HF_ERR_NOT_CONVERGED;
    for (int n = 0;; ++n) {
      spmm(c, m, X, W);                                                   // step 3 / 4d
      HF_LAUNCH(c, HF_PROF_VECTOR, k_sub<<<nb, 256, 0, s>>>((int64_t)blk, B, W, R));
      double res = 0;
      if ((r2 = max_col_ratio(c, m, R, bnorm, &res))) return r2;
      h.push_back(res);
      it = n;
      if (!(res > c->opts.gcr_tol)) { rc = HF_OK; break; }
      if (n == maxit) break;
      if ((r2 = precond(c, m, R, W, tmp))) return r2;                     // 4a-4b
      HF_LAUNCH(c, HF_PROF_VECTOR, k_addto<<<nb, 256, 0, s>>>((int64_t)blk, W, X));   // 4c
    }
  }
  HF_CUDA_TRY(cudaGetLastError());
  HF_CUDA_TRY(cudaStreamSynchronize(s));
  if (hist) for (size_t k = 0; k < h.size() && k <= (size_t)maxit; ++k) hist[k] = h[k];
  if (iters) *iters = it;
  return rc;
}

int hf_precond_impl(hf_ctx* c, int m, const double* R, double* W) {
  if (!c || m < 1 || !R || !W) return HF_ERR_ARG;
  if (!c->factored) return HF_ERR_STATE;
  const size_t blk = (size_t)c->L * m;
  int rc;
  if ((rc = hf_ensure(c->d_solve, (blk * 3 + 64) * 8))) return rc;
  if ((rc = precond(c, m, R, W, c->d_solve.p))) return rc;
  return sweep_status(c);
}

// dJ/dKbar_ij = -sum_r lam_i^r x_j^r on the stored pattern (adjoint of the solve); one warp per row
__global__ void k_values_adjoint(int64_t L, int m, const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                                 const double* __restrict__ x, int64_t ldx, const double* __restrict__ lam,
                                 int64_t ldl, double* __restrict__ grad) {
  int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (row >= L) return;
  for (int64_t e = rowptr[row] + lane; e < rowptr[row + 1]; e += 32) {
    const int j = col[e];
    double g = 0.0;
    for (int r = 0; r < m; ++r) g += lam[row + r * ldl] * x[j + r * ldx];
    grad[e] = -g;
  }
}

int hf_values_adjoint_impl(hf_ctx* c, int m, const double* x, int64_t ldx, const double* lam, int64_t ldl,
                           double* grad) {
  if (!c || m < 1 || !x || !lam || !grad || ldx < c->L || ldl < c->L) return HF_ERR_ARG;
  if (!c->factored) return HF_ERR_STATE;
  cudaStream_t s = hf_stream(c);
  c->work_flops[HF_PROF_SCHUR] += 2.0 * (double)c->nnz * m;
  HF_LAUNCH(c, HF_PROF_SCHUR, k_values_adjoint<<<nblk(c->L * 32, 256), 256, 0, s>>>(c->L, m, (const int64_t*)c->d_rowptr.p,
                                                                                  (const int32_t*)c->d_col.p, x, ldx, lam, ldl, grad));
  HF_CUDA_TRY(cudaGetLastError());
  HF_CUDA_TRY(cudaStreamSynchronize(s));
  return HF_OK;
}

// ---------------------------------------------------------------------------
// Q^-1 without device allocation.  All scratch of the solve lives in this file-scope
// device array, which every GPU that loads the library holds until the process exits.
// ---------------------------------------------------------------------------
#define HF_NOALLOC_SCRATCH_BYTES (64ull << 20)
static __device__ __align__(256) unsigned char g_precond_scratch[HF_NOALLOC_SCRATCH_BYTES];

static void* g_precond_scratch_addr[64] = {nullptr};   // device address of the array, per device

int hf_precond_noalloc_impl(hf_ctx* c, int m, const double* R, double* W) {
  if (!c || m < 1 || !R || !W) return HF_ERR_ARG;
  if (!c->factored) return HF_ERR_STATE;
  int dev = 0;
  HF_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return HF_ERR_ARG;
  const bool dbl = c->prec == HF_PREC_FP64;
  const size_t esz = dbl ? 8 : 4;
  const size_t tmp_bytes = dbl ? (size_t)c->L * m * 8 : (size_t)c->L * m * 4 * 3;
  const size_t tmp_round = (tmp_bytes + 255) / 256 * 256;
  const size_t vec_bytes = sweep_vec_bytes(c, m, esz) + sweep_sync_bytes(c, m);
  if (tmp_round + vec_bytes > HF_NOALLOC_SCRATCH_BYTES) return HF_ERR_ARG;
  static std::mutex addr_mu;
  std::lock_guard<std::mutex> addr_lock(addr_mu);
  if (!g_precond_scratch_addr[dev]) {
    // host code only has a stand-in for the array's name: ask the runtime for the address
    // on this device (once per device, with that device current)
    void* p = nullptr;
    HF_CUDA_TRY(cudaGetSymbolAddress(&p, g_precond_scratch));
    g_precond_scratch_addr[dev] = p;
  }
  unsigned char* base = (unsigned char*)g_precond_scratch_addr[dev];
  const bool prof = c->prof_on;
  c->prof_on = false;                  // event bookkeeping could create events: keep it off here
  int rc = precond_on(c, m, R, W, base, base + tmp_round);
  c->prof_on = prof;
  if (rc) return rc;
  return sweep_status(c);
}

// Kernel basis of K-bar (mixed form; after hf_schur): L x kernel_dim column-major on the device.
int hf_kernel_basis_impl(hf_ctx* c, double* basis, int64_t ldb) {
  if (!c->schured) return HF_ERR_STATE;
  if (c->prec != HF_PREC_MIXED) return HF_ERR_STATE;
  const int M = (int)c->M, kd = c->kernel_dim;
  if (kd == 0) return HF_OK;
  if (!basis || ldb < c->L) return HF_ERR_ARG;
  cudaStream_t s = hf_stream(c);
  int rc;
  if ((rc = hf_ensure(c->d_small, ((size_t)M * kd + M + 64) * 8))) return rc;
  double* N2 = (double*)c->d_small.p;
  double* w = N2 + (size_t)M * kd;
  HF_LAUNCH(c, HF_PROF_DENSE_LDLT, k_s22_nullvecs<<<1, 256, 0, s>>>(M, (const double*)c->d_bk_lf.p, (const int*)c->d_bk_perm.p,
                                                               (const int*)c->d_bk_blk.p, (const double*)c->d_bk_dval.p,
                                                               (const int*)c->d_bk_null.p, kd, N2, w));
  HF_LAUNCH(c, HF_PROF_VECTOR, k_kernel_basis<<<dim3(nblk(c->L, 256), kd), 256, 0, s>>>(c->L, M, kd, (const double*)c->d_x12.p, N2,
                                                                              (const int32_t*)c->d_lam2pos.p,
                                                                              (const double*)c->d_q.p, basis, ldb));
  HF_CUDA_TRY(cudaGetLastError());
  HF_CUDA_TRY(cudaStreamSynchronize(s));
  return HF_OK;
}
