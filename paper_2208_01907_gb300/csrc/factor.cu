// Alg. 1 step 1 on the GPU: diagonal scaling (Sec. 2), multifrontal LDL^T along the
// dissection tree with symmetric max-|diag| pivoting and threshold postponing
// (Sec. 2.1-2.2), refactorization of the postponed set Lambda_0 and enlargement of
// the hard part (Sec. 2.2).
//
// Layout: every front t is a dense ld x ld column-major matrix in one arena; only
// its lower triangle is stored and updated.  Rows are ordered
// [Lambda_t | static structure | rows delayed from the children].  Pivoting permutes
// the first n rows (the candidates); after the front is done, columns [0, k) hold the
// factor (unit L below the diagonal, D on it) and the trailing block [k, f)^2 is the
// contribution passed to the parent by extend-add.
#include "common.cuh"
#include "tcgen05.cuh"

#include <cuda_bf16.h>

#include <cooperative_groups.h>
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <mutex>
#include <vector>

namespace {

constexpr int TB = 64;            // trailing-update tile
constexpr int TK = 16;            // trailing-update k chunk

// ---------------------------------------------------------------------------
// Sec. 2: Q_ii = 1/sqrt(|Kbar_ii|) (1 if zero) and K = Q Kbar Q.
// With row signs J (the LDU form Kbar = J S, S symmetric, Sec. 4.2) the rows are
// scaled by J Q instead: K = J Q Kbar Q = Q S Q, the symmetric matrix whose Schur
// complements are J times those of Q Kbar Q (same pivots and split, Sec. 2.1).
// ---------------------------------------------------------------------------
__global__ void k_scale_diag(int64_t L, const int64_t* __restrict__ diagpos, const double* __restrict__ vals,
                             double* __restrict__ q, const int8_t* __restrict__ rsign, double* __restrict__ qrow) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= L) return;
  double d = vals[diagpos[i]];
  const double qi = (d != 0.0) ? 1.0 / sqrt(fabs(d)) : 1.0;
  q[i] = qi;
  if (rsign) qrow[i] = rsign[i] < 0 ? -qi : qi;
}

// qrow: the row scale (Q, or J Q with row signs); q: the column scale Q
__global__ void k_scale_vals(int64_t L, const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                             const double* __restrict__ vals, const double* __restrict__ qrow,
                             const double* __restrict__ q, double* __restrict__ kval, int* __restrict__ flags) {
  int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (row >= L) return;
  double qi = qrow[row];
  bool bad = false;
  for (int64_t e = rowptr[row] + lane; e < rowptr[row + 1]; e += 32) {
    double v = vals[e];
    if (!isfinite(v)) bad = true;
    kval[e] = qi * v * q[col[e]];
  }
  if (bad) flags[FLAG_NUMERIC] = 1;
}

// ---------------------------------------------------------------------------
// Per level: delayed-row counts and front orders, extend-add maps
// ---------------------------------------------------------------------------
__global__ void k_level_prep(const NodeDesc* __restrict__ nd, NodeState* __restrict__ st, int t0, int cnt,
                             int* __restrict__ flags) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= cnt) return;
  int t = t0 + i;
  NodeDesc d = nd[t];
  int D = 0, off[2] = {0, 0};
  int ch[2] = {d.child0, d.child1};
  for (int s = 0; s < 2; ++s) {
    if (ch[s] < 0) continue;
    off[s] = D;
    // postponed candidates of the child plus the rows it received from its own children
    D += (nd[ch[s]].n - st[ch[s]].k) + st[ch[s]].D;
  }
  if (D > d.dc) { flags[FLAG_DELAY_OVERFLOW] = 1; D = d.dc; }
  NodeState S;
  S.k = 0; S.kp0 = 0; S.D = D; S.f = d.n + d.s + D; S.stopped = 0; S.dref = 1.0;   // reading R2
  S.ksolve = 0; S.nmoved = 0; S.delay_off0 = off[0]; S.delay_off1 = off[1];
  S.nact = d.cand_all ? S.f : d.n;
  st[t] = S;
}

// contribution rows of each child -> rows of this front; delayed rows get their ids
__global__ void k_level_maps(const NodeDesc* __restrict__ nd, const NodeState* __restrict__ st, int t0,
                             int32_t* __restrict__ rowid, const int32_t* __restrict__ smap,
                             int32_t* __restrict__ cbmap) {
  int t = t0 + blockIdx.x;
  NodeDesc d = nd[t];
  const int f = st[t].f;
  int ch[2] = {d.child0, d.child1};
  int off[2] = {st[t].delay_off0, st[t].delay_off1};
  for (int s = 0; s < 2; ++s) {
    int c = ch[s];
    if (c < 0) continue;
    NodeDesc dc = nd[c];
    int kc = st[c].k, fc = st[c].f;
    int base = d.n + d.s + off[s];
    for (int a = threadIdx.x; a < fc - kc; a += blockDim.x) {
      int p = kc + a;
      int tgt;
      if (p < dc.n) tgt = base + (p - kc);                                  // postponed in the child
      else if (p < dc.n + dc.s) tgt = smap[dc.smap_off + (p - dc.n)];       // static structure
      else tgt = base + (dc.n - kc) + (p - dc.n - dc.s);                    // delayed through the child
      if (tgt >= f) tgt = -1;                                               // only after an overflow
      cbmap[dc.row_off + a] = tgt;
      if (tgt >= d.n + d.s) rowid[d.row_off + tgt] = rowid[dc.row_off + p];
    }
  }
}

// ---------------------------------------------------------------------------
// Front assembly: zero, scatter scaled K entries, extend-add the children
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_front_zero(const NodeDesc* __restrict__ nd, const NodeState* __restrict__ st, int t0,
                             T* __restrict__ arena) {
  int t = t0 + blockIdx.y;
  NodeDesc d = nd[t];
  const int64_t f = st[t].f;
  T* F = arena + d.front_off;
  for (int64_t c = blockIdx.x; c < f; c += gridDim.x)
    for (int64_t r = c + threadIdx.x; r < f; r += blockDim.x) F[r + c * d.ld] = T(0);
}

template <typename T>
__global__ void k_front_asm(const NodeDesc* __restrict__ nd, int t0, const AsmEntry* __restrict__ al,
                            const double* __restrict__ kval, T* __restrict__ arena) {
  int t = t0 + blockIdx.y;
  NodeDesc d = nd[t];
  T* F = arena + d.front_off;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < d.asm_cnt; e += (int64_t)gridDim.x * blockDim.x) {
    AsmEntry a = al[d.asm_off + e];
    F[a.r + (int64_t)a.c * d.ld] = (T)kval[a.csr];
  }
}

template <typename T>
__global__ void k_extend_add(const NodeDesc* __restrict__ nd, const NodeState* __restrict__ st, int t0, int slot,
                             const int32_t* __restrict__ cbmap, T* __restrict__ arena) {
  int t = t0 + blockIdx.y;
  NodeDesc d = nd[t];
  int c = slot == 0 ? d.child0 : d.child1;
  if (c < 0) return;
  NodeDesc dc = nd[c];
  const int kc = st[c].k, m = st[c].f - kc;
  const T* CB = arena + dc.front_off + kc + (int64_t)kc * dc.ld;
  const int32_t* map = cbmap + dc.row_off;
  T* F = arena + d.front_off;
  // four entries of a column per pass, all loads before the stores: the map is one to one,
  // so the four targets are distinct and the loads need not wait for the stores before them
  constexpr int U = 4;
  for (int a = blockIdx.x; a < m; a += gridDim.x) {
    const int ta = map[a];
    if (ta < 0) continue;
    const T* cba = CB + (int64_t)a * dc.ld;
    for (int b0 = a + threadIdx.x; b0 < m; b0 += U * blockDim.x) {
      T v[U], o[U];
      int64_t pos[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int b = b0 + u * blockDim.x;
        const int tb = b < m ? map[b] : -1;
        pos[u] = -1;
        if (tb >= 0) {
          pos[u] = max(ta, tb) + (int64_t)min(ta, tb) * d.ld;
          v[u] = cba[b];
          o[u] = F[pos[u]];
        }
      }
#pragma unroll
      for (int u = 0; u < U; ++u)
        if (pos[u] >= 0) F[pos[u]] = o[u] + v[u];
    }
  }
}

// Term magnitudes G of the front rows (reading R3b): |K_ii| for the rows of Lambda_t,
// plus what the children accumulated for their contribution rows.
template <typename T>
__global__ void k_g_assemble(const NodeDesc* __restrict__ nd, const NodeState* __restrict__ st, int t0,
                             const int32_t* __restrict__ rowid, const int32_t* __restrict__ cbmap,
                             const int64_t* __restrict__ diagpos, const double* __restrict__ kval,
                             T* __restrict__ G, int32_t* __restrict__ pos0) {
  const int t = t0 + blockIdx.x;
  const NodeDesc d = nd[t];
  const int f = st[t].f;
  const int nown = d.cand_all ? 0 : d.n;
  T* Gt = G + d.row_off;
  for (int i = threadIdx.x; i < f; i += blockDim.x) {
    Gt[i] = (i < nown) ? (T)fabs(kval[diagpos[rowid[d.row_off + i]]]) : T(0);
    pos0[d.row_off + i] = i;                  // pivoting permutes this with the rows
  }
  __syncthreads();
  for (int slot = 0; slot < 2; ++slot) {
    const int c = slot == 0 ? d.child0 : d.child1;
    if (c < 0) continue;
    const NodeDesc dc = nd[c];
    const int kc = st[c].k, m = st[c].f - kc;
    const T* Gc = G + dc.row_off + kc;
    for (int a = threadIdx.x; a < m; a += blockDim.x) {
      int tg = cbmap[dc.row_off + a];
      if (tg >= 0) Gt[tg] += Gc[a];
    }
    __syncthreads();
  }
}

// symmetric swap of rows/columns a < b of a lower-stored front (order f)
template <typename T>
__device__ __forceinline__ void sym_swap(T* F, int64_t ld, int f, int a, int b, int tid, int nt) {
  const int nA = a, nB = b - a - 1, nC = f - b - 1;
  const int tot = nA + nB + nC + 1;
  for (int e = tid; e < tot; e += nt) {
    int64_t x, y;
    if (e < nA) { x = a + e * ld; y = b + e * ld; }                            // rows a, b left of a
    else if (e < nA + nB) { int j = a + 1 + (e - nA); x = j + a * ld; y = b + j * ld; }
    else if (e < nA + nB + nC) { int i = b + 1 + (e - nA - nB); x = i + a * ld; y = i + b * ld; }
    else { x = a + a * ld; y = b + b * ld; }
    T tmp = F[x]; F[x] = F[y]; F[y] = tmp;
  }
}

// sum_{c < n} a[c sa] * b[c] in four interleaved partial sums (c mod 4), added pairwise at
// the end: the chain of dependent multiply-adds is a quarter of the length of a sequential
// sum; the loads are issued eight at a time so that their latency overlaps.  Both panel
// kernels sum in this order, so they compute the same factor.
template <typename T>
__device__ __forceinline__ T dot4(const T* __restrict__ a, int64_t sa, const T* __restrict__ b, int n) {
  T s0 = T(0), s1 = T(0), s2 = T(0), s3 = T(0);
  int c = 0;
  for (; c + 8 <= n; c += 8) {
    T x[8], y[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) { x[u] = a[(c + u) * sa]; y[u] = b[c + u]; }
    s0 += x[0] * y[0]; s1 += x[1] * y[1]; s2 += x[2] * y[2]; s3 += x[3] * y[3];
    s0 += x[4] * y[4]; s1 += x[5] * y[5]; s2 += x[6] * y[6]; s3 += x[7] * y[7];
  }
  for (; c + 4 <= n; c += 4) {
    s0 += a[c * sa] * b[c]; s1 += a[(c + 1) * sa] * b[c + 1];
    s2 += a[(c + 2) * sa] * b[c + 2]; s3 += a[(c + 3) * sa] * b[c + 3];
  }
  if (c < n) s0 += a[c * sa] * b[c];
  if (c + 1 < n) s1 += a[(c + 1) * sa] * b[c + 1];
  if (c + 2 < n) s2 += a[(c + 2) * sa] * b[c + 2];
  return (s0 + s1) + (s2 + s3);
}

// ---------------------------------------------------------------------------
// Panel factorization with symmetric max-|diag| pivoting and the ratio test
// (Sec. 2.1-2.2).  One CTA per front; up to nb pivots; columns of the panel are
// computed left-looking, the rest of the front is updated by k_trailing.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_panel(const NodeDesc* __restrict__ nd, NodeState* __restrict__ st, int t0,
                        T* __restrict__ arena, int32_t* __restrict__ rowid, T* __restrict__ Gall,
                        int32_t* __restrict__ pos0all, int nb, double tau, double tau_null, int cap) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ T red_k[32];
  __shared__ int red_i[32], red_p[32];
  __shared__ int s_q, s_act;
  const int t = t0 + blockIdx.x;
  const NodeDesc d = nd[t];
  NodeState* S = st + t;
  const int f = S->f;
  const int ncand = d.cand_all ? f : d.n;
  const int k0 = S->k;
  int nact = S->nact;
  const int tid = threadIdx.x, nt = blockDim.x;
  if (f - k0 <= cap) return;               // handled by the shared-memory cluster kernel
  if (S->stopped || k0 >= nact) {
    if (tid == 0) S->kp0 = k0;
    return;
  }
  T* F = arena + d.front_off;
  T* G = Gall + d.row_off;
  const int64_t ld = d.ld;
  int32_t* rid = rowid + d.row_off;
  int32_t* pos0 = pos0all + d.row_off;
  T* w = (T*)smem_raw;                        // nb entries
  T* dg = w + nb;                             // ncand entries (front positions)
  int* sid = (int*)(dg + ncand);              // ncand entries
  for (int i = k0 + tid; i < nact; i += nt) {
    dg[i] = F[i + i * ld];
    sid[i] = rid[i];
  }
  double dref = S->dref;
  int k = k0;
  bool stopped = false;
  __syncthreads();
  while (k < k0 + nb && k < nact) {
    // 1. argmax |dg| over the active candidates, ties to the smaller original index (R5)
    T bk = T(-2);
    int bi = 0x7fffffff, bp = -1;
    for (int i = k + tid; i < nact; i += nt) {
      const T kk = piv_key_t(dg[i]);
      if (better_t(kk, sid[i], bk, bi)) { bk = kk; bi = sid[i]; bp = i; }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      T ok = __shfl_xor_sync(0xffffffffu, bk, o);
      int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      int op = __shfl_xor_sync(0xffffffffu, bp, o);
      if (better_t(ok, oi, bk, bi)) { bk = ok; bi = oi; bp = op; }
    }
    if ((tid & 31) == 0) { red_k[tid >> 5] = bk; red_i[tid >> 5] = bi; red_p[tid >> 5] = bp; }
    __syncthreads();
    if (tid == 0) {
      for (int wv = 1; wv < (nt + 31) / 32; ++wv)
        if (better_t(red_k[wv], red_i[wv], bk, bi)) { bk = red_k[wv]; bi = red_i[wv]; bp = red_p[wv]; }
      // ratio test |d_{i+1} / d_i| < tau stops the set (R2/R3; NaN fails it); the
      // optional null-pivot test |d| < tau * G postpones this candidate alone (R3b)
      int act = 0;
      if (!((double)bk >= tau * dref)) act = 1;
      else if (!((double)bk >= tau_null * (double)G[bp])) act = 2;
      s_act = act;
      s_q = bp;
    }
    __syncthreads();
    const int act = s_act, q = s_q;
    if (act == 1) { stopped = true; break; }
    if (act == 2) {
      // move the null candidate to the end of the active range
      const int last = nact - 1;
      if (q != last) {
        sym_swap(F, ld, f, q, last, tid, nt);
        if (tid == 0) {
          T td = dg[q]; dg[q] = dg[last]; dg[last] = td;
          int ti = sid[q]; sid[q] = sid[last]; sid[last] = ti;
          int tr = rid[q]; rid[q] = rid[last]; rid[last] = tr;
          int tp = pos0[q]; pos0[q] = pos0[last]; pos0[last] = tp;
          T tg = G[q]; G[q] = G[last]; G[last] = tg;
        }
      }
      --nact;
      __syncthreads();
      continue;
    }
    // 2. symmetric swap k <-> q in lower storage
    if (q != k) {
      sym_swap(F, ld, f, k, q, tid, nt);
      if (tid == 0) {
        T td = dg[k]; dg[k] = dg[q]; dg[q] = td;
        int ti = sid[k]; sid[k] = sid[q]; sid[q] = ti;
        int tr = rid[k]; rid[k] = rid[q]; rid[q] = tr;
        int tp = pos0[k]; pos0[k] = pos0[q]; pos0[q] = tp;
        T tg = G[k]; G[k] = G[q]; G[q] = tg;
      }
    }
    __syncthreads();
    // 3. w_t = d_t * L(k, t) for the panel columns already done
    for (int c = k0 + tid; c < k; c += nt) w[c - k0] = F[c + c * ld] * F[k + c * ld];
    __syncthreads();
    // 4. current column k: c_i = A(i, k) - sum_t L(i, t) d_t L(k, t)
    for (int i = k + tid; i < f; i += nt)
      F[i + k * ld] = F[i + k * ld] - dot4(F + i + (int64_t)k0 * ld, ld, w, k - k0);
    __syncthreads();
    const T dk = F[k + k * ld];
    // 5. L(i, k) = c_i / d_k, the candidates' diagonals and the term magnitudes
    for (int i = k + 1 + tid; i < f; i += nt) {
      T c = F[i + k * ld];
      T l = c / dk;
      F[i + k * ld] = l;
      if (i < nact) dg[i] -= l * c;
      G[i] += fabs(l * c);
    }
    if (tid == 0) dref = fabs((double)dk);     // used by the deciding thread only
    ++k;
    __syncthreads();
  }
  if (tid == 0) {
    S->kp0 = k0;
    S->k = k;
    S->dref = dref;
    S->nact = nact;
    if (stopped) S->stopped = 1;
  }
}

// ---------------------------------------------------------------------------
// The same panel step with the panel resident in distributed shared memory: a
// cluster of C CTAs per front, CTA r owning the front positions
// [k0 + r R, k0 + (r+1) R) of the rows [k0, f).  Each CTA keeps, for its rows, the
// panel columns computed so far (row-major, stride nb+1) and the per-row data
// (running candidate diagonal, diagonal entry, term magnitude, ids).
//
// One cluster barrier per pivot.  Before it, every CTA pushes into every CTA's
// (double-buffered) slots: its best candidate (key, id, G, diagonal, panel row),
// and the owners of positions k and nact-1 push those rows.  After it, every CTA
// takes the same decision (R2, R3, the optional R3b, R5) from its local slots, forms
// w_c = d_c L(q, c), computes d_k itself (the same operations as the owner's) and
// processes its own rows: the symmetric swap k <-> q is fused into the load of the new
// column k, then L(i, k), the diagonals and the magnitudes.  The arithmetic per element
// is that of k_panel, in the same order.  A front larger than C * Rcap rows is left to
// k_panel (which skips the fronts handled here).
// ---------------------------------------------------------------------------
// smallest float >= x (for a float g, g >= x exactly when g >= ceil_float(x); NaN stays NaN)
__device__ __forceinline__ float ceil_float(double x) {
  float f = (float)x;
  if ((double)f < x) f = nextafterf(f, INFINITY);
  return f;
}

// the ratio-test threshold in the factor's type: g >= x exactly when g >= thr_up<T>(x)
template <typename T> __device__ __forceinline__ T thr_up(double x);
template <> __device__ __forceinline__ float thr_up<float>(double x) { return ceil_float(x); }
template <> __device__ __forceinline__ double thr_up<double>(double x) { return x; }

// the data pushed with a candidate row into a slot of every CTA of the cluster
template <typename T> struct __align__(16) PclMeta {
  T key, G, diag, dg;                          // pivot key, term magnitude, diagonal entry, running diagonal
  int sid, pos, rid, p0;                       // original index, front position, row id, position before pivoting
};
template <typename T>
__device__ __forceinline__ void pcl_store_meta(PclMeta<T>* dst, const PclMeta<T>& m) {
  const int4* src = reinterpret_cast<const int4*>(&m);
  int4* d = reinterpret_cast<int4*>(dst);
#pragma unroll
  for (int u = 0; u < (int)(sizeof(PclMeta<T>) / 16); ++u) d[u] = src[u];
}

constexpr int PCL_THREADS = 512;
constexpr int PCL_RPT = 2;                    // rows per thread: Rcap <= PCL_RPT * PCL_THREADS
constexpr int PCL_CMAX = 16;
constexpr int PCL_SLOTS = PCL_CMAX + 2;       // candidates of C CTAs, row k, row nact-1
constexpr int PCL_SWAPS = 256;                // listed row interchanges staged in shared memory

template <typename T> struct PclLayout {
  // bytes of dynamic shared memory for Rcap rows and panel width nb
  static size_t bytes(int Rcap, int nb) {
    const size_t per_row = (size_t)(nb + 1) * sizeof(T) + 3 * sizeof(T) + 3 * sizeof(int);
    return (size_t)Rcap * per_row + 2 * (size_t)nb * sizeof(T) + push_bytes(nb) + 64;
  }
  static size_t push_bytes(int nb) {
    return 2 * (size_t)PCL_SLOTS * ((size_t)nb * sizeof(T) + 3 * sizeof(T) + sizeof(double) + 4 * sizeof(int));
  }
};

template <typename T>
__global__ void __launch_bounds__(PCL_THREADS, 1)
k_panel_cl(const NodeDesc* __restrict__ nd, NodeState* __restrict__ st, int t0, T* __restrict__ arena,
           int32_t* __restrict__ rowid, T* __restrict__ Gall, int32_t* __restrict__ pos0all, int nb, double tau,
           double tau_null, int C, int Rcap, int4* __restrict__ swlist, int* __restrict__ swcount) {
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ T red_k[32];
  __shared__ int red_i[32], red_p[32];
  __shared__ int s_swa[PCL_SWAPS], s_swb[PCL_SWAPS];
  __shared__ T s_thr;                          // tau |previous pivot| rounded up to T
  const int rank = (int)cl.block_rank();
  const int t = t0 + (int)(blockIdx.x / (unsigned)C);
  const NodeDesc d = nd[t];
  NodeState* S = st + t;
  const int f = S->f;
  const int k0 = S->k;
  int nact = S->nact;
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31;
  // the same decisions in every CTA of the cluster
  if (S->stopped || k0 >= nact || f - k0 > C * Rcap) {
    if (rank == 0 && tid == 0 && (S->stopped || k0 >= nact)) S->kp0 = k0;
    return;
  }
  T* F = arena + d.front_off;
  T* Gg = Gall + d.row_off;
  const int64_t ld = d.ld;
  int32_t* rid = rowid + d.row_off;
  int32_t* pos0 = pos0all + d.row_off;
  const int ps = nb + 1;
  const int swbase = swcount[t];                       // read before the cluster barrier below
  // dynamic shared memory
  T* P = (T*)smem_raw;                         // Rcap x ps: panel rows
  T* dgl = P + (size_t)Rcap * ps;              // running candidate diagonal
  T* Gl = dgl + Rcap;                          // term magnitudes
  T* diagl = Gl + Rcap;                        // diagonal entries F(p, p)
  T* wv = diagl + Rcap;                        // nb
  T* dpiv = wv + nb;                           // nb: pivots of this panel
  T* prow = dpiv + nb;                         // [2][SLOTS][nb] pushed panel rows
  // [2][SLOTS] pushed row data, one 16-byte aligned record per slot (stored with vector stores)
  PclMeta<T>* pm = (PclMeta<T>*)(((uintptr_t)(prow + 2 * PCL_SLOTS * nb) + 15) & ~(uintptr_t)15);
  int* sidl = (int*)(pm + 2 * PCL_SLOTS);      // Rcap
  int* ridl = sidl + Rcap;                     // Rcap
  int* pos0l = ridl + Rcap;                    // Rcap
  const int R = (f - k0 + C - 1) / C;
  const int p0 = k0 + rank * R, p1 = min(f, p0 + R);
  auto owner = [&](int p) { return (p - k0) / R; };
  for (int p = p0 + tid; p < p1; p += nt) {
    const int l = p - p0;
    const T dv = F[p + (int64_t)p * ld];
    diagl[l] = dv;
    dgl[l] = dv;
    Gl[l] = Gg[p];
    sidl[l] = rid[p];
    ridl[l] = rid[p];
    pos0l[l] = pos0[p];
  }
  double dref = S->dref;                       // kept by the last thread
  if (tid == nt - 1) s_thr = thr_up<T>(tau * dref);
  int k = k0;
  bool stopped = false;
  int it = 0;
  cl.sync();
  // push the row at own position p into slot `slot` of buffer `buf` of every CTA
  auto push_row = [&](int buf, int slot, int p, T key, int kk) {
    const int l = p - p0;
    const int base = buf * PCL_SLOTS + slot;
    for (int e = tid; e < C * kk; e += nt) {
      const int r = e / kk, c = e - r * kk;
      cl.map_shared_rank(prow, r)[(size_t)base * nb + c] = P[(size_t)l * ps + c];
    }
    if (tid < C) {
      PclMeta<T> mt;
      mt.key = key; mt.G = Gl[l]; mt.diag = diagl[l]; mt.dg = dgl[l];
      mt.sid = sidl[l]; mt.pos = p; mt.rid = ridl[l]; mt.p0 = pos0l[l];
      pcl_store_meta(cl.map_shared_rank(pm, tid) + base, mt);
    }
  };
  // The row interchanges of the columns of earlier panels, [0, k0), are not needed by this
  // panel nor by any later step of the front's factorization: they are appended, in order
  // and tagged with this panel's k0, to the front's interchange list, and the columns are
  // put in their final row order once, after the front's last panel (k_swap_sigma,
  // k_swap_apply), instead of two strided accesses per column and pivot here.
  int4* gl = swlist + 2 * d.row_off;                   // 2 ld entries: <= ld pivots + ld postponements
  const int gcap = 2 * (int)ld;
  int nsw = 0, gsw = swbase;
  auto defer_swap = [&](int a, int b) {               // uniform across the block
    if (nsw == PCL_SWAPS) {
      __syncthreads();
      if (rank == 0)
        for (int i = tid; i < nsw; i += nt)
          if (gsw + i < gcap) gl[gsw + i] = make_int4(s_swa[i], s_swb[i], k0, 0);
      __syncthreads();
      gsw += nsw;
      nsw = 0;
    }
    if (tid == 0) { s_swa[nsw] = a; s_swb[nsw] = b; }
    ++nsw;
  };

  // rows are owned by fixed threads: position p belongs to thread (p - p0) % nt, so the
  // column updates of one pivot and the argmax of the next touch only the thread's rows
  while (k < k0 + nb && k < nact) {
    const int buf = it & 1;
    const int kk = k - k0;
    // 1. argmax over the own candidates [k, nact), ties to the smaller original index (R5)
    T bk = T(-2);
    int bi = 0x7fffffff, bp = -1;
#pragma unroll
    for (int j = 0; j < PCL_RPT; ++j) {
      const int p = p0 + tid + j * nt;
      if (p >= k && p < nact && p < p1) {
        const T kv = piv_key_t(dgl[p - p0]);
        const int si = sidl[p - p0];
        if (better_t(kv, si, bk, bi)) { bk = kv; bi = si; bp = p; }
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      T ok = __shfl_xor_sync(0xffffffffu, bk, o);
      int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      int op = __shfl_xor_sync(0xffffffffu, bp, o);
      if (better_t(ok, oi, bk, bi)) { bk = ok; bi = oi; bp = op; }
    }
    if (lane == 0) { red_k[tid >> 5] = bk; red_i[tid >> 5] = bi; red_p[tid >> 5] = bp; }
    __syncthreads();
    {
      // every warp reduces the warps' candidates itself (the same result everywhere), so
      // no second block barrier publishes it
      const int nw = (nt + 31) / 32;
      bk = lane < nw ? red_k[lane] : T(-2);
      bi = lane < nw ? red_i[lane] : 0x7fffffff;
      bp = lane < nw ? red_p[lane] : -1;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        T ok = __shfl_xor_sync(0xffffffffu, bk, o);
        int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        int op = __shfl_xor_sync(0xffffffffu, bp, o);
        if (better_t(ok, oi, bk, bi)) { bk = ok; bi = oi; bp = op; }
      }
    }
    // 2. pushes: own candidate, and rows k / nact-1 by their owners
    {
      const int pbest = bp;
      const int base = buf * PCL_SLOTS + rank;
      if (pbest >= 0) {
        push_row(buf, rank, pbest, bk, kk);
      } else if (tid < C) {
        PclMeta<T> mt = {};
        mt.key = T(-2); mt.sid = 0x7fffffff; mt.pos = -1;
        pcl_store_meta(cl.map_shared_rank(pm, tid) + base, mt);
      }
      if (owner(k) == rank) push_row(buf, PCL_CMAX, k, T(0), kk);
      // row nact-1 is read only when a candidate is postponed alone (the null-pivot test)
      if (tau_null > 0.0 && owner(nact - 1) == rank) push_row(buf, PCL_CMAX + 1, nact - 1, T(0), kk);
    }
    if (C > 1) cl.sync(); else __syncthreads();                            // the only cluster barrier
    // 3. the decision from the local slots, taken by every warp (the same in every warp and
    // every CTA, so no block barrier publishes it): the argmax over the C slots by the lanes
    // (the order is strict: ids are unique), the FP64 null-pivot test by lane 0
    const int sb = buf * PCL_SLOTS;
    int act, wslot;
    {
      T gk = T(-2);
      int gi = 0x7fffffff, gw = -1;
      if (lane < C && pm[sb + lane].pos >= 0) { gk = pm[sb + lane].key; gi = pm[sb + lane].sid; gw = lane; }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const T ok = __shfl_xor_sync(0xffffffffu, gk, o);
        const int oi = __shfl_xor_sync(0xffffffffu, gi, o);
        const int ow = __shfl_xor_sync(0xffffffffu, gw, o);
        if (better_t(ok, oi, gk, gi)) { gk = ok; gi = oi; gw = ow; }
      }
      // ratio test (R2/R3) against the threshold in the factor's type (exact: gk is a T,
      // s_thr the smallest T >= tau |d_prev|); the null-pivot test (R3b) only when asked for
      int a2 = 0;
      if (!(gk >= s_thr)) a2 = 1;
      else if (tau_null > 0.0) {
        if (lane == 0) a2 = ((double)gk >= tau_null * (double)pm[sb + gw].G) ? 0 : 2;
        a2 = __shfl_sync(0xffffffffu, a2, 0);
      }
      act = a2;
      wslot = gw;
    }
    const int wsl = sb + wslot;
    const int q = wslot >= 0 ? pm[wsl].pos : -1;
    if (act == 1) { stopped = true; break; }
    if (act == 2) {
      // 4a. postpone the null candidate: swap q <-> b = nact-1 (both candidates)
      const int b = nact - 1;
      if (q != b) {
        const int bsl = sb + PCL_CMAX + 1;
        // rows q and b over the trailing columns [k, q), spread over the cluster (ordered
        // before any later use by the next cluster barrier); over [0, k0): deferred
        for (int e = rank * nt + tid; e < q - k; e += C * nt) {
          const int j = k + e;
          const int64_t x = q + (int64_t)j * ld, y = b + (int64_t)j * ld;
          const T tmp = F[x]; F[x] = F[y]; F[y] = tmp;
        }
        defer_swap(q, b);
        if (owner(q) == rank) {
          const int l = q - p0;
          for (int c = tid; c < kk; c += nt) P[(size_t)l * ps + c] = prow[(size_t)bsl * nb + c];
          if (tid == 0) {
            dgl[l] = pm[bsl].dg; Gl[l] = pm[bsl].G; diagl[l] = pm[bsl].diag;
            sidl[l] = pm[bsl].sid; ridl[l] = pm[bsl].rid; pos0l[l] = pm[bsl].p0;
          }
        }
        if (owner(b) == rank) {
          const int l = b - p0;
          for (int c = tid; c < kk; c += nt) P[(size_t)l * ps + c] = prow[(size_t)wsl * nb + c];
          if (tid == 0) {
            dgl[l] = pm[wsl].dg; Gl[l] = pm[wsl].G; diagl[l] = pm[wsl].diag;
            sidl[l] = pm[wsl].sid; ridl[l] = pm[wsl].rid; pos0l[l] = pm[wsl].p0;
          }
        }
        // middle (j in (q, b): (j, q) <-> (b, j)) and lower (i > b: (i, q) <-> (i, b)) parts by row owners
#pragma unroll
        for (int j = 0; j < PCL_RPT; ++j) {
          const int p = p0 + tid + j * nt;
          if (p > q && p < p1 && p != b) {
            const int64_t x = p + (int64_t)q * ld;
            const int64_t y = p < b ? b + (int64_t)p * ld : p + (int64_t)b * ld;
            const T tmp = F[x]; F[x] = F[y]; F[y] = tmp;
          }
        }
      }
      --nact;
      ++it;
      __syncthreads();
      continue;
    }
    // 4. loads first, as soon as q is known: the new column k of the own rows (swap fused),
    // in flight while the rows of positions k and q are exchanged below; the interchange of
    // rows k and q over the earlier panels' columns [0, k0) is listed for the end of the panel
    T v[PCL_RPT];
    int64_t wy[PCL_RPT];
    T wx[PCL_RPT];
#pragma unroll
    for (int j = 0; j < PCL_RPT; ++j) {
      const int p = p0 + tid + j * nt;
      wy[j] = -1;
      v[j] = T(0);
      if (p > k && p < p1) {
        if (q == k) {
          v[j] = F[p + (int64_t)k * ld];
        } else if (p != q) {
          const int64_t x = p + (int64_t)k * ld;
          wy[j] = p > q ? p + (int64_t)q * ld : q + (int64_t)p * ld;
          v[j] = F[wy[j]];
          wx[j] = F[x];
        } else {
          v[j] = F[q + (int64_t)k * ld];
        }
      }
    }
    if (q != k) defer_swap(k, q);                      // rows k and q over [0, k0)
    // 5. pivot q -> position k: w from the winner's row, new contents of positions k and q
    const T* rq = prow + (size_t)wsl * nb;
    const int ksl = sb + PCL_CMAX;
    const T* rk = prow + (size_t)ksl * nb;
    for (int c = tid; c < kk; c += nt) wv[c] = dpiv[c] * rq[c];
    if (owner(k) == rank) {
      const int l = k - p0;
      for (int c = tid; c < kk; c += nt) P[(size_t)l * ps + c] = rq[c];
      if (tid == 0) {
        sidl[l] = pm[wsl].sid; ridl[l] = pm[wsl].rid; pos0l[l] = pm[wsl].p0; Gl[l] = pm[wsl].G;
      }
    }
    if (q != k && owner(q) == rank) {
      const int l = q - p0;
      for (int c = tid; c < kk; c += nt) P[(size_t)l * ps + c] = rk[c];
      if (tid == 0) {
        dgl[l] = pm[ksl].dg; Gl[l] = pm[ksl].G; diagl[l] = pm[ksl].diag;
        sidl[l] = pm[ksl].sid; ridl[l] = pm[ksl].rid; pos0l[l] = pm[ksl].p0;
      }
    }
    __syncthreads();
    // d_k by every thread: the owner's operations on the winner's row
    const T dk = pm[wsl].diag - dot4(rq, 1, wv, kk);
    // 6. c_i = A(i, k) - sum_c L(i, c) w_c; L(i, k) = c_i / d_k; diagonals and magnitudes
#pragma unroll
    for (int j = 0; j < PCL_RPT; ++j) {
      const int p = p0 + tid + j * nt;
      if (p > k && p < p1) {
        const int l = p - p0;
        T* Pr = P + (size_t)l * ps;
        // the sum does not wait for the column's load, which is still in flight
        const T acc = v[j] - dot4(Pr, 1, wv, kk);
        if (wy[j] >= 0) F[wy[j]] = wx[j];
        const T lv = acc / dk;
        Pr[kk] = lv;
        if (p < nact) dgl[l] -= lv * acc;
        Gl[l] += fabs(lv * acc);
      } else if (p == k && p < p1) {                   // position k, if this CTA owns it
        P[(size_t)(k - p0) * ps + kk] = dk;
      }
    }
    if (tid == 0) dpiv[kk] = dk;
    // the next threshold, in FP64, by the last thread: it has the fewest rows of the CTA,
    // so this latency stays off the pivot's critical path
    if (tid == nt - 1) {
      dref = fabs((double)dk);
      s_thr = thr_up<T>(tau * dref);
    }
    ++k;
    ++it;
  }
  // write back: computed panel columns (lower part), diagonals of the unpivoted rows, row data
  __syncthreads();
  if (rank == 0) {                                     // the rest of this panel's interchanges
    for (int i = tid; i < nsw; i += nt)
      if (gsw + i < gcap) gl[gsw + i] = make_int4(s_swa[i], s_swb[i], k0, 0);
    if (tid == 0) swcount[t] = min(gcap, gsw + nsw);
  }
  const int kdone = k - k0;
  for (int c = 0; c < kdone; ++c)
    for (int p = max(p0, k0 + c) + tid; p < p1; p += nt)
      F[p + (int64_t)(k0 + c) * ld] = P[(size_t)(p - p0) * ps + c];
  for (int p = max(p0, k) + tid; p < p1; p += nt) F[p + (int64_t)p * ld] = diagl[p - p0];
  for (int p = p0 + tid; p < p1; p += nt) {
    const int l = p - p0;
    Gg[p] = Gl[l];
    rid[p] = ridl[l];
    pos0[p] = pos0l[l];
  }
  if (rank == 0 && tid == 0) {
    S->kp0 = k0;
    S->k = k;
    S->nact = nact;
    if (stopped) S->stopped = 1;
  }
  if (rank == 0 && tid == nt - 1) S->dref = dref;
  cl.sync();                               // no CTA leaves while its shared memory may be written
}

// ---------------------------------------------------------------------------
// Final row order of the factor columns of the cluster-panel fronts.  The panel lists its
// row interchanges (a, b) tagged with its first column k0 instead of applying them to the
// columns [0, k0) of earlier panels.  A column c must receive, in list order, every
// interchange tagged k0 > c: walking the list backwards one panel at a time, the map
// sigma (new row pos takes old row sigma[pos]) of the interchanges after panel g is
// sigma_g = s_g o sigma_{g+1}, s_g the panel's own composition (tabulated by applying its
// interchanges, in order, to an identity array).  k_swap_sigma stores sigma_g per panel;
// k_swap_apply gathers each column through shared memory (coalesced reads and writes).
// ---------------------------------------------------------------------------
constexpr size_t SW_SMEM = 200 * 1024;   // fronts of up to 25,600 rows
// sig layout per front (stride sf): groups g = 0.. (last panel first), each sg ints:
// [tag k0, sigma[0 .. f)]
constexpr int SW_THREADS = 1024;
constexpr int SW_WIN = 256;              // list entries staged in shared memory at a time
__global__ void __launch_bounds__(SW_THREADS) k_swap_sigma(const NodeDesc* __restrict__ nd, const NodeState* __restrict__ st,
                                                    int t0, const int4* __restrict__ swlist,
                                                    const int* __restrict__ swcount, int* __restrict__ sig, int64_t sf,
                                                    int sg, int gcap, int* __restrict__ ngrp) {
  extern __shared__ int sw_smem[];
  __shared__ int2 lst[SW_WIN];
  __shared__ int s_cut;
  const int t = t0 + blockIdx.x;
  const int n = swcount[t];
  const int tid = threadIdx.x, nt = blockDim.x;
  if (n <= 0) { if (tid == 0) ngrp[blockIdx.x] = 0; return; }
  const NodeDesc d = nd[t];
  const int f = st[t].f;
  const int4* list = swlist + 2 * d.row_off;
  int* sigma = sw_smem;            // f
  int* img = sw_smem + f;          // f: composition of one panel's interchanges
  int* out = sig + (int64_t)blockIdx.x * sf;
  for (int p = tid; p < f; p += nt) { sigma[p] = p; img[p] = p; }
  __syncthreads();
  int g = 0;
  int i = n - 1;
  while (i >= 0 && g < gcap) {
    // entries [j, i]: one panel (the run of entry i's tag), found a window at a time: the
    // last entry before i with another tag ends the run
    const int tag = list[i].z;
    int j = i;
    for (;;) {
      const int lo = max(0, j - SW_WIN);
      if (tid == 0) s_cut = -1;
      __syncthreads();
      for (int e = lo + tid; e < j; e += nt)
        if (list[e].z != tag) atomicMax(&s_cut, e);
      __syncthreads();
      const int cut = s_cut;
      __syncthreads();
      if (cut >= 0) { j = cut + 1; break; }
      j = lo;
      if (lo == 0) break;
    }
    // the panel's interchanges, in order, on img: staged into shared memory, applied by one
    // thread (each may touch the rows of the ones before it)
    for (int e0 = j; e0 <= i; e0 += SW_WIN) {
      const int ne = min(SW_WIN, i - e0 + 1);
      for (int e = tid; e < ne; e += nt) {
        const int4 v = list[e0 + e];
        lst[e] = make_int2(v.x, v.y);
      }
      __syncthreads();
      if (tid == 0)
        for (int e = 0; e < ne; ++e) {
          const int a = lst[e].x, b = lst[e].y;
          const int x = img[a]; img[a] = img[b]; img[b] = x;
        }
      __syncthreads();
    }
    for (int p = tid; p < f; p += nt) sigma[p] = img[sigma[p]];
    __syncthreads();
    int* og = out + (int64_t)g * sg;
    if (tid == 0) og[0] = tag;
    for (int p = tid; p < f; p += nt) og[1 + p] = sigma[p];
    // img back to the identity on the rows the panel touched (same values from any thread)
    for (int e = j + tid; e <= i; e += nt) {
      const int4 v = list[e];
      img[v.x] = v.x;
      img[v.y] = v.y;
    }
    __syncthreads();
    ++g;
    i = j - 1;
  }
  if (tid == 0) ngrp[blockIdx.x] = g;
}

// One column c of a front per block: the rows [c + 1, f) take their final order.
template <typename T>
__global__ void __launch_bounds__(256) k_swap_apply(const NodeDesc* __restrict__ nd, const NodeState* __restrict__ st,
                                                    int t0, T* __restrict__ arena, const int* __restrict__ sig,
                                                    int64_t sf, int sg, const int* __restrict__ ngrp) {
  extern __shared__ __align__(16) unsigned char sw_buf[];
  const int ng = ngrp[blockIdx.y];
  if (ng == 0) return;
  const int t = t0 + blockIdx.y;
  const int c = blockIdx.x;
  const int k = st[t].k, f = st[t].f;
  if (c >= k) return;
  const int* base = sig + (int64_t)blockIdx.y * sf;
  // m = the panels with tag > c; the tags decrease with g, so m is one past the last such g
  // (all tags read at once, not one after another)
  __shared__ int s_m;
  if (threadIdx.x == 0) s_m = 0;
  __syncthreads();
  for (int g = threadIdx.x; g < ng; g += blockDim.x)
    if (base[(int64_t)g * sg] > c) atomicMax(&s_m, g + 1);
  __syncthreads();
  const int m = s_m;
  if (m == 0) return;
  const int* sigma = base + (int64_t)(m - 1) * sg + 1;
  const NodeDesc d = nd[t];
  T* col = arena + d.front_off + (int64_t)c * d.ld;
  T* buf = (T*)sw_buf;
  const int r0 = c + 1;
  for (int p = r0 + threadIdx.x; p < f; p += blockDim.x) buf[p - r0] = col[p];
  __syncthreads();
  for (int p = r0 + threadIdx.x; p < f; p += blockDim.x) {
    const int q = sigma[p];                            // in [c + 1, f): interchanges tagged > c
    if (q != p && q >= r0 && q < f) col[p] = buf[q - r0];
  }
}

// ---------------------------------------------------------------------------
// Trailing update of the front: A[k1:f, k1:f] -= W D W^T (lower tiles only),
// W = L[k1:f, k0:k1], D = diag(d_k0..d_k1-1)   (rank-nb Schur update, Sec. 2.1)
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) k_trailing(const NodeDesc* __restrict__ nd, const NodeState* __restrict__ st,
                                                  int t0, T* __restrict__ arena) {
  const int t = t0 + blockIdx.z;
  const NodeDesc d = nd[t];
  const int k0 = st[t].kp0, k1 = st[t].k, f = st[t].f;
  if (k1 <= k0) return;
  const int bi = blockIdx.x, bj = blockIdx.y;
  if (bj > bi) return;
  const int r0 = k1 + bi * TB, c0 = k1 + bj * TB;
  if (r0 >= f) return;
  T* F = arena + d.front_off;
  const int64_t ld = d.ld;
  __shared__ T As[TK][TB + 1];
  __shared__ T Bs[TK][TB + 1];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  T acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = T(0);
  for (int kc = k0; kc < k1; kc += TK) {
    for (int e = threadIdx.x; e < TK * TB; e += 256) {
      int kk = e / TB, rr = e % TB;
      int c = kc + kk;
      T a = T(0), b = T(0);
      if (c < k1) {
        int r = r0 + rr;
        if (r < f) a = F[r + c * ld];
        int r2 = c0 + rr;
        if (r2 < f) b = F[r2 + c * ld] * F[c + c * ld];
      }
      As[kk][rr] = a;
      Bs[kk][rr] = b;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < TK; ++kk) {
      T av[4], bv[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) av[i] = As[kk][tx + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) bv[j] = Bs[kk][ty + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] += av[i] * bv[j];
    }
    __syncthreads();
  }
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    int c = c0 + ty + 16 * j;
    if (c >= f) continue;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      int r = r0 + tx + 16 * i;
      if (r < f && r >= c) F[r + c * ld] -= acc[i][j];
    }
  }
}

// ---------------------------------------------------------------------------
// The same trailing update on the tensor cores (the precision form of the FP32 factor).
// Each FP32 operand is split exactly into three BF16 parts, x = x0 + x1 + x2 with
// x0 = bf16(x), x1 = bf16(x - x0), x2 = bf16(x - x0 - x1) (24 significant bits), and
// the six products of total order <= 2 accumulate in FP32 in TMEM: the order-0 product
// x0 y0 in one accumulator, the five of orders 1 and 2 (at most 2^-8 of it) in a second,
// the two added in registers, so the tensor core's FP32 accumulation never adds terms of
// very different magnitude.  The dropped products are below 2^-24 of |W| |D| |W|^T, the
// rounding level of the FP32 SIMT update.
//
// One persistent CTA per SM takes the 128 x 128 tiles of the lower trailing blocks of
// all fronts of the level in a fixed order (tile u, u + grid, ...).  Warp roles:
//   warp 0  one thread issues the bulk copies of a tile's pre-split operands into one of
//           two shared-memory stages (the parts are laid out so that a tile's rows of one
//           part and k-group are one contiguous block)
//   warp 1  allocates TMEM (two accumulator pairs of 2 x 128 columns) and one thread
//           issues the 24 MMAs of a tile (M = N = 128, K = 16, kind::f16)
//   warps 2-9  the epilogue: TMEM -> registers, C -= acc0 + acc1 on the lower triangle
//           (two warps per TMEM lane quarter, 64 columns each)
// so the copies of tile u+1 and the epilogue of tile u-1 overlap the MMAs of tile u.
// Every mbarrier wait is bounded; a wait that gives up sets the error flag and an abort
// word that ends every role, each role waits (bounded) for its own work in flight, and
// the TMEM is freed before the CTA returns.
// ---------------------------------------------------------------------------
constexpr int TT_M = 128, TT_K = 64;                 // tile rows; k = the panel's columns
constexpr int TT_EPI = 8;                           // epilogue warps: two per TMEM lane quarter
constexpr int TT_THREADS = 64 + 32 * TT_EPI;
static_assert(TT_THREADS % 32 == 0 && TT_THREADS <= 32 * 32, "the tile prefix scans one warp total per lane");
constexpr int TT_PART = TT_M * TT_K * 2;            // 16 KB: one BF16 part of 128 rows x 64 k
constexpr int TT_MAXF = 4096;                       // fronts per level the tile map holds
constexpr int TT_COLS = 512;                        // TMEM columns allocated (all of them)
constexpr int TT_SPIN = 1 << 22;
constexpr int TT_MIN_ROWS = 256;                    // levels with smaller fronts keep the SIMT update

// Tile shape and accumulation of one form of the kernel: TN columns per tile; the order-0
// products x0 y0 of the tile's k range are summed by the tensor core in KS accumulators
// (k-steps of 16 split evenly over them), the order-1 and order-2 products in one more;
// the KS + 1 partial sums are added in registers.  NBUF accumulator sets fit the TMEM.
template <int TN, int KS> struct TtCfg {
  static constexpr int B_PART = TN * TT_K * 2;
  static constexpr int STAGE = 3 * TT_PART + 3 * B_PART;
  static constexpr int ACOLS = (KS + 1) * TN;                  // TMEM columns of one accumulator set
  static constexpr int NBUF = 2 * ACOLS <= TT_COLS ? 2 : 1;
  static constexpr int SMEM = 2 * STAGE + (TT_MAXF + 1) * 4 + 1024;
  static constexpr int R = TT_M / TN;                          // column blocks per row block
  static constexpr uint32_t IDESC = tc::bf16_idesc(TT_M, TN);
  static_assert(ACOLS <= TT_COLS && TT_K / 16 % KS == 0 && TT_M % TN == 0, "tile form");
};
__device__ __forceinline__ void split3(float x, uint32_t& h0, uint32_t& h1, uint32_t& h2) {
  const __nv_bfloat16 b0 = __float2bfloat16_rn(x);
  const float r1 = x - __bfloat162float(b0);
  const __nv_bfloat16 b1 = __float2bfloat16_rn(r1);
  const float r2 = r1 - __bfloat162float(b1);
  const __nv_bfloat16 b2 = __float2bfloat16_rn(r2);
  h0 = __bfloat16_as_ushort(b0);
  h1 = __bfloat16_as_ushort(b1);
  h2 = __bfloat16_as_ushort(b2);
}

// Split of the panel, once per panel step: rows [k1, f) of W = L[:, k0:k1) and of W D
// into three BF16 parts each, stored per front as [part 0..5][k-group 0..7][row][8 BF16]
// (16 bytes per row and k-group; row = front position), i.e. already in the K-major
// core-matrix layout of a tile, so that a tile of consecutive rows is one contiguous
// block per part and k-group.
__global__ void __launch_bounds__(256) k_trailing_split(const NodeDesc* __restrict__ nd,
                                                         const NodeState* __restrict__ st, int t0,
                                                         const float* __restrict__ arena, uint4* __restrict__ parts) {
  const int t = t0 + blockIdx.y;
  const int k0 = st[t].kp0, k1 = st[t].k, f = st[t].f;
  if (k1 <= k0) return;
  const NodeDesc d = nd[t];
  const float* F = arena + d.front_off;
  const int64_t ld = d.ld;
  const int K = min(k1 - k0, TT_K);
  __shared__ float dk[TT_K];
  if (threadIdx.x < TT_K) dk[threadIdx.x] = threadIdx.x < K ? F[(k0 + threadIdx.x) * (ld + 1)] : 0.f;
  __syncthreads();
  uint4* P = parts + d.row_off * 48;                           // 6 parts x 8 k-groups per row
  // a warp takes 32 consecutive rows of one k-group: the column reads and the 16-byte part
  // writes of a warp are contiguous
  const int kg = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int rb = k1 + blockIdx.x * 32; rb < f; rb += gridDim.x * 32) {
    const int r = rb + lane;
    if (r >= f) continue;
    float w[8], b[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int k = kg * 8 + q;
      const float x = k < K ? F[r + (int64_t)(k0 + k) * ld] : 0.f;
      w[q] = x;
      b[q] = x * dk[k];
    }
    uint32_t p[6][4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      uint32_t a0, a1, a2, c0, c1, c2;
      split3(w[2 * q], a0, a1, a2);
      split3(w[2 * q + 1], c0, c1, c2);
      p[0][q] = a0 | (c0 << 16); p[1][q] = a1 | (c1 << 16); p[2][q] = a2 | (c2 << 16);
      split3(b[2 * q], a0, a1, a2);
      split3(b[2 * q + 1], c0, c1, c2);
      p[3][q] = a0 | (c0 << 16); p[4][q] = a1 | (c1 << 16); p[5][q] = a2 | (c2 << 16);
    }
#pragma unroll
    for (int part = 0; part < 6; ++part)
      P[((int64_t)(part * 8 + kg)) * ld + r] = make_uint4(p[part][0], p[part][1], p[part][2], p[part][3]);
  }
}

__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
               :: "r"(dst), "l"(src), "r"(bytes), "r"(bar) : "memory");
}

// tile u of the level -> (front slot, row block bi, column block bj < R (bi + 1)): fronts by
// the prefix of their tile counts, then the lower tile index within the front (row block bi
// of 128 rows holds the R (bi + 1) column blocks of TT_M / R columns that reach its last row)
struct TtTile { int slot, bi, bj; };
__device__ __forceinline__ TtTile tt_tile(const int* pre, int cnt, int u, int R) {
  int lo = 0, hi = cnt - 1;                           // last slot with pre[slot] <= u
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (pre[mid] <= u) lo = mid; else hi = mid - 1;
  }
  const int v = u - pre[lo];
  int bi = (int)((sqrtf(8.f * (float)v / (float)R + 1.f) - 1.f) * 0.5f);
  while (R * (bi + 1) * (bi + 2) / 2 <= v) ++bi;
  while (bi > 0 && R * bi * (bi + 1) / 2 > v) --bi;
  return {lo, bi, v - R * bi * (bi + 1) / 2};
}

// bounded wait on an mbarrier phase; false when it gave up (abort word set) or another
// role already gave up
__device__ __forceinline__ bool tt_wait(uint32_t bar, uint32_t par, volatile int* abort_w, int* flags) {
  for (int it = 0; it < TT_SPIN; ++it) {
    if (tc::mbar_try(bar, par)) return true;
    if (*abort_w) return false;
  }
  *abort_w = 1;
  atomicExch(flags + FLAG_TC_TIMEOUT, 1);
  return false;
}

// the same wait for the clean-up of an aborted CTA: ignores the abort word
__device__ __forceinline__ void tt_drain(uint32_t bar, uint32_t par) {
  for (int it = 0; it < TT_SPIN; ++it)
    if (tc::mbar_try(bar, par)) return;
}

__device__ __forceinline__ void tt_bar_init(uint64_t* b, int count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(tc::smem_u32(b)), "r"(count));
}

template <int TN, int KS>
__global__ void __launch_bounds__(TT_THREADS, 1) k_trailing_tc(const NodeDesc* __restrict__ nd,
                                                             const NodeState* __restrict__ st, int t0, int cnt,
                                                             float* __restrict__ arena,
                                                             const uint4* __restrict__ parts,
                                                             int* __restrict__ flags) {
  using Cfg = TtCfg<TN, KS>;
  constexpr int NB = Cfg::NBUF;
  constexpr int CW = TN / 2;                                   // columns per epilogue warp
  extern __shared__ __align__(1024) unsigned char tt_raw[];
  unsigned char* stages = (unsigned char*)(((uintptr_t)tt_raw + 1023) & ~(uintptr_t)1023);
  int* pre = (int*)(stages + 2 * Cfg::STAGE);                // cnt + 1 tile prefix counts
  __shared__ uint32_t tslot;
  __shared__ __align__(8) uint64_t bar_full[2], bar_empty[2], bar_tfull[2], bar_tempty[2];
  __shared__ int seg[TT_THREADS / 32 + 1];
  __shared__ int abort_s;
  volatile int* abort_w = &abort_s;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  // tiles of every front of the level: n = f - k1 trailing rows, nt = ceil(n / 128) row
  // blocks, R nt (nt + 1) / 2 lower tiles; prefix over the fronts (segments of threads)
  const int per = (cnt + TT_THREADS - 1) / TT_THREADS;
  const int a0 = min(cnt, tid * per), a1 = min(cnt, a0 + per);
  int sum = 0;
  for (int i = a0; i < a1; ++i) {
    const int k0 = st[t0 + i].kp0, k1 = st[t0 + i].k, f = st[t0 + i].f;
    const int n = k1 > k0 ? f - k1 : 0;
    const int nt = (n + TT_M - 1) / TT_M;
    pre[i] = Cfg::R * nt * (nt + 1) / 2;
    sum += pre[i];
  }
  // exclusive prefix of the threads' sums: a shuffle scan in each warp, then one over the
  // warp totals
  constexpr int NW = TT_THREADS / 32;
  int incl = sum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) seg[warp] = incl;
  if (tid == 0) {
    abort_s = 0;
    for (int s = 0; s < 2; ++s) {
      tt_bar_init(&bar_full[s], 1);
      tt_bar_init(&bar_empty[s], 1);
      tt_bar_init(&bar_tfull[s], 1);
      tt_bar_init(&bar_tempty[s], TT_EPI);                   // one arrival per epilogue warp
    }
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" :: "r"(tc::smem_u32(&tslot)), "r"(TT_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  __syncthreads();
  if (warp == 0) {
    const int wv = lane < NW ? seg[lane] : 0;
    int wi = wv;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, wi, o);
      if (lane >= o) wi += y;
    }
    __syncwarp();                                             // every lane has read seg
    if (lane < NW) seg[lane] = wi - wv;                       // first tile of warp `lane`'s fronts
    if (lane == NW - 1) seg[NW] = wi;                         // tiles of the level
  }
  __syncthreads();
  {
    int acc = seg[warp] + incl - sum;
    for (int i = a0; i < a1; ++i) { const int v = pre[i]; pre[i] = acc; acc += v; }
    if (tid == 0) pre[cnt] = seg[NW];
  }
  asm volatile("tcgen05.fence::after_thread_sync;");
  __syncthreads();
  const uint32_t tmem = tslot;
  const int total = pre[cnt];
  // a contiguous run of tiles per CTA: consecutive tiles of a row block share the A operand
  // (the panel's rows i0..i0+127), which then stays in the stage instead of being copied again
  const int G = (int)gridDim.x;
  const int chunk = (total + G - 1) / G;
  const int u0 = (int)blockIdx.x * chunk;
  const int ntile = max(0, min(chunk, total - u0));

  if (warp == 0) {
    // ---- producer: bulk copies of the pre-split parts of tile it into stage it % 2, the 48
    // copies (3 parts x 8 k-groups for each operand) issued by the 32 lanes of the warp
    int issued = 0;
    // where the parts of tile it come from: the front's parts, its leading dimension, the
    // first rows of the A (i0) and B (j0) operands.  Found one tile ahead (the tile map's
    // search and the front's fields are dependent loads), while the copies are in flight
    struct TtSrc { const uint4* P; int64_t ld; int i0, j0, akey; };
    int akey0 = -1, akey1 = -1;                                 // the A operand held by each stage
    auto src_of = [&](int it) {
      const TtTile tl = tt_tile(pre, cnt, u0 + it, Cfg::R);
      const int t = t0 + tl.slot;
      const int k1 = st[t].k;
      TtSrc r;
      r.akey = tl.slot * 65536 + tl.bi;
      r.ld = nd[t].ld;
      r.P = parts + nd[t].row_off * 48;
      r.i0 = k1 + tl.bi * TT_M;
      r.j0 = k1 + tl.bj * TN;
      return r;
    };
    TtSrc nx = {};
    if (ntile > 0) nx = src_of(0);
    for (int it = 0; it < ntile; ++it) {
      const int s = it & 1;
      const TtSrc cu = nx;
      int ok = 1;
      if (it >= 2 && lane == 0) ok = tt_wait(tc::smem_u32(&bar_empty[s]), ((it >> 1) + 1) & 1, abort_w, flags) ? 1 : 0;
      if (!__shfl_sync(0xffffffffu, ok, 0)) break;
      const int64_t ld = cu.ld;
      const uint4* P = cu.P;
      const int i0 = cu.i0, j0 = cu.j0;
      const uint32_t bf = tc::smem_u32(&bar_full[s]);
      const uint32_t sa = tc::smem_u32(stages + s * Cfg::STAGE);
      // the stage's A operand is that of the tile two before (the same stage): kept if it
      // is this tile's too, only the B operand is copied
      const bool copy_a = (s ? akey1 : akey0) != cu.akey;
      if (s) akey1 = cu.akey; else akey0 = cu.akey;
      if (lane == 0)
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(bf),
                     "r"(copy_a ? Cfg::STAGE : 3 * Cfg::B_PART) : "memory");
      __syncwarp();
      for (int e = lane + (copy_a ? 0 : 24); e < 48; e += 32) {
        const int op = e / 24, part = (e % 24) / 8, kg = e % 8;
        if (op == 0)
          bulk_g2s(sa + part * TT_PART + kg * (TT_M * 16), P + (int64_t)(part * 8 + kg) * ld + i0, TT_M * 16, bf);
        else
          bulk_g2s(sa + 3 * TT_PART + part * Cfg::B_PART + kg * (TN * 16),
                   P + (int64_t)((part + 3) * 8 + kg) * ld + j0, TN * 16, bf);
      }
      if (it + 1 < ntile) nx = src_of(it + 1);
      issued = it + 1;
    }
    if (lane == 0 && *abort_w)                               // own copies still in flight
      for (int it = max(0, issued - 2); it < issued; ++it) tt_drain(tc::smem_u32(&bar_full[it & 1]), (it >> 1) & 1);
  } else if (warp == 1 && lane == 0) {
    // ---- MMA issuer: 6 products x 4 k-steps into accumulator set it % NB
    const int ps[6] = {0, 0, 1, 0, 1, 2}, qs[6] = {0, 1, 0, 2, 1, 0};
    int done_it = 0;
    for (int it = 0; it < ntile; ++it) {
      const int s = it & 1, ab = NB == 2 ? (it & 1) : 0, use = it / NB;
      if (!tt_wait(tc::smem_u32(&bar_full[s]), (it >> 1) & 1, abort_w, flags)) break;
      if (use >= 1 && !tt_wait(tc::smem_u32(&bar_tempty[ab]), (use - 1) & 1, abort_w, flags)) break;
      asm volatile("tcgen05.fence::after_thread_sync;");
      const uint32_t sa = tc::smem_u32(stages + s * Cfg::STAGE), sb = sa + 3 * TT_PART;
      const uint32_t acc = tmem + (uint32_t)(ab * Cfg::ACOLS);
#pragma unroll 1
      for (int ks = 0; ks < TT_K / 16; ++ks) {
        const int a0c = ks / (TT_K / 16 / KS);                  // which order-0 accumulator
#pragma unroll
        for (int u = 0; u < 6; ++u) {
          const uint64_t ad = tc::smem_desc(sa + ps[u] * TT_PART + ks * (2 * TT_M * 16), 16 * TT_M, 128);
          const uint64_t bd = tc::smem_desc(sb + qs[u] * Cfg::B_PART + ks * (2 * TN * 16), 16 * TN, 128);
          const bool first = u == 0 ? (ks % (TT_K / 16 / KS) == 0) : (ks == 0 && u == 1);
          tc::mma_bf16(acc + (uint32_t)((u == 0 ? a0c : KS) * TN), ad, bd, Cfg::IDESC, first ? 0u : 1u);
        }
      }
      tc::mma_commit(tc::smem_u32(&bar_empty[s]));          // stage s may be refilled
      tc::mma_commit(tc::smem_u32(&bar_tfull[ab]));         // accumulator set ab is complete
      done_it = it + 1;
    }
    if (done_it > 0) {                                        // own MMAs done before the TMEM is freed
      const int last = done_it - 1;
      tt_drain(tc::smem_u32(&bar_tfull[NB == 2 ? (last & 1) : 0]), (last / NB) & 1);
    }
  } else if (warp >= 2) {
    // ---- epilogue: rows i0 + 32 q4 + lane, columns j0 + CW h .. + CW of the tile,
    // C -= (acc0_0 + .. + acc0_KS-1) + acc1 on the lower triangle
    const int q4 = warp & 3;                                  // the TMEM lane quarter this warp may read
    const int h = (warp - 2) >> 2;                            // which half of the tile's columns
    // this thread's row of tile it: front, leading dimension, row i, first column j0, and
    // qmax (columns q <= qmax are in the lower triangle of the front)
    struct EpiRow { float* F; int64_t ld; int i, j0, qmax; };
    auto row_of = [&](int it) {
      const TtTile tl = tt_tile(pre, cnt, u0 + it, Cfg::R);
      const int t = t0 + tl.slot;
      const int k1 = st[t].k, f = st[t].f;
      EpiRow e;
      e.F = arena + nd[t].front_off;
      e.ld = nd[t].ld;
      e.i = k1 + tl.bi * TT_M + q4 * 32 + lane;
      e.j0 = k1 + tl.bj * TN + h * CW;
      e.qmax = e.i < f ? min(e.i, f - 1) - e.j0 : -1;
      return e;
    };
    auto load_row = [&](const EpiRow& e, float* v) {
      const float* pc = e.F + e.i + (int64_t)e.j0 * e.ld;
#pragma unroll
      for (int q = 0; q < CW; ++q) {
        v[q] = q <= e.qmax ? *pc : 0.f;
        pc += e.ld;
      }
    };
    // C of a tile is loaded one tile ahead: while this tile's MMAs run and its accumulator
    // is read and stored
    float cv[CW], cvn[CW];
    EpiRow cur = {};
    if (ntile > 0) {
      cur = row_of(0);
      load_row(cur, cv);
    }
    for (int it = 0; it < ntile; ++it) {
      const int ab = NB == 2 ? (it & 1) : 0, use = it / NB;
      EpiRow nxt = cur;
      if (it + 1 < ntile) {
        nxt = row_of(it + 1);
        load_row(nxt, cvn);
      }
      int ok = 1;
      if (lane == 0) ok = tt_wait(tc::smem_u32(&bar_tfull[ab]), use & 1, abort_w, flags) ? 1 : 0;
      ok = __shfl_sync(0xffffffffu, ok, 0);
      if (!ok) break;
      asm volatile("tcgen05.fence::after_thread_sync;");
      const uint32_t ta = tmem + ((uint32_t)(q4 * 32) << 16) + (uint32_t)(ab * Cfg::ACOLS + h * CW);
      float* pw = cur.F + cur.i + (int64_t)cur.j0 * cur.ld;
#pragma unroll
      for (int ch = 0; ch < CW / 16; ++ch) {
        const int c0 = ch * 16;
        float v[16];
        uint32_t r[16];
        tc::tmem_ld16(ta + (uint32_t)c0, r);
#pragma unroll
        for (int q = 0; q < 16; ++q) v[q] = __uint_as_float(r[q]);
#pragma unroll
        for (int a = 1; a <= KS; ++a) {                       // the other order-0 sums, then acc1
          tc::tmem_ld16(ta + (uint32_t)(a * TN + c0), r);
#pragma unroll
          for (int q = 0; q < 16; ++q) v[q] += __uint_as_float(r[q]);
        }
        if (ch == CW / 16 - 1) {                              // this warp's part read: release it
          asm volatile("tcgen05.fence::before_thread_sync;");
          __syncwarp();
          if (lane == 0)
            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" :: "r"(tc::smem_u32(&bar_tempty[ab])) : "memory");
        }
#pragma unroll
        for (int q = 0; q < 16; ++q) {
          if (c0 + q <= cur.qmax) *pw = cv[c0 + q] - v[q];
          pw += cur.ld;
        }
      }
      cur = nxt;
#pragma unroll
      for (int q = 0; q < CW; ++q) cv[q] = cvn[q];
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 1) {
    __syncwarp();
    asm volatile("tcgen05.fence::after_thread_sync;");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(TT_COLS));
  }
}

// After the factorization the contribution maps of every child are re-expressed in the
// parent's pivoted row order (the solves work in that order).
__global__ void k_cbmap_post(const NodeDesc* __restrict__ nd, const NodeState* __restrict__ st,
                             const int32_t* __restrict__ pos0, int32_t* __restrict__ inv,
                             int32_t* __restrict__ cbmap) {
  const int p = blockIdx.x;
  const NodeDesc d = nd[p];
  const int nperm = d.cand_all ? st[p].f : d.n;
  for (int i = threadIdx.x; i < nperm; i += blockDim.x) inv[d.row_off + pos0[d.row_off + i]] = i;
  __syncthreads();
  for (int slot = 0; slot < 2; ++slot) {
    const int ch = slot == 0 ? d.child0 : d.child1;
    if (ch < 0) continue;
    const NodeDesc dc = nd[ch];
    const int mc = st[ch].f - st[ch].k;
    for (int a = threadIdx.x; a < mc; a += blockDim.x) {
      int tg = cbmap[dc.row_off + a];
      if (tg >= 0 && tg < nperm) cbmap[dc.row_off + a] = inv[d.row_off + tg];
    }
  }
}

// The contribution maps read the other way, for the gathers of the triangular sweeps:
// gmap[slot][row of front p] = the contribution row a of p's child `slot` mapped to that row
// (-1 where none), after the factorization's final maps and states.
__global__ void k_gmap_build(const NodeDesc* __restrict__ nd, const NodeState* __restrict__ st,
                             const int32_t* __restrict__ cbmap, int32_t* __restrict__ gmap, int64_t rows) {
  const int p = blockIdx.x;
  const NodeDesc d = nd[p];
  for (int slot = 0; slot < 2; ++slot) {
    const int ch = slot == 0 ? d.child0 : d.child1;
    if (ch < 0) continue;
    const NodeDesc dc = nd[ch];
    const int mc = st[ch].f - st[ch].k;
    for (int a = threadIdx.x; a < mc; a += blockDim.x) {
      const int tg = cbmap[dc.row_off + a];
      if (tg >= 0) gmap[slot * rows + d.row_off + tg] = a;
    }
  }
}

// ---------------------------------------------------------------------------
// Enlargement (Sec. 2.2, reading R13) and collection of Lambda_2
// ---------------------------------------------------------------------------
__global__ void k_finalize(const NodeDesc* __restrict__ nd, NodeState* __restrict__ st, int nn, int n_enlarge,
                           const int32_t* __restrict__ rowid, int32_t* __restrict__ lam2, int64_t* __restrict__ counts) {
  const int tid = threadIdx.x;
  for (int t = tid; t <= nn; t += blockDim.x) { st[t].ksolve = st[t].k; st[t].nmoved = 0; }
  __syncthreads();
  if (tid == 0) {
    int rem = n_enlarge;
    for (int t = nn; t >= 0 && rem > 0; --t) {
      int take = min(rem, st[t].k);
      st[t].nmoved = take;
      st[t].ksolve = st[t].k - take;
      rem -= take;
    }
    int64_t M = 0, piv = 0;
    const NodeDesc r = nd[nn];
    const int ksr = st[nn].k, fsr = st[nn].f;
    for (int i = ksr; i < fsr; ++i) lam2[M++] = rowid[r.row_off + i];
    for (int t = 0; t <= nn; ++t) {
      piv += st[t].k;
      for (int i = st[t].ksolve; i < st[t].k; ++i) lam2[M++] = rowid[nd[t].row_off + i];
    }
    counts[0] = M;
    counts[1] = fsr;          // #Lambda_0
    counts[2] = piv;
  }
}

// ---------------------------------------------------------------------------
// S22 taken from the factor (HF_PREC_FP64 / HF_PREC_FP32 forms): with T the moved
// pivots (a suffix of the elimination order) and H the unfactorized rows,
// S22 = L_(T+H),T D_T L_(T+H),T^T + (0 (+) S_H)   (block LDL^T of the trailing matrix, Eq. 1)
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_s22_from_factor(const NodeDesc* __restrict__ nd, const NodeState* __restrict__ st, int nn,
                                  const T* __restrict__ arena, const int32_t* __restrict__ rowid,
                                  const int32_t* __restrict__ lam2pos, int M, double* __restrict__ S22,
                                  int* __restrict__ flags) {
  const int tid = threadIdx.x;
  for (int e = tid; e < M * M; e += blockDim.x) S22[e] = 0.0;
  __syncthreads();
  {   // unfactorized block of the Lambda_0 stage front
    const NodeDesc r = nd[nn];
    const T* F = arena + r.front_off;
    const int ksr = st[nn].k, fsr = st[nn].f;
    const int m = fsr - ksr;
    for (int e = tid; e < m * m; e += blockDim.x) {
      int a = e / m, b = e % m;
      if (b < a) continue;
      int ia = ksr + a, ib = ksr + b;
      double v = (double)F[ib + (int64_t)ia * r.ld];
      int ga = rowid[r.row_off + ia], gb = rowid[r.row_off + ib];
      int pa = ga >= 0 ? lam2pos[ga] : -1, pb = gb >= 0 ? lam2pos[gb] : -1;
      if (pa < 0 || pb < 0) { flags[FLAG_NUMERIC] = 2; continue; }
      S22[pa * M + pb] = v;
      S22[pb * M + pa] = v;
    }
  }
  __syncthreads();
  // moved pivots, one column at a time (at most n_enlarge of them)
  for (int t = nn; t >= 0; --t) {
    const int ks = st[t].ksolve, k = st[t].k;
    if (ks == k) continue;
    const NodeDesc dn = nd[t];
    const T* F = arena + dn.front_off;
    const int f = st[t].f;
    for (int j = ks; j < k; ++j) {
      const double dj = (double)F[j + (int64_t)j * dn.ld];
      const int m = f - j;                    // rows j..f-1 (row j carries the unit diagonal)
      for (int e = tid; e < m * m; e += blockDim.x) {
        int a = e / m, b = e % m;
        if (b < a) continue;
        int ia = j + a, ib = j + b;
        double la = (a == 0) ? 1.0 : (double)F[ia + (int64_t)j * dn.ld];
        double lb = (b == 0) ? 1.0 : (double)F[ib + (int64_t)j * dn.ld];
        int ga = rowid[dn.row_off + ia], gb = rowid[dn.row_off + ib];
        int pa = ga >= 0 ? lam2pos[ga] : -1, pb = gb >= 0 ? lam2pos[gb] : -1;
        if (pa < 0 || pb < 0) { flags[FLAG_NUMERIC] = 2; continue; }
        double v = la * dj * lb;
        S22[pa * M + pb] += v;
        if (pa != pb) S22[pb * M + pa] += v;
      }
      __syncthreads();
    }
  }
}

template <typename T>
int run_levels(hf_ctx* c) {
  cudaStream_t s = hf_stream(c);
  const NodeDesc* nd = (const NodeDesc*)c->d_nodes.p;
  NodeState* st = (NodeState*)c->d_state.p;
  T* arena = (T*)c->d_front.p;
  T* gmag = (T*)c->d_gmag.p;
  int32_t* rowid = (int32_t*)c->d_rowid.p;
  int* flags = (int*)c->d_flags.p;
  const int nb = std::max(1, std::min(c->opts.panel, 256));
  const int nn = c->n_nodes;
  constexpr size_t PCL_SMEM = 220 * 1024;
  static bool attr_set[2] = {false, false};
  static int max_cluster[2] = {0, 0};
  static int active_clusters[2][PCL_CMAX + 1] = {};   // co-resident clusters of each size
  static std::mutex attr_mu;                 // contexts may be driven from several host threads
  static int num_sms = 0;
  int cmax = 0;
  {
  std::lock_guard<std::mutex> attr_lock(attr_mu);   // the one-time set-up only, not the launches
  if (!num_sms) {
    int dev = 0;
    HF_CUDA_TRY(cudaGetDevice(&dev));
    HF_CUDA_TRY(cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev));
    num_sms = std::max(1, num_sms);
  }
  if (!attr_set[sizeof(T) == 8]) {
    HF_CUDA_TRY(cudaFuncSetAttribute(k_panel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024));
    HF_CUDA_TRY(cudaFuncSetAttribute(k_panel_cl<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)PCL_SMEM));
    HF_CUDA_TRY(cudaFuncSetAttribute(k_trailing_tc<128, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, TtCfg<128, 1>::SMEM));
    HF_CUDA_TRY(cudaFuncSetAttribute(k_trailing_tc<128, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, TtCfg<128, 2>::SMEM));
    HF_CUDA_TRY(cudaFuncSetAttribute(k_trailing_tc<64, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, TtCfg<64, 2>::SMEM));
    HF_CUDA_TRY(cudaFuncSetAttribute(k_trailing_tc<64, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, TtCfg<64, 4>::SMEM));
    HF_CUDA_TRY(cudaFuncSetAttribute(k_swap_sigma, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SW_SMEM));
    HF_CUDA_TRY(cudaFuncSetAttribute(k_swap_apply<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SW_SMEM));
    if (cudaFuncSetAttribute(k_panel_cl<T>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess)
      (void)cudaGetLastError();
    // clusters of each size (<= 16) that can be resident at once with the full
    // shared-memory panel; the largest size with at least one
    for (int cs = PCL_CMAX; cs >= 1; --cs) {
      cudaLaunchConfig_t q = {};
      q.gridDim = dim3(cs);
      q.blockDim = dim3(PCL_THREADS);
      q.dynamicSmemBytes = PCL_SMEM;
      cudaLaunchAttribute at[1];
      at[0].id = cudaLaunchAttributeClusterDimension;
      at[0].val.clusterDim.x = cs; at[0].val.clusterDim.y = 1; at[0].val.clusterDim.z = 1;
      q.attrs = at; q.numAttrs = 1;
      int ncl = 0;
      if (cudaOccupancyMaxActiveClusters(&ncl, k_panel_cl<T>, &q) == cudaSuccess && ncl > 0) {
        active_clusters[sizeof(T) == 8][cs] = ncl;
        max_cluster[sizeof(T) == 8] = std::max(max_cluster[sizeof(T) == 8], cs);
      } else {
        (void)cudaGetLastError();
      }
    }
    attr_set[sizeof(T) == 8] = true;
  }
  cmax = max_cluster[sizeof(T) == 8];
  }
  const int* ncl_of = active_clusters[sizeof(T) == 8];
  // the optional null-pivot test (R3b) compares |d| with tau_null * G; 0 switches it off
  // (|d| >= 0 always holds; a NaN pivot already fails the ratio test)
  const double tau_null = c->opts.null_test ? c->tau : 0.0;
  // trailing updates of the FP32 factor on the tensor cores (3 x BF16 split) when selected
  const bool use_tc = sizeof(T) == 4 && c->opts.trailing == 0;
  // HF_TC_MIN_ROWS=n: smallest largest-front order of a level that takes the tensor cores
  // (default TT_MIN_ROWS; 0 = every level; diagnostic)
  const char* tmr = std::getenv("HF_TC_MIN_ROWS");
  const int tc_min_rows = tmr ? std::max(0, std::atoi(tmr)) : TT_MIN_ROWS;
  // HF_TC_FORM=n: tile form of the tensor-core update (0: 128 x 128 tiles, order-0 products in
  // one accumulator; 1: 128 x 128, two; 2: 128 x 64, two; 3: 128 x 64, one per k-step of 16,
  // the default: the fewer products one tensor-core FP32 sum takes, the closer the update is
  // to the FP32 SIMT one; diagnostic)
  const char* tfm = std::getenv("HF_TC_FORM");
  const int tc_form = tfm ? std::atoi(tfm) : 3;
  // HF_LEVEL_TIMES=1: time the panel and trailing launches of every level (diagnostic)
  const char* lt = std::getenv("HF_LEVEL_TIMES");
  const bool level_times = lt && lt[0] == '1';
  // HF_PANEL_KERNEL=global: one CTA per front with the panel in global memory (for comparison)
  const char* pk = std::getenv("HF_PANEL_KERNEL");
  const bool panel_global = pk && pk[0] == 'g';
  // HF_PANEL_ROWS=n: at most n rows per CTA of the cluster panel, so that small fronts take
  // the larger clusters of large ones (the same arithmetic spread over more CTAs; diagnostic)
  const char* pr = std::getenv("HF_PANEL_ROWS");
  const int rows_cap = pr ? std::max(1, std::atoi(pr)) : 0;
  c->path_cluster = 0;
  c->path_global = 0;
  c->lev_panel_global.assign(c->m + 1, 0);
  for (int lev = c->m; lev >= 0; --lev) {
    const int t0 = c->level_start[lev], cnt = c->level_count[lev];
    int maxn = 0, maxld = 0;
    int64_t maxasm = 0;
    bool has_children = false;
    for (int t = t0; t < t0 + cnt; ++t) {
      const NodeDesc& d = c->nodes[t];
      maxn = std::max(maxn, d.cand_all ? d.ld : d.n);
      maxld = std::max(maxld, d.ld);
      maxasm = std::max<int64_t>(maxasm, d.asm_cnt);
      has_children |= (d.child0 >= 0);
    }
    HF_LAUNCH(c, HF_PROF_ASSEMBLE, k_level_prep<<<(cnt + 127) / 128, 128, 0, s>>>(nd, st, t0, cnt, flags));
    if (has_children)
      HF_LAUNCH(c, HF_PROF_ASSEMBLE, k_level_maps<<<cnt, 1024, 0, s>>>(nd, st, t0, rowid, (const int32_t*)c->d_smap.p, (int32_t*)c->d_cbmap.p));
    // blocks per front: enough for the largest front, but about 4,864 in all for a level of
    // many fronts (the kernels loop over columns or entries, so fewer blocks each do more;
    // a level of 1,024 fronts with one block per column made 400k blocks of a few stores)
    const int per_front = std::max(1, 4864 / cnt);
    {
      int bx = std::min({std::max(1, maxld), 512, per_front});
      HF_LAUNCH(c, HF_PROF_ASSEMBLE, k_front_zero<T><<<dim3(bx, cnt), 256, 0, s>>>(nd, st, t0, arena));
    }
    if (maxasm > 0) {
      int bx = (int)std::min<int64_t>(std::min<int64_t>((maxasm + 255) / 256, 1024), per_front);
      HF_LAUNCH(c, HF_PROF_ASSEMBLE, k_front_asm<T><<<dim3(bx, cnt), 256, 0, s>>>(nd, t0, (const AsmEntry*)c->d_asm.p,
                                                   (const double*)c->d_kval.p, arena));
    }
    if (has_children) {
      int bx = std::min({std::max(1, maxld), 1024, 2 * per_front});     // 128-thread blocks
      for (int slot = 0; slot < 2; ++slot)
        HF_LAUNCH(c, HF_PROF_ASSEMBLE, k_extend_add<T><<<dim3(bx, cnt), 128, 0, s>>>(nd, st, t0, slot, (const int32_t*)c->d_cbmap.p, arena));
    }
    HF_LAUNCH(c, HF_PROF_ASSEMBLE, k_g_assemble<T><<<cnt, 1024, 0, s>>>(nd, st, t0, rowid, (const int32_t*)c->d_cbmap.p,
                                        (const int64_t*)c->d_diagpos.p, (const double*)c->d_kval.p, gmag,
                                        (int32_t*)c->d_pos0.p));
    // panel in distributed shared memory for the fronts a cluster of <= cmax CTAs can hold;
    // larger ones (if any) by the global-memory kernel in the same step
    const int nbc = sizeof(T) == 8 ? std::min(nb, 32) : nb;
    const size_t per_row = (size_t)(nbc + 1) * sizeof(T) + 3 * sizeof(T) + 3 * sizeof(int);
    const size_t fixed = PclLayout<T>::bytes(0, nbc);
    int Rcap = std::min((int)((PCL_SMEM - fixed) / per_row), PCL_RPT * PCL_THREADS);
    if (rows_cap > 0) Rcap = std::min(Rcap, rows_cap);
    // fewest CTAs per front whose shared memory holds the level's largest front
    int C = std::max(1, std::min(cmax, (maxld + Rcap - 1) / Rcap));
    bool level_global = panel_global;
    if (rows_cap == 0 && !panel_global && cmax > 0 && maxld > 0) {
      // a pivot costs less when every thread holds one row: more CTAs per front, as long
      // as the level's clusters are resident at once (measured at 40^3 elasticity: the
      // root 22.7 -> 21.2 ms with 10 CTAs instead of 7, the two fronts of the level below
      // 16.3 -> 14.5 ms with 15 instead of 10)
      const int C1 = (maxld + PCL_THREADS - 1) / PCL_THREADS;
      if (C1 > C && C1 <= cmax && ncl_of[C1] >= cnt) C = C1;
      // levels of many small fronts whose clusters would run in more than two waves: the
      // global-memory panel (one small CTA per front, all fronts at once) is faster there
      // (1,024 fronts of <= 432 rows: 3.19 -> 2.35 ms; 128 fronts of <= 1,572 rows, three
      // waves: 2.14 -> 1.91 ms; 64 fronts in 1.7 waves: 3.23 ms with clusters, 4.60 without)
      if (ncl_of[C] > 0 && cnt > 2 * ncl_of[C]) level_global = true;
    }
    const bool use_cl = cmax > 0 && maxld > 0 && !level_global;
    const int cap = use_cl ? C * Rcap : -1;
    const bool use_gl = !use_cl || maxld > cap;
    if (use_cl) c->path_cluster = std::max(c->path_cluster, C);
    if (use_gl) c->path_global++;
    c->lev_panel_global[lev] = use_cl ? 0 : 1;       // fronts of a mixed level: counted as cluster
    const int nbl = use_cl ? nbc : nb;
    const int npan = (maxn + nbl - 1) / nbl;
    const size_t smem = (size_t)nbl * sizeof(T) + (size_t)maxn * (sizeof(T) + sizeof(int));
    if (use_gl && smem > 220 * 1024) return HF_ERR_CAPACITY;
    const int pthreads = maxld > 1024 ? 1024 : 256;
    // tensor-core trailing update for the levels of large fronts (a panel of <= 64 pivots,
    // the tile map of <= TT_MAXF fronts): one persistent CTA per SM, at most one per tile
    const bool tc_level = use_tc && nbl <= TT_K && cnt <= TT_MAXF && maxld >= tc_min_rows;
    unsigned tc_grid = 1;
    if (tc_level) {
      const int64_t nt = (maxld + TT_M - 1) / TT_M;
      tc_grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>((int64_t)cnt * 2 * nt * (nt + 1) / 2, num_sms));
    }
    const int tiles = (maxld + TB - 1) / TB;
    int4* swl = (int4*)c->d_swlist.p;
    int* swc = (int*)c->d_swcount.p;
    cudaLaunchConfig_t lc = {};
    cudaLaunchAttribute la[1];
    if (use_cl) {
      lc.gridDim = dim3((unsigned)(cnt * C));
      lc.blockDim = dim3(PCL_THREADS);
      lc.dynamicSmemBytes = PCL_SMEM;
      lc.stream = s;
      la[0].id = cudaLaunchAttributeClusterDimension;
      la[0].val.clusterDim.x = (unsigned)C; la[0].val.clusterDim.y = 1; la[0].val.clusterDim.z = 1;
      lc.attrs = la; lc.numAttrs = 1;
    }
    cudaEvent_t lev_e0 = nullptr, lev_e1 = nullptr;
    if (level_times) {
      cudaEventCreate(&lev_e0); cudaEventCreate(&lev_e1);
      cudaEventRecord(lev_e0, s);
    }
    for (int p = 0; p < npan; ++p) {
      if (use_cl)
        HF_LAUNCH(c, HF_PROF_PANEL, HF_CUDA_TRY(cudaLaunchKernelEx(&lc, k_panel_cl<T>, nd, st, t0, arena, rowid, gmag,
                                                                   (int32_t*)c->d_pos0.p, nbl, c->tau, tau_null, C, Rcap,
                                                                   swl, swc)));
      if (use_gl)
        HF_LAUNCH(c, HF_PROF_PANEL_GLOBAL, k_panel<T><<<cnt, pthreads, smem, s>>>(nd, st, t0, arena, rowid, gmag,
                                                                           (int32_t*)c->d_pos0.p, nbl, c->tau, tau_null, cap));
      if (tc_level) {
        uint4* parts = (uint4*)c->d_tparts.p;
        HF_LAUNCH(c, HF_PROF_TC_PREP, k_trailing_split<<<dim3((unsigned)std::min({1024, (maxld + 31) / 32, std::max(1, 4864 / cnt)}), cnt), 256, 0, s>>>(
                                           nd, st, t0, (const float*)arena, parts));
        float* fa = (float*)arena;
        switch (tc_form) {
          case 1: HF_LAUNCH(c, HF_PROF_TRAILING, k_trailing_tc<128, 2><<<tc_grid, TT_THREADS, TtCfg<128, 2>::SMEM, s>>>(
                                                     nd, st, t0, cnt, fa, parts, flags)); break;
          case 2: HF_LAUNCH(c, HF_PROF_TRAILING, k_trailing_tc<64, 2><<<tc_grid, TT_THREADS, TtCfg<64, 2>::SMEM, s>>>(
                                                     nd, st, t0, cnt, fa, parts, flags)); break;
          case 3: HF_LAUNCH(c, HF_PROF_TRAILING, k_trailing_tc<64, 4><<<tc_grid, TT_THREADS, TtCfg<64, 4>::SMEM, s>>>(
                                                     nd, st, t0, cnt, fa, parts, flags)); break;
          default: HF_LAUNCH(c, HF_PROF_TRAILING, k_trailing_tc<128, 1><<<tc_grid, TT_THREADS, TtCfg<128, 1>::SMEM, s>>>(
                                                     nd, st, t0, cnt, fa, parts, flags)); break;
        }
      } else
        HF_LAUNCH(c, HF_PROF_TRAILING, k_trailing<T><<<dim3(tiles, tiles, cnt), 256, 0, s>>>(nd, st, t0, arena));
    }
    if (use_cl) {
      // the listed interchanges of this level's cluster-panel fronts, in their final order
      if ((size_t)2 * maxld * sizeof(int) > SW_SMEM || (size_t)maxld * sizeof(T) > SW_SMEM) return HF_ERR_CAPACITY;
      const int gcap = npan + 1;
      const int sg = maxld + 1;
      const int64_t sf = (int64_t)gcap * sg;
      int rc2;
      if ((rc2 = hf_ensure(c->d_swsig, (size_t)cnt * sf * sizeof(int) + ((size_t)cnt + 1) * sizeof(int) + 64))) return rc2;
      int* sig = (int*)c->d_swsig.p;
      int* ngrp = sig + (size_t)cnt * sf;
      HF_LAUNCH(c, HF_PROF_PANEL_SWAP, k_swap_sigma<<<cnt, SW_THREADS, (size_t)2 * maxld * sizeof(int), s>>>(
                                      nd, st, t0, (const int4*)swl, swc, sig, sf, sg, gcap, ngrp));
      HF_LAUNCH(c, HF_PROF_PANEL_SWAP, k_swap_apply<T><<<dim3((unsigned)maxld, (unsigned)cnt), 256, (size_t)maxld * sizeof(T), s>>>(
                                      nd, st, t0, arena, sig, sf, sg, ngrp));
    }
    if (level_times) {
      float ms = 0;
      cudaEventRecord(lev_e1, s);
      cudaEventSynchronize(lev_e1);
      cudaEventElapsedTime(&ms, lev_e0, lev_e1);
      std::fprintf(stderr, "level %d: fronts %d max n %d max ld %d cluster %d (cap %d) global %d panels %d: %.3f ms\n",
                   lev, cnt, maxn, maxld, use_cl ? C : 0, cap, use_gl ? 1 : 0, npan, ms);
      cudaEventDestroy(lev_e0); cudaEventDestroy(lev_e1);
    }
    HF_CUDA_TRY(cudaGetLastError());
  }
  (void)nn;
  return HF_OK;
}

// algorithmic work of the trailing updates of a finished factorization (host state)
static void trailing_work(hf_ctx* c, size_t esz) {
  const double nb = std::max(1, std::min(c->opts.panel, 256));
  double fl = 0, by = 0;
  for (const NodeState& S : c->state_host) {
    for (double k0 = 0; k0 < S.k; k0 += nb) {
      double k1 = std::min<double>(S.k, k0 + nb), n = S.f - k1;
      fl += (k1 - k0) * n * (n + 1);
      by += n * (n + 1) / 2 * 2 * esz + n * (k1 - k0) * esz;   // C read+write, panel read
    }
  }
  c->work_flops[HF_PROF_TRAILING] += fl;
  c->work_bytes[HF_PROF_TRAILING] += by;
  // panels: column k of a panel costs 2 (f - k) (k - k0) for the left-looking products plus
  // 3 (f - k) for the division, diagonal and magnitude updates; the panel block is read and
  // written once
  // (to the class of the panel kernel that the front's level took)
  for (size_t t = 0; t < c->state_host.size(); ++t) {
    const NodeState& S = c->state_host[t];
    const int lev = c->nodes[t].level;
    const int cls = lev >= 0 && lev < (int)c->lev_panel_global.size() && c->lev_panel_global[lev]
                        ? HF_PROF_PANEL_GLOBAL : HF_PROF_PANEL;
    double pf = 0, pb = 0;
    for (double k = 0; k < S.k; k += 1) {
      const double kk = std::fmod(k, nb), rows = S.f - k;
      pf += 2.0 * rows * kk + 3.0 * rows;
      if (kk == 0) pb += 2.0 * rows * std::min(nb, (double)S.k - k) * esz;
    }
    c->work_flops[cls] += pf;
    c->work_bytes[cls] += pb;
  }
}

}  // namespace

// Device upload of the analysis results (first factorization, or after a re-layout).
static int upload_analysis(hf_ctx* c) {
  cudaStream_t s = hf_stream(c);
  const int nn = c->n_nodes;
  auto up = [&](DevBuf& b, const void* src, size_t bytes) -> int {
    int rc = hf_ensure(b, std::max<size_t>(bytes, 16));
    if (rc) return rc;
    if (bytes) HF_CUDA_TRY(cudaMemcpyAsync(b.p, src, bytes, cudaMemcpyHostToDevice, s));
    return HF_OK;
  };
  int rc;
  if ((rc = up(c->d_rowptr, c->rowptr.data(), c->rowptr.size() * 8))) return rc;
  if ((rc = up(c->d_col, c->col.data(), c->col.size() * 4))) return rc;
  if ((rc = up(c->d_diagpos, c->diagpos.data(), c->diagpos.size() * 8))) return rc;
  if ((rc = up(c->d_nodes, c->nodes.data(), c->nodes.size() * sizeof(NodeDesc)))) return rc;
  if ((rc = up(c->d_rowid_static, c->rowid_static.data(), c->rowid_static.size() * 4))) return rc;
  if ((rc = up(c->d_smap, c->smap.data(), c->smap.size() * 4))) return rc;
  if ((rc = up(c->d_asm, c->asm_list.data(), c->asm_list.size() * sizeof(AsmEntry)))) return rc;
  if ((rc = hf_ensure(c->d_state, (size_t)(nn + 1) * sizeof(NodeState)))) return rc;
  if ((rc = hf_ensure(c->d_rowid, c->rowid_static.size() * 4 + 16))) return rc;
  if ((rc = hf_ensure(c->d_cbmap, c->rowid_static.size() * 4 + 16))) return rc;
  if ((rc = hf_ensure(c->d_flags, FLAG_COUNT * sizeof(int) + 64))) return rc;
  if ((rc = hf_ensure(c->d_q, c->L * 8))) return rc;
  if ((rc = hf_ensure(c->d_qrow, c->L * 8))) return rc;
  if ((rc = hf_ensure(c->d_kval, c->nnz * 8))) return rc;
  if ((rc = hf_ensure(c->d_lam2pos, c->L * 4))) return rc;
  if ((rc = hf_ensure(c->d_lam2, c->L * 4 + 16))) return rc;
  return HF_OK;
}

int hf_factorize_impl(hf_ctx* c, const double* vals, double tau) {
  if (!c || !vals || !(tau > 0)) return HF_ERR_ARG;
  cudaStream_t s = hf_stream(c);
  c->tau = tau;
  c->prec = c->opts.precision;
  c->factored = false;
  c->schured = false;
  const bool dbl = (c->prec == HF_PREC_FP64);
  int rc;
  bool uploaded = c->d_nodes.p != nullptr;
  for (int attempt = 0; attempt < 16; ++attempt) {
    if (!uploaded) {
      if ((rc = upload_analysis(c))) return rc;
      uploaded = true;
    }
    const size_t esz = dbl ? 8 : 4;
    if ((rc = hf_ensure(c->d_front, (size_t)c->front_elems * esz + 64))) return rc;
    if ((rc = hf_ensure(c->d_gmag, (size_t)c->row_elems * esz + 64))) return rc;
    // pre-split panel parts of the tensor-core trailing update: 768 bytes per front row, plus
    // one tile of rows past the last front (tiles may read beyond a front's rows)
    if (!dbl && c->opts.trailing == 0 && (rc = hf_ensure(c->d_tparts, ((size_t)c->row_elems + TT_M) * 768 + 256))) return rc;
    if ((rc = hf_ensure(c->d_pos0, (size_t)c->row_elems * 4 + 64))) return rc;
    if ((rc = hf_ensure(c->d_invpos, (size_t)c->row_elems * 4 + 64))) return rc;
    // listed row interchanges of the cluster panels: 2 ld entries per front, one count per front
    if ((rc = hf_ensure(c->d_swlist, (size_t)c->row_elems * 2 * sizeof(int4) + 64))) return rc;
    if ((rc = hf_ensure(c->d_swcount, ((size_t)c->n_nodes + 1) * sizeof(int) + 64))) return rc;
    HF_CUDA_TRY(cudaMemsetAsync(c->d_swcount.p, 0, ((size_t)c->n_nodes + 1) * sizeof(int), s));
    HF_CUDA_TRY(cudaMemsetAsync(c->d_flags.p, 0, FLAG_COUNT * sizeof(int) + 64, s));
    HF_CUDA_TRY(cudaMemcpyAsync(c->d_rowid.p, c->d_rowid_static.p, c->rowid_static.size() * 4,
                                cudaMemcpyDeviceToDevice, s));
    const int64_t L = c->L;
    const int8_t* rsign = c->has_rsign ? (const int8_t*)c->d_rsign.p : nullptr;
    const double* qrow = (const double*)(c->has_rsign ? c->d_qrow.p : c->d_q.p);
    HF_LAUNCH(c, HF_PROF_SCALE, k_scale_diag<<<(unsigned)((L + 255) / 256), 256, 0, s>>>(L, (const int64_t*)c->d_diagpos.p, vals, (double*)c->d_q.p,
                                                                                      rsign, (double*)c->d_qrow.p));
    HF_LAUNCH(c, HF_PROF_SCALE, k_scale_vals<<<(unsigned)((L * 32 + 255) / 256), 256, 0, s>>>(L, (const int64_t*)c->d_rowptr.p, (const int32_t*)c->d_col.p,
                                                          vals, qrow, (const double*)c->d_q.p, (double*)c->d_kval.p,
                                                          (int*)c->d_flags.p));
    HF_CUDA_TRY(cudaGetLastError());
    rc = dbl ? run_levels<double>(c) : run_levels<float>(c);
    if (rc) return rc;
    HF_LAUNCH(c, HF_PROF_LAMBDA, k_cbmap_post<<<c->n_nodes + 1, 256, 0, s>>>((const NodeDesc*)c->d_nodes.p,
                                                                            (const NodeState*)c->d_state.p,
                                                                            (const int32_t*)c->d_pos0.p,
                                                                            (int32_t*)c->d_invpos.p,
                                                                            (int32_t*)c->d_cbmap.p));
    int64_t* counts = (int64_t*)((int*)c->d_flags.p + FLAG_COUNT);
    HF_LAUNCH(c, HF_PROF_LAMBDA, k_finalize<<<1, 256, 0, s>>>((const NodeDesc*)c->d_nodes.p, (NodeState*)c->d_state.p, c->n_nodes,
                                 c->opts.n_enlarge, (const int32_t*)c->d_rowid.p, (int32_t*)c->d_lam2.p, counts));
    // the child contributions of every front row, read by the sweeps' gathers
    if ((rc = hf_ensure(c->d_gmap, (size_t)c->row_elems * 2 * sizeof(int32_t) + 64))) return rc;
    HF_CUDA_TRY(cudaMemsetAsync(c->d_gmap.p, 0xFF, (size_t)c->row_elems * 2 * sizeof(int32_t), s));
    HF_LAUNCH(c, HF_PROF_LAMBDA, k_gmap_build<<<c->n_nodes + 1, 256, 0, s>>>((const NodeDesc*)c->d_nodes.p,
                                                                            (const NodeState*)c->d_state.p,
                                                                            (const int32_t*)c->d_cbmap.p,
                                                                            (int32_t*)c->d_gmap.p, c->row_elems));
    HF_CUDA_TRY(cudaGetLastError());
    int hflags[FLAG_COUNT];
    int64_t hcounts[3];
    HF_CUDA_TRY(cudaMemcpyAsync(hflags, c->d_flags.p, sizeof(hflags), cudaMemcpyDeviceToHost, s));
    HF_CUDA_TRY(cudaMemcpyAsync(hcounts, counts, sizeof(hcounts), cudaMemcpyDeviceToHost, s));
    HF_CUDA_TRY(cudaStreamSynchronize(s));
    if (hflags[FLAG_NUMERIC]) return HF_ERR_NUMERIC;
    if (hflags[FLAG_TC_TIMEOUT]) return HF_ERR_TIMEOUT;
    if (hflags[FLAG_DELAY_OVERFLOW]) {
      // grow the capacity for postponed rows and lay the fronts out again
      c->opts.delay_cap = std::max(1, c->opts.delay_cap) * 2;
      c->delay_retries++;
      hf_layout_fronts(c);
      uploaded = false;
      continue;
    }
    c->M = hcounts[0];
    c->n_lambda0 = hcounts[1];
    c->N = c->L - c->M;
    c->lambda2.resize(c->M);
    if (c->M) HF_CUDA_TRY(cudaMemcpy(c->lambda2.data(), c->d_lam2.p, c->M * 4, cudaMemcpyDeviceToHost));
    std::sort(c->lambda2.begin(), c->lambda2.end());
    c->state_host.resize(c->n_nodes + 1);
    HF_CUDA_TRY(cudaMemcpy(c->state_host.data(), c->d_state.p, c->state_host.size() * sizeof(NodeState),
                           cudaMemcpyDeviceToHost));
    // sorted Lambda_2 and the position map
    std::vector<int32_t> pos(c->L, -1);
    for (int64_t i = 0; i < c->M; ++i) pos[c->lambda2[i]] = (int32_t)i;
    HF_CUDA_TRY(cudaMemcpyAsync(c->d_lam2pos.p, pos.data(), c->L * 4, cudaMemcpyHostToDevice, s));
    if (c->M) HF_CUDA_TRY(cudaMemcpyAsync(c->d_lam2.p, c->lambda2.data(), c->M * 4, cudaMemcpyHostToDevice, s));
    HF_CUDA_TRY(cudaStreamSynchronize(s));
    int64_t nz = 0;
    for (int t = 0; t <= c->n_nodes; ++t) {
      const NodeState& S = c->state_host[t];
      nz += (int64_t)S.k * (S.f - S.k) + (int64_t)S.k * (S.k - 1) / 2;
    }
    c->nnz_factor = nz;
    if ((rc = hf_sweep_plan(c))) return rc;
    if ((rc = hf_diag_inverses(c))) return rc;
    c->front_prec = c->prec;
    c->factored = true;
    trailing_work(c, dbl ? 8 : 4);
    return HF_OK;
  }
  return HF_ERR_OOM;
}

// S22 from the factor (non-mixed forms)
int hf_s22_from_factor(hf_ctx* c) {
  cudaStream_t s = hf_stream(c);
  int M = (int)c->M;
  int rc;
  if ((rc = hf_ensure(c->d_s22, (size_t)M * M * 8 + 16))) return rc;
  if (M == 0) return HF_OK;
  if (c->prec == HF_PREC_FP64)
    HF_LAUNCH(c, HF_PROF_LAMBDA, k_s22_from_factor<double><<<1, 1024, 0, s>>>((const NodeDesc*)c->d_nodes.p, (const NodeState*)c->d_state.p,
                                                 c->n_nodes, (const double*)c->d_front.p, (const int32_t*)c->d_rowid.p,
                                                 (const int32_t*)c->d_lam2pos.p, M, (double*)c->d_s22.p,
                                                 (int*)c->d_flags.p));
  else
    HF_LAUNCH(c, HF_PROF_LAMBDA, k_s22_from_factor<float><<<1, 1024, 0, s>>>((const NodeDesc*)c->d_nodes.p, (const NodeState*)c->d_state.p,
                                                c->n_nodes, (const float*)c->d_front.p, (const int32_t*)c->d_rowid.p,
                                                (const int32_t*)c->d_lam2pos.p, M, (double*)c->d_s22.p,
                                                (int*)c->d_flags.p));
  HF_CUDA_TRY(cudaGetLastError());
  return HF_OK;
}
