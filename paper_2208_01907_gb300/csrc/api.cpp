// C ABI entry points (include/hf.h): argument checks, call order, host getters.
#include "hf_internal.h"

#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <cstdlib>
#include <atomic>
#include <thread>
#include <vector>

int hf_factorize_impl(hf_ctx* c, const double* vals, double tau);
int hf_schur_impl(hf_ctx* c);
int hf_solve_impl(hf_ctx* c, int nrhs, const double* b, int64_t ldb, double* x, int64_t ldx);
int hf_precond_impl(hf_ctx* c, int m, const double* R, double* W);
int hf_precond_noalloc_impl(hf_ctx* c, int m, const double* R, double* W);
int hf_gram_fp64_impl(hf_ctx* c, int64_t L, int ma, int mb, const double* A, const double* B, double* G, double scale);
int hf_k11_iterate_impl(hf_ctx* c, int method, int m, const double* B, double* X, int maxit, double* hist, int* iters);
int hf_update_fp64_impl(hf_ctx* c, int64_t L, int m, const double* A, const double* C, double* Y, const double* Yinit,
                        double sgn);
int hf_kernel_basis_impl(hf_ctx* c, double* basis, int64_t ldb);
int hf_values_adjoint_impl(hf_ctx* c, int m, const double* x, int64_t ldx, const double* lam, int64_t ldl,
                           double* grad);

static thread_local char g_cuda_msg[256] = "";

int hf_cuda_error(cudaError_t e) {
  std::snprintf(g_cuda_msg, sizeof(g_cuda_msg), "%s", cudaGetErrorString(e));
  if (e == cudaErrorMemoryAllocation) { cudaGetLastError(); return HF_ERR_OOM; }
  return HF_ERR_CUDA;
}

const char* hf_last_cuda_message() { return g_cuda_msg; }

int hf_ensure(DevBuf& b, size_t bytes) {
  if (b.p && b.bytes >= bytes) return HF_OK;
  if (b.p) { cudaFree(b.p); b.p = nullptr; b.bytes = 0; }
  cudaError_t e = cudaMalloc(&b.p, bytes);
  if (e != cudaSuccess) { b.p = nullptr; return hf_cuda_error(e); }
  b.bytes = bytes;
  return HF_OK;
}

void hf_release(DevBuf& b) {
  if (b.p) cudaFree(b.p);
  b.p = nullptr;
  b.bytes = 0;
}

ProfScope::ProfScope(hf_ctx* ctx, int k) : c(ctx), cls(k), idx(0), on(ctx && ctx->prof_on) {
  if (!c) return;
  c->launches[cls]++;
  if (!on) return;
  while (c->ev_pool.size() < c->ev_used + 2) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) { on = false; return; }
    c->ev_pool.push_back(e);
  }
  idx = c->ev_used;
  c->ev_used += 2;
  cudaEventRecord(c->ev_pool[idx], (cudaStream_t)c->opts.cuda_stream);
}

ProfScope::~ProfScope() {
  if (!on) return;
  cudaEventRecord(c->ev_pool[idx + 1], (cudaStream_t)c->opts.cuda_stream);
  c->prof_recs.push_back({cls, idx});
}

namespace {

int batch_workers(int n) {
  int w = 8;
  if (const char* e = std::getenv("HF_BATCH_WORKERS")) w = std::max(1, std::atoi(e));
  return std::max(1, std::min(w, n));
}

// Runs op(i) for the n contexts on a pool of host threads.  Each worker owns a
// non-blocking stream, used by contexts created on the default stream.
template <typename Op>
int run_batched(hf_ctx* const* ctxs, int n, int32_t* status, Op op) {
  if (!ctxs || n < 0) return HF_ERR_ARG;
  if (n == 0) return HF_OK;
  {
    std::vector<hf_ctx*> v(ctxs, ctxs + n);
    for (hf_ctx* c : v) if (!c) return HF_ERR_ARG;
    std::sort(v.begin(), v.end());
    if (std::adjacent_find(v.begin(), v.end()) != v.end()) return HF_ERR_ARG;
  }
  int dev = 0;
  {
    const cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return hf_cuda_error(e);
  }
  const int W = batch_workers(n);
  std::vector<cudaStream_t> streams(W, nullptr);
  for (int w = 0; w < W; ++w) {
    cudaError_t e = cudaStreamCreateWithFlags(&streams[w], cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      for (int u = 0; u < w; ++u) cudaStreamDestroy(streams[u]);
      return hf_cuda_error(e);
    }
  }
  std::vector<int32_t> st(n, HF_OK);
  std::atomic<int> next(0);
  auto worker = [&](int w) {
    cudaSetDevice(dev);
    for (;;) {
      const int i = next.fetch_add(1);
      if (i >= n) break;
      hf_ctx* c = ctxs[i];
      void* saved = c->opts.cuda_stream;
      if (!saved) c->opts.cuda_stream = streams[w];
      int rc = op(i);
      const cudaError_t e = cudaStreamSynchronize((cudaStream_t)c->opts.cuda_stream);
      if (rc == HF_OK && e != cudaSuccess) rc = hf_cuda_error(e);
      c->opts.cuda_stream = saved;
      st[i] = rc;
    }
  };
  std::vector<std::thread> threads;
  threads.reserve(W);
  for (int w = 0; w < W; ++w) threads.emplace_back(worker, w);
  for (auto& t : threads) t.join();
  for (int w = 0; w < W; ++w) cudaStreamDestroy(streams[w]);
  int first = HF_OK;
  for (int i = 0; i < n; ++i) {
    if (status) status[i] = st[i];
    if (first == HF_OK && st[i] != HF_OK) first = st[i];
  }
  return first;
}

}  // namespace

extern "C" {

int hf_profile(hf_ctx* c, int enable) {
  if (!c) return HF_ERR_ARG;
  c->prof_on = enable != 0;
  c->prof_recs.clear();
  c->ev_used = 0;
  for (auto& v : c->launches) v = 0;
  for (auto& v : c->work_flops) v = 0;
  for (auto& v : c->work_bytes) v = 0;
  return HF_OK;
}

int hf_get_profile(hf_ctx* c, double* ms, int64_t* launches, double* flops, double* bytes) {
  if (!c) return HF_ERR_ARG;
  if (cudaStreamSynchronize((cudaStream_t)c->opts.cuda_stream) != cudaSuccess) return HF_ERR_CUDA;
  double acc[HF_NPROF] = {0};
  for (auto& r : c->prof_recs) {
    float t = 0;
    if (cudaEventElapsedTime(&t, c->ev_pool[r.second], c->ev_pool[r.second + 1]) == cudaSuccess) acc[r.first] += t;
  }
  if (ms) for (int i = 0; i < HF_NPROF; ++i) ms[i] = acc[i];
  if (launches) for (int i = 0; i < HF_NPROF; ++i) launches[i] = c->launches[i];
  if (flops) for (int i = 0; i < HF_NPROF; ++i) flops[i] = c->work_flops[i];
  if (bytes) for (int i = 0; i < HF_NPROF; ++i) bytes[i] = c->work_bytes[i];
  c->prof_recs.clear();
  c->ev_used = 0;
  for (auto& v : c->launches) v = 0;
  for (auto& v : c->work_flops) v = 0;
  for (auto& v : c->work_bytes) v = 0;
  return HF_OK;
}

const char* hf_profile_name(int cls) {
  static const char* names[HF_NPROF] = {"scale", "assemble", "panel", "trailing", "lambda0",
                                        "trsv_fwd", "trsv_bwd", "spmm", "gram", "block_update",
                                        "schur", "dense_ldlt", "vector", "panel_swap", "sweep_io",
                                        "tc_prep", "diag_inverse", "panel_global"};
  return (cls >= 0 && cls < HF_NPROF) ? names[cls] : "unknown";
}

int hf_default_opts(hf_opts* o) {
  if (!o) return HF_ERR_ARG;
  std::memset(o, 0, sizeof(*o));
  o->tau = 1e-2;
  o->n_enlarge = 4;
  o->precision = HF_PREC_MIXED;
  o->gcr_tol = 1e-14;
  o->gcr_maxit = 40;
  o->kernel_eps = 1e-10;
  o->kernel_gap = 1e4;
  o->nd_leaf = 256;
  o->nd_levels = 0;
  o->delay_cap = 256;
  o->panel = 64;
  o->cuda_stream = nullptr;
  o->fp64_gemm = 0;
  o->trailing = 0;
  o->null_test = 0;
  o->spin_limit = 0;
  return HF_OK;
}

int hf_set_spin_limit(hf_ctx* c, int limit) {
  if (!c || limit < 0) return HF_ERR_ARG;
  c->opts.spin_limit = limit;
  return HF_OK;
}

const char* hf_error_string(int code) {
  switch (code) {
    case HF_OK: return "ok";
    case HF_ERR_ARG: return "invalid argument";
    case HF_ERR_STATE: return "call order violated";
    case HF_ERR_PATTERN: return "invalid sparsity pattern";
    case HF_ERR_NUMERIC: return "non-finite input values";
    case HF_ERR_NOT_CONVERGED: return "block GCR did not converge";
    case HF_ERR_TIMEOUT: return "device wait timed out";
    case HF_ERR_CUDA: return "CUDA error";
    case HF_ERR_OOM: return "device out of memory";
    case HF_ERR_CAPACITY: return "front too large for the panel kernels (too many postponed rows)";
    default: return "unknown error";
  }
}

int hf_analyze(int64_t L, const int64_t* rowptr, const int32_t* col, const double* coords, int dim,
               const hf_opts* opts, hf_ctx** out) {
  if (opts) {
    if (!(opts->tau > 0) || opts->n_enlarge < 0 || opts->gcr_maxit < 1 || opts->nd_leaf < 1 ||
        opts->panel < 1 || opts->delay_cap < 0 || opts->nd_levels < 0 || opts->nd_levels > 24 ||
        opts->spin_limit < 0 || opts->null_test < 0 || opts->null_test > 1)
      return HF_ERR_ARG;
    if (opts->precision < HF_PREC_MIXED || opts->precision > HF_PREC_FP32) return HF_ERR_ARG;
  }
  return hf_analyze_impl(L, rowptr, col, coords, dim, opts, out);
}

int hf_factorize(hf_ctx* c, const double* vals, double tau) {
  if (!c || !vals || !(tau > 0)) return HF_ERR_ARG;
  return hf_factorize_impl(c, vals, tau);
}

int hf_set_row_signs(hf_ctx* c, const int8_t* sign) {
  if (!c) return HF_ERR_ARG;
  if (sign)
    for (int64_t i = 0; i < c->L; ++i)
      if (sign[i] != 1 && sign[i] != -1) return HF_ERR_ARG;   // state unchanged
  c->factored = false;
  c->schured = false;
  c->has_rsign = false;
  if (!sign) return HF_OK;
  int rc;
  if ((rc = hf_ensure(c->d_rsign, (size_t)c->L + 16))) return rc;
  cudaStream_t s = (cudaStream_t)c->opts.cuda_stream;
  cudaError_t e = cudaMemcpyAsync(c->d_rsign.p, sign, (size_t)c->L, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);   // the caller may free its array on return
  if (e != cudaSuccess) return hf_cuda_error(e);
  c->has_rsign = true;
  return HF_OK;
}

int hf_schur(hf_ctx* c) {
  if (!c) return HF_ERR_ARG;
  return hf_schur_impl(c);
}

int hf_solve(hf_ctx* c, int nrhs, const double* b, int64_t ldb, double* x, int64_t ldx) {
  if (!c) return HF_ERR_ARG;
  return hf_solve_impl(c, nrhs, b, ldb, x, ldx);
}

int hf_precond(hf_ctx* c, int m, const double* R, double* W) {
  if (!c) return HF_ERR_ARG;
  return hf_precond_impl(c, m, R, W);
}

int hf_values_adjoint(hf_ctx* c, int nrhs, const double* x, int64_t ldx, const double* lam, int64_t ldl,
                      double* grad_vals) {
  if (!c) return HF_ERR_ARG;
  return hf_values_adjoint_impl(c, nrhs, x, ldx, lam, ldl, grad_vals);
}

int hf_k11_iterate(hf_ctx* c, int method, int m, const double* B, double* X, int maxit, double* hist, int* iters) {
  if (!c) return HF_ERR_ARG;
  return hf_k11_iterate_impl(c, method, m, B, X, maxit, hist, iters);
}

int hf_gram_fp64(hf_ctx* c, int64_t L, int ma, int mb, const double* A, const double* B, double* G, double scale) {
  if (!c) return HF_ERR_ARG;
  return hf_gram_fp64_impl(c, L, ma, mb, A, B, G, scale);
}

int hf_update_fp64(hf_ctx* c, int64_t L, int m, const double* A, const double* C, double* Y, const double* Yinit,
                   double sgn) {
  if (!c) return HF_ERR_ARG;
  return hf_update_fp64_impl(c, L, m, A, C, Y, Yinit, sgn);
}

int hf_precond_noalloc(hf_ctx* c, int m, const double* R, double* W) {
  if (!c) return HF_ERR_ARG;
  return hf_precond_noalloc_impl(c, m, R, W);
}

int hf_get_info(hf_ctx* c, hf_info* info) {
  if (!c || !info) return HF_ERR_ARG;
  std::memset(info, 0, sizeof(*info));
  info->L = c->L;
  info->N = c->N;
  info->M = c->M;
  info->n_lambda0 = c->n_lambda0;
  info->nnz_factor = c->nnz_factor;
  info->n_nodes = c->n_nodes;
  info->levels = c->m;
  info->kernel_dim = c->kernel_dim;
  info->gcr_iters = c->gcr_iters;
  info->solve_iters = c->solve_iters;
  info->gcr_relres = c->gcr_relres;
  info->solve_relres = c->solve_relres;
  double fl = 0;
  for (size_t t = 0; t < c->state_host.size(); ++t) {
    double k = c->state_host[t].k, f = c->state_host[t].f;
    // sum over pivots j of (f - j - 1)^2 multiply-adds in the Schur updates
    fl += 2.0 * (k * (f - 1) * (f - 1) - (f - 1) * k * (k - 1) + k * (k - 1) * (2 * k - 1) / 6.0) / 2.0;
  }
  info->factor_flops = fl;
  {
    const double nb = std::max(1, std::min(c->opts.panel, 256));
    double tf = 0;
    int64_t se = 0;
    for (size_t t = 0; t < c->state_host.size(); ++t) {
      const double k = c->state_host[t].k, f = c->state_host[t].f, ks = c->state_host[t].ksolve;
      for (double k0 = 0; k0 < k; k0 += nb) {
        double k1 = std::min(k, k0 + nb), n = f - k1;
        tf += (k1 - k0) * n * (n + 1);
      }
      se += (int64_t)(f * ks - ks * (ks + 1) / 2);
      info->sweep_blocks = std::max(info->sweep_blocks, (int32_t)((c->state_host[t].ksolve + 63) / 64));
    }
    info->trailing_flops = tf;
    info->solve_factor_entries = se;
  }
  info->panel_cluster = c->path_cluster;
  info->panel_global = c->path_global;
  info->ldlt_kernel = c->path_ldlt;
  info->gcr_restarts = c->gcr_restarts;
  info->front_bytes = c->d_front.p ? (int64_t)c->d_front.bytes : 0;
  info->delay_retries = c->delay_retries;
  info->precision = c->prec;
  return HF_OK;
}

int hf_get_split(hf_ctx* c, int32_t* pivot_order, int32_t* lambda2, hf_info* info) {
  if (!c) return HF_ERR_ARG;
  if (!c->factored) return HF_ERR_STATE;
  if (lambda2 && c->M) std::memcpy(lambda2, c->lambda2.data(), c->M * 4);
  if (pivot_order) {
    std::vector<int32_t> rid(c->row_elems);
    if (cudaMemcpy(rid.data(), c->d_rowid.p, rid.size() * 4, cudaMemcpyDeviceToHost) != cudaSuccess)
      return HF_ERR_CUDA;
    int64_t p = 0;
    for (int t = 0; t <= c->n_nodes; ++t) {
      const NodeState& S = c->state_host[t];
      for (int i = 0; i < S.ksolve; ++i) pivot_order[p++] = rid[c->nodes[t].row_off + i];
    }
    for (int32_t v : c->lambda2) pivot_order[p++] = v;
    if (p != c->L) return HF_ERR_STATE;
  }
  if (info) return hf_get_info(c, info);
  return HF_OK;
}

int hf_get_tree(hf_ctx* c, int32_t* parent, int64_t* set_ptr, int32_t* set_idx) {
  if (!c) return HF_ERR_ARG;
  const int nn = c->n_nodes;
  if (parent)
    for (int t = 0; t < nn; ++t) parent[t] = (c->nodes[t].parent >= nn) ? -1 : c->nodes[t].parent;
  if (set_ptr) std::memcpy(set_ptr, c->set_ptr.data(), (nn + 1) * sizeof(int64_t));
  if (set_idx) std::memcpy(set_idx, c->set_idx.data(), c->set_idx.size() * 4);
  return HF_OK;
}

int hf_get_pivots(hf_ctx* c, int64_t* node_ptr, int32_t* piv, int32_t* moved, int32_t* n_moved) {
  if (!c) return HF_ERR_ARG;
  if (!c->factored) return HF_ERR_STATE;
  std::vector<int32_t> rid(c->row_elems);
  if (cudaMemcpy(rid.data(), c->d_rowid.p, rid.size() * 4, cudaMemcpyDeviceToHost) != cudaSuccess)
    return HF_ERR_CUDA;
  const int nn = c->n_nodes;
  int64_t p = 0;
  int nm = 0;
  if (node_ptr) node_ptr[0] = 0;
  for (int t = 0; t <= nn; ++t) {
    const NodeState& S = c->state_host[t];
    for (int i = 0; i < S.k; ++i) {
      if (piv) piv[p] = rid[c->nodes[t].row_off + i];
      ++p;
    }
    if (node_ptr) node_ptr[t + 1] = p;
  }
  // moved entries in elimination order
  for (int t = 0; t <= nn; ++t) {
    const NodeState& S = c->state_host[t];
    for (int i = S.ksolve; i < S.k; ++i) {
      if (moved) moved[nm] = rid[c->nodes[t].row_off + i];
      ++nm;
    }
  }
  if (n_moved) *n_moved = nm;
  return HF_OK;
}

int hf_get_pivot_events(hf_ctx* c, int64_t* node_ptr, int32_t* cand, int32_t* counts) {
  if (!c || !node_ptr) return HF_ERR_ARG;
  if (!c->factored) return HF_ERR_STATE;
  const int nn = c->n_nodes;
  std::vector<int32_t> rid;
  if (cand) {
    rid.resize(c->row_elems);
    if (cudaMemcpy(rid.data(), c->d_rowid.p, rid.size() * 4, cudaMemcpyDeviceToHost) != cudaSuccess)
      return HF_ERR_CUDA;
  }
  node_ptr[0] = 0;
  int64_t p = 0;
  for (int t = 0; t <= nn; ++t) {
    const NodeState& S = c->state_host[t];
    const int ncand = c->nodes[t].cand_all ? S.f : c->nodes[t].n;
    for (int i = 0; i < ncand; ++i) {
      if (cand) cand[p] = rid[c->nodes[t].row_off + i];
      ++p;
    }
    node_ptr[t + 1] = p;
    if (counts) { counts[2 * t] = S.k; counts[2 * t + 1] = S.nact; }
  }
  return HF_OK;
}

int hf_get_factor(hf_ctx* c, int64_t* col_ptr, int32_t* row_idx, double* val, double* d) {
  if (!c || !col_ptr) return HF_ERR_ARG;
  if (!c->factored) return HF_ERR_STATE;
  const int nn = c->n_nodes;
  int64_t p = 0, j = 0;
  col_ptr[0] = 0;
  for (int t = 0; t <= nn; ++t) {
    const NodeState& S = c->state_host[t];
    for (int i = 0; i < S.k; ++i) { p += S.f - i - 1; col_ptr[++j] = p; }
  }
  if (!row_idx && !val && !d) return HF_OK;
  std::vector<int32_t> rid(c->row_elems);
  if (cudaMemcpy(rid.data(), c->d_rowid.p, rid.size() * 4, cudaMemcpyDeviceToHost) != cudaSuccess)
    return HF_ERR_CUDA;
  const bool dbl = c->front_prec == HF_PREC_FP64;
  j = 0;
  p = 0;
  for (int t = 0; t <= nn; ++t) {
    const NodeState& S = c->state_host[t];
    const NodeDesc& nd = c->nodes[t];
    if (S.k == 0) continue;
    const size_t esz = dbl ? 8 : 4;
    std::vector<unsigned char> buf((size_t)nd.ld * S.k * esz);
    if (cudaMemcpy(buf.data(), (const unsigned char*)c->d_front.p + nd.front_off * esz, buf.size(),
                   cudaMemcpyDeviceToHost) != cudaSuccess)
      return HF_ERR_CUDA;
    auto at = [&](int r, int cc) -> double {
      size_t o = (size_t)r + (size_t)cc * nd.ld;
      return dbl ? ((const double*)buf.data())[o] : (double)((const float*)buf.data())[o];
    };
    for (int i = 0; i < S.k; ++i) {
      if (d) d[j] = at(i, i);
      for (int r = i + 1; r < S.f; ++r) {
        if (row_idx) row_idx[p] = rid[nd.row_off + r];
        if (val) val[p] = at(r, i);
        ++p;
      }
      ++j;
    }
  }
  return HF_OK;
}

int hf_get_x12(hf_ctx* c, double* x12, int64_t ldx12) {
  if (!c || !x12 || ldx12 < c->M) return HF_ERR_ARG;
  if (!c->schured || c->prec != HF_PREC_MIXED) return HF_ERR_STATE;
  if (c->M == 0) return HF_OK;
  cudaError_t e = cudaMemcpy2D(x12, ldx12 * 8, c->d_x12.p, c->M * 8, c->M * 8, c->L, cudaMemcpyDeviceToDevice);
  return e == cudaSuccess ? HF_OK : hf_cuda_error(e);
}

int hf_get_kernel_basis(hf_ctx* c, double* basis, int64_t ldb) {
  if (!c) return HF_ERR_ARG;
  return hf_kernel_basis_impl(c, basis, ldb);
}

int hf_get_s22(hf_ctx* c, double* s22) {
  if (!c || !s22) return HF_ERR_ARG;
  if (!c->schured) return HF_ERR_STATE;
  if (c->M == 0) return HF_OK;
  cudaError_t e = cudaMemcpy(s22, c->d_s22.p, c->M * c->M * 8, cudaMemcpyDeviceToDevice);
  return e == cudaSuccess ? HF_OK : hf_cuda_error(e);
}

int hf_get_s22_factor(hf_ctx* c, int32_t* perm, double* lf, int32_t* dblk, double* dval, int32_t* null_piv) {
  if (!c) return HF_ERR_ARG;
  if (!c->schured) return HF_ERR_STATE;
  const int64_t M = c->M;
  if (M == 0) return HF_OK;
  cudaError_t e = cudaSuccess;
  if (perm && e == cudaSuccess) e = cudaMemcpy(perm, c->d_bk_perm.p, M * 4, cudaMemcpyDeviceToHost);
  if (lf && e == cudaSuccess) e = cudaMemcpy(lf, c->d_bk_lf.p, M * M * 8, cudaMemcpyDeviceToHost);
  if (dblk && e == cudaSuccess) e = cudaMemcpy(dblk, c->d_bk_blk.p, M * 4, cudaMemcpyDeviceToHost);
  if (dval && e == cudaSuccess) e = cudaMemcpy(dval, c->d_bk_dval.p, M * 16, cudaMemcpyDeviceToHost);
  if (null_piv && e == cudaSuccess) e = cudaMemcpy(null_piv, c->d_bk_null.p, M * 4, cudaMemcpyDeviceToHost);
  return e == cudaSuccess ? HF_OK : hf_cuda_error(e);
}

int hf_factorize_batched(hf_ctx* const* ctxs, int n, const double* const* vals_dev, double tau, int32_t* status) {
  if (!vals_dev) return HF_ERR_ARG;
  return run_batched(ctxs, n, status, [&](int i) { return hf_factorize(ctxs[i], vals_dev[i], tau); });
}

int hf_schur_batched(hf_ctx* const* ctxs, int n, int32_t* status) {
  return run_batched(ctxs, n, status, [&](int i) { return hf_schur(ctxs[i]); });
}

int hf_solve_batched(hf_ctx* const* ctxs, int n, int nrhs, const double* const* b_dev, const int64_t* ldb,
                     double* const* x_dev, const int64_t* ldx, int32_t* status) {
  if (!b_dev || !x_dev) return HF_ERR_ARG;
  return run_batched(ctxs, n, status, [&](int i) {
    const int64_t lb = ldb ? ldb[i] : ctxs[i]->L, lx = ldx ? ldx[i] : ctxs[i]->L;
    return hf_solve(ctxs[i], nrhs, b_dev[i], lb, x_dev[i], lx);
  });
}

void hf_free(hf_ctx* c) {
  if (!c) return;
  DevBuf* bufs[] = {&c->d_rowptr, &c->d_col, &c->d_diagpos, &c->d_nodes, &c->d_state, &c->d_rowid,
                    &c->d_rowid_static, &c->d_smap, &c->d_asm, &c->d_cbmap, &c->d_q, &c->d_kval,
                    &c->d_front, &c->d_flags, &c->d_lam2pos, &c->d_lam2, &c->d_vec, &c->d_x12,
                    &c->d_s22, &c->d_bk_lf, &c->d_bk_perm, &c->d_bk_blk, &c->d_bk_dval, &c->d_bk_null,
                    &c->d_work, &c->d_small, &c->d_ozslice, &c->d_gsmall, &c->d_k12, &c->d_solve, &c->d_gmag,
                    &c->d_pos0, &c->d_invpos, &c->d_ozint, &c->d_tparts, &c->d_dinv, &c->d_gmap, &c->d_bpart, &c->d_swlist,
                    &c->d_swcount, &c->d_swplan, &c->d_swsig, &c->d_rsign, &c->d_qrow};
  for (DevBuf* b : bufs) hf_release(*b);
  for (DevBuf& b : c->d_hist) hf_release(b);
  for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
  delete c;
}

}  // extern "C"
