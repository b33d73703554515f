// Internal state of an hf_ctx: host-side analysis results and device buffers.
#pragma once
#include "hf.h"

#include <cuda_runtime_api.h>

#include <cstdint>
#include <cstddef>
#include <string>
#include <vector>

typedef struct CUstream_st* hf_stream_t;

// Per-front static description, uploaded once (layout shared by host and device).
struct NodeDesc {
  int32_t n;          // |Lambda_t|: pivot candidates (Sec. 2.2); 0 for the Lambda_0 stage node
  int32_t s;          // rows of the static structure (ancestor indices coupled to Lambda_t)
  int32_t dc;         // capacity for postponed rows delayed into this front
  int32_t ld;         // leading dimension of the dense front (>= n + s + dc, multiple of 4)
  int32_t parent;     // elimination-order index of the parent, -1 for the Lambda_0 stage node
  int32_t child0;     // -1 if absent
  int32_t child1;     // -1 if absent
  int32_t cand_all;   // 1 for the Lambda_0 stage node: every row is a pivot candidate
  int64_t front_off;  // element offset of the front in the front arena (ld * ld elements)
  int64_t row_off;    // offset into the row-id arrays (ld entries)
  int64_t smap_off;   // offset into smap (s entries): parent front row of each structure row
  int64_t asm_off;    // offset into the assembly list
  int64_t asm_cnt;    // entries of the assembly list
  int32_t level;      // tree depth: 1 = root .. m = leaves; 0 = Lambda_0 stage
  int32_t pad;
};

// Per-front dynamic state, written by the factorization kernels.
struct NodeState {
  int32_t k;          // pivots eliminated so far (tilde-Lambda_t)
  int32_t kp0;        // first pivot of the panel just factorized (for the trailing update)
  int32_t D;          // rows delayed into this front by the children
  int32_t f;          // current front order n + s + D
  int32_t stopped;    // 1 once the ratio test postponed the rest of Lambda_t
  double dref;        // |previous pivot| for the ratio test (Sec. 2.2); 1.0 initially
  int32_t ksolve;     // pivots that belong to K11 (k minus entries moved into Lambda_2)
  int32_t nmoved;     // entries of this front moved into Lambda_2 by the enlargement
  int32_t delay_off0; // first delayed slot taken by child 0's rows
  int32_t delay_off1; // first delayed slot taken by child 1's rows
  int32_t nact;       // candidates [k, nact) still active; [nact, n) were skipped as null pivots
};

// Assembly entry: front position (row, col) receives K[csr] (scaled).
struct AsmEntry {
  int32_t r, c;
  int64_t csr;
};

struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
};

struct hf_ctx {
  hf_opts opts;
  // ---- pattern and analysis (host) ----
  int64_t L = 0, nnz = 0;
  std::vector<int64_t> rowptr;
  std::vector<int32_t> col;
  std::vector<int64_t> diagpos;      // CSR index of the diagonal of each row
  int m = 0;                         // tree levels
  int n_nodes = 0;                   // 2^m - 1 tree nodes (elimination order), plus one Lambda_0 node
  std::vector<NodeDesc> nodes;       // n_nodes + 1 entries; the last is the Lambda_0 stage node
  std::vector<int32_t> set_idx;      // Lambda_t concatenated in elimination order
  std::vector<int64_t> set_ptr;
  std::vector<int32_t> struct_idx;   // static structure rows of every front, concatenated
  std::vector<int64_t> struct_ptr;
  std::vector<int32_t> rowid_static; // per front: [Lambda_t | structure | delayed (-1)]
  std::vector<int32_t> smap;
  std::vector<AsmEntry> asm_list;
  std::vector<int> level_start, level_count;   // by depth 0..m (0 = Lambda_0 stage)
  int64_t front_elems = 0, row_elems = 0;
  double static_flops = 0;
  int delay_retries = 0;
  // ---- device: pattern and maps ----
  DevBuf d_rowptr, d_col, d_diagpos, d_nodes, d_state, d_rowid, d_rowid_static, d_smap, d_asm;
  DevBuf d_cbmap;                    // per front: parent row of each contribution row (ld entries)
  DevBuf d_q, d_kval;                // scaling diag(Q) and scaled K values (FP64)
  DevBuf d_rsign, d_qrow;            // row signs J (int8, L) and the row scale J Q (FP64, L)
  bool has_rsign = false;            // K = J Q Kbar Q is factorized (the LDU form Kbar = J S)
  DevBuf d_front;                    // front arena (float or double)
  DevBuf d_bpart;                    // per-block partial maxima of the cooperative S22 LDL^T
  DevBuf d_tparts;                   // BF16 parts of the current panel (tensor-core trailing update)
  DevBuf d_gmag;                     // per front row: |K_ii| + accumulated |l|^2 |d| (null-pivot test)
  DevBuf d_pos0;                     // per front row: its position before pivoting
  DevBuf d_invpos;                   // inverse of d_pos0 (scratch)
  DevBuf d_swlist, d_swcount;        // row interchanges listed by the cluster panel (per front)
  DevBuf d_swsig;                    // per level: row maps of the listed interchanges (scratch)
  int front_prec = -1;               // precision the arena was sized for
  DevBuf d_flags;                    // int flags: [0] delay overflow, [1] numeric error
  DevBuf d_lam2pos;                  // L ints: position in Lambda_2 or -1
  DevBuf d_lam2;                     // M ints ascending
  DevBuf d_vec;                      // per-front solve vectors (+ the sweep flags and tickets)
  size_t vec_cap = 0;
  DevBuf d_swplan;                   // dataflow sweeps: work items (forward, backward), block bases
  DevBuf d_dinv;                     // dataflow sweeps: inverse of every 64 x 64 unit lower diagonal block
  DevBuf d_gmap;                     // per front row and child slot: the child's contribution row mapped there, or -1
  std::vector<int> sw_fwd_start, sw_fwd_cnt, sw_bwd_start, sw_bwd_cnt;   // per level: item range
  int sw_blocks = 0;                 // 64-row diagonal blocks of all fronts
  // ---- split (host copy) ----
  bool factored = false, schured = false;
  int prec = HF_PREC_MIXED;
  double tau = 1e-2;
  int64_t N = 0, M = 0, n_lambda0 = 0;
  std::vector<int32_t> lambda2;      // ascending
  std::vector<NodeState> state_host;
  // ---- Schur / Krylov (device, FP64) ----
  DevBuf d_x12, d_s22, d_bk_lf, d_bk_perm, d_bk_blk, d_bk_dval, d_bk_null;
  int kernel_dim = 0;
  double s22_noise = 0;              // error estimate of S22 used by the kernel rule
  int gcr_iters = 0, solve_iters = 0;
  double gcr_relres = 0, solve_relres = 0;
  int64_t nnz_factor = 0;
  DevBuf d_work;                     // Krylov workspace
  std::vector<DevBuf> d_hist;        // block-GCR history P_0, Q_0, P_1, Q_1, ... (grown on demand)
  size_t work_cap = 0;
  DevBuf d_ozslice;                  // BF16 slices of the operands of the emulated FP64 products
  DevBuf d_small;                    // small matrices / partial sums
  size_t small_cap = 0;
  // ---- tracing ----
  bool prof_on = false;
  int64_t launches[HF_NPROF] = {0};
  double work_flops[HF_NPROF] = {0};   // algorithmic flops of the counted launches
  double work_bytes[HF_NPROF] = {0};   // algorithmic bytes of the counted launches
  std::vector<cudaEvent_t> ev_pool;   // recycled start/stop events
  size_t ev_used = 0;
  std::vector<std::pair<int, size_t>> prof_recs;   // (class, index of the start event)
  DevBuf d_gsmall;                   // block GCR small matrices (M_n, coefficients)
  DevBuf d_k12;                      // K12 block (L x M), the right-hand sides of Alg. 1 step 3
  DevBuf d_ozint;                    // scaling exponents of the emulated FP64 products
  DevBuf d_solve;                    // hf_solve scratch
  // ---- code paths of the last calls (hf_info) ----
  int path_cluster = 0;              // largest panel cluster of the last factorization
  int path_global = 0;               // levels that ran the global-memory panel
  int path_ldlt = 0;                 // S22 LDL^T kernel of the last hf_schur (hf_info.ldlt_kernel)
  int gcr_restarts = 0;              // block GCR runs restarted with native FP64 products (hf_info)
  std::vector<char> lev_panel_global;  // per tree level: 1 when its panels took k_panel
};

// analyze.cpp
int hf_analyze_impl(int64_t L, const int64_t* rowptr, const int32_t* col, const double* coords,
                    int dim, const hf_opts* opts, hf_ctx** out);
void hf_layout_fronts(hf_ctx* c);

// krylov.cu: work-item lists of the dataflow sweeps, from the host front state
int hf_sweep_plan(hf_ctx* c);   // capacities, ld, offsets (depends on opts.delay_cap)
int hf_diag_inverses(hf_ctx* c);   // inverses of the diagonal blocks of the FP32 factor (after the plan)

// Counts a kernel launch of class `cls` and, when profiling, brackets it with events.
struct ProfScope {
  hf_ctx* c;
  int cls;
  size_t idx;
  bool on;
  ProfScope(hf_ctx* ctx, int k);
  ~ProfScope();
};
#define HF_LAUNCH(ctx, cls, ...)        \
  do {                                  \
    ProfScope hf_ps_(ctx, cls);         \
    __VA_ARGS__;                        \
  } while (0)
