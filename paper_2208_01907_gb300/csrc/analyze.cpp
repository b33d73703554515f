// Host analysis: nested-dissection bisection tree (Sec. 2.2, Fig. 1), front row
// structures of the elimination tree, extend-add maps and assembly lists.
// Runs on the host only and touches no GPU.
#include "hf_internal.h"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <numeric>

namespace {

struct Analyzer {
  int64_t L;
  const int64_t* rp;
  const int32_t* ci;
  const double* coords;
  int dim;
  int m;
  std::vector<std::vector<int32_t>> sets;   // by heap id (1 .. 2^m - 1)
  std::vector<int32_t> stamp;
  int32_t stamp_val = 0;
  std::vector<int32_t> level_of;            // BFS scratch
  std::vector<int32_t> queue;

  // recursive bisection of `verts` into the sets of heap node l and its subtree
  void bisect(int l, std::vector<int32_t>& verts, int level) {
    if (level == m || verts.empty()) {
      sets[l] = verts;
      if (level < m) {
        std::vector<int32_t> e1, e2;
        bisect(2 * l, e1, level + 1);
        bisect(2 * l + 1, e2, level + 1);
      }
      return;
    }
    std::vector<int32_t> lower, upper;
    bool ok = coords ? split_geometric(verts, lower, upper) : split_graph(verts, lower, upper);
    if (!ok) {            // cannot bisect: the whole set is the separator
      sets[l] = verts;
      std::vector<int32_t> e1, e2;
      bisect(2 * l, e1, level + 1);
      bisect(2 * l + 1, e2, level + 1);
      return;
    }
    // vertex separator: vertices of `lower` that touch `upper`
    int32_t up = ++stamp_val;
    for (int32_t v : upper) stamp[v] = up;
    std::vector<int32_t> sep, low2;
    for (int32_t v : lower) {
      bool touch = false;
      for (int64_t e = rp[v]; e < rp[v + 1] && !touch; ++e) touch = (stamp[ci[e]] == up);
      (touch ? sep : low2).push_back(v);
    }
    std::sort(sep.begin(), sep.end());
    sets[l] = sep;
    verts.clear();
    verts.shrink_to_fit();
    bisect(2 * l, low2, level + 1);
    bisect(2 * l + 1, upper, level + 1);
  }

  // coordinate bisection at the middle distinct value of the widest axis
  bool split_geometric(const std::vector<int32_t>& verts, std::vector<int32_t>& lower,
                       std::vector<int32_t>& upper) {
    int ax = 0;
    double best = -1;
    for (int d = 0; d < dim; ++d) {
      double lo = INFINITY, hi = -INFINITY;
      for (int32_t v : verts) {
        double x = coords[(int64_t)v * dim + d];
        lo = std::min(lo, x);
        hi = std::max(hi, x);
      }
      if (hi - lo > best) { best = hi - lo; ax = d; }
    }
    std::vector<double> vals(verts.size());
    for (size_t i = 0; i < verts.size(); ++i) vals[i] = coords[(int64_t)verts[i] * dim + ax];
    std::sort(vals.begin(), vals.end());
    vals.erase(std::unique(vals.begin(), vals.end()), vals.end());
    if (vals.size() < 2) return false;
    double med = vals[(vals.size() + 1) / 2];
    for (int32_t v : verts) (coords[(int64_t)v * dim + ax] < med ? lower : upper).push_back(v);
    return true;
  }

  std::vector<int32_t> vis;                 // BFS visited marks (own stamp counter)
  int32_t vis_val = 0;

  // BFS from `start` restricted to vertices stamped `in`; fills level_of and queue
  int32_t bfs(int32_t start, int32_t in, int32_t& nlev) {
    int32_t vv = ++vis_val;
    queue.clear();
    queue.push_back(start);
    vis[start] = vv;
    level_of[start] = 0;
    size_t h = 0;
    int32_t last = start;
    while (h < queue.size()) {
      int32_t v = queue[h++];
      last = v;
      for (int64_t e = rp[v]; e < rp[v + 1]; ++e) {
        int32_t u = ci[e];
        if (stamp[u] == in && vis[u] != vv) {
          vis[u] = vv;
          level_of[u] = level_of[v] + 1;
          queue.push_back(u);
        }
      }
    }
    nlev = level_of[last] + 1;
    return last;
  }

  // graph bisection: middle BFS level from a pseudo-peripheral vertex; vertices the
  // BFS does not reach (other components) go to the upper half
  bool split_graph(const std::vector<int32_t>& verts, std::vector<int32_t>& lower,
                   std::vector<int32_t>& upper) {
    int32_t in = ++stamp_val;
    for (int32_t v : verts) stamp[v] = in;
    int32_t nlev;
    int32_t a = bfs(verts[0], in, nlev);
    a = bfs(a, in, nlev);
    bfs(a, in, nlev);
    const int32_t vv = vis_val;
    if (nlev < 3) return false;
    std::vector<int64_t> cnt(nlev, 0);
    int64_t reached = 0;
    for (int32_t v : verts) if (vis[v] == vv) { cnt[level_of[v]]++; reached++; }
    int64_t half = reached / 2, acc = 0;
    int cut = 1;
    for (int t = 0; t < nlev; ++t) {
      acc += cnt[t];
      if (acc >= half) { cut = t; break; }
    }
    cut = std::max(1, std::min(cut, nlev - 2));
    // lower = levels <= cut; its boundary layer (level cut) becomes the separator
    for (int32_t v : verts)
      ((vis[v] == vv && level_of[v] <= cut) ? lower : upper).push_back(v);
    return !lower.empty() && !upper.empty();
  }
};

inline int depth_of(int64_t heap) { int d = 0; while (heap) { heap >>= 1; ++d; } return d; }

}  // namespace

void hf_layout_fronts(hf_ctx* c) {
  const int nn = c->n_nodes;
  int cap = std::max(0, c->opts.delay_cap);
  int64_t off = 0, roff = 0;
  double flops = 0;
  for (int t = 0; t <= nn; ++t) {
    NodeDesc& d = c->nodes[t];
    int64_t dc = 0;
    if (t == nn) {
      const NodeDesc& r = c->nodes[nn - 1];
      dc = (int64_t)r.n + r.dc;
    } else {
      for (int ch : {d.child0, d.child1})
        if (ch >= 0) dc += (int64_t)c->nodes[ch].n + c->nodes[ch].dc;
    }
    d.dc = (int32_t)std::min<int64_t>(dc, cap);
    if (t == nn) d.dc = (int32_t)std::min<int64_t>(dc, std::max(cap, 1));
    int64_t f = (int64_t)d.n + d.s + d.dc;
    d.ld = (int32_t)((f + 3) / 4 * 4);
    if (d.ld == 0) d.ld = 4;
    d.front_off = off;
    off += (int64_t)d.ld * d.ld;
    d.row_off = roff;
    roff += d.ld;
    double n = d.n, s = d.s;
    flops += (n * n * n) / 3.0 + n * n * s + n * s * s;   // LDL^T of the static front
  }
  c->front_elems = off;
  c->row_elems = roff;
  c->static_flops = flops;
  // static row ids: [Lambda_t | structure | -1 ...]
  c->rowid_static.assign(roff, -1);
  for (int t = 0; t < nn; ++t) {
    const NodeDesc& d = c->nodes[t];
    int32_t* r = c->rowid_static.data() + d.row_off;
    for (int i = 0; i < d.n; ++i) r[i] = c->set_idx[c->set_ptr[t] + i];
    if (!c->struct_ptr.empty())
      for (int i = 0; i < d.s; ++i) r[d.n + i] = c->struct_idx[c->struct_ptr[t] + i];
  }
}

int hf_analyze_impl(int64_t L, const int64_t* rowptr, const int32_t* col, const double* coords,
                    int dim, const hf_opts* opts, hf_ctx** out) {
  if (!out || L <= 0 || !rowptr || !col) return HF_ERR_ARG;
  if (coords && (dim < 1 || dim > 3)) return HF_ERR_ARG;
  if (L >= (int64_t)INT32_MAX) return HF_ERR_ARG;
  *out = nullptr;
  // ---- validate the pattern ----
  if (rowptr[0] != 0) return HF_ERR_PATTERN;
  for (int64_t i = 0; i < L; ++i)
    if (rowptr[i + 1] < rowptr[i]) return HF_ERR_PATTERN;
  const int64_t nnz = rowptr[L];
  std::vector<int64_t> diagpos(L, -1);
  for (int64_t i = 0; i < L; ++i) {
    for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) {
      int32_t j = col[e];
      if (j < 0 || j >= L) return HF_ERR_PATTERN;
      if (e > rowptr[i] && col[e - 1] >= j) return HF_ERR_PATTERN;
      if (j == i) diagpos[i] = e;
    }
    if (diagpos[i] < 0) return HF_ERR_PATTERN;
  }
  for (int64_t i = 0; i < L; ++i)
    for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) {
      int32_t j = col[e];
      if (!std::binary_search(col + rowptr[j], col + rowptr[j + 1], (int32_t)i)) return HF_ERR_PATTERN;
    }

  hf_ctx* c = new (std::nothrow) hf_ctx();
  if (!c) return HF_ERR_OOM;
  if (opts) c->opts = *opts; else hf_default_opts(&c->opts);
  c->tau = c->opts.tau;
  c->prec = c->opts.precision;
  c->L = L;
  c->nnz = nnz;
  c->rowptr.assign(rowptr, rowptr + L + 1);
  c->col.assign(col, col + nnz);
  c->diagpos = diagpos;

  // ---- nested dissection (Sec. 2.2): complete m-level bisection tree ----
  int leaf = std::max(1, c->opts.nd_leaf);
  int m = c->opts.nd_levels;
  if (m <= 0) {
    m = 1;
    while (m < 24 && (double)L / std::ldexp(1.0, m - 1) > leaf) ++m;
  }
  m = std::min(m, 24);
  c->m = m;
  Analyzer A;
  A.L = L; A.rp = rowptr; A.ci = col; A.coords = coords; A.dim = dim; A.m = m;
  A.sets.resize((size_t)1 << m);
  A.stamp.assign(L, 0);
  A.level_of.assign(L, 0);
  A.vis.assign(L, 0);
  {
    std::vector<int32_t> all(L);
    std::iota(all.begin(), all.end(), 0);
    A.bisect(1, all, 1);
  }
  // elimination order: deepest level first, left to right (Fig. 1: 4,5,6,7,2,3,1)
  const int nn = (1 << m) - 1;
  c->n_nodes = nn;
  std::vector<int> heap_of(nn), pos_of_heap(nn + 1);
  {
    int t = 0;
    c->level_start.assign(m + 1, 0);
    c->level_count.assign(m + 1, 0);
    for (int lev = m; lev >= 1; --lev) {
      c->level_start[lev] = t;
      c->level_count[lev] = 1 << (lev - 1);
      for (int l = 1 << (lev - 1); l < (1 << lev); ++l) { heap_of[t] = l; pos_of_heap[l] = t; ++t; }
    }
    c->level_start[0] = nn;
    c->level_count[0] = 1;
  }
  c->nodes.assign(nn + 1, NodeDesc{});
  c->set_ptr.assign(nn + 2, 0);
  c->set_idx.clear();
  c->set_idx.reserve(L);
  std::vector<int32_t> owner(L, -1);
  for (int t = 0; t < nn; ++t) {
    const auto& s = A.sets[heap_of[t]];
    c->set_ptr[t + 1] = c->set_ptr[t] + (int64_t)s.size();
    for (int32_t v : s) { c->set_idx.push_back(v); owner[v] = t; }
  }
  c->set_ptr[nn + 1] = c->set_ptr[nn];
  if ((int64_t)c->set_idx.size() != L) { delete c; return HF_ERR_PATTERN; }
  A.sets.clear();

  for (int t = 0; t < nn; ++t) {
    NodeDesc& d = c->nodes[t];
    int l = heap_of[t];
    d.n = (int32_t)(c->set_ptr[t + 1] - c->set_ptr[t]);
    d.level = depth_of(l);
    d.parent = (l == 1) ? nn : pos_of_heap[l >> 1];
    d.child0 = (d.level < m) ? pos_of_heap[2 * l] : -1;
    d.child1 = (d.level < m) ? pos_of_heap[2 * l + 1] : -1;
    d.cand_all = 0;
  }
  {
    NodeDesc& d = c->nodes[nn];     // Lambda_0 stage: refactorization of the postponed set
    d.n = 0; d.s = 0; d.level = 0; d.parent = -1; d.child0 = nn - 1; d.child1 = -1; d.cand_all = 1;
  }

  // ---- front structures: ancestors coupled to Lambda_t through the filled graph ----
  auto is_strict_ancestor = [&](int a_t, int t) {
    int64_t a = heap_of[a_t], s = heap_of[t];
    int da = depth_of(a), ds = depth_of(s);
    if (da >= ds) return false;
    return (s >> (ds - da)) == a;
  };
  std::vector<std::vector<int32_t>> strc(nn);
  std::vector<int32_t> mark(L, -1);
  for (int t = 0; t < nn; ++t) {
    std::vector<int32_t>& S = strc[t];
    for (int64_t i = c->set_ptr[t]; i < c->set_ptr[t + 1]; ++i) {
      int32_t v = c->set_idx[i];
      for (int64_t e = rowptr[v]; e < rowptr[v + 1]; ++e) {
        int32_t u = col[e];
        int o = owner[u];
        if (o != t && mark[u] != t && is_strict_ancestor(o, t)) { mark[u] = t; S.push_back(u); }
      }
    }
    for (int ch : {c->nodes[t].child0, c->nodes[t].child1}) {
      if (ch < 0) continue;
      for (int32_t u : strc[ch])
        if (owner[u] != t && mark[u] != t) { mark[u] = t; S.push_back(u); }
    }
    std::sort(S.begin(), S.end(), [&](int32_t a, int32_t b) {
      return owner[a] != owner[b] ? owner[a] < owner[b] : a < b;
    });
    c->nodes[t].s = (int32_t)S.size();
  }
  c->struct_ptr.assign(nn + 1, 0);
  for (int t = 0; t < nn; ++t) c->struct_ptr[t + 1] = c->struct_ptr[t] + (int64_t)strc[t].size();
  c->struct_idx.clear();
  c->struct_idx.reserve(c->struct_ptr[nn]);
  for (int t = 0; t < nn; ++t) c->struct_idx.insert(c->struct_idx.end(), strc[t].begin(), strc[t].end());
  hf_layout_fronts(c);
  // structure rows into the static row ids; extend-add maps; assembly lists
  std::vector<int32_t> fpos(L, -1);
  c->smap.clear();
  c->asm_list.clear();
  c->asm_list.reserve((size_t)(nnz * 3 / 2 + 16));
  for (int t = 0; t < nn; ++t) {
    NodeDesc& d = c->nodes[t];
    const int32_t* r = c->rowid_static.data() + d.row_off;
    for (int i = 0; i < d.n + d.s; ++i) fpos[r[i]] = i;
    for (int ch : {d.child0, d.child1}) {
      if (ch < 0) continue;
      c->nodes[ch].smap_off = (int64_t)c->smap.size();
      for (int32_t u : strc[ch]) c->smap.push_back(fpos[u]);
    }
    d.asm_off = (int64_t)c->asm_list.size();
    for (int i = 0; i < d.n; ++i) {
      int32_t v = r[i];
      for (int64_t e = rowptr[v]; e < rowptr[v + 1]; ++e) {
        int32_t u = col[e];
        int o = owner[u];
        if (o == t) {                       // inside Lambda_t: lower triangle only
          if (fpos[u] <= i) c->asm_list.push_back({i, fpos[u], e});
        } else if (is_strict_ancestor(o, t)) {   // structure row (always below Lambda_t)
          c->asm_list.push_back({fpos[u], i, e});
        }
      }
    }
    d.asm_cnt = (int64_t)c->asm_list.size() - d.asm_off;
    for (int i = 0; i < d.n + d.s; ++i) fpos[r[i]] = -1;
  }
  c->nodes[nn - 1].smap_off = (int64_t)c->smap.size();   // root: empty structure
  c->nodes[nn].smap_off = (int64_t)c->smap.size();
  c->nodes[nn].asm_off = (int64_t)c->asm_list.size();
  c->nodes[nn].asm_cnt = 0;
  *out = c;
  return HF_OK;
}
