"""ctypes binding of the C ABI in include/hf.h (argument marshalling only).

Every numerical step runs in libhf.so.  Device buffers are torch CUDA tensors
(PyTorch supplies device memory and the stream); host buffers are numpy arrays.
Loading fails loudly when the library has not been built: there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libhf.so")

HF_OK, HF_ERR_ARG, HF_ERR_STATE, HF_ERR_PATTERN, HF_ERR_NUMERIC = 0, 1, 2, 3, 4
HF_ERR_NOT_CONVERGED, HF_ERR_TIMEOUT, HF_ERR_CUDA, HF_ERR_OOM, HF_ERR_CAPACITY = 5, 6, 7, 8, 9
HF_PREC_MIXED, HF_PREC_FP64, HF_PREC_FP32 = 0, 1, 2

#: every symbol declared in include/hf.h
EXPORTED = (
    "hf_default_opts", "hf_error_string", "hf_analyze", "hf_factorize", "hf_schur", "hf_solve",
    "hf_get_split", "hf_get_info", "hf_get_tree", "hf_get_pivots", "hf_get_factor", "hf_get_x12",
    "hf_get_s22", "hf_get_s22_factor", "hf_get_pivot_events", "hf_precond", "hf_profile",
    "hf_get_profile", "hf_profile_name", "hf_values_adjoint", "hf_precond_noalloc",
    "hf_factorize_batched", "hf_schur_batched", "hf_solve_batched", "hf_get_kernel_basis",
    "hf_gram_fp64", "hf_update_fp64", "hf_k11_iterate", "hf_set_row_signs", "hf_set_spin_limit", "hf_free",
)
HF_NPROF = 18


class hf_opts(C.Structure):
    _fields_ = [
        ("tau", C.c_double), ("n_enlarge", C.c_int), ("precision", C.c_int),
        ("gcr_tol", C.c_double), ("gcr_maxit", C.c_int), ("kernel_eps", C.c_double),
        ("kernel_gap", C.c_double), ("nd_leaf", C.c_int), ("nd_levels", C.c_int),
        ("delay_cap", C.c_int), ("panel", C.c_int), ("cuda_stream", C.c_void_p),
        ("fp64_gemm", C.c_int), ("trailing", C.c_int), ("null_test", C.c_int), ("spin_limit", C.c_int),
    ]


class hf_info(C.Structure):
    _fields_ = [
        ("L", C.c_int64), ("N", C.c_int64), ("M", C.c_int64), ("n_lambda0", C.c_int64),
        ("nnz_factor", C.c_int64), ("n_nodes", C.c_int64), ("levels", C.c_int32),
        ("kernel_dim", C.c_int32), ("gcr_iters", C.c_int32), ("solve_iters", C.c_int32),
        ("gcr_relres", C.c_double), ("solve_relres", C.c_double), ("factor_flops", C.c_double),
        ("front_bytes", C.c_int64), ("delay_retries", C.c_int32), ("precision", C.c_int32),
        ("trailing_flops", C.c_double), ("solve_factor_entries", C.c_int64),
        ("panel_cluster", C.c_int32), ("panel_global", C.c_int32), ("sweep_blocks", C.c_int32),
        ("ldlt_kernel", C.c_int32), ("gcr_restarts", C.c_int32),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class HFError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        super().__init__(f"{where}: {lib().hf_error_string(code).decode()} (code {code})")


_lib = None


def lib():
    """Load libhf.so (raises if it is missing: there is no CPU fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"libhf.so not built ({LIB_PATH}); run __graft_entry__.build()")
    L = C.CDLL(LIB_PATH)
    vp, i64, i32, dbl = C.c_void_p, C.c_int64, C.c_int, C.c_double
    L.hf_default_opts.argtypes = [C.POINTER(hf_opts)]
    L.hf_error_string.argtypes = [i32]
    L.hf_error_string.restype = C.c_char_p
    L.hf_analyze.argtypes = [i64, vp, vp, vp, i32, C.POINTER(hf_opts), C.POINTER(vp)]
    L.hf_factorize.argtypes = [vp, vp, dbl]
    L.hf_set_row_signs.argtypes = [vp, vp]
    L.hf_set_spin_limit.argtypes = [vp, i32]
    L.hf_schur.argtypes = [vp]
    L.hf_solve.argtypes = [vp, i32, vp, i64, vp, i64]
    L.hf_get_split.argtypes = [vp, vp, vp, C.POINTER(hf_info)]
    L.hf_get_info.argtypes = [vp, C.POINTER(hf_info)]
    L.hf_get_tree.argtypes = [vp, vp, vp, vp]
    L.hf_get_pivots.argtypes = [vp, vp, vp, vp, vp]
    L.hf_get_factor.argtypes = [vp, vp, vp, vp, vp]
    L.hf_get_pivot_events.argtypes = [vp, vp, vp, vp]
    L.hf_precond.argtypes = [vp, i32, vp, vp]
    L.hf_profile.argtypes = [vp, i32]
    L.hf_values_adjoint.argtypes = [vp, i32, vp, i64, vp, i64, vp]
    L.hf_precond_noalloc.argtypes = [vp, i32, vp, vp]
    L.hf_get_profile.argtypes = [vp, vp, vp, vp, vp]
    L.hf_profile_name.argtypes = [i32]
    L.hf_profile_name.restype = C.c_char_p
    L.hf_get_x12.argtypes = [vp, vp, i64]
    L.hf_get_s22.argtypes = [vp, vp]
    L.hf_get_s22_factor.argtypes = [vp, vp, vp, vp, vp, vp]
    L.hf_free.argtypes = [vp]
    L.hf_free.restype = None
    L.hf_get_kernel_basis.argtypes = [vp, vp, i64]
    L.hf_gram_fp64.argtypes = [vp, i64, i32, i32, vp, vp, vp, dbl]
    L.hf_k11_iterate.argtypes = [vp, i32, i32, vp, vp, i32, vp, vp]
    L.hf_update_fp64.argtypes = [vp, i64, i32, vp, vp, vp, vp, dbl]
    pp = C.POINTER(C.c_void_p)
    L.hf_factorize_batched.argtypes = [pp, i32, pp, dbl, vp]
    L.hf_schur_batched.argtypes = [pp, i32, vp]
    L.hf_solve_batched.argtypes = [pp, i32, i32, pp, vp, pp, vp, vp]
    for name in EXPORTED:
        if name not in ("hf_error_string", "hf_free", "hf_profile_name"):
            getattr(L, name).restype = i32
    _lib = L
    return L


def _check(rc, where, allow=()):
    if rc != HF_OK and rc not in allow:
        raise HFError(rc, where)
    return rc


def _ptr(a):
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return C.c_void_p(a.data_ptr())
    return a.ctypes.data_as(C.c_void_p)


def _dev(t, name, numel, rows=None, cols=None):
    """Pointer of a device operand after checking what the C ABI cannot: a contiguous
    float64 CUDA tensor with at least `numel` entries (and `rows` rows / `cols` columns
    when it is 2-D).  The library reads and writes exactly that many entries."""
    if not hasattr(t, "data_ptr") or not getattr(t, "is_cuda", False):
        raise TypeError(f"{name}: expected a CUDA tensor, got {type(t).__name__}")
    if str(t.dtype) != "torch.float64":
        raise TypeError(f"{name}: expected float64, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name}: expected a contiguous tensor")
    if t.numel() < numel:
        raise ValueError(f"{name}: holds {t.numel()} entries, the call needs {numel}")
    if t.dim() == 2 and ((rows is not None and t.shape[0] != rows) or (cols is not None and t.shape[1] != cols)):
        raise ValueError(f"{name}: shape {tuple(t.shape)} does not match ({rows}, {cols})")
    return C.c_void_p(t.data_ptr())


def default_opts(**kw) -> hf_opts:
    o = hf_opts()
    _check(lib().hf_default_opts(C.byref(o)), "hf_default_opts")
    for k, v in kw.items():
        if k == "cuda_stream":
            v = C.c_void_p(v)
        setattr(o, k, v)
    return o


class HybridFactor:
    """One context of the C ABI: hf_analyze / hf_factorize / hf_schur / hf_solve / hf_free."""

    def __init__(self, L, rowptr, col, coords=None, **opts):
        self.L = int(L)
        self._rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
        self._col = np.ascontiguousarray(col, dtype=np.int32)
        crd = None if coords is None else np.ascontiguousarray(coords, dtype=np.float64)
        dim = 0 if crd is None else crd.shape[1]
        self.opts = default_opts(**opts)
        h = C.c_void_p()
        _check(lib().hf_analyze(self.L, _ptr(self._rowptr), _ptr(self._col), _ptr(crd), dim,
                                C.byref(self.opts), C.byref(h)), "hf_analyze")
        self._h = h
        self.generation = 0      # bumped by every factorize(): which factor the context holds

    # -- lifecycle ---------------------------------------------------------
    def free(self):
        if getattr(self, "_h", None) and self._h.value:
            lib().hf_free(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    # -- the four calls ----------------------------------------------------
    def factorize(self, vals_dev, tau=None):
        """vals_dev: torch float64 CUDA tensor with the CSR values of K-bar."""
        t = self.opts.tau if tau is None else tau
        v = _dev(vals_dev, "vals", self._col.shape[0])
        self.generation += 1
        _check(lib().hf_factorize(self._h, v, float(t)), "hf_factorize")

    def set_spin_limit(self, limit):
        """Polls of a bounded wait of the triangular sweeps before HF_ERR_TIMEOUT (0 = built in)."""
        _check(lib().hf_set_spin_limit(self._h, int(limit)), "hf_set_spin_limit")
        self.opts.spin_limit = int(limit)

    def set_row_signs(self, sign):
        """sign: host array of L entries in {+1, -1} (Kbar = diag(sign) S, S symmetric), or None."""
        if sign is None:
            self._rsign = None
            _check(lib().hf_set_row_signs(self._h, None), "hf_set_row_signs")
            return
        self._rsign = np.ascontiguousarray(sign, dtype=np.int8)
        if self._rsign.shape != (self.L,):
            raise ValueError(f"row signs: expected {self.L} entries, got shape {self._rsign.shape}")
        _check(lib().hf_set_row_signs(self._h, _ptr(self._rsign)), "hf_set_row_signs")

    @property
    def has_row_signs(self):
        return getattr(self, "_rsign", None) is not None

    def schur(self):
        return _check(lib().hf_schur(self._h), "hf_schur", allow=(HF_ERR_NOT_CONVERGED,))

    def solve(self, b_dev, x_dev):
        """b_dev, x_dev: torch float64 CUDA tensors, column-major L x nrhs (shape (nrhs, L) contiguous)."""
        nrhs = 1 if b_dev.dim() == 1 else b_dev.shape[0]
        b = _dev(b_dev, "b", self.L * nrhs, cols=self.L)
        x = _dev(x_dev, "x", self.L * nrhs, cols=self.L)
        if b.value == x.value:
            raise ValueError("x may not alias b")
        return _check(lib().hf_solve(self._h, nrhs, b, self.L, x, self.L),
                      "hf_solve", allow=(HF_ERR_NOT_CONVERGED,))

    def kernel_basis(self, torch):
        """Kernel basis of K-bar as a (kernel_dim, L) CUDA float64 tensor (rows = basis vectors)."""
        kd = self.info()["kernel_dim"]
        out = torch.zeros((max(kd, 0), self.L), dtype=torch.float64, device="cuda")
        if kd:
            _check(lib().hf_get_kernel_basis(self._h, _ptr(out), self.L), "hf_get_kernel_basis")
        return out

    def precond(self, R_dev, W_dev):
        """W = Q^-1 R (Sec. 3.2) on row-major L x m torch float64 CUDA tensors (scaled unknowns)."""
        m = 1 if R_dev.dim() == 1 else R_dev.shape[1]
        R, W = _dev(R_dev, "R", self.L * m, rows=self.L), _dev(W_dev, "W", self.L * m, rows=self.L)
        _check(lib().hf_precond(self._h, m, R, W), "hf_precond")

    def profile(self, enable=True):
        _check(lib().hf_profile(self._h, 1 if enable else 0), "hf_profile")

    def get_profile(self):
        """{class: (device ms, launches, algorithmic flops, algorithmic bytes)} since the last call."""
        ms = np.zeros(HF_NPROF)
        ln = np.zeros(HF_NPROF, np.int64)
        fl = np.zeros(HF_NPROF)
        by = np.zeros(HF_NPROF)
        _check(lib().hf_get_profile(self._h, _ptr(ms), _ptr(ln), _ptr(fl), _ptr(by)), "hf_get_profile")
        return {lib().hf_profile_name(i).decode(): (float(ms[i]), int(ln[i]), float(fl[i]), float(by[i]))
                for i in range(HF_NPROF)}

    def precond_noalloc(self, R_dev, W_dev):
        """Same as precond(), with all scratch in the library's fixed device array (no allocation)."""
        m = 1 if R_dev.dim() == 1 else R_dev.shape[1]
        R, W = _dev(R_dev, "R", self.L * m, rows=self.L), _dev(W_dev, "W", self.L * m, rows=self.L)
        _check(lib().hf_precond_noalloc(self._h, m, R, W), "hf_precond_noalloc")

    def k11_iterate(self, method, B_dev, X_dev, maxit=40):
        """K11 X = B by block GCR (method 0, Alg. 5), GCR per column (1, Alg. 4) or
        iterative refinement (2, Alg. 3); returns (rc, iterations, residual history)."""
        m = 1 if B_dev.dim() == 1 else B_dev.shape[1]
        B, X = _dev(B_dev, "B", self.L * m, rows=self.L), _dev(X_dev, "X", self.L * m, rows=self.L)
        hist = np.zeros(max(int(maxit), 0) + 1)
        it = C.c_int(0)
        rc = lib().hf_k11_iterate(self._h, int(method), m, B, X, int(maxit), _ptr(hist), C.byref(it))
        _check(rc, "hf_k11_iterate", allow=(HF_ERR_NOT_CONVERGED,))
        return rc, it.value, hist[:it.value + 1].copy()

    def gram_fp64(self, A_dev, B_dev, G_dev, scale=1.0):
        """G = scale * A^T B (Alg. 5's Gram products) on row-major L x ma / L x mb float64 CUDA tensors."""
        L, ma = A_dev.shape
        mb = B_dev.shape[1]
        A, B = _dev(A_dev, "A", L * ma, rows=L), _dev(B_dev, "B", L * mb, rows=L)
        G = _dev(G_dev, "G", ma * mb)
        _check(lib().hf_gram_fp64(self._h, L, ma, mb, A, B, G, float(scale)), "hf_gram_fp64")

    def update_fp64(self, A_dev, C_dev, Y_dev, Yinit_dev=None, sgn=1.0):
        """Y = (Yinit or Y) + sgn * A C (Alg. 5's block updates), row-major float64 CUDA tensors."""
        L, m = A_dev.shape
        A, Cm = _dev(A_dev, "A", L * m, rows=L), _dev(C_dev, "C", m * m)
        Y = _dev(Y_dev, "Y", L * m, rows=L)
        yi = _dev(Yinit_dev, "Yinit", L * m, rows=L) if Yinit_dev is not None else None
        _check(lib().hf_update_fp64(self._h, L, m, A, Cm, Y, yi, float(sgn)), "hf_update_fp64")

    def values_adjoint(self, x_dev, lam_dev, grad_dev):
        """grad[e] = -sum_r lam[row_e, r] x[col_e, r] (tensors (nrhs, L) contiguous = column-major L x nrhs)."""
        nrhs = 1 if x_dev.dim() == 1 else x_dev.shape[0]
        x = _dev(x_dev, "x", self.L * nrhs, cols=self.L)
        lam = _dev(lam_dev, "lam", self.L * nrhs, cols=self.L)
        g = _dev(grad_dev, "grad", self._col.shape[0])
        _check(lib().hf_values_adjoint(self._h, nrhs, x, self.L, lam, self.L, g), "hf_values_adjoint")

    # -- getters -----------------------------------------------------------
    def info(self) -> dict:
        inf = hf_info()
        _check(lib().hf_get_info(self._h, C.byref(inf)), "hf_get_info")
        return inf.as_dict()

    def split(self):
        inf = self.info()
        order = np.zeros(self.L, np.int32)
        lam2 = np.zeros(max(inf["M"], 1), np.int32)
        _check(lib().hf_get_split(self._h, _ptr(order), _ptr(lam2), None), "hf_get_split")
        return order, lam2[:inf["M"]]

    def tree(self):
        nn = self.info()["n_nodes"]
        parent = np.zeros(nn, np.int32)
        ptr = np.zeros(nn + 1, np.int64)
        idx = np.zeros(self.L, np.int32)
        _check(lib().hf_get_tree(self._h, _ptr(parent), _ptr(ptr), _ptr(idx)), "hf_get_tree")
        return parent, [idx[ptr[t]:ptr[t + 1]].astype(np.int64) for t in range(nn)]

    def pivots(self):
        nn = self.info()["n_nodes"]
        ptr = np.zeros(nn + 2, np.int64)
        piv = np.zeros(self.L, np.int32)
        moved = np.zeros(max(64, int(self.opts.n_enlarge)), np.int32)
        nm = C.c_int32()
        _check(lib().hf_get_pivots(self._h, _ptr(ptr), _ptr(piv), _ptr(moved), C.byref(nm)), "hf_get_pivots")
        per = [piv[ptr[t]:ptr[t + 1]].astype(np.int64) for t in range(nn + 1)]
        return per[:nn], per[nn], moved[:nm.value].astype(np.int64)

    def pivot_events(self):
        """Per front (tree nodes, then the Lambda_0 stage): (eliminated, stopped, skipped) index arrays."""
        nn = self.info()["n_nodes"]
        ptr = np.zeros(nn + 2, np.int64)
        _check(lib().hf_get_pivot_events(self._h, _ptr(ptr), None, None), "hf_get_pivot_events")
        cand = np.zeros(max(int(ptr[-1]), 1), np.int32)
        cnt = np.zeros(2 * (nn + 1), np.int32)
        _check(lib().hf_get_pivot_events(self._h, _ptr(ptr), _ptr(cand), _ptr(cnt)), "hf_get_pivot_events")
        out = []
        for t in range(nn + 1):
            c = cand[ptr[t]:ptr[t + 1]].astype(np.int64)
            k, na = int(cnt[2 * t]), int(cnt[2 * t + 1])
            out.append((c[:k], c[k:na], c[na:][::-1]))
        return out

    def factor(self):
        per, sr, _ = self.pivots()
        npiv = int(sum(len(p) for p in per)) + len(sr)
        cp = np.zeros(npiv + 1, np.int64)
        _check(lib().hf_get_factor(self._h, _ptr(cp), None, None, None), "hf_get_factor")
        ri = np.zeros(max(cp[-1], 1), np.int32)
        va = np.zeros(max(cp[-1], 1), np.float64)
        d = np.zeros(max(npiv, 1), np.float64)
        _check(lib().hf_get_factor(self._h, _ptr(cp), _ptr(ri), _ptr(va), _ptr(d)), "hf_get_factor")
        return cp, ri, va, d[:npiv]

    def x12(self, torch_mod):
        M = self.info()["M"]
        out = torch_mod.zeros((self.L, max(M, 1)), dtype=torch_mod.float64, device="cuda")
        _check(lib().hf_get_x12(self._h, _ptr(out), max(M, 1)), "hf_get_x12")
        return out[:, :M]

    def s22(self, torch_mod):
        M = self.info()["M"]
        out = torch_mod.zeros((max(M, 1), max(M, 1)), dtype=torch_mod.float64, device="cuda")
        if M:
            _check(lib().hf_get_s22(self._h, _ptr(out)), "hf_get_s22")
        return out[:M, :M]

    def s22_factor(self):
        M = self.info()["M"]
        perm = np.zeros(max(M, 1), np.int32)
        lf = np.zeros((max(M, 1), max(M, 1)))
        blk = np.zeros(max(M, 1), np.int32)
        dval = np.zeros((max(M, 1), 2))
        nul = np.zeros(max(M, 1), np.int32)
        _check(lib().hf_get_s22_factor(self._h, _ptr(perm), _ptr(lf), _ptr(blk), _ptr(dval), _ptr(nul)),
               "hf_get_s22_factor")
        return perm[:M], lf[:M, :M], blk[:M], dval[:M], nul[:M]


# -- batched form ---------------------------------------------------------
def _ptrs(items):
    return (C.c_void_p * len(items))(*[int(x) for x in items])


def _batched_check(rc, st, where, allow=()):
    bad = [(i, int(v)) for i, v in enumerate(st) if v != HF_OK and v not in allow]
    if bad:
        i, v = bad[0]
        raise HFError(v, f"{where} (system {i})")
    if rc != HF_OK and rc not in allow:
        raise HFError(rc, where)            # rejected before any system ran
    return [int(v) for v in st]


def factorize_batched(factors, vals_list, tau=1e-2):
    """hf_factorize on every (HybridFactor, CUDA values) pair, run concurrently."""
    n = len(factors)
    if len(vals_list) != n:
        raise ValueError("one values tensor per system")
    vp = [_dev(v, f"vals[{i}]", f._col.shape[0]).value for i, (f, v) in enumerate(zip(factors, vals_list))]
    st = np.zeros(n, np.int32)
    rc = lib().hf_factorize_batched(_ptrs([f._h.value for f in factors]), n, _ptrs(vp), float(tau), _ptr(st))
    return _batched_check(rc, st, "hf_factorize_batched")


def schur_batched(factors):
    n = len(factors)
    st = np.zeros(n, np.int32)
    rc = lib().hf_schur_batched(_ptrs([f._h.value for f in factors]), n, _ptr(st))
    return _batched_check(rc, st, "hf_schur_batched", allow=(HF_ERR_NOT_CONVERGED,))


def solve_batched(factors, bs, xs):
    """bs[i], xs[i]: CUDA float64 tensors of shape (nrhs, L_i), the same nrhs for all."""
    n = len(factors)
    if len(bs) != n or len(xs) != n:
        raise ValueError("one right-hand side and one solution tensor per system")
    nrhs = 1 if bs[0].dim() == 1 else bs[0].shape[0]
    bp = [_dev(b, f"bs[{i}]", f.L * nrhs, cols=f.L).value for i, (f, b) in enumerate(zip(factors, bs))]
    xp = [_dev(x, f"xs[{i}]", f.L * nrhs, cols=f.L).value for i, (f, x) in enumerate(zip(factors, xs))]
    st = np.zeros(n, np.int32)
    rc = lib().hf_solve_batched(_ptrs([f._h.value for f in factors]), n, nrhs, _ptrs(bp), None, _ptrs(xp), None,
                                _ptr(st))
    return _batched_check(rc, st, "hf_solve_batched", allow=(HF_ERR_NOT_CONVERGED,))
