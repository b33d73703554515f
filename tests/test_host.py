"""CPU-only checks of the library: it loads, exports every declared symbol, and
its host analysis (nested dissection, Sec. 2.2) is correct.  No GPU call."""
import os
import re

import numpy as np
import pytest

import oracle as O
from workloads import diffusion2d, stokes3d, elasticity3d

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _hf():
    import paper_2208_01907_gb300 as hf
    if not os.path.exists(hf.LIB_PATH):
        from paper_2208_01907_gb300.build import build
        build()
    return hf


def test_library_exports_every_declared_symbol():
    hf = _hf()
    L = hf.lib()
    header = open(os.path.join(ROOT, "include", "hf.h")).read()
    declared = set(re.findall(r"^\s*(?:int|void|const char\*)\s+(hf_\w+)\s*\(", header, re.M))
    assert declared == set(hf.EXPORTED)
    for name in declared:
        assert hasattr(L, name), name


def test_default_opts_and_error_strings():
    hf = _hf()
    o = hf.default_opts()
    assert o.tau == 1e-2 and o.n_enlarge == 4 and o.precision == hf.HF_PREC_MIXED
    assert o.null_test == 0 and o.spin_limit == 0         # the ratio test of Sec. 2.2 alone
    assert hf.lib().hf_error_string(5) == b"block GCR did not converge"
    # every code of the header's enum has its own message, mirrored by the binding
    header = open(os.path.join(ROOT, "include", "hf.h")).read()
    codes = {n: int(v) for n, v in re.findall(r"(HF_(?:OK|ERR_\w+)) = (\d+)", header)}
    assert sorted(codes.values()) == list(range(len(codes)))
    msgs = [hf.lib().hf_error_string(v) for v in codes.values()]
    assert len(set(msgs)) == len(codes) and b"unknown error" not in msgs
    for n, v in codes.items():
        assert getattr(hf.hf, n) == v, n


def test_binding_mirrors_the_header_structs_and_profile_classes():
    # the ctypes structs and the profile class count follow include/hf.h field by field
    import ctypes
    hf = _hf()
    header = open(os.path.join(ROOT, "include", "hf.h")).read()

    def fields(struct):
        body = re.search(r"typedef struct \{([^{}]*)\}\s*" + struct + ";", header).group(1)
        body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
        return [m.group(2) for m in re.finditer(r"(\w+\*?)\s+(\w+)\s*;", body)]

    assert fields("hf_opts") == [f for f, _ in hf.hf.hf_opts._fields_]
    assert fields("hf_info") == [f for f, _ in hf.hf.hf_info._fields_]
    enum = re.search(r"HF_PROF_SCALE = 0,(.*?)HF_NPROF", header, re.S).group(1)
    enum = re.sub(r"/\*.*?\*/", "", enum, flags=re.S)
    assert hf.hf.HF_NPROF == 1 + len(re.findall(r"HF_PROF_\w+", enum))
    names = [hf.lib().hf_profile_name(i).decode() for i in range(hf.hf.HF_NPROF)]
    assert len(set(names)) == hf.hf.HF_NPROF and "unknown" not in names
    assert hf.lib().hf_profile_name(hf.hf.HF_NPROF) == b"unknown"


def test_host_analysis_reproduces_fig1():
    hf = _hf()
    s = diffusion2d(7, 7, n_islands=0)
    H = hf.HybridFactor(s.L, s.rowptr, s.col, s.coords, nd_levels=3)
    parent, sets = H.tree()
    heap = [4, 5, 6, 7, 2, 3, 1]                 # elimination order of Fig. 1
    assert parent.tolist() == [4, 4, 5, 5, 6, 6, -1]
    pairs = {p for p in O.tree_block_pattern(s.to_scipy(), {heap[t]: sets[t] for t in range(7)}) if p[0] > p[1]}
    golden = set()
    for line in open(os.path.join(ROOT, "tests", "golden", "fig1_blocks.txt")):
        if line.strip() and not line.startswith("#"):
            golden.add(tuple(map(int, line.split())))
    assert pairs == golden


@pytest.mark.parametrize("maker,coords", [(lambda: diffusion2d(33, 21, n_islands=0), True),
                                          (lambda: stokes3d(6), True),
                                          (lambda: elasticity3d(6, n_incl=1, incl=2), True),
                                          (lambda: diffusion2d(25, 25, n_islands=0), False)])
def test_host_analysis_separators(maker, coords):
    hf = _hf()
    s = maker()
    H = hf.HybridFactor(s.L, s.rowptr, s.col, s.coords if coords else None, nd_leaf=40)
    parent, sets = H.tree()
    nn = len(sets)
    owner = np.full(s.L, -1)
    for t, v in enumerate(sets):
        owner[v] = t
    assert (owner >= 0).all()
    children = {t: [] for t in range(nn)}
    for t, p in enumerate(parent):
        if p >= 0:
            children[p].append(t)

    def subtree(t):
        out = {t}
        for c in children[t]:
            out |= subtree(c)
        return out
    A = s.to_scipy().tocoo()
    for t in range(nn):
        if len(children[t]) == 2:
            a, b = subtree(children[t][0]), subtree(children[t][1])
            cross = np.isin(owner[A.row], list(a)) & np.isin(owner[A.col], list(b))
            assert not cross.any()


def test_pattern_validation():
    hf = _hf()
    s = diffusion2d(4, 4, n_islands=0)
    col = s.col.copy()
    col[[1, 2]] = col[[2, 1]]                    # unsorted row
    with pytest.raises(hf.HFError) as e:
        hf.HybridFactor(s.L, s.rowptr, col, s.coords)
    assert e.value.code == 3
    # drop one off-diagonal entry: pattern no longer symmetric
    import scipy.sparse as sp
    A = s.to_scipy().tolil()
    A[0, 1] = 0
    A = A.tocsr()
    A.eliminate_zeros()
    with pytest.raises(hf.HFError) as e:
        hf.HybridFactor(s.L, A.indptr.astype(np.int64), A.indices.astype(np.int32), s.coords)
    assert e.value.code == 3
    with pytest.raises(hf.HFError) as e:
        hf.HybridFactor(s.L, s.rowptr, s.col, s.coords, tau=-1.0)
    assert e.value.code == 1


def test_binding_fails_loudly_without_the_library(monkeypatch, tmp_path):
    # no CPU fallback: with libhf.so absent the first call into the library raises
    import paper_2208_01907_gb300.hf as binding
    s = diffusion2d(6, 6, n_islands=0)
    A = s.to_scipy()
    monkeypatch.setattr(binding, "_lib", None)
    monkeypatch.setattr(binding, "LIB_PATH", str(tmp_path / "libhf.so"))
    with pytest.raises(RuntimeError, match="not built"):
        binding.lib()
    with pytest.raises(RuntimeError, match="not built"):
        binding.HybridFactor(A.shape[0], A.indptr, A.indices, s.coords)


def test_product_path_never_reaches_the_oracle():
    # the package neither imports the oracle nor names it in code; importing it leaves
    # the oracle unloaded (checked in a fresh interpreter)
    import subprocess
    import sys
    pkg = os.path.join(ROOT, "paper_2208_01907_gb300")
    for dirpath, _, files in os.walk(pkg):
        for name in files:
            if name.endswith((".py", ".cu", ".cuh", ".cpp", ".h")):
                text = open(os.path.join(dirpath, name)).read()
                assert not re.search(r"^\s*(from|import)\s+oracle\b", text, re.M), name
                assert "oracle/" not in text and "import_module(\"oracle" not in text, name
    code = ("import sys, paper_2208_01907_gb300, paper_2208_01907_gb300.shard; "
            "assert not any(m == 'oracle' or m.startswith('oracle.') for m in sys.modules)")
    subprocess.run([sys.executable, "-c", code], cwd=ROOT, check=True)


def test_bench_kernel_work_rates():
    # per-class rates of the bench line: GFLOP and GB per step, TFLOP/s and GB/s over the class's time
    import sys
    sys.path.insert(0, ROOT)
    import bench
    prof = {"trsv_fwd": (180.0, 477, 1.8e12, 15.0e9), "scale": (0.2, 3, 0.0, 0.0), "gram": (0.0, 9, 1e9, 2e9)}
    w = bench.kernel_work(prof, 3)
    assert set(w) == {"trsv_fwd", "gram"}
    assert w["trsv_fwd"] == {"gflop": 600.0, "gbytes": 5.0, "tflop_s": 10.0, "gb_s": 83.3}
    assert w["gram"]["tflop_s"] is None and w["gram"]["gb_s"] is None


def test_analysis_edge_cases():
    # empty and malformed inputs are refused on the host; the smallest systems analyse
    import ctypes as C
    hf = _hf()
    L = hf.lib()
    o = hf.default_opts()
    h = C.c_void_p()
    rp = np.array([0], dtype=np.int64)
    cl = np.zeros(1, dtype=np.int32)
    assert L.hf_analyze(0, rp.ctypes.data, cl.ctypes.data, None, 0, C.byref(o), C.byref(h)) == 1   # L = 0
    s = diffusion2d(4, 4, n_islands=0)
    with pytest.raises(hf.HFError) as e:                       # coordinates of dimension 4
        hf.HybridFactor(s.L, s.rowptr, s.col, np.zeros((s.L, 4)))
    assert e.value.code == 1
    col = s.col.copy()
    col[-1] = s.L                                              # column out of range
    with pytest.raises(hf.HFError) as e:
        hf.HybridFactor(s.L, s.rowptr, col, s.coords)
    assert e.value.code == 3
    rp = s.rowptr.copy()
    rp[0] = 1                                                  # row pointers not starting at 0
    with pytest.raises(hf.HFError) as e:
        hf.HybridFactor(s.L, rp, s.col, s.coords)
    assert e.value.code == 3
    import scipy.sparse as sp
    A = s.to_scipy().tolil()
    A.setdiag(0)
    A = A.tocsr()
    A.eliminate_zeros()                                        # rows without a stored diagonal
    with pytest.raises(hf.HFError) as e:
        hf.HybridFactor(s.L, A.indptr.astype(np.int64), A.indices.astype(np.int32), s.coords)
    assert e.value.code == 3
    # one unknown, and two disconnected unknowns without coordinates: one tree each way
    for n, rp, cl in ((1, [0, 1], [0]), (2, [0, 1, 2], [0, 1])):
        H = hf.HybridFactor(n, np.array(rp), np.array(cl))
        parent, sets = H.tree()
        assert sorted(np.concatenate(sets).tolist()) == list(range(n))
        assert sum(1 for p in parent if p < 0) == 1
        H.free()


class _FakeCuda:
    """Stands in for a CUDA tensor in argument checks that must fail before any library call."""

    def __init__(self, shape, dtype="torch.float64", contiguous=True, ptr=1 << 20):
        self.shape, self.dtype, self._c, self._p, self.is_cuda = tuple(shape), dtype, contiguous, ptr, True

    def data_ptr(self):
        return self._p

    def dim(self):
        return len(self.shape)

    def numel(self):
        return int(np.prod(self.shape))

    def is_contiguous(self):
        return self._c


def test_binding_checks_device_operands():
    # the C ABI cannot see a device buffer's size or type: the binding refuses what would make
    # the library read or write past a tensor, before calling it
    import torch
    hf = _hf()
    s = diffusion2d(6, 6, n_islands=0)
    H = hf.HybridFactor(s.L, s.rowptr, s.col, s.coords)
    nnz = s.col.shape[0]
    with pytest.raises(TypeError, match="CUDA"):
        H.factorize(torch.zeros(nnz, dtype=torch.float64))             # host tensor
    with pytest.raises(TypeError, match="float64"):
        H.factorize(_FakeCuda((nnz,), dtype="torch.float32"))
    with pytest.raises(ValueError, match="contiguous"):
        H.factorize(_FakeCuda((nnz,), contiguous=False))
    with pytest.raises(ValueError, match="entries"):
        H.factorize(_FakeCuda((nnz - 1,)))
    b = _FakeCuda((2, s.L))
    with pytest.raises(ValueError, match="shape"):
        H.solve(_FakeCuda((2, s.L + 1)), b)
    with pytest.raises(ValueError, match="alias"):
        H.solve(b, b)
    with pytest.raises(ValueError, match="entries|shape"):
        H.precond(_FakeCuda((3, s.L)), _FakeCuda((3, s.L)))            # transposed layout
    with pytest.raises(ValueError, match="shape"):
        H.k11_iterate(0, _FakeCuda((s.L + 1, 2)), _FakeCuda((s.L + 1, 2)))
    with pytest.raises(ValueError, match="entries"):
        H.gram_fp64(_FakeCuda((s.L, 4)), _FakeCuda((s.L, 5)), _FakeCuda((19,)))
    with pytest.raises(ValueError, match="entries"):
        H.values_adjoint(_FakeCuda((s.L,)), _FakeCuda((s.L,)), _FakeCuda((nnz - 1,)))
    with pytest.raises(ValueError, match="row signs"):
        H.set_row_signs(np.ones(s.L - 1, dtype=np.int8))
    with pytest.raises(ValueError, match="per system"):
        hf.factorize_batched([H, H], [_FakeCuda((nnz,))])
    H.free()


@pytest.mark.parametrize("maker", [lambda: stokes3d(32, seed=2),                         # the benchmark workload
                                   lambda: elasticity3d(40, seed=3)],                     # elasticity 40^3
                         ids=["stokes32", "elasticity40"])
def test_host_analysis_full_size(maker):
    # Sec. 2.2 at the full sizes: the sets partition the unknowns and every coupling of K
    # joins a node to itself or to one of its ancestors (each set separates its subtrees)
    hf = _hf()
    s = maker()
    H = hf.HybridFactor(s.L, s.rowptr, s.col, s.coords)
    parent, sets = H.tree()
    info = H.info()
    nn = len(sets)
    assert nn == info["n_nodes"] == 2 ** info["levels"] - 1
    owner = np.full(s.L, -1)
    for t, v in enumerate(sets):
        assert (owner[v] == -1).all()
        owner[v] = t
    assert (owner >= 0).all()
    children = [[] for _ in range(nn)]
    roots = [t for t in range(nn) if parent[t] < 0]
    for t, p in enumerate(parent):
        if p >= 0:
            children[p].append(t)
    assert len(roots) == 1
    tin, tout, clock, stack = np.zeros(nn, np.int64), np.zeros(nn, np.int64), 0, [(roots[0], 0)]
    while stack:                                               # Euler tour of the tree
        t, state = stack.pop()
        if state == 0:
            tin[t] = clock
            clock += 1
            stack.append((t, 1))
            stack.extend((c, 0) for c in children[t])
        else:
            tout[t] = clock
    rows = np.repeat(np.arange(s.L), np.diff(s.rowptr))
    a, b = owner[rows], owner[s.col]
    anc = ((tin[a] <= tin[b]) & (tin[b] < tout[a])) | ((tin[b] <= tin[a]) & (tin[a] < tout[b]))
    assert anc.all()
    leaves = [t for t in range(nn) if not children[t]]
    assert max(len(sets[t]) for t in leaves) <= 2 * H.opts.nd_leaf
    H.free()


def test_device_entries_fail_cleanly_without_a_gpu():
    # on a machine without a GPU the host-only analysis works and every call that needs the
    # device returns an error code (no crash, no CPU fallback)
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    hf = _hf()
    s = diffusion2d(6, 6, n_islands=0)
    H = hf.HybridFactor(s.L, s.rowptr, s.col, s.coords)
    with pytest.raises(hf.HFError) as e:
        H.set_row_signs(np.ones(s.L, dtype=np.int8))
    assert e.value.code in (7, 8)                               # HF_ERR_CUDA / HF_ERR_OOM
    for call in (H.schur, H.split, H.pivots):
        with pytest.raises(hf.HFError) as e:
            call()
        assert e.value.code == 2                                # HF_ERR_STATE: nothing factorized
    assert H.info()["L"] == s.L
    H.free()


def test_bench_fit_and_rooflines():
    # the oracle's growth exponent is the least-squares slope in log-log; the per-kernel
    # roofline divides the counted work of exactly the profiled launches by their time
    import sys
    sys.path.insert(0, ROOT)
    import bench
    pts = [(1000, 2.0), (2000, 2.0 * 2 ** 1.7), (4000, 2.0 * 4 ** 1.7)]
    assert abs(bench.fit_exponent(pts) - 1.7) < 1e-12
    assert abs(bench.extrapolate(2.0, 1000, 8000, 1.7) - 2.0 * 8 ** 1.7) < 1e-9
    prof = {"trsv_fwd": (20.0, 40, 1e9, 34e9), "gram": (4.0, 2, 1e11, 1e9), "block_update": (6.0, 3, 2e11, 1e9),
            "panel": (30.0, 60, 3e9, 1e9)}
    r = bench.kernel_rooflines(prof, 2, trailing_tc=False)
    assert r["k_sweep_df<1>"]["bound"] == "hbm"
    assert abs(r["k_sweep_df<1>"]["achieved"] - 34e9 / 0.02 / 1e9) < 1e-6
    oz = r["k_oz_mma"]
    assert oz["ms_per_step"] == 5.0 and oz["launches_per_step"] == 2.5
    assert abs(oz["achieved"] - 36 * 3e11 / 0.01 / 1e12) < 1e-6
    assert r["k_panel_cl"]["bound"] == "alu" and r["k_panel_cl"]["ms_per_step"] == 15.0
