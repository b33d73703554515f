"""Parity on the code paths that only the full-size workloads reach, at sizes the dense
oracle still replays.

The full-size fronts take panels spread over thread-block clusters of up to 16 CTAs,
the global-memory panel for fronts a cluster cannot hold, triangular sweeps with long
chains of 64-row diagonal blocks, and the cooperative S22 LDL^T for M in the hundreds.
Each test below drives one of those paths on a system small enough for the oracle
(diagnostic knobs that change how the work is spread, never what is computed: rows per
CTA of the cluster panel, the global panel for every front, large dissection leaves, a
threshold that postpones everything), proves from hf_info that the path ran, and checks
the split bit for bit against the oracle's replay, S22 and X12 to 1e-10, the kernel
dimension and the backward error of the solve.
"""
import numpy as np
import pytest

import oracle as O
from workloads import diffusion2d, stokes3d, elasticity3d
from gpu_common import run_gpu, replay, rel_fro

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _check_against_oracle(s, out, tau, kdim):
    H, info = out["H"], out["info"]
    q, K, fac, moved = replay(s, H, tau)
    assert fac.violations == []
    order, lam2 = H.split()
    assert lam2.tolist() == fac.lambda2.tolist()
    assert order[:fac.N].tolist() == fac.lambda1_order.tolist()
    assert moved.tolist() == fac.moved.tolist()
    if fac.M and fac.N:
        S22 = H.s22(torch).cpu().numpy()
        assert rel_fro(S22, O.schur_direct(K, fac.lambda2)) <= 1e-10
        X12 = H.x12(torch).cpu().numpy()
        Xref = O.x12_direct(K, fac.lambda2)
        assert np.abs(X12 - Xref).max() <= 1e-10 * max(np.abs(Xref).max(), 1.0)
    elif fac.M:                                       # everything postponed: S22 = K
        S22 = H.s22(torch).cpu().numpy()
        assert rel_fro(S22, K.toarray()) <= 1e-14
    assert info["kernel_dim"] == kdim
    assert O.backward_error(s.to_scipy(), out["x"], out["b"]) <= 1e-12
    return fac


def test_cluster_panel_of_sixteen_ctas_and_global_panel(monkeypatch):
    # 32 rows per CTA: fronts of 257..512 rows take clusters of 9..16 CTAs, larger ones the
    # global-memory panel; the front's factorization may switch from the global to the
    # cluster panel as its trailing part shrinks
    s = stokes3d(10, seed=2)
    monkeypatch.setenv("HF_PANEL_ROWS", "32")
    out = run_gpu(s, tau=1e-2, null_test=1)
    info = out["info"]
    assert info["panel_cluster"] >= 8
    assert info["panel_global"] >= 1
    _check_against_oracle(s, out, 1e-2, 3)


def test_global_memory_panel_for_every_front(monkeypatch):
    # the two panel kernels sum in the same order: the same pivots and the same factor, bit
    # for bit, whichever holds a front
    s = elasticity3d(8, n_incl=2, incl=2, seed=3)
    monkeypatch.setenv("HF_PANEL_ROWS", "96")           # clusters of several CTAs
    ref = run_gpu(s, tau=1e-2)
    assert ref["info"]["panel_cluster"] >= 2 and ref["info"]["panel_global"] == 0
    monkeypatch.delenv("HF_PANEL_ROWS")
    monkeypatch.setenv("HF_PANEL_KERNEL", "global")
    out = run_gpu(s, tau=1e-2)
    assert out["info"]["panel_cluster"] == 0 and out["info"]["panel_global"] >= 1
    for a, b in zip(ref["H"].factor(), out["H"].factor()):
        np.testing.assert_array_equal(a, b)
    _check_against_oracle(s, out, 1e-2, 6)


def test_long_chains_of_diagonal_blocks_in_the_sweeps():
    # dissection leaves of up to 2048 unknowns: a front solves >= 16 diagonal blocks in a
    # chain in every sweep; the preconditioner is compared with the oracle's
    s = stokes3d(12, seed=2)
    out = run_gpu(s, tau=1e-2, nd_leaf=2048)
    info = out["info"]
    assert info["sweep_blocks"] >= 16
    fac = _check_against_oracle(s, out, 1e-2, 3)
    H, K = out["H"], O.scale_matrix(s.to_scipy())[1]
    _, lam2 = H.split()
    X = np.random.default_rng(2).standard_normal((s.L, 70))
    X[lam2] = 0
    A = O.k11_operator(K, lam2)
    R = torch.tensor(A(X), device="cuda")
    W = torch.zeros_like(R)
    H.precond(R, W)
    Wo = O.precond_apply(fac, A(X))
    assert np.linalg.norm(W.cpu().numpy() - Wo) <= 1e-3 * np.linalg.norm(Wo)


@pytest.mark.parametrize("n,kind", [(12, 1), (26, 2)])
def test_s22_ldlt_cluster_and_cooperative_forms(n, kind):
    # tau = 2 postpones every index, so S22 is the whole scaled K: M = 144 runs the
    # cluster-resident LDL^T, M = 676 the cooperative one over all SMs; pivots as the oracle's
    s = diffusion2d(n, n, n_islands=1, island=3, contrast=1e6, dirichlet_x=True, seed=8)
    out = run_gpu(s, tau=2.0, nd_leaf=64)
    H, info = out["H"], out["info"]
    assert info["M"] == s.L and info["ldlt_kernel"] == kind
    S22 = H.s22(torch).cpu().numpy()
    perm, lf, blk, dval, nul = H.s22_factor()
    operm, oLf, oblocks = O.bunch_parlett(S22)
    assert perm.tolist() == operm.tolist()
    np.testing.assert_allclose(lf, oLf, atol=1e-8 * max(1.0, np.abs(oLf).max()))
    assert info["kernel_dim"] == 0
    _check_against_oracle(s, out, 2.0, 0)


@pytest.mark.parametrize("n", [10, 12])
def test_elasticity_replay_at_the_largest_oracle_sizes(n):
    # the full-size workload's equations (Q1 elasticity, stiff inclusions, 6 rigid modes)
    s = elasticity3d(n, n_incl=n // 3, incl=2, seed=3)
    out = run_gpu(s, tau=1e-2)
    _check_against_oracle(s, out, 1e-2, 6)


def test_stokes_replay_at_fourteen_cubed():
    s = stokes3d(14, seed=2)
    out = run_gpu(s, tau=1e-2, null_test=1)
    _check_against_oracle(s, out, 1e-2, 3)
