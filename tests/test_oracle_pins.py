"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: closed forms,
the Fig. 1 pattern, brute-force Schur complements from dense inverses,
determinant identities, Krylov least-squares optima, SVD nullities, finite
differences.  A plausible mistake (dropped term, wrong sign or index,
transposed operand) in the oracle fails at least one of them.
"""
import math
import os

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp

import oracle as O
from workloads import diffusion2d, stokes3d, stokes3d_ldu, elasticity3d, darcy2d, consistent_rhs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rand_spd(n, rng, cond=10.0):
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    ev = np.exp(rng.uniform(0, math.log(cond), n))
    return (Q * ev) @ Q.T


def _rand_sym(n, rng):
    A = rng.standard_normal((n, n))
    return A + A.T


# --------------------------------------------------------------------------- Sec. 2 scaling
def test_scaling_closed_form():
    A = sp.csr_matrix(np.array([[4.0, 1.0, 0.0, 2.0],
                                [1.0, -9.0, 3.0, 0.0],
                                [0.0, 3.0, 0.0, 1.0],
                                [2.0, 0.0, 1.0, 0.25]]))
    q, K = O.scale_matrix(A)
    np.testing.assert_allclose(q, [0.5, 1 / 3, 1.0, 2.0])
    np.testing.assert_allclose(K.diagonal(), [1.0, -1.0, 0.0, 1.0])     # diag in {-1, 0, 1}
    np.testing.assert_allclose(K.toarray()[0, 3], 2.0 * 0.5 * 2.0)      # q_i K_ij q_j
    np.testing.assert_allclose(K.toarray()[1, 2], 3.0 / 3.0)


def test_scaling_preserves_solution():
    s = diffusion2d(8, 8, n_islands=0, dirichlet_x=True)
    Kb = s.to_scipy().toarray()
    q, K = O.scale_matrix(s.to_scipy())
    b = np.random.default_rng(0).standard_normal(s.L)
    x_direct = np.linalg.solve(Kb, b)
    x_scaled = q * np.linalg.solve(K.toarray(), q * b)                  # x-bar = Q x with K x = Q b
    np.testing.assert_allclose(x_scaled, x_direct, rtol=1e-12)


# --------------------------------------------------------------------------- Sec. 2.2 / Fig. 1
def _fig1_pairs():
    pairs = set()
    with open(os.path.join(GOLDEN, "fig1_blocks.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                i, j = map(int, line.split())
                pairs.add((i, j))
    return pairs


def test_nd_fig1_block_pattern():
    s = diffusion2d(7, 7, n_islands=0)
    sets, order = O.nested_dissection(s.to_scipy(), s.coords, 3)
    assert order == [4, 5, 6, 7, 2, 3, 1]
    got = {p for p in O.tree_block_pattern(s.to_scipy(), sets) if p[0] > p[1]}
    assert got == _fig1_pairs()
    assert sorted(np.concatenate(list(sets.values()))) == list(range(s.L))


@pytest.mark.parametrize("maker", [lambda: diffusion2d(20, 17, n_islands=0),
                                   lambda: stokes3d(5),
                                   lambda: elasticity3d(6, n_incl=1, incl=2)])
def test_nd_separators(maker):
    s = maker()
    A = s.to_scipy().tocoo()
    m = 4
    sets, _ = O.nested_dissection(s.to_scipy(), s.coords, m)
    owner = np.full(s.L, -1)
    for l, v in sets.items():
        owner[v] = l

    def subtree(l):
        out = {l}
        if 2 * l < 2 ** m:
            out |= subtree(2 * l) | subtree(2 * l + 1)
        return out

    # removing Lambda_l disconnects its two subtrees: no edge joins them
    for l in range(1, 2 ** (m - 1)):
        left, right = subtree(2 * l), subtree(2 * l + 1)
        a = np.isin(owner[A.row], list(left)) & np.isin(owner[A.col], list(right))
        assert not a.any(), f"node {l} is not a separator"


# --------------------------------------------------------------------------- Sec. 2.1-2.2 factorization
def test_hand_case_pivot_order_and_postponing():
    # K = diag(0.5, 1.0, 0.003), one index set, tau = 1e-2, n = 1:
    # pivots 1 (1.0) then 0 (ratio 0.5) ; 2 fails 0.003/0.5 < tau -> Lambda_0 = {2};
    # the Lambda_0 refactorization postpones it too (0.003 < tau * 1); enlargement moves 0.
    K = sp.csr_matrix(np.diag([0.5, 1.0, 0.003]))
    fac = O.threshold_factorize(K, [np.array([0, 1, 2])], tau=1e-2, n_enlarge=1)
    assert fac.node_pivots[0].tolist() == [1, 0]
    assert fac.node_postponed[0].tolist() == [2]
    assert fac.lam0.tolist() == [2]
    assert fac.lam0_pivots.tolist() == []
    assert fac.moved.tolist() == [0]
    assert fac.lambda2.tolist() == [0, 2]
    assert fac.lambda1_order.tolist() == [1]


def test_hand_case_tie_break_and_first_pivot_reference():
    # equal diagonals: the smaller index goes first (R5); |d_1| < tau postpones the whole set (R2)
    K = sp.csr_matrix(np.diag([1.0, 1.0, 1.0]))
    fac = O.threshold_factorize(K, [np.array([2, 0, 1])], tau=0.5, n_enlarge=0)
    assert fac.node_pivots[0].tolist() == [0, 1, 2]
    K2 = sp.csr_matrix(np.diag([0.004, 0.003]))
    fac2 = O.threshold_factorize(K2, [np.array([0, 1])], tau=1e-2, n_enlarge=0)
    assert fac2.node_pivots[0].tolist() == [] and fac2.lambda2.tolist() == [0, 1]


def test_hand_case_ratio_to_previous_pivot():
    # R3: each pivot is measured against the previous pivot of its set, not against 1 or
    # the first pivot.  diag(1, 0.05, 0.004, 3e-5), tau = 1e-2: ratios 0.05, 0.08, 0.0075,
    # so 0.004 is accepted although it is below tau * 1, and 3e-5 is postponed.
    K = sp.csr_matrix(np.diag([1.0, 0.05, 0.004, 3e-5]))
    fac = O.threshold_factorize(K, [np.array([0, 1, 2, 3])], tau=1e-2, n_enlarge=0)
    assert fac.node_pivots[0].tolist() == [0, 1, 2]
    assert fac.node_postponed[0].tolist() == [3]
    # R2 on the refactorization of Lambda_0: its first pivot is compared with 1 again
    assert fac.lam0_pivots.tolist() == [] and fac.lambda2.tolist() == [3]
    # the reference restarts at 1 in every set: the second set's 0.004 fails against 1,
    # although it is within tau of the previous set's last pivot 0.05 ...
    fac2 = O.threshold_factorize(sp.csr_matrix(np.diag([1.0, 0.05, 0.004])),
                                 [np.array([0, 1]), np.array([2])], tau=1e-2, n_enlarge=0)
    assert fac2.node_pivots[1].tolist() == [] and fac2.lambda2.tolist() == [2]
    # ... and passes against 1 when tau allows it, whatever the previous set ended with
    fac3 = O.threshold_factorize(sp.csr_matrix(np.diag([1.0, 1e-3, 0.5])),
                                 [np.array([0, 1]), np.array([2])], tau=1e-2, n_enlarge=0)
    assert fac3.node_pivots[0].tolist() == [0] and fac3.node_pivots[1].tolist() == [2]


def test_pivot_sequence_matches_brute_force_schur():
    # At every step the chosen pivot is the max |diag| of the exact Schur complement,
    # formed here from scratch with a dense inverse, and d equals that diagonal entry.
    rng = np.random.default_rng(7)
    for trial in range(6):
        n = 7
        A = _rand_sym(n, rng) * 0.3 + np.diag(rng.uniform(0.5, 3.0, n) * rng.choice([-1, 1], n))
        fac = O.threshold_factorize(sp.csr_matrix(A), [np.arange(n)], tau=1e-6, n_enlarge=0)
        elim = []
        for q in fac.node_pivots[0]:
            rest = [i for i in range(n) if i not in elim]
            if elim:
                S = A[np.ix_(rest, rest)] - A[np.ix_(rest, elim)] @ np.linalg.solve(A[np.ix_(elim, elim)], A[np.ix_(elim, rest)])
            else:
                S = A[np.ix_(rest, rest)]
            dg = np.abs(np.diag(S))
            assert rest[int(np.argmax(dg))] == q
            np.testing.assert_allclose(fac.d[int(q)], S[rest.index(q), rest.index(q)], rtol=2e-5)
            elim.append(int(q))


def test_factor_reconstructs_eq1():
    # Eq. (1): the recorded unit-L, D satisfy Pi^T K Pi = L D L^T on the eliminated indices
    s = diffusion2d(12, 12, n_islands=1, island=3, contrast=1e3, seed=3)
    q, K = O.scale_matrix(s.to_scipy())
    sets, order = O.nested_dissection(K, s.coords, 3)
    fac = O.threshold_factorize(K, [sets[l] for l in order], tau=1e-2, n_enlarge=4)
    elim = np.concatenate([*fac.node_pivots, fac.lam0_pivots]).astype(int)
    pos = {int(g): i for i, g in enumerate(elim)}
    n = len(elim)
    Lm = np.eye(n)
    D = np.zeros(n)
    for g in elim:
        j = pos[int(g)]
        D[j] = fac.d[int(g)]
        rows, vals = fac.lcol[int(g)]
        for r, v in zip(rows, vals):
            if int(r) in pos:
                Lm[pos[int(r)], j] = v
    Kd = K.toarray()[np.ix_(elim, elim)]
    err = np.abs(Lm @ np.diag(D) @ Lm.T - Kd).max() / np.abs(Kd).max()
    assert err < 1e-5                                           # float32 factorization
    assert fac.M >= 4 and len(set(fac.lambda1_order) & set(fac.lambda2)) == 0
    assert len(fac.lambda1_order) + fac.M == s.L


def test_tau_limits():
    s = diffusion2d(10, 10, n_islands=0, dirichlet_x=True)
    q, K = O.scale_matrix(s.to_scipy())
    sets, order = O.nested_dissection(K, s.coords, 3)
    nodes = [sets[l] for l in order]
    small = O.threshold_factorize(K, nodes, tau=1e-30, n_enlarge=4)
    assert len(small.lam0) == 0 and small.M == 4                 # nothing postponed, only the n moved
    big = O.threshold_factorize(K, nodes, tau=2.0, n_enlarge=4)
    assert big.M == s.L and len(big.lam0) == s.L                 # every first pivot fails |d| < 2 * 1


# --------------------------------------------------------------------------- Sec. 3 preconditioner / GCR
def _cfg1_small():
    s = diffusion2d(16, 16, n_islands=2, island=3, contrast=1e8, seed=4)
    q, K = O.scale_matrix(s.to_scipy())
    sets, order = O.nested_dissection(K, s.coords, 4)
    fac = O.threshold_factorize(K, [sets[l] for l in order], tau=1e-2, n_enlarge=4)
    return s, q, K, fac


def test_precond_approximates_inverse():
    s, q, K, fac = _cfg1_small()
    A = O.k11_operator(K, fac.lambda2)
    rng = np.random.default_rng(1)
    X = rng.standard_normal((s.L, 3))
    X[fac.lambda2] = 0
    Y = O.precond_apply(fac, A(X))
    err = np.linalg.norm(Y - X) / np.linalg.norm(X)
    assert err < 1e-3                                            # Q^-1 K11 ~ I (Sec. 3.3)


def test_block_gcr_invariants_and_solution():
    s, q, K, fac = _cfg1_small()
    A = O.k11_operator(K, fac.lambda2)
    lam1 = np.setdiff1d(np.arange(s.L), fac.lambda2)
    B = np.zeros((s.L, fac.M))
    B[lam1] = K.toarray()[np.ix_(lam1, fac.lambda2)]
    X, hist, P, Qs = O.block_gcr(A, lambda R: O.precond_apply(fac, R), B, tol=1e-15, maxit=20)
    Xd = O.x12_direct(K, fac.lambda2)
    assert np.abs(X - Xd).max() / np.abs(Xd).max() < 1e-12
    for n in range(len(P)):
        np.testing.assert_allclose(Qs[n], A(P[n]), atol=1e-10 * np.abs(Qs[n]).max())  # q_n = A p_n
    for m_ in range(len(P)):
        for n in range(m_ + 1, len(P)):
            cross = np.abs(Qs[m_].T @ Qs[n]).max()
            scale = np.linalg.norm(Qs[m_]) * np.linalg.norm(Qs[n])
            assert cross <= 1e-8 * scale                          # (A p_m, A p_n) = 0, m != n
    assert hist[-1] <= 1e-15 and len(hist) <= 8


def test_gcr_unpreconditioned_is_krylov_minimal_residual():
    # Q = I: GCR minimises |b - A x| over x in span{b, A b, ..., A^(n-1) b} (Sec. 3.4)
    rng = np.random.default_rng(3)
    n = 30
    Am = _rand_spd(n, rng, 50.0) + 0.3 * _rand_sym(n, rng)
    b = rng.standard_normal(n)
    A = lambda v: Am @ v
    for its in range(1, 6):
        x, hist, _, _ = O.gcr_single(A, lambda v: np.zeros_like(v) + v, b, tol=0.0, maxit=its)
        # GCR with x0 = Q^-1 b = b: after `its` steps x is in b + span{r0, ..., A^(its-1) r0}
        r0 = b - Am @ b
        Kry = np.stack([np.linalg.matrix_power(Am, k) @ r0 for k in range(its)], axis=1)
        c = np.linalg.lstsq(Am @ Kry, r0, rcond=None)[0]
        best = np.linalg.norm(r0 - Am @ Kry @ c) / np.linalg.norm(b)
        assert abs(hist[-1] - best) <= 1e-9 * max(best, 1e-12) + 1e-14


def test_block_gcr_single_rhs_equals_alg4():
    s, q, K, fac = _cfg1_small()
    A = O.k11_operator(K, fac.lambda2)
    Qi = lambda R: O.precond_apply(fac, R)
    lam1 = np.setdiff1d(np.arange(s.L), fac.lambda2)
    b = np.zeros(s.L)
    b[lam1] = np.random.default_rng(2).standard_normal(len(lam1))
    xb, hb, _, _ = O.block_gcr(A, Qi, b[:, None], tol=1e-15, maxit=6)
    xs, hs, _, _ = O.gcr_single(A, Qi, b, tol=1e-15, maxit=6)
    n = min(len(hb), len(hs))
    np.testing.assert_allclose(hb[:n], hs[:n], rtol=1e-6, atol=1e-16)
    np.testing.assert_allclose(xb[:, 0], xs, rtol=1e-10, atol=1e-12 * np.abs(xs).max())


def test_iterative_refinement_residuals_follow_the_closed_form():
    # Sec. 3.3: with a fixed linear Q^-1, r_n = (I - A Q^-1)^n r_0 and the iterate lies in
    # x_0 + span{Q^-1 r_0, (Q^-1 A) Q^-1 r_0, ...}; here Q^-1 is an inexact inverse (Jacobi)
    rng = np.random.default_rng(7)
    n = 25
    Am = _rand_spd(n, rng, 20.0)
    Qm = np.diag(1.0 / np.diag(Am))
    A = lambda V: Am @ V
    Qinv = lambda V: Qm @ V
    B = rng.standard_normal((n, 2))
    X, hist = O.iterative_refinement(A, Qinv, B, tol=0.0, maxit=6)
    r0 = B - Am @ (Qm @ B)
    Tm = np.eye(n) - Am @ Qm
    for k in range(7):
        rk = np.linalg.matrix_power(Tm, k) @ r0
        want = np.max(np.linalg.norm(rk, axis=0) / np.linalg.norm(B, axis=0))
        assert abs(hist[k] - want) <= 1e-12 * max(want, 1e-300) + 1e-15
    # the iterate: x_6 = x_0 + sum_{j<6} (Q^-1 (I - A Q^-1)^j) r_0
    xs = Qm @ B + sum(Qm @ np.linalg.matrix_power(Tm, j) @ r0 for j in range(6))
    np.testing.assert_allclose(X, xs, rtol=1e-12, atol=1e-14)


def test_iterative_refinement_exact_preconditioner_and_gcr_not_worse():
    # exact Q: x_0 is the solution; inexact Q: GCR's residual (minimal over the same Krylov
    # space, Sec. 3.4) is never above IR's at the same step
    s, q, K, fac = _cfg1_small()
    A = O.k11_operator(K, fac.lambda2)
    Qi = lambda R: O.precond_apply(fac, R)
    lam1 = np.setdiff1d(np.arange(s.L), fac.lambda2)
    K11 = K.toarray()[np.ix_(lam1, lam1)]

    def exact(R):
        out = np.zeros_like(R)
        out[lam1] = np.linalg.solve(K11, R[lam1])
        return out
    b = np.zeros(s.L)
    b[lam1] = np.random.default_rng(4).standard_normal(len(lam1))
    _, he = O.iterative_refinement(A, exact, b[:, None], tol=0.0, maxit=1)
    assert he[0] < 1e-10
    _, hi = O.iterative_refinement(A, Qi, b[:, None], tol=0.0, maxit=4)
    _, hg, _, _ = O.gcr_single(A, Qi, b, tol=0.0, maxit=4)
    for k in range(1, min(len(hi), len(hg))):
        if hi[k] > 1e-13:                                       # above the FP64 floor
            assert hg[k] <= hi[k] * (1 + 1e-6)


def test_block_gcr_exact_preconditioner_converges_at_x0():
    s, q, K, fac = _cfg1_small()
    A = O.k11_operator(K, fac.lambda2)
    lam1 = np.setdiff1d(np.arange(s.L), fac.lambda2)
    K11 = K.toarray()[np.ix_(lam1, lam1)]

    def exact(R):
        out = np.zeros_like(R)
        out[lam1] = np.linalg.solve(K11, R[lam1])
        return out
    B = np.zeros((s.L, fac.M))
    B[lam1] = K.toarray()[np.ix_(lam1, fac.lambda2)]
    X, hist, _, _ = O.block_gcr(A, exact, B, tol=1e-15, maxit=5)
    assert hist[0] < 1e-10


# --------------------------------------------------------------------------- Eq. 2 Schur complement
def test_schur_matches_dense_inverse_and_determinant():
    rng = np.random.default_rng(5)
    for _ in range(4):
        n = 12
        A = _rand_sym(n, rng) + np.diag(rng.uniform(3, 6, n))
        lam2 = np.sort(rng.choice(n, 4, replace=False))
        lam1 = np.setdiff1d(np.arange(n), lam2)
        S = O.schur_direct(sp.csr_matrix(A), lam2)
        Sref = A[np.ix_(lam2, lam2)] - A[np.ix_(lam2, lam1)] @ np.linalg.inv(A[np.ix_(lam1, lam1)]) @ A[np.ix_(lam1, lam2)]
        np.testing.assert_allclose(S, Sref, rtol=1e-12, atol=1e-12)
        # det K = det K11 det S22 (block LDU, Eq. 1)
        np.testing.assert_allclose(np.linalg.det(A), np.linalg.det(A[np.ix_(lam1, lam1)]) * np.linalg.det(S), rtol=1e-9)


def test_schur_of_cfg1_small_via_gcr_equals_direct():
    s, q, K, fac = _cfg1_small()
    res = O.run_hybrid(s.to_scipy(), _nodes_cfg1(), 1e-2, use_gcr=True)
    S_direct = O.schur_direct(res["K"], res["fac"].lambda2)
    assert np.linalg.norm(res["S22"] - S_direct) / np.linalg.norm(S_direct) < 1e-12


def _nodes_cfg1():
    s = diffusion2d(16, 16, n_islands=2, island=3, contrast=1e8, seed=4)
    q, K = O.scale_matrix(s.to_scipy())
    sets, order = O.nested_dissection(K, s.coords, 4)
    return [sets[l] for l in order]


# --------------------------------------------------------------------------- Alg. 1 step 5 Bunch-Kaufman
def test_bunch_kaufman_reconstruction_and_inertia():
    rng = np.random.default_rng(9)
    for n in (1, 2, 5, 17, 40):
        A = _rand_sym(n, rng)
        perm, Lf, blocks = O.bunch_kaufman(A)
        np.testing.assert_allclose(O.bk_reconstruct(perm, Lf, blocks), A, atol=1e-11 * np.abs(A).max())
        # Sylvester: inertia of D equals inertia of A
        ev = np.linalg.eigvalsh(A)
        dev = np.concatenate([np.linalg.eigvalsh(B) for _, _, B in blocks])
        assert (dev > 0).sum() == (ev > 0).sum() and (dev < 0).sum() == (ev < 0).sum()
        # LAPACK's Bunch-Kaufman (sytrf, through scipy.linalg.ldl) picks the same 1x1 / 2x2 blocks
        _, d, _ = sla.ldl(A, lower=True)
        sizes, i = [], 0
        while i < n:
            z = 2 if (i + 1 < n and d[i + 1, i] != 0) else 1
            sizes.append(z)
            i += z
        assert sizes == [z for _, z, _ in blocks]
        Dm = np.zeros((n, n))
        for s0, z, B in blocks:
            Dm[s0:s0 + z, s0:s0 + z] = B
        np.testing.assert_allclose(np.sort(np.abs(np.diag(Dm))), np.sort(np.abs(np.diag(d))), rtol=1e-8)


def test_bunch_kaufman_zero_diagonal_needs_2x2():
    A = np.array([[0.0, 1.0], [1.0, 0.0]])
    perm, Lf, blocks = O.bunch_kaufman(A)
    assert len(blocks) == 1 and blocks[0][1] == 2
    # the LAPACK Bunch-Kaufman routine (sytrf) makes the same choice
    lu, d, p = sla.ldl(A, lower=True)
    assert abs(d[1, 0]) > 0


def test_bunch_kaufman_solve_matches_dense():
    rng = np.random.default_rng(11)
    A = _rand_sym(9, rng)
    y = rng.standard_normal((9, 2))
    bk = O.bunch_kaufman(A)
    np.testing.assert_allclose(O.bk_solve(*bk, y, 0), np.linalg.solve(A, y), rtol=1e-9, atol=1e-10)


# --------------------------------------------------------------------------- kernel detection
@pytest.mark.parametrize("maker,expect", [
    (lambda: diffusion2d(16, 16, n_islands=2, island=3, contrast=1e8, seed=4), 1),
    (lambda: diffusion2d(14, 14, n_islands=0, dirichlet_x=True), 0),
    (lambda: stokes3d(5), 3),
    (lambda: elasticity3d(5, n_incl=1, incl=2), 6),
    (lambda: darcy2d(12, 12, n_islands=1, island=3), 1),
])
def test_kernel_dimension_matches_svd(maker, expect):
    s = maker()
    Kb = s.to_scipy()
    sv = np.linalg.svd(Kb.toarray(), compute_uv=False)
    null_svd = int((sv < 1e-12 * sv[0]).sum())
    assert null_svd == expect
    q, K = O.scale_matrix(Kb)
    dim = s.coords.shape[1]
    m = max(2, int(math.ceil(math.log2(s.L / 64))) + 1)
    sets, order = O.nested_dissection(K, s.coords, m)
    res = O.run_hybrid(Kb, [sets[l] for l in order], 1e-2)
    assert res["kdim"] == expect


# --------------------------------------------------------------------------- Alg. 2 solve
def test_kernel_dimension_rule_hand_cases():
    # R10 on hand-made pivot magnitudes: the tail after the largest gap >= gap_min whose
    # tail lies at or below max(kernel_eps * scale, noise), scale = max(max pivot, ref)
    assert O.kernel_dimension([1.0, 0.5, 1e-13, 1e-14]) == 2                 # gap 5e12
    assert O.kernel_dimension([1.0, 9e-11, 1e-22]) == 1                      # the larger of two gaps wins
    assert O.kernel_dimension([1.0, 0.5, 1e-8, 1e-9]) == 0                   # nothing below 1e-10
    assert O.kernel_dimension([1.0, 0.5, 1e-8, 1e-9], noise=1e-7) == 2       # the S22 error estimate
    assert O.kernel_dimension([1.0, 0.5, 1e-8, 1e-9], noise=1e-7, gap_min=1e9) == 0
    assert O.kernel_dimension([1e-12, 1e-13], ref=1.0) == 2                  # all null against the unit diagonal
    assert O.kernel_dimension([1e-12, 1e-13]) == 0                           # relative to themselves: no gap
    assert O.kernel_dimension([1e-12, 1e-25]) == 1
    assert O.kernel_dimension([0.0, 0.0]) == 2 and O.kernel_dimension([]) == 0
    assert O.kernel_dimension([3.0, 2.0, 1.0]) == 0


def test_hybrid_solve_exact_on_nonsingular():
    s = diffusion2d(12, 12, n_islands=1, island=3, contrast=1e6, dirichlet_x=True, seed=2)
    Kb = s.to_scipy()
    q, K = O.scale_matrix(Kb)
    sets, order = O.nested_dissection(K, s.coords, 3)
    res = O.run_hybrid(Kb, [sets[l] for l in order], 1e-2)
    b = np.random.default_rng(0).standard_normal((s.L, 2))
    x = q[:, None] * O.hybrid_solve(res["K"], res["fac"].lambda2, res["X12"], res["bk"], res["kdim"], q[:, None] * b)
    xr = np.linalg.solve(Kb.toarray(), b)
    assert np.abs(x - xr).max() / np.abs(xr).max() < 1e-9
    assert O.backward_error(Kb, x, b) < 1e-14


def test_hybrid_solve_singular_consistent():
    s = diffusion2d(16, 16, n_islands=2, island=3, contrast=1e8, seed=4)
    Kb = s.to_scipy()
    res = O.run_hybrid(Kb, _nodes_cfg1(), 1e-2, use_gcr=True)
    b = consistent_rhs(s, 3)
    q = res["q"]
    x = q[:, None] * O.hybrid_solve(res["K"], res["fac"].lambda2, res["X12"], res["bk"], res["kdim"], q[:, None] * b)
    assert O.backward_error(Kb, x, b) < 1e-14


def test_residual_measures_closed_form():
    # |r|_2/|b|_2 and the normwise backward error |r|_inf / (|K|_inf |x|_inf + |b|_inf) on a
    # 2x2 case worked by hand: K = [[2, -1], [0.5, 3]], x = [1, 0], b = [2, 0.496]:
    # r = K x - b = [0, 0.004], |K|_inf = max row sum 3.5 (the column sums are 2.5 and 4),
    # |x|_inf = 1, |b|_inf = 2.
    Kb = sp.csr_matrix(np.array([[2.0, -1.0], [0.5, 3.0]]))
    x = np.array([[1.0], [0.0]])
    b = np.array([[2.0], [0.496]])
    assert abs(O.relative_residual(Kb, x, b) - 0.004 / math.hypot(2.0, 0.496)) < 1e-15
    assert abs(O.backward_error(Kb, x, b) - 0.004 / (3.5 * 1.0 + 2.0)) < 1e-16
    # scaling x and b together leaves the measure unchanged
    assert abs(O.backward_error(Kb, 10 * x, 10 * b) - O.backward_error(Kb, x, b)) < 1e-16
    # max over columns
    X2 = np.hstack([x, x])
    B2 = np.hstack([b, np.array([[2.0], [0.5]])])
    assert O.backward_error(Kb, X2, B2) == O.backward_error(Kb, x, b)


def test_s22_noise_estimates_the_schur_error():
    # Perturb X12 by D on Lambda_1: S22 changes by exactly -K21 D, and the estimate
    # factor * |K21 Q^-1 (K12 - K11 X12)|_max reads it through Q^-1 K11 ~ I (Sec. 3.3).
    s, q, K, fac = _cfg1_small()
    lam1 = np.setdiff1d(np.arange(s.L), fac.lambda2)
    X12 = O.x12_direct(K, fac.lambda2)
    assert O.s22_noise(K, fac, X12, factor=1.0) < 1e-12
    D = np.zeros_like(X12)
    D[lam1] = np.random.default_rng(8).standard_normal((len(lam1), fac.M)) * 1e-6
    dS = O.schur_direct(K, fac.lambda2, X12 + D) - O.schur_direct(K, fac.lambda2, X12)
    est = O.s22_noise(K, fac, X12 + D, factor=1.0)
    assert abs(est - np.abs(dS).max()) <= 1e-2 * np.abs(dS).max()
    assert abs(O.s22_noise(K, fac, X12 + D) - 100.0 * est) <= 1e-12 * est


# --------------------------------------------------------------------------- adjoint
def test_adjoint_gradient_matches_central_differences():
    n = 6
    rng = np.random.default_rng(5)
    theta = rng.standard_normal(n * n)
    b = rng.uniform(-1, 1, n * n)
    xs = rng.uniform(-1, 1, n * n)

    def J(th):
        s = diffusion2d(n, n, n_islands=0, dirichlet_x=True, kcell=np.exp(th))
        x = np.linalg.solve(s.to_scipy().toarray(), b)
        return O.diffusion_objective(x, xs), x, s

    _, x, s = J(theta)
    lam = np.linalg.solve(s.to_scipy().toarray().T, x - xs)
    g = O.adjoint_gradient(n, n, theta, x, lam)
    for _ in range(4):
        d = rng.standard_normal(n * n)
        h = 1e-6
        fd = (J(theta + h * d)[0] - J(theta - h * d)[0]) / (2 * h)
        np.testing.assert_allclose(g @ d, fd, rtol=1e-5)


# --------------------------------------------------------------------------- R3b null-pivot test
def test_null_pivot_test_skips_cancelled_pivot():
    # index 2 keeps 1.5e-3 of a diagonal built from terms of size ~2: the ratio test to the
    # previous pivot (0.5) passes at tau = 1e-3.  Sec. 2.2 postpones on that ratio alone, so
    # by default all three are eliminated and only the enlargement (n = 1) moves index 2.
    a = np.sqrt(1 - 1.5e-3)
    K = sp.csr_matrix(np.array([[0.5, 0, 0], [0, 1.0, a], [0, a, 1.0]]))
    lit = O.threshold_factorize(K, [np.array([0, 1, 2])], tau=1e-3, n_enlarge=1)
    assert lit.node_pivots[0].tolist() == [1, 0, 2]
    assert lit.node_skipped[0].tolist() == [] and lit.lam0.tolist() == []
    assert lit.lambda2.tolist() == [2]
    # the optional cancellation (null) test R3b skips index 2 instead
    fac = O.threshold_factorize(K, [np.array([0, 1, 2])], tau=1e-3, n_enlarge=1, null_test=True)
    assert fac.node_pivots[0].tolist() == [1, 0]
    assert fac.node_skipped[0].tolist() == [2]
    assert fac.lam0_skipped.tolist() == [2] and fac.lam0_pivots.tolist() == []
    assert fac.lambda2.tolist() == [0, 2]


# --------------------------------------------------------------------------- R11 Bunch-Parlett
def test_bunch_parlett_reconstruction_inertia_and_bound():
    rng = np.random.default_rng(21)
    alpha = (1 + math.sqrt(17)) / 8
    for n in (1, 2, 6, 19, 41):
        A = _rand_sym(n, rng)
        if n > 3:
            A[np.arange(n), np.arange(n)] *= 1e-3          # forces 2x2 pivots
        perm, Lf, blocks = O.bunch_parlett(A)
        np.testing.assert_allclose(O.bk_reconstruct(perm, Lf, blocks), A, atol=1e-11 * np.abs(A).max())
        ev = np.linalg.eigvalsh(A)
        dev = np.concatenate([np.linalg.eigvalsh(B) for _, _, B in blocks])
        assert (dev > 0).sum() == (ev > 0).sum() and (dev < 0).sum() == (ev < 0).sum()
        assert np.abs(Lf).max() <= 1.0 / (1.0 - alpha) + 1e-9   # complete-pivoting growth bound on L
        if n > 3:
            assert any(z == 2 for _, z, _ in blocks)


def test_bunch_parlett_choice_matches_brute_force():
    # R11 complete pivoting, checked step by step on Schur complements formed from scratch:
    # a 1x1 pivot is the largest |diagonal| of the remaining block and is at least alpha
    # times its largest off-diagonal; a 2x2 pivot holds that largest off-diagonal entry.
    rng = np.random.default_rng(23)
    alpha = (1 + math.sqrt(17)) / 8
    seen = set()
    for trial in range(8):
        n = 9
        A = _rand_sym(n, rng)
        A[np.arange(n), np.arange(n)] *= rng.choice([1e-3, 1.0, 3.0])
        perm, Lf, blocks = O.bunch_parlett(A)
        Ap = A[np.ix_(perm, perm)]
        for s0, z, B in blocks:
            S = Ap[s0:, s0:] - (Ap[s0:, :s0] @ np.linalg.solve(Ap[:s0, :s0], Ap[:s0, s0:]) if s0 else 0)
            mu0 = np.abs(np.diag(S)).max()
            off = np.abs(S - np.diag(np.diag(S)))
            mu1 = off.max()
            np.testing.assert_allclose(B, S[:z, :z], rtol=1e-9, atol=1e-12)
            if z == 1:
                assert abs(B[0, 0]) >= mu0 * (1 - 1e-12) and mu0 >= alpha * mu1 * (1 - 1e-12)
            else:
                assert mu0 < alpha * mu1 * (1 + 1e-12) and abs(B[1, 0]) >= mu1 * (1 - 1e-12)
            seen.add(z)
    assert seen == {1, 2}


def test_pivot_magnitudes_of_2x2_blocks():
    # a 2x2 pivot counts by the magnitudes of its eigenvalues, not its diagonal:
    # [[0, 1], [1, 0]] (+) [0] has a one-dimensional kernel, and the block itself is regular
    A = np.zeros((3, 3))
    A[0, 1] = A[1, 0] = 1.0
    perm, Lf, blocks = O.bunch_parlett(A)
    mags, owners = O.pivot_magnitudes(blocks)
    assert sorted(z for _, z, _ in blocks) == [1, 2]
    np.testing.assert_allclose(np.sort(mags), [0.0, 1.0, 1.0])
    assert O.kernel_dimension(mags) == 1
    B = np.array([[2.0, 5.0], [5.0, -1.0]])
    m2, _ = O.pivot_magnitudes([(0, 2, B)])
    np.testing.assert_allclose(np.sort(m2), np.sort(np.abs(np.linalg.eigvalsh(B))))


def test_bunch_parlett_is_rank_revealing():
    rng = np.random.default_rng(22)
    for n, r in ((8, 5), (12, 6), (20, 17)):
        U, _ = np.linalg.qr(rng.standard_normal((n, n)))
        lam = np.concatenate([rng.uniform(1, 2, r) * rng.choice([-1, 1], r), np.zeros(n - r)])
        A = (U * lam) @ U.T
        perm, Lf, blocks = O.bunch_parlett(A)
        mags, owners = O.pivot_magnitudes(blocks)
        order_mags = np.concatenate([np.abs(np.linalg.eigvalsh(B)) if z == 2 else [abs(B[0, 0])] for _, z, B in blocks])
        assert (order_mags[r:] < 1e-12).all() and (order_mags[:r] > 1e-4).all()   # null pivots last
        assert O.kernel_dimension(mags) == n - r
        # Bunch-Kaufman (partial pivoting) does not promise this ordering


# --------------------------------------------------------------------------- LDU form (U != L^T)
def _rand_unsym(n, rng):
    return rng.standard_normal((n, n)) * 0.3 + np.diag(rng.uniform(0.5, 3.0, n) * rng.choice([-1, 1], n))


def _convection_diffusion(n, seed=0, peclet=0.4):
    # diffusion with islands plus a skew-symmetric part on the same pattern: K-bar != K-bar^T
    s = diffusion2d(n, n, n_islands=1, island=3, contrast=1e4, dirichlet_x=True, seed=seed)
    K = s.to_scipy().tocsr()
    U = sp.triu(K, 1).tocoo()
    rng = np.random.default_rng(seed)
    w = peclet * np.abs(U.data) * rng.uniform(0.5, 1.0, U.nnz)
    N = sp.coo_matrix((np.concatenate([w, -w]), (np.concatenate([U.row, U.col]), np.concatenate([U.col, U.row]))),
                      shape=K.shape)
    return s, (K + N).tocsr()


def test_ldu_reconstructs_eq1_unsymmetric():
    # Eq. (1) in its LDU form: Pi^T K Pi = L D U with unit L (columns) and unit U (rows)
    rng = np.random.default_rng(31)
    for _ in range(4):
        n = 11
        A = _rand_unsym(n, rng)
        fac = O.threshold_factorize(sp.csr_matrix(A), [np.arange(n)], tau=1e-6, n_enlarge=0)
        elim = fac.node_pivots[0].astype(int)
        pos = {int(g): i for i, g in enumerate(elim)}
        m = len(elim)
        Lm, Um, D = np.eye(m), np.eye(m), np.zeros(m)
        for g in elim:
            j = pos[int(g)]
            D[j] = fac.d[int(g)]
            for r, v in zip(*fac.lcol[int(g)]):
                if int(r) in pos:
                    Lm[pos[int(r)], j] = v
            for r, v in zip(*fac.urow[int(g)]):
                if int(r) in pos:
                    Um[j, pos[int(r)]] = v
        Ad = A[np.ix_(elim, elim)]
        assert np.abs(np.tril(Lm, -1)).max() > 0 and np.abs(Lm - Um.T).max() > 1e-3   # really unsymmetric
        assert np.abs(Lm @ np.diag(D) @ Um - Ad).max() / np.abs(Ad).max() < 1e-5


def test_ldu_pivots_match_brute_force_unsymmetric_schur():
    rng = np.random.default_rng(32)
    for _ in range(6):
        n = 8
        A = _rand_unsym(n, rng)
        fac = O.threshold_factorize(sp.csr_matrix(A), [np.arange(n)], tau=1e-6, n_enlarge=0)
        elim = []
        for q in fac.node_pivots[0]:
            rest = [i for i in range(n) if i not in elim]
            S = A[np.ix_(rest, rest)]
            if elim:
                S = S - A[np.ix_(rest, elim)] @ np.linalg.solve(A[np.ix_(elim, elim)], A[np.ix_(elim, rest)])
            assert rest[int(np.argmax(np.abs(np.diag(S))))] == q
            np.testing.assert_allclose(fac.d[int(q)], S[rest.index(q), rest.index(q)], rtol=2e-5)
            elim.append(int(q))


def test_sign_form_factorizes_like_the_symmetric_matrix():
    # K-bar = J S (J = diag(I, -I), S symmetric): every Schur complement of Q K-bar Q is J times
    # that of Q S Q, so the pivots, the split and X12 are those of S, d and l change sign with
    # J, u does not, S22 = J2 S22(S), and K-bar x = b is S x = J b (Sec. 2.1 rank-1 update).
    s = stokes3d_ldu(4, delta=0.01)
    S = stokes3d(4, delta=0.01)
    J = s.meta["row_sign"].astype(np.float64)
    Ku, Ks = s.to_scipy(), S.to_scipy()
    assert abs(Ku - Ku.T).max() > 0 and abs(Ks - Ks.T).max() == 0
    qu, K1 = O.scale_matrix(Ku)
    qs, K2 = O.scale_matrix(Ks)
    np.testing.assert_array_equal(qu, qs)
    sets, order = O.nested_dissection(K2, S.coords, 3)
    nodes = [sets[l] for l in order]
    fu = O.threshold_factorize(K1, nodes, tau=1e-2)
    fs = O.threshold_factorize(K2, nodes, tau=1e-2)
    for a, b in zip(fu.node_pivots, fs.node_pivots):
        np.testing.assert_array_equal(a, b)
    np.testing.assert_array_equal(fu.lambda2, fs.lambda2)
    for g in fs.d:
        assert fu.d[g] == J[g] * fs.d[g]
        ru, lu = fu.lcol[g]
        rs, ls = fs.lcol[g]
        np.testing.assert_array_equal(ru, rs)
        np.testing.assert_array_equal(lu, (J[rs] * J[g] * ls).astype(ls.dtype))
        np.testing.assert_array_equal(fu.urow[g][1], fs.urow[g][1])
    ru_ = O.run_hybrid(Ku, nodes, 1e-2)
    rs_ = O.run_hybrid(Ks, nodes, 1e-2)
    lam2 = fs.lambda2
    np.testing.assert_allclose(ru_["S22"], J[lam2][:, None] * rs_["S22"], atol=1e-11 * np.abs(rs_["S22"]).max())
    assert len(ru_["bk"]) == 4 and len(rs_["bk"]) == 3 and ru_["kdim"] == rs_["kdim"] == 3


def test_lu_complete_reconstruction_and_pivot_choice():
    rng = np.random.default_rng(33)
    for n in (1, 2, 5, 9, 16):
        A = rng.standard_normal((n, n))
        prow, pcol, Lf, U = O.lu_complete(A)
        np.testing.assert_allclose(O.lu_reconstruct(prow, pcol, Lf, U), A, atol=1e-12 * np.abs(A).max())
        assert np.abs(Lf).max() <= 1.0 + 1e-12                        # complete pivoting: |l| <= 1
        Ap = A[np.ix_(prow, pcol)]
        for k in range(n):                                             # brute-force Schur complements
            Sk = Ap[k:, k:] - (Ap[k:, :k] @ np.linalg.solve(Ap[:k, :k], Ap[:k, k:]) if k else 0)
            assert abs(U[k, k]) >= np.abs(Sk).max() * (1 - 1e-10)
            np.testing.assert_allclose(U[k, k:], Sk[0], rtol=1e-9, atol=1e-12 * np.abs(A).max())


def test_lu_complete_is_rank_revealing_and_pseudo_solves():
    rng = np.random.default_rng(34)
    for n, r in ((8, 5), (12, 9), (20, 17)):
        X, Y = rng.standard_normal((n, r)), rng.standard_normal((r, n))
        A = X @ Y
        prow, pcol, Lf, U = O.lu_complete(A)
        mags = np.abs(np.diag(U))
        assert (mags[r:] < 1e-10 * mags[0]).all() and (mags[:r] > 1e-6 * mags[0]).all()
        assert O.kernel_dimension(mags) == n - r
        y = A @ rng.standard_normal((n, 2))                            # consistent
        x = O.lu_pseudo_solve(prow, pcol, Lf, U, y, n - r)
        np.testing.assert_allclose(A @ x, y, atol=1e-9 * np.abs(y).max())
    A = rng.standard_normal((9, 9))
    y = rng.standard_normal((9, 3))
    np.testing.assert_allclose(O.lu_pseudo_solve(*O.lu_complete(A), y, 0), np.linalg.solve(A, y), rtol=1e-9, atol=1e-10)


def test_unsymmetric_precond_and_gcr():
    s, Kb = _convection_diffusion(14, seed=3)
    q, K = O.scale_matrix(Kb)
    sets, order = O.nested_dissection(K, s.coords, 3)
    fac = O.threshold_factorize(K, [sets[l] for l in order], tau=1e-2, n_enlarge=4)
    A = O.k11_operator(K, fac.lambda2)
    X = np.random.default_rng(1).standard_normal((s.L, 3))
    X[fac.lambda2] = 0
    Y = O.precond_apply(fac, A(X))
    assert np.linalg.norm(Y - X) / np.linalg.norm(X) < 1e-3            # Q^-1 K11 ~ I with U != L^T
    lam1 = np.setdiff1d(np.arange(s.L), fac.lambda2)
    B = np.zeros((s.L, fac.M))
    B[lam1] = K.toarray()[np.ix_(lam1, fac.lambda2)]
    Xg, hist, _, _ = O.block_gcr(A, lambda R: O.precond_apply(fac, R), B, tol=1e-15, maxit=20)
    Xd = O.x12_direct(K, fac.lambda2)
    assert np.abs(Xg - Xd).max() / np.abs(Xd).max() < 1e-12


def test_unsymmetric_hybrid_solve():
    # nonsingular convection-diffusion: the exact solution; the singular Stokes LDU form of
    # Sec. 4.2 with a consistent right-hand side: backward error at FP64 rounding, kernel 3
    s, Kb = _convection_diffusion(12, seed=4)
    q, K = O.scale_matrix(Kb)
    sets, order = O.nested_dissection(K, s.coords, 3)
    res = O.run_hybrid(Kb, [sets[l] for l in order], 1e-2, use_gcr=True)
    assert len(res["bk"]) == 4 and res["kdim"] == 0
    b = np.random.default_rng(0).standard_normal((s.L, 2))
    x = q[:, None] * O.hybrid_solve(res["K"], res["fac"].lambda2, res["X12"], res["bk"], res["kdim"], q[:, None] * b)
    xr = np.linalg.solve(Kb.toarray(), b)
    assert np.abs(x - xr).max() / np.abs(xr).max() < 1e-9
    t = stokes3d_ldu(4, delta=0.01)
    Kt = t.to_scipy()
    qt, K2 = O.scale_matrix(Kt)
    sets, order = O.nested_dissection(K2, t.coords, 3)
    res = O.run_hybrid(Kt, [sets[l] for l in order], 1e-2, use_gcr=True)
    assert res["kdim"] == 3
    b = consistent_rhs(t, 5, nrhs=2)
    x = qt[:, None] * O.hybrid_solve(res["K"], res["fac"].lambda2, res["X12"], res["bk"], res["kdim"], qt[:, None] * b)
    assert O.backward_error(Kt, x, b) < 1e-14


# --------------------------------------------------------------------------- replay admissibility
def test_replay_admits_the_rule_and_flags_other_choices():
    # replaying the oracle's own decisions is admissible; a pivot order that takes a clearly
    # smaller diagonal first, or an early stop, is reported; a near-tie inside the rounding
    # of the compared values (relative slack) is admitted
    K = sp.csr_matrix(np.diag([1.0, 0.5, 0.25, 0.2]))
    nodes = [np.array([0, 1, 2, 3])]
    own = O.threshold_factorize(K, nodes, tau=1e-2, n_enlarge=0)
    rp = {"node_pivots": [own.node_pivots[0]], "node_skipped": [np.zeros(0, np.int64)],
          "lam0_pivots": own.lam0_pivots, "lam0_skipped": np.zeros(0, np.int64)}
    assert O.threshold_factorize(K, nodes, 1e-2, 0, replay=rp).violations == []
    bad = dict(rp, node_pivots=[np.array([1, 0, 2, 3])])
    v = O.threshold_factorize(K, nodes, 1e-2, 0, replay=bad).violations
    assert any("< max" in m for m in v)
    stop = dict(rp, node_pivots=[np.array([0, 1])], lam0_pivots=np.array([2, 3]))
    assert any("stopped" in m for m in O.threshold_factorize(K, nodes, 1e-2, 0, replay=stop).violations)
    Kt = sp.csr_matrix(np.diag([1.0, 1.0 - 2e-5, 0.5]))
    tie = {"node_pivots": [np.array([1, 0, 2])], "node_skipped": [np.zeros(0, np.int64)],
           "lam0_pivots": np.zeros(0, np.int64), "lam0_skipped": np.zeros(0, np.int64)}
    assert O.threshold_factorize(Kt, [np.array([0, 1, 2])], 1e-2, 0, replay=tie).violations == []
