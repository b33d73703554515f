"""Plain CPU restatement of the hybrid factorization, step by step in the paper's order.

Test infrastructure only (see the package docstring).  Notation follows the
paper: K-bar the user matrix, Q the diagonal scaling, K = Q K-bar Q (Sec. 2),
Lambda_l the index sets of the nested-dissection tree (Sec. 2.2), tau the
postponing threshold, Lambda_0 the postponed set, Lambda_1 / Lambda_2 the
moderate / hard split with N = #Lambda_1, M = #Lambda_2 (Alg. 1), X12 the
solution of K11 X12 = K12 (Alg. 1 step 3), S22 the Schur complement (Eq. 2).

Readings of passages where the paper is silent or garbled (each also listed in
the design notes):
  R1  Q_ii = 1/sqrt(|K-bar_ii|), so diag(K) is in {-1, 0, 1}  (Sec. 2).
  R2  The first pivot of every index set is compared against 1: it is
      postponed if |d_1| < tau (the unit diagonal after scaling).
  R3  The ratio test compares each pivot with the previous pivot of the
      same index set: postpone when |d_{i+1} / d_i| < tau (Sec. 2.2).
  R4  Lambda_2 = the postponed part of Lambda_0 after enlargement,
      Lambda_1 = all other indices (Sec. 2.2 prints the same hat twice).
  R5  Ties in max |diag| go to the smallest original index.
  R6  GCR: beta uses (A w_{n+1}, A p_m), the form that gives the
      A-orthogonality the paper states (Sec. 3.4).
  R7  Block GCR: B_mn = -Q_m^T Z_{n+1}, P_{n+1} = W_{n+1} + sum_m P_m M_m^-1 B_mn,
      and Q_{n+1} likewise (Sec. 3.5).
  R8  Block GCR starts as Alg. 4 (X0 = Q^-1 B) and stops when every column
      satisfies |r_k| / |b_k| <= tol.
  R3b Optional null-pivot test, not in the paper and off by default
      (null_test=False): Sec. 2.2 postpones on the ratio test alone.  When
      asked for, a candidate whose current diagonal is below tau times the
      magnitude of the terms it was formed from (|K_ii| plus the accumulated
      |l_ik|^2 |d_k| of earlier eliminations) counts as cancelled: it is
      postponed on its own (skipped) and the elimination of the set goes on.
  R14 The GPU path forms q_{n+1} = A p_{n+1} by a product with A instead of the
      recurrence q_{n+1} = z_{n+1} + sum beta q_m (Sec. 3.4 keeps the
      recurrence to save one SpMV for a single rhs; with M rhs the recurrence
      costs N M^2 n flops against nnz M for the product).  Both equal A p;
      the oracle keeps the paper's recurrence.
  R10 Kernel detection: pivot magnitudes of the S22 LDL^T sorted; the kernel
      is the tail after the largest ratio gap >= gap_min whose tail lies
      below kernel_eps * max.
  R11 S22 is factorized with symmetric complete (Bunch-Parlett) pivoting,
      1x1 or 2x2 blocks, alpha = (1+sqrt 17)/8: the largest entries of the
      whole remaining block go first, so null pivots come last (rank
      revealing, as the kernel detection needs).
  R15 An unsymmetric S22 (the LDU form with U != L^T, e.g. the saddle point
      [A B^T; -B delta D] of Sec. 4.2) is factorized by Gaussian elimination
      with complete pivoting, the unsymmetric counterpart of R11: the entry of
      largest magnitude of the whole remaining block goes first, so null
      pivots come last; the kernel rule R10 reads |u_kk|.
  R13 The enlargement moves the last n = 4 entries of the elimination order
      into hat-Lambda_0.  These are the last entries of tilde-Lambda_0 when it
      holds at least n of them; when tilde-Lambda_0 is shorter (every
      Lambda_0 pivot failed the threshold) the move continues backwards into
      the last eliminated pivots, so S22 still gets an image space of n
      regular pivots to compare the null pivots against (Sec. 2.2).
"""
from __future__ import annotations

from dataclasses import dataclass, field
import math

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

__all__ = [
    "scale_matrix", "nested_dissection", "tree_block_pattern", "threshold_factorize",
    "FactorResult", "precond_apply", "k11_operator", "block_gcr", "gcr_single", "iterative_refinement",
    "schur_direct", "x12_direct", "bunch_kaufman", "bunch_parlett", "bk_reconstruct", "pivot_magnitudes",
    "kernel_dimension", "bk_solve", "hybrid_solve", "relative_residual", "backward_error",
    "run_hybrid", "s22_noise", "adjoint_gradient", "diffusion_objective",
    "lu_complete", "lu_reconstruct", "lu_pseudo_solve",
]


# ---------------------------------------------------------------------------
# Sec. 2: diagonal scaling K = Q K-bar Q
# ---------------------------------------------------------------------------
def scale_matrix(Kbar: sp.csr_matrix):
    """Return (q, K) with q = diag(Q), Q_ii = 1/sqrt(|K-bar_ii|) when nonzero else 1 (Sec. 2, R1)."""
    d = Kbar.diagonal()
    q = np.ones(Kbar.shape[0])
    nz = d != 0
    q[nz] = 1.0 / np.sqrt(np.abs(d[nz]))
    Q = sp.diags(q)
    K = (Q @ Kbar @ Q).tocsr()
    return q, K


# ---------------------------------------------------------------------------
# Sec. 2.2: nested dissection with an m-level bisection tree (oracle's own)
# ---------------------------------------------------------------------------
def nested_dissection(K: sp.csr_matrix, coords: np.ndarray, m: int):
    """Split {0..L-1} into 2^m - 1 sets Lambda_l of an m-level bisection tree (Sec. 2.2, Fig. 1).

    Nodes are numbered as in Fig. 1: root 1, children of l are 2l and 2l+1.
    Each interior set is a vertex separator: the vertices of the lower half
    (coordinate below the median of the widest axis) that touch the upper half.
    Returns (sets, order) where sets[l] is an index array for l = 1 .. 2^m - 1
    and order lists the node ids in elimination order, deepest level first
    (Fig. 1 eliminates 4, 5, 6, 7, 2, 3, 1).
    """
    L = K.shape[0]
    adj = K.tocsr()
    sets = {}

    def split(l, verts, level):
        if level == m:
            sets[l] = np.sort(verts)
            return
        if len(verts) == 0:
            sets[l] = verts
            split(2 * l, verts, level + 1)
            split(2 * l + 1, verts, level + 1)
            return
        c = coords[verts]
        ax = int(np.argmax(c.max(axis=0) - c.min(axis=0)))
        vals = np.unique(c[:, ax])
        if len(vals) == 1:                      # cannot bisect: the whole set is the separator
            sets[l] = np.sort(verts)
            empty = np.zeros(0, dtype=np.int64)
            split(2 * l, empty, level + 1)
            split(2 * l + 1, empty, level + 1)
            return
        med = vals[(len(vals) + 1) // 2]
        lower = verts[c[:, ax] < med]
        upper = verts[c[:, ax] >= med]
        inupper = np.zeros(L, bool)
        inupper[upper] = True
        sep = [v for v in lower if inupper[adj.indices[adj.indptr[v]:adj.indptr[v + 1]]].any()]
        sep = np.array(sep, dtype=np.int64)
        insep = np.zeros(L, bool)
        insep[sep] = True
        lower = lower[~insep[lower]]
        sets[l] = np.sort(sep)
        split(2 * l, lower, level + 1)
        split(2 * l + 1, upper, level + 1)

    split(1, np.arange(L, dtype=np.int64), 1)
    order = [l for lev in range(m, 0, -1) for l in range(2 ** (lev - 1), 2 ** lev)]
    return sets, order


def tree_block_pattern(K: sp.csr_matrix, sets: dict):
    """Set of (i, j) node pairs whose block K[Lambda_i, Lambda_j] has a nonzero (Fig. 1)."""
    L = K.shape[0]
    owner = np.full(L, -1)
    for l, s in sets.items():
        owner[s] = l
    C = K.tocoo()
    pairs = set(zip(owner[C.row].tolist(), owner[C.col].tolist()))
    return pairs


# ---------------------------------------------------------------------------
# Sec. 2.1-2.2 and Alg. 1 step 1: lower-precision LDL^T with symmetric
# pivoting and threshold postponing along the dissection tree
# ---------------------------------------------------------------------------
@dataclass
class FactorResult:
    node_pivots: list                 # per tree node (elimination order): chosen indices in order
    node_postponed: list              # per tree node: tilde/hat split -> hat part
    lam0: np.ndarray                  # Lambda_0, union of the postponed sets
    lam0_pivots: np.ndarray           # tilde-Lambda_0 in the order of the refactorization
    moved: np.ndarray                 # the entries moved from tilde-Lambda_0 to hat-Lambda_0
    lambda1_order: np.ndarray         # Pi_1: elimination order of Lambda_1
    lambda2: np.ndarray               # Lambda_2, sorted
    d: dict = field(default_factory=dict)       # pivot value (float32) per eliminated index
    lcol: dict = field(default_factory=dict)    # index -> (rows, float32 values) of L (column)
    urow: dict = field(default_factory=dict)    # index -> (rows, float32 values) of U (row); = lcol if K = K^T
    violations: list = field(default_factory=list)

    @property
    def N(self):
        return len(self.lambda1_order)

    @property
    def M(self):
        return len(self.lambda2)


def _eliminate(S, G, remaining, q, fac, symmetric):
    """One rank-1 Schur update with weight 1/d on the remaining indices (Sec. 2.1).

    The LDU form: the pivot's column (below) and row (right) enter the update
    separately, S' = S - col d^-1 row, with l = col / d and u = row / d.  For a
    symmetric S the column is the row (LDL^T) and only the row is read.
    G accumulates, per index, |K_ii| plus the magnitudes |l_i u_i d| of the
    updates its diagonal received (used by the null-pivot test R3b).
    """
    d = S[q, q]
    remaining[q] = False
    if symmetric:
        rows = np.flatnonzero((S[q] != 0) & remaining)
        col = row = S[q, rows].copy()
    else:
        rows = np.flatnonzero(((S[:, q] != 0) | (S[q] != 0)) & remaining)
        col = S[rows, q].copy()
        row = S[q, rows].copy()
    if rows.size:
        S[np.ix_(rows, rows)] -= np.outer(col, row) / d
        G[rows] += np.abs(col * (row / d))
    fac.d[int(q)] = d
    fac.lcol[int(q)] = (rows, col / d)
    fac.urow[int(q)] = (rows, row / d)
    return d


def _factor_set(S, G, remaining, cand, tau, fac, replay=None, slack=1e-4, null_test=False, tag="",
                symmetric=False):
    """Symmetric max-|diag| pivoting with threshold postponing on one index set (Sec. 2.1-2.2).

    Each step takes the candidate of largest |diag| (R5 ties).  If it fails the
    ratio test (R2/R3) the rest of the set is postponed (stop).  With the
    optional null-pivot test (R3b, null_test=True) a candidate that passes the
    ratio test but fails that test is postponed alone (skip).
    Returns (chosen, postponed, skipped).

    Replay mode: ``replay = (accepted sequence, set of skipped indices)`` chosen
    by another implementation.  The oracle follows it: it skips the listed
    candidates when they come up as the maximum and accepts the listed pivots
    in order, recording any step that this rule would not admit.  The decisions
    are taken in the lower precision (Alg. 1 step 1), so a comparison counts as
    admissible within the rounding of the values compared: a relative slack, plus
    slack times the magnitude G of the terms each diagonal was formed from (the
    size of its rounding error when cancellation has made it small).
    """
    cand = list(np.asarray(cand, dtype=np.int64))
    chosen, skipped = [], []
    d_ref = 1.0                                   # R2: first pivot compared with the unit diagonal
    seq, skip_set = (None, set()) if replay is None else (list(replay[0]), set(int(x) for x in replay[1]))
    step = 0
    while cand:
        dg = np.abs(np.array([S[c, c] for c in cand], dtype=np.float64))
        dg[np.isnan(dg)] = -1.0
        best = max(range(len(cand)), key=lambda t: (dg[t], -cand[t]))   # R5 tie -> smallest index
        if seq is None:
            t = best
            if not (dg[t] >= tau * d_ref):                           # R3 ratio test (NaN stops)
                break
            if null_test and not (dg[t] >= tau * float(G[cand[t]])):  # R3b null pivot: skip it
                skipped.append(cand.pop(t))
                continue
        else:
            bq = cand[best]
            if bq in skip_set and step <= len(seq):
                # the other implementation skipped this candidate when it was the maximum
                if null_test and dg[best] > tau * float(G[bq]) * (1 + slack):
                    fac.violations.append(f"{tag}: skipped {bq} passes the null test")
                skipped.append(cand.pop(best))
                continue
            if step >= len(seq):
                if dg[best] >= tau * d_ref * (1 + slack) + slack * float(G[bq]) and \
                        not (null_test and dg[best] < tau * float(G[bq])):
                    fac.violations.append(f"{tag}: replay stopped at step {step} but oracle ratio "
                                          f"{dg[best] / d_ref:.6g} >= tau")
                break
            q = int(seq[step])
            if q not in cand:
                fac.violations.append(f"{tag}: replay pivot {q} is not a candidate")
                break
            t = cand.index(q)
            if dg[t] < (1 - slack) * dg[best] - slack * (float(G[q]) + float(G[bq])):
                fac.violations.append(f"{tag}: step {step} pivot {q} |d|={dg[t]:.8g} < max {dg[best]:.8g}")
            if dg[t] < tau * d_ref * (1 - slack) - slack * float(G[q]):
                fac.violations.append(f"{tag}: step {step} pivot {q} fails the ratio test")
            if null_test and dg[t] < tau * float(G[q]) * (1 - slack):
                fac.violations.append(f"{tag}: step {step} pivot {q} fails the null test")
        q = cand.pop(t)
        d = _eliminate(S, G, remaining, q, fac, symmetric)
        d_ref = abs(float(d))
        chosen.append(q)
        step += 1
    if seq is not None:
        if step < len(seq):
            fac.violations.append(f"{tag}: oracle could not follow replay past step {step}")
        missing = skip_set - set(skipped)
        if missing:
            fac.violations.append(f"{tag}: replay skipped {sorted(missing)[:5]} never came up as maximum")
    postponed = np.array(sorted(set(cand) | set(skipped)), dtype=np.int64)
    return np.array(chosen, dtype=np.int64), postponed, np.array(skipped, dtype=np.int64)


def _symmetric(K) -> bool:
    """K = K^T up to rounding: max |K - K^T| <= 1e-14 max |K|.

    An assembled or scaled matrix can differ from its transpose in the last bits
    (element sums taken in another order, (q_i k_ij) q_j against (q_j k_ji) q_i); for
    the method it is symmetric (LDL^T, Bunch-Parlett).  The row-sign form
    [A B^T; -B delta D] differs by 2|B| and takes the LDU route (R15).
    """
    K = sp.csr_matrix(K)
    return bool(abs(K - K.T).max() <= 1e-14 * abs(K).max())


def threshold_factorize(K: sp.csr_matrix, nodes: list, tau: float, n_enlarge: int = 4,
                        replay: dict | None = None, slack: float = 1e-4, dtype=np.float32,
                        null_test: bool = False) -> FactorResult:
    """Alg. 1 step 1: factor along the tree, postpone, refactor Lambda_0, enlarge.

    ``nodes``: index arrays Lambda_l in elimination order (children before parents).
    ``dtype``: the lower precision of the factorization (float32 for the mixed
    form; float64 reproduces the plain double form of Table 1).
    ``replay``: optional {"node_pivots": [...], "node_skipped": [...],
    "lam0_pivots": [...], "lam0_skipped": [...]} chosen by another implementation;
    the oracle follows it and records any choice that this rule would not admit.
    ``null_test``: add the optional null-pivot test R3b to the ratio test of Sec. 2.2.
    """
    L = K.shape[0]
    S = K.toarray().astype(dtype)                  # current Schur complement
    symmetric = _symmetric(K)
    G = np.abs(np.diag(S)).copy()                  # R3b magnitude of the terms in each diagonal
    remaining = np.ones(L, dtype=bool)
    fac = FactorResult([], [], None, None, None, None, None)
    fac.node_skipped = []
    for t, lam in enumerate(nodes):
        rp = None if replay is None else (replay["node_pivots"][t], replay["node_skipped"][t])
        ch, pp, sk = _factor_set(S, G, remaining, lam, tau, fac, rp, slack, null_test, tag=f"node{t}",
                                 symmetric=symmetric)
        fac.node_pivots.append(ch)
        fac.node_postponed.append(pp)
        fac.node_skipped.append(sk)
    lam0 = np.concatenate(fac.node_postponed) if fac.node_postponed else np.zeros(0, np.int64)
    fac.lam0 = np.sort(lam0)
    rp = None if replay is None else (replay["lam0_pivots"], replay["lam0_skipped"])
    ch0, hat0, sk0 = _factor_set(S, G, remaining, fac.lam0, tau, fac, rp, slack, null_test, tag="lambda0",
                                 symmetric=symmetric)
    fac.lam0_pivots = ch0
    fac.lam0_skipped = sk0
    # R13: move the last n entries of the elimination order into hat-Lambda_0.  They are
    # the last entries of tilde-Lambda_0 whenever it holds n or more of them.
    order = np.concatenate([*fac.node_pivots, ch0]).astype(np.int64)
    nmove = min(n_enlarge, len(order))
    fac.moved = order[len(order) - nmove:]
    fac.lambda2 = np.sort(np.concatenate([hat0, fac.moved]))         # R4
    fac.lambda1_order = order[:len(order) - nmove]
    return fac


# ---------------------------------------------------------------------------
# Sec. 3.1-3.2: the lower-precision solve Q^-1 used as preconditioner
# ---------------------------------------------------------------------------
def precond_apply(fac: FactorResult, R: np.ndarray) -> np.ndarray:
    """e = Q^-1 r: cast r to float32, solve L D U e = r with the float32 factor of K11, cast back.

    The factor of K11 in the order Pi_1 is the recorded factor restricted to
    Lambda_1 rows and columns (Eq. 1 with the leading block).  Rows of
    Lambda_2 are zero on input and output.
    """
    L = R.shape[0]
    in1 = np.ones(L, dtype=bool)
    in1[fac.lambda2] = False
    dt = np.asarray(next(iter(fac.d.values()))).dtype if fac.d else np.float32
    y = np.array(R, dtype=dt, copy=True).reshape(L, -1)
    y[~in1] = 0
    order = fac.lambda1_order
    for p in order:                                   # forward, unit lower triangular
        rows, l = fac.lcol[int(p)]
        keep = in1[rows]
        y[rows[keep]] -= np.outer(l[keep], y[p])
    for p in order:                                   # diagonal
        y[p] /= fac.d[int(p)]
    for p in order[::-1]:                             # backward, unit upper triangular U
        rows, u = fac.urow[int(p)]
        keep = in1[rows]
        y[p] -= u[keep] @ y[rows[keep]]
    return y.astype(np.float64).reshape(R.shape)


def k11_operator(K: sp.csr_matrix, lambda2: np.ndarray):
    """v -> K11 v in the full index space: rows and columns of Lambda_2 masked to zero."""
    L = K.shape[0]
    in1 = np.ones(L, dtype=bool)
    in1[lambda2] = False
    D1 = sp.diags(in1.astype(np.float64))
    K11 = (D1 @ K @ D1).tocsr()
    return lambda V: K11 @ V


# ---------------------------------------------------------------------------
# Sec. 3.4 Alg. 4 (single rhs) and Sec. 3.5 "Algorithm 5" (block GCR)
# ---------------------------------------------------------------------------
def iterative_refinement(A, Qinv, B, tol=1e-14, maxit=50):
    """Iterative refinement, Alg. 3 (Sec. 3.3), on the columns of B at once.

    Steps 1-2: x_0 = Q^-1 b (the lower-precision solve, here the operator Qinv);
    step 3: r_0 = b - A x_0; step 4: e_n = Q^-1 r_n, x_{n+1} = x_n + e_n,
    r_{n+1} = b - A x_{n+1} (the true residual, FP64), until max_k |r_k|/|b_k| <= tol.
    Returns (X, history of max column relative residuals, hist[0] for x_0).
    """
    X = Qinv(B)
    nb = np.linalg.norm(B, axis=0)
    nb[nb == 0] = 1.0
    hist = []
    for n in range(maxit + 1):
        R = B - A(X)
        hist.append(float(np.max(np.linalg.norm(R, axis=0) / nb)))
        if hist[-1] <= tol or n == maxit:
            break
        X = X + Qinv(R)
    return X, hist


def gcr_single(A, Qinv, b, tol=1e-14, maxit=100):
    """Right-preconditioned GCR, Alg. 4, keeping q = A p by recurrence (R6)."""
    x = Qinv(b)
    r = b - A(x)
    w = Qinv(r)
    p, q = [w], [A(w)]
    nb = np.linalg.norm(b)
    hist = [np.linalg.norm(r) / nb]
    for n in range(maxit):
        qn = q[n]
        alpha = (r @ qn) / (qn @ qn)
        x = x + alpha * p[n]
        r = r - alpha * qn
        hist.append(np.linalg.norm(r) / nb)
        if hist[-1] <= tol:
            break
        w = Qinv(r)
        z = A(w)
        pn, qn1 = w.copy(), z.copy()
        for m in range(n + 1):
            beta = -(z @ q[m]) / (q[m] @ q[m])
            pn += beta * p[m]
            qn1 += beta * q[m]
        p.append(pn)
        q.append(qn1)
    return x, hist, p, q


def block_gcr(A, Qinv, B, tol=1e-14, maxit=50, rcond=1e-15):
    """Right-preconditioned block GCR for A X = B, M right-hand sides (Sec. 3.5, R7, R8).

    M_n = Q_n^T Q_n, A_n = Q_n^T R_n, X_{n+1} = X_n + P_n M_n^-1 A_n,
    R_{n+1} = R_n - Q_n M_n^-1 A_n, B_mn = -Q_m^T Z_{n+1},
    P_{n+1} = W_{n+1} + sum_m P_m M_m^-1 B_mn,  Q_{n+1} = Z_{n+1} + sum_m Q_m M_m^-1 B_mn.
    M_n^-1 is applied by least squares so a rank-deficient M_n (converged
    columns) does not break the iteration.
    Returns (X, history of max column relative residuals, P list, Q list).
    """
    X = Qinv(B)
    R = B - A(X)
    W = Qinv(R)
    P, Qs, Ms = [W], [A(W)], []
    nb = np.linalg.norm(B, axis=0)
    nb[nb == 0] = 1.0
    hist = [float(np.max(np.linalg.norm(R, axis=0) / nb))]

    def msolve(Mm, Y):
        return np.linalg.lstsq(Mm, Y, rcond=rcond)[0]

    for n in range(maxit):
        Mn = Qs[n].T @ Qs[n]
        Ms.append(Mn)
        An = Qs[n].T @ R
        C = msolve(Mn, An)
        X = X + P[n] @ C
        R = R - Qs[n] @ C
        hist.append(float(np.max(np.linalg.norm(R, axis=0) / nb)))
        if hist[-1] <= tol:
            break
        W = Qinv(R)
        Z = A(W)
        Pn, Qn = W.copy(), Z.copy()
        for m in range(n + 1):
            G = msolve(Ms[m], -(Qs[m].T @ Z))
            Pn += P[m] @ G
            Qn += Qs[m] @ G
        P.append(Pn)
        Qs.append(Qn)
    return X, hist, P, Qs


# ---------------------------------------------------------------------------
# Alg. 1 steps 2-4: K12 block, X12 and the Schur complement (Eq. 2)
# ---------------------------------------------------------------------------
def _blocks(K: sp.csr_matrix, lambda2):
    L = K.shape[0]
    in1 = np.ones(L, dtype=bool)
    in1[lambda2] = False
    lam1 = np.flatnonzero(in1)
    K = K.tocsr()
    return lam1, K[lam1][:, lam1].tocsc(), K[lam1][:, lambda2], K[lambda2][:, lam1], K[lambda2][:, lambda2]


def x12_direct(K: sp.csr_matrix, lambda2):
    """X12 = K11^-1 K12 by a direct FP64 sparse LU (the plain definition of Alg. 1 step 3)."""
    lam1, K11, K12, _, _ = _blocks(K, lambda2)
    X = np.zeros((K.shape[0], len(lambda2)))
    if len(lambda2):
        lu = spla.splu(K11)
        X[lam1] = lu.solve(K12.toarray())
    return X


def schur_direct(K: sp.csr_matrix, lambda2, X12=None):
    """S22 = K22 - K21 K11^-1 K12 in FP64 (Eq. 2 / Alg. 1 step 4)."""
    lam1, _, _, K21, K22 = _blocks(K, lambda2)
    if X12 is None:
        X12 = x12_direct(K, lambda2)
    return K22.toarray() - K21 @ X12[lam1]


# ---------------------------------------------------------------------------
# Alg. 1 step 5: higher-precision symmetric factorization of S22 with 2x2 pivots
# ---------------------------------------------------------------------------
def bunch_parlett(A):
    """Symmetric LDL^T with complete (Bunch-Parlett) pivoting, alpha = (1+sqrt 17)/8 (R11).

    At each step, over the remaining block: mu0 = max |a_ii|, mu1 = max_{i>j} |a_ij|
    (ties: smallest index; off-diagonal ties: smallest column, then row).  If
    mu0 >= alpha mu1 the largest diagonal is a 1x1 pivot, otherwise the largest
    off-diagonal pair (i, j) forms a 2x2 pivot.
    Returns (perm, Lf, blocks): P^T A P = Lf D Lf^T, row i of the factor = row perm[i] of A.
    """
    A = np.array(A, dtype=np.float64, copy=True)
    n = A.shape[0]
    alpha = (1.0 + math.sqrt(17.0)) / 8.0
    perm = np.arange(n)
    Lf = np.eye(n)
    blocks = []

    def swap(i, j):
        if i == j:
            return
        A[[i, j], :] = A[[j, i], :]
        A[:, [i, j]] = A[:, [j, i]]
        Lf[[i, j], :i] = Lf[[j, i], :i]
        perm[[i, j]] = perm[[j, i]]

    k = 0
    while k < n:
        dgs = np.abs(np.diag(A)[k:])
        i0 = int(np.argmax(dgs))
        mu0 = dgs[i0]
        mu1, bi, bj = 0.0, -1, -1
        for j in range(k, n):                     # column-major scan of the strict lower triangle
            if j + 1 < n:
                colv = np.abs(A[j + 1:, j])
                r = int(np.argmax(colv))
                if colv[r] > mu1:
                    mu1, bi, bj = colv[r], j + 1 + r, j
        if mu0 == 0.0 and mu1 == 0.0:
            blocks.append((k, 1, np.array([[0.0]])))
            k += 1
            continue
        if mu0 >= alpha * mu1:
            swap(k, k + i0)
            d = A[k, k]
            l = A[k + 1:, k] / d
            A[k + 1:, k + 1:] -= np.outer(l, A[k + 1:, k])
            Lf[k + 1:, k] = l
            blocks.append((k, 1, np.array([[d]])))
            k += 1
        else:
            swap(k, bj)
            swap(k + 1, bi)
            D = A[k:k + 2, k:k + 2].copy()
            C = A[k + 2:, k:k + 2]
            l = np.linalg.solve(D, C.T).T
            A[k + 2:, k + 2:] -= l @ C.T
            Lf[k + 2:, k:k + 2] = l
            blocks.append((k, 2, D))
            k += 2
    return perm, Lf, blocks


def bunch_kaufman(A):
    """Textbook Bunch-Kaufman LDL^T (partial pivoting), kept to pin the block formulas."""
    A = np.array(A, dtype=np.float64, copy=True)
    n = A.shape[0]
    alpha = (1.0 + math.sqrt(17.0)) / 8.0
    perm = np.arange(n)
    Lf = np.eye(n)
    blocks = []

    def swap(i, j):
        if i == j:
            return
        A[[i, j], :] = A[[j, i], :]
        A[:, [i, j]] = A[:, [j, i]]
        Lf[[i, j], :i] = Lf[[j, i], :i]
        perm[[i, j]] = perm[[j, i]]

    k = 0
    while k < n:
        akk = abs(A[k, k])
        if k + 1 < n:
            col = np.abs(A[k + 1:, k])
            r = k + 1 + int(np.argmax(col))
            lam = col.max()
        else:
            r, lam = k, 0.0
        size = 1
        if max(akk, lam) == 0.0:
            pass
        elif akk >= alpha * lam:
            pass
        else:
            offr = np.abs(np.concatenate([A[r, k:r], A[r + 1:, r]]))
            sigma = offr.max() if offr.size else 0.0
            if akk * sigma >= alpha * lam * lam:
                pass
            elif abs(A[r, r]) >= alpha * sigma:
                swap(k, r)
            else:
                swap(k + 1, r)
                size = 2
        if size == 1:
            d = A[k, k]
            if d != 0.0:
                l = A[k + 1:, k] / d
                A[k + 1:, k + 1:] -= np.outer(l, A[k + 1:, k])
                Lf[k + 1:, k] = l
            blocks.append((k, 1, np.array([[d]])))
            k += 1
        else:
            D = A[k:k + 2, k:k + 2].copy()
            C = A[k + 2:, k:k + 2]
            l = np.linalg.solve(D, C.T).T
            A[k + 2:, k + 2:] -= l @ C.T
            Lf[k + 2:, k:k + 2] = l
            blocks.append((k, 2, D))
            k += 2
    return perm, Lf, blocks


def bk_reconstruct(perm, Lf, blocks):
    """A = P Lf D Lf^T P^T from the factors of bunch_parlett / bunch_kaufman."""
    n = len(perm)
    D = np.zeros((n, n))
    for s, z, B in blocks:
        D[s:s + z, s:s + z] = B
    Ap = Lf @ D @ Lf.T
    A = np.empty_like(Ap)
    A[np.ix_(perm, perm)] = Ap
    return A


def pivot_magnitudes(blocks):
    """|pivot| per 1x1 block and |eigenvalues| per 2x2 block, with (block, slot) owners."""
    mags, owners = [], []
    for b, (s, z, B) in enumerate(blocks):
        if z == 1:
            mags.append(abs(B[0, 0])); owners.append((b, 0))
        else:
            ev = np.linalg.eigvalsh(B)
            for t in range(2):
                mags.append(abs(ev[t])); owners.append((b, t))
    return np.array(mags), owners


def kernel_dimension(mags, kernel_eps=1e-10, gap_min=1e4, ref=0.0, noise=0.0):
    """R10: the tail after the largest ratio gap >= gap_min whose tail is <= the null threshold.

    threshold = max(kernel_eps * scale, noise) with scale = max(max pivot magnitude, ref);
    ref is max |diag(K22)| of the scaled K (1 unless every hard index has a zero
    diagonal): S22 is a difference of O(1) terms, so its null pivots are small
    relative to the unit diagonal even when S22 itself is small.  ``noise`` is an
    estimate of the error of S22 (100 |K21 Q^-1 (K12 - K11 X12)|_max for an
    iterative X12): pivots at or below it cannot be told from zero.
    """
    if len(mags) == 0:
        return 0
    s = np.sort(np.asarray(mags))[::-1]
    scale = max(s[0], ref)
    if scale == 0:
        return len(s)
    thr = max(kernel_eps * scale, noise)
    best, dim = 0.0, 0
    for i in range(0 if s[0] <= thr else 1, len(s)):
        if s[i] > thr:
            continue
        if i == 0:                                 # every pivot is null relative to the unit scale
            return len(s)
        ratio = math.inf if s[i] == 0 else s[i - 1] / s[i]
        if ratio >= gap_min and ratio > best:
            best, dim = ratio, len(s) - i
    return dim


def bk_solve(perm, Lf, blocks, y, kdim):
    # (works for the factors of bunch_parlett and bunch_kaufman alike)
    """x = S^+ y with the kdim smallest pivot magnitudes treated as zero (kernel pivots)."""
    n = len(perm)
    mags, owners = pivot_magnitudes(blocks)
    zero = set(owners[i] for i in np.argsort(mags)[:kdim]) if kdim else set()
    y = np.asarray(y, dtype=np.float64).reshape(n, -1)
    z = np.linalg.solve(Lf, y[perm])
    for b, (s, sz, B) in enumerate(blocks):
        if sz == 1:
            z[s] = 0.0 if (b, 0) in zero or B[0, 0] == 0 else z[s] / B[0, 0]
        else:
            ev, V = np.linalg.eigh(B)
            inv = np.array([0.0 if ((b, t) in zero or ev[t] == 0) else 1.0 / ev[t] for t in range(2)])
            z[s:s + 2] = V @ (inv[:, None] * (V.T @ z[s:s + 2]))
    w = np.linalg.solve(Lf.T, z)
    x = np.empty_like(w)
    x[perm] = w
    return x


def lu_complete(A):
    """Gaussian elimination with complete pivoting, A[prow][:, pcol] = Lf U (R15).

    Each step takes the entry of largest magnitude of the remaining block (ties:
    smallest column, then smallest row) and moves it to the diagonal by one row and
    one column interchange.  A remaining block that is exactly zero ends the
    elimination (its pivots are zero).
    Returns (prow, pcol, Lf, U): row i of the factor is row prow[i] of A and
    column j is column pcol[j] of A; Lf is unit lower and U upper triangular.
    """
    A = np.array(A, dtype=np.float64, copy=True)
    n = A.shape[0]
    prow, pcol = np.arange(n), np.arange(n)
    Lf = np.eye(n)
    for k in range(n):
        j, i = divmod(int(np.argmax(np.abs(A[k:, k:]).T)), n - k)   # column by column
        i, j = i + k, j + k
        A[[k, i], :] = A[[i, k], :]
        Lf[[k, i], :k] = Lf[[i, k], :k]
        prow[[k, i]] = prow[[i, k]]
        A[:, [k, j]] = A[:, [j, k]]
        pcol[[k, j]] = pcol[[j, k]]
        d = A[k, k]
        if d == 0.0:
            break
        l = A[k + 1:, k] / d
        A[k + 1:, k + 1:] -= np.outer(l, A[k, k + 1:])
        A[k + 1:, k] = 0.0
        Lf[k + 1:, k] = l
    return prow, pcol, Lf, np.triu(A)


def lu_reconstruct(prow, pcol, Lf, U):
    """A from the factors of lu_complete."""
    A = np.empty_like(U)
    A[np.ix_(prow, pcol)] = Lf @ U
    return A


def lu_pseudo_solve(prow, pcol, Lf, U, y, kdim):
    """x with A x = y on the image, the kdim smallest |u_kk| treated as zero (kernel pivots)."""
    n = len(prow)
    y = np.asarray(y, dtype=np.float64).reshape(n, -1)
    z = np.linalg.solve(Lf, y[prow])
    zero = set(np.argsort(np.abs(np.diag(U)))[:kdim].tolist()) if kdim else set()
    w = np.zeros_like(z)
    for k in range(n - 1, -1, -1):
        if k in zero or U[k, k] == 0.0:
            continue
        w[k] = (z[k] - U[k, k + 1:] @ w[k + 1:]) / U[k, k]
    x = np.empty_like(w)
    x[pcol] = w
    return x


# ---------------------------------------------------------------------------
# Alg. 2: forward / backward substitution of the hybrid factorization
# ---------------------------------------------------------------------------
def hybrid_solve(K: sp.csr_matrix, lambda2, X12, bk, kdim, b):
    """Alg. 2 in the scaled space: y1 = K11^-1 b1, y2 = b2 - K21 y1, S22 x2 = y2, x1 = y1 - X12 x2."""
    lam1, K11, _, K21, _ = _blocks(K, lambda2)
    b = np.asarray(b, dtype=np.float64).reshape(K.shape[0], -1)
    x = np.zeros_like(b)
    y1 = spla.splu(K11).solve(b[lam1]) if len(lam1) else np.zeros((0, b.shape[1]))
    y2 = b[lambda2] - K21 @ y1
    if not len(lambda2):
        x2 = y2
    elif len(bk) == 4:                            # lu_complete factors of an unsymmetric S22
        x2 = lu_pseudo_solve(*bk, y2, kdim)
    else:
        x2 = bk_solve(*bk, y2, kdim)
    x[lam1] = y1 - X12[lam1] @ x2
    x[lambda2] = x2
    return x


def relative_residual(Kbar: sp.csr_matrix, x, b):
    """|K-bar x - b|_2 / |b|_2 per column (max over columns)."""
    r = Kbar @ x - b
    return float(np.max(np.linalg.norm(r, axis=0) / np.linalg.norm(b, axis=0)))


def backward_error(Kbar: sp.csr_matrix, x, b):
    """Normwise backward error |K-bar x - b|_inf / (|K-bar|_inf |x|_inf + |b|_inf), max over columns."""
    x = np.asarray(x).reshape(Kbar.shape[0], -1)
    b = np.asarray(b).reshape(Kbar.shape[0], -1)
    r = Kbar @ x - b
    nK = float(abs(Kbar).sum(axis=1).max())
    out = []
    for j in range(x.shape[1]):
        out.append(np.abs(r[:, j]).max() / (nK * np.abs(x[:, j]).max() + np.abs(b[:, j]).max()))
    return float(max(out))


def run_hybrid(Kbar: sp.csr_matrix, nodes, tau, n_enlarge=4, replay=None, kernel_eps=1e-10,
               gap_min=1e4, use_gcr=False, gcr_tol=1e-14, gcr_maxit=50, dtype=np.float32,
               null_test=False):
    """Alg. 1 end to end: scale, threshold factorization, X12, S22, its dense factor, kernel dim.

    S22 is factorized by Bunch-Parlett (R11) when K-bar is symmetric and by LU with
    complete pivoting (R15) otherwise.
    """
    q, K = scale_matrix(Kbar)
    fac = threshold_factorize(K, nodes, tau, n_enlarge, replay, dtype=dtype, null_test=null_test)
    if use_gcr and fac.M:
        lam1, _, K12, _, _ = _blocks(K, fac.lambda2)
        B = np.zeros((K.shape[0], fac.M))
        B[lam1] = K12.toarray()
        X12, hist, _, _ = block_gcr(k11_operator(K, fac.lambda2), lambda R: precond_apply(fac, R),
                                    B, gcr_tol, gcr_maxit)
    else:
        X12, hist = x12_direct(K, fac.lambda2), None
    S22 = schur_direct(K, fac.lambda2, X12)
    noise = s22_noise(K, fac, X12) if (use_gcr and fac.M) else 0.0
    symmetric = _symmetric(Kbar)
    if not fac.M:
        bk, mags = (np.zeros(0, int), np.zeros((0, 0)), []), np.zeros(0)
    elif symmetric:
        bk = bunch_parlett(S22)
        mags = pivot_magnitudes(bk[2])[0]
    else:
        bk = lu_complete(S22)
        mags = np.abs(np.diag(bk[3]))
    ref = float(np.abs(K.diagonal()[fac.lambda2]).max()) if fac.M else 0.0
    kdim = kernel_dimension(mags, kernel_eps, gap_min, ref, noise) if fac.M else 0
    return dict(q=q, K=K, fac=fac, X12=X12, S22=S22, bk=bk, kdim=kdim, gcr_hist=hist, noise=noise)


def s22_noise(K: sp.csr_matrix, fac: FactorResult, X12, factor=100.0):
    """Error estimate of S22 = K22 - K21 X12 for an iterative X12 (used by R10).

    The error of X12 is K11^-1 R with R = K12 - K11 X12; the preconditioner
    stands in for K11^-1, so E = K21 Q^-1 R and the estimate is factor * max|E|.
    """
    lam1, _, K12, K21, _ = _blocks(K, fac.lambda2)
    B = np.zeros((K.shape[0], fac.M))
    B[lam1] = K12.toarray()
    R = B - k11_operator(K, fac.lambda2)(X12)
    W = precond_apply(fac, R)
    return factor * float(np.abs(K21 @ W[lam1]).max())


# ---------------------------------------------------------------------------
# Adjoint (diffusion with per-cell log coefficient theta): dJ/dtheta
# ---------------------------------------------------------------------------
def diffusion_objective(x, x_star):
    """J = 1/2 |x - x*|^2."""
    return 0.5 * float(np.sum((x - x_star) ** 2))


def adjoint_gradient(nx, ny, theta, x, lam, dirichlet_x=True):
    """dJ/dtheta for K-bar(theta) x = b, J = 1/2|x - x*|^2, with lam = K-bar^-T (x - x*).

    dJ/dtheta_c = -lam^T (dK-bar/dtheta_c) x.  A face (a, b) with
    transmissibility t = 2 k_a k_b / (k_a + k_b), k = exp(theta), contributes
    t (u_a - u_b)(v_a - v_b) to u^T K-bar v and dt/dtheta_a = 2 k_a k_b^2 / (k_a + k_b)^2.
    A Dirichlet ghost face of cell c contributes 2 k_c u_c v_c.
    """
    k = np.exp(np.asarray(theta, dtype=np.float64)).reshape(ny, nx)
    X = np.asarray(x).reshape(ny, nx)
    Lm = np.asarray(lam).reshape(ny, nx)
    g = np.zeros((ny, nx))
    for axis in (1, 0):
        if axis == 1:
            ka, kb = k[:, :-1], k[:, 1:]
            dx, dl = X[:, :-1] - X[:, 1:], Lm[:, :-1] - Lm[:, 1:]
        else:
            ka, kb = k[:-1, :], k[1:, :]
            dx, dl = X[:-1, :] - X[1:, :], Lm[:-1, :] - Lm[1:, :]
        s = (ka + kb) ** 2
        da = 2 * ka * kb * kb / s
        db = 2 * kb * ka * ka / s
        prod = dx * dl
        if axis == 1:
            g[:, :-1] -= da * prod
            g[:, 1:] -= db * prod
        else:
            g[:-1, :] -= da * prod
            g[1:, :] -= db * prod
    if dirichlet_x:
        g[:, 0] -= 2 * k[:, 0] * X[:, 0] * Lm[:, 0]
        g[:, -1] -= 2 * k[:, -1] * X[:, -1] * Lm[:, -1]
    return g.ravel()
