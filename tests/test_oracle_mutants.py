"""The oracle's pins catch plausible mistakes: each case plants one in a copy of the oracle.

A mutant is the oracle's source with one edit (a dropped term, a flipped sign, a
wrong index or operand, an off-by-one), compiled into a throwaway module on the
CPU.  The pins of tests/test_oracle_pins.py run against it with the module
swapped in, and every pin listed for the mutant must fail.  The unedited source,
compiled the same way, must pass the same pins, so a failure comes from the edit
and not from the mechanism.
"""
import os
import sys
import types

import pytest

import test_oracle_pins as pins
from workloads import diffusion2d, stokes3d

# a planted mistake may produce NaN on purpose (a square root of a negative diagonal)
pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")

SRC_PATH = os.path.join(os.path.dirname(__file__), os.pardir, "oracle", "hybrid.py")
with open(SRC_PATH) as _f:
    SRC = _f.read()


def _compile(src, tag):
    name = f"_oracle_mutant_{tag}"
    mod = types.ModuleType(name)
    mod.__file__ = SRC_PATH
    sys.modules[name] = mod                    # dataclasses look the module up by name
    try:
        exec(compile(src, f"{SRC_PATH}<{tag}>", "exec"), mod.__dict__)
    finally:
        del sys.modules[name]
    return mod


def _mutate(old, new, nth=0):
    """Replace the nth occurrence of ``old`` (which must occur) with ``new``."""
    at = -1
    for _ in range(nth + 1):
        at = SRC.find(old, at + 1)
        assert at >= 0, f"mutation target not found: {old!r}"
    return SRC[:at] + new + SRC[at + len(old):]


PINS = {
    "scaling_closed_form": pins.test_scaling_closed_form,
    "scaling_preserves_solution": pins.test_scaling_preserves_solution,
    "nd_fig1": pins.test_nd_fig1_block_pattern,
    "nd_separators": lambda: pins.test_nd_separators(lambda: stokes3d(5)),
    "hand_postponing": pins.test_hand_case_pivot_order_and_postponing,
    "hand_tie_break": pins.test_hand_case_tie_break_and_first_pivot_reference,
    "hand_ratio_previous": pins.test_hand_case_ratio_to_previous_pivot,
    "brute_force_schur": pins.test_pivot_sequence_matches_brute_force_schur,
    "eq1": pins.test_factor_reconstructs_eq1,
    "null_pivot": pins.test_null_pivot_test_skips_cancelled_pivot,
    "precond": pins.test_precond_approximates_inverse,
    "gcr_block": pins.test_block_gcr_invariants_and_solution,
    "gcr_krylov": pins.test_gcr_unpreconditioned_is_krylov_minimal_residual,
    "gcr_alg4": pins.test_block_gcr_single_rhs_equals_alg4,
    "ir_closed_form": pins.test_iterative_refinement_residuals_follow_the_closed_form,
    "schur_dense": pins.test_schur_matches_dense_inverse_and_determinant,
    "bp_reconstruct": pins.test_bunch_parlett_reconstruction_inertia_and_bound,
    "bp_rank": pins.test_bunch_parlett_is_rank_revealing,
    "bp_brute_force": pins.test_bunch_parlett_choice_matches_brute_force,
    "pivot_mags": pins.test_pivot_magnitudes_of_2x2_blocks,
    "bk_reconstruct": pins.test_bunch_kaufman_reconstruction_and_inertia,
    "bk_solve": pins.test_bunch_kaufman_solve_matches_dense,
    "kernel_svd": lambda: pins.test_kernel_dimension_matches_svd(
        lambda: diffusion2d(16, 16, n_islands=2, island=3, contrast=1e8, seed=4), 1),
    "solve_nonsingular": pins.test_hybrid_solve_exact_on_nonsingular,
    "solve_singular": pins.test_hybrid_solve_singular_consistent,
    "residual_measures": pins.test_residual_measures_closed_form,
    "s22_noise": pins.test_s22_noise_estimates_the_schur_error,
    "adjoint_fd": pins.test_adjoint_gradient_matches_central_differences,
    "ldu_eq1": pins.test_ldu_reconstructs_eq1_unsymmetric,
    "ldu_brute_force": pins.test_ldu_pivots_match_brute_force_unsymmetric_schur,
    "sign_form": pins.test_sign_form_factorizes_like_the_symmetric_matrix,
    "lu_choice": pins.test_lu_complete_reconstruction_and_pivot_choice,
    "lu_rank": pins.test_lu_complete_is_rank_revealing_and_pseudo_solves,
    "precond_unsym": pins.test_unsymmetric_precond_and_gcr,
    "solve_unsym": pins.test_unsymmetric_hybrid_solve,
    "kernel_rule": pins.test_kernel_dimension_rule_hand_cases,
    "tau_limits": pins.test_tau_limits,
}

# (id, text in the oracle, planted replacement, occurrence, pins that must fail)
MUTANTS = [
    # Sec. 2 scaling
    ("scale_no_sqrt", "q[nz] = 1.0 / np.sqrt(np.abs(d[nz]))", "q[nz] = 1.0 / np.abs(d[nz])", 0,
     ["scaling_closed_form"]),
    ("scale_one_sided", "K = (Q @ Kbar @ Q).tocsr()", "K = (Q @ Kbar).tocsr()", 0,
     ["scaling_closed_form"]),
    # Sec. 2.2 nested dissection
    ("nd_overlap", "lower = verts[c[:, ax] < med]", "lower = verts[c[:, ax] <= med]", 0, ["nd_fig1"]),
    ("nd_separator_all", "inupper[adj.indices[adj.indptr[v]:adj.indptr[v + 1]]].any()",
     "inupper[adj.indices[adj.indptr[v]:adj.indptr[v + 1]]].all()", 0, ["nd_separators", "nd_fig1"]),
    ("nd_root_first", "for lev in range(m, 0, -1)", "for lev in range(1, m + 1)", 0, ["nd_fig1"]),
    # Sec. 2.1 elimination
    ("elim_sign", "S[np.ix_(rows, rows)] -= np.outer(col, row) / d",
     "S[np.ix_(rows, rows)] += np.outer(col, row) / d", 0, ["brute_force_schur", "eq1"]),
    ("elim_l_unscaled", "fac.lcol[int(q)] = (rows, col / d)", "fac.lcol[int(q)] = (rows, col)", 0,
     ["eq1", "precond"]),
    ("null_test_not_accumulated", "G[rows] += np.abs(col * (row / d))",
     "G[rows] = np.abs(col * (row / d))", 0, ["null_pivot"]),
    ("null_test_on_by_default", "null_test: bool = False) -> FactorResult:",
     "null_test: bool = True) -> FactorResult:", 0, ["null_pivot"]),
    # Sec. 2.2 pivoting and postponing
    ("ratio_against_one", "if not (dg[t] >= tau * d_ref):", "if not (dg[t] >= tau):", 0,
     ["hand_ratio_previous"]),
    ("ratio_against_first", "        d_ref = abs(float(d))\n",
     "        d_ref = abs(float(d)) if step == 0 else d_ref\n", 0, ["hand_ratio_previous"]),
    ("ratio_carried_across_sets", "    d_ref = 1.0                                   # R2",
     "    d_ref = abs(float(fac.d[next(reversed(fac.d))])) if fac.d else 1.0  # R2", 0,
     ["hand_ratio_previous"]),
    ("tie_to_largest", "key=lambda t: (dg[t], -cand[t])", "key=lambda t: (dg[t], cand[t])", 0,
     ["hand_tie_break"]),
    ("pivot_min_diag", "best = max(range(len(cand))", "best = min(range(len(cand))", 0,
     ["brute_force_schur", "hand_postponing"]),
    ("enlarge_moves_first", "fac.moved = order[len(order) - nmove:]", "fac.moved = order[:nmove]", 0,
     ["hand_postponing"]),
    # Sec. 3.1-3.2 preconditioner
    ("precond_bwd_sign", "y[p] -= u[keep] @ y[rows[keep]]", "y[p] += u[keep] @ y[rows[keep]]", 0,
     ["precond"]),
    ("precond_diag_mul", "y[p] /= fac.d[int(p)]", "y[p] *= fac.d[int(p)]", 0, ["precond"]),
    ("precond_bwd_order", "for p in order[::-1]:", "for p in order:", 0, ["precond"]),
    # Sec. 3.3-3.5 iterations
    ("ir_no_precond", "X = X + Qinv(R)", "X = X + R", 0, ["ir_closed_form"]),
    ("ir_zero_start", "    X = Qinv(B)\n    nb = np.linalg.norm(B, axis=0)\n    nb[nb == 0] = 1.0\n    hist = []",
     "    X = 0 * B\n    nb = np.linalg.norm(B, axis=0)\n    nb[nb == 0] = 1.0\n    hist = []", 0,
     ["ir_closed_form"]),
    ("gcr_alpha_p", "alpha = (r @ qn) / (qn @ qn)", "alpha = (r @ p[n]) / (qn @ qn)", 0, ["gcr_krylov"]),
    ("gcr_beta_w", "beta = -(z @ q[m]) / (q[m] @ q[m])", "beta = -(w @ q[m]) / (q[m] @ q[m])", 0,
     ["gcr_krylov"]),
    ("bgcr_residual_with_p", "R = R - Qs[n] @ C", "R = R - P[n] @ C", 0, ["gcr_block"]),
    ("bgcr_beta_sign", "G = msolve(Ms[m], -(Qs[m].T @ Z))", "G = msolve(Ms[m], (Qs[m].T @ Z))", 0,
     ["gcr_block"]),
    ("bgcr_q_from_p", "Qn += Qs[m] @ G", "Qn += P[m] @ G", 0, ["gcr_block"]),
    # Eq. 2 Schur complement
    ("schur_sign", "return K22.toarray() - K21 @ X12[lam1]", "return K22.toarray() + K21 @ X12[lam1]", 0,
     ["schur_dense"]),
    # Alg. 1 step 5: Bunch-Parlett / Bunch-Kaufman
    ("bp_update_sign", "A[k + 1:, k + 1:] -= np.outer(l, A[k + 1:, k])",
     "A[k + 1:, k + 1:] += np.outer(l, A[k + 1:, k])", 0, ["bp_reconstruct"]),
    ("bp_swap_keeps_l", "Lf[[i, j], :i] = Lf[[j, i], :i]", "pass", 0, ["bp_reconstruct"]),
    ("bp_first_column_only", "for j in range(k, n):", "for j in range(k, k + 1):", 0, ["bp_brute_force"]),
    ("bk_2x2_transposed", "l = np.linalg.solve(D, C.T).T", "l = np.linalg.solve(D.T, C).T", 1,
     ["bk_reconstruct"]),
    ("bk_solve_transposed", "z = np.linalg.solve(Lf, y[perm])", "z = np.linalg.solve(Lf.T, y[perm])", 0,
     ["bk_solve"]),
    # R10 kernel detection
    ("kernel_gap_reversed", "if ratio >= gap_min and ratio > best:", "if ratio <= gap_min and ratio > best:", 0,
     ["kernel_svd", "bp_rank"]),
    ("kernel_off_by_one", "best, dim = ratio, len(s) - i", "best, dim = ratio, len(s) - i - 1", 0,
     ["kernel_svd", "bp_rank"]),
    ("kernel_largest_zeroed", "np.argsort(mags)[:kdim]", "np.argsort(mags)[::-1][:kdim]", 0,
     ["solve_singular"]),
    ("pivot_mags_diag", "mags.append(abs(ev[t])); owners.append((b, t))",
     "mags.append(abs(B[t, t])); owners.append((b, t))", 0, ["pivot_mags"]),
    # Alg. 2 solve
    ("solve_y2_sign", "y2 = b[lambda2] - K21 @ y1", "y2 = b[lambda2] + K21 @ y1", 0, ["solve_nonsingular"]),
    ("solve_x1_sign", "x[lam1] = y1 - X12[lam1] @ x2", "x[lam1] = y1 + X12[lam1] @ x2", 0,
     ["solve_nonsingular"]),
    # measures and the S22 error estimate
    ("backward_error_no_b", "(nK * np.abs(x[:, j]).max() + np.abs(b[:, j]).max())",
     "(nK * np.abs(x[:, j]).max())", 0, ["residual_measures"]),
    ("noise_without_precond", "W = precond_apply(fac, R)", "W = R", 0, ["s22_noise"]),
    # LDU form (U != L^T) and the unsymmetric S22 (R15)
    ("elim_row_as_column", "row = S[q, rows].copy()", "row = S[rows, q].copy()", 1,
     ["ldu_eq1", "ldu_brute_force"]),
    ("elim_u_unscaled", "fac.urow[int(q)] = (rows, row / d)", "fac.urow[int(q)] = (rows, row)", 0,
     ["ldu_eq1", "precond_unsym"]),
    ("precond_bwd_uses_l", "rows, u = fac.urow[int(p)]", "rows, u = fac.lcol[int(p)]", 0, ["precond_unsym"]),
    ("lu_column_not_swapped", "A[:, [k, j]] = A[:, [j, k]]", "pass", 0, ["lu_choice"]),
    ("lu_partial_pivoting", "j, i = divmod(int(np.argmax(np.abs(A[k:, k:]).T)), n - k)",
     "j, i = 0, int(np.argmax(np.abs(A[k:, k])))", 0, ["lu_choice"]),
    ("lu_update_uses_column", "A[k + 1:, k + 1:] -= np.outer(l, A[k, k + 1:])",
     "A[k + 1:, k + 1:] -= np.outer(l, A[k + 1:, k])", 0, ["lu_choice"]),
    ("lu_solve_row_perm", "    x[pcol] = w\n", "    x[prow] = w\n", 0, ["lu_rank"]),
    ("s22_dispatch_inverted", "    elif symmetric:\n", "    elif not symmetric:\n", 0,
     ["sign_form", "solve_unsym"]),
    # more: pattern, masks, measures, rule constants, forward solves
    ("pattern_row_for_col", "pairs = set(zip(owner[C.row].tolist(), owner[C.col].tolist()))",
     "pairs = set(zip(owner[C.row].tolist(), owner[C.row].tolist()))", 0, ["nd_fig1"]),
    ("k11_rows_not_masked", "    in1[lambda2] = False\n    D1 = sp.diags", "    D1 = sp.diags", 0, ["gcr_block"]),
    ("kernel_noise_dropped", "thr = max(kernel_eps * scale, noise)", "thr = kernel_eps * scale", 0, ["kernel_rule"]),
    ("kernel_ref_dropped", "scale = max(s[0], ref)", "scale = s[0]", 0, ["kernel_rule"]),
    ("backward_error_one_norm", "nK = float(abs(Kbar).sum(axis=1).max())", "nK = float(abs(Kbar).sum(axis=0).max())", 0,
     ["residual_measures"]),
    ("precond_fwd_sign", "y[rows[keep]] -= np.outer(l[keep], y[p])", "y[rows[keep]] += np.outer(l[keep], y[p])", 0,
     ["precond"]),
    ("enlarge_one_short", "nmove = min(n_enlarge, len(order))", "nmove = min(n_enlarge - 1, len(order))", 0,
     ["hand_postponing", "tau_limits"]),
    ("lam0_first_node_only", "lam0 = np.concatenate(fac.node_postponed) if", "lam0 = np.concatenate(fac.node_postponed[:1]) if",
     0, ["tau_limits"]),
    ("bk_sigma_test", "if akk * sigma >= alpha * lam * lam:", "if akk * sigma >= alpha * lam:", 0, ["bk_reconstruct"]),
    ("gcr_x_with_q", "x = x + alpha * p[n]", "x = x + alpha * q[n]", 0, ["gcr_alg4"]),
    ("scale_no_abs", "q[nz] = 1.0 / np.sqrt(np.abs(d[nz]))", "q[nz] = 1.0 / np.sqrt(d[nz])", 0, ["scaling_closed_form"]),
    ("solve_x2_unsolved", "    x[lambda2] = x2\n", "    x[lambda2] = y2\n", 0, ["solve_nonsingular"]),
    ("lu_zero_largest", "zero = set(np.argsort(np.abs(np.diag(U)))[:kdim].tolist())",
     "zero = set(np.argsort(np.abs(np.diag(U)))[::-1][:kdim].tolist())", 0, ["lu_rank"]),
    ("pivot_mags_signed", "mags.append(abs(B[0, 0])); owners.append((b, 0))", "mags.append(B[0, 0]); owners.append((b, 0))",
     0, ["bp_rank"]),
    ("adjoint_sign", "            g[:, :-1] -= da * prod", "            g[:, :-1] += da * prod", 0, ["adjoint_fd"]),
    # adjoint
    ("adjoint_swapped_derivative", "db = 2 * kb * ka * ka / s", "db = 2 * ka * kb * kb / s", 0, ["adjoint_fd"]),
    ("adjoint_dirichlet_half", "g[:, 0] -= 2 * k[:, 0] * X[:, 0] * Lm[:, 0]",
     "g[:, 0] -= k[:, 0] * X[:, 0] * Lm[:, 0]", 0, ["adjoint_fd"]),
]


def _run_pin(monkeypatch, mod, pin):
    monkeypatch.setattr(pins, "O", mod)
    PINS[pin]()


def test_unmutated_copy_passes_every_pin(monkeypatch):
    mod = _compile(SRC, "identity")
    for pin in PINS:
        _run_pin(monkeypatch, mod, pin)


@pytest.mark.parametrize("mid,old,new,nth,caught_by", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_is_caught(monkeypatch, mid, old, new, nth, caught_by):
    mod = _compile(_mutate(old, new, nth), mid)
    for pin in caught_by:
        with pytest.raises(Exception):
            _run_pin(monkeypatch, mod, pin)
