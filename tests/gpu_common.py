"""Helpers shared by the GPU tests: run the C ABI on a system, replay it in the oracle."""
from __future__ import annotations

import numpy as np

import oracle as O


def run_gpu(system, tau=1e-2, nrhs=1, rhs_seed=3, rhs_mode="uniform", solve=True, **opts):
    import torch
    import paper_2208_01907_gb300 as hf
    from workloads import consistent_rhs

    H = hf.HybridFactor(system.L, system.rowptr, system.col, system.coords, **opts)
    vals = torch.tensor(system.val, device="cuda", dtype=torch.float64)
    H.factorize(vals, tau)
    rc = H.schur()
    out = dict(H=H, schur_rc=rc, info=H.info())
    if solve:
        b = consistent_rhs(system, rhs_seed, nrhs, rhs_mode)
        bt = torch.tensor(np.ascontiguousarray(b.T), device="cuda")
        xt = torch.zeros_like(bt)
        out["solve_rc"] = H.solve(bt, xt)
        out["b"] = b
        out["x"] = xt.cpu().numpy().T.copy()
    out["info"] = H.info()
    return out


def replay(system, H, tau, n_enlarge=4, slack=1e-4, dtype=np.float32, null_test=None):
    """Oracle factorization on the GPU's tree, following the GPU's pivot decisions, under the
    rule the context ran with (the ratio test of Sec. 2.2, plus R3b if H asked for it)."""
    if null_test is None:
        null_test = bool(H.opts.null_test)
    _, sets = H.tree()
    ev = H.pivot_events()
    _, _, moved = H.pivots()
    q, K = O.scale_matrix(system.to_scipy())
    rp = {"node_pivots": [e[0] for e in ev[:-1]], "node_skipped": [e[2] for e in ev[:-1]],
          "lam0_pivots": ev[-1][0], "lam0_skipped": ev[-1][2]}
    fac = O.threshold_factorize(K, sets, tau, n_enlarge, replay=rp, slack=slack, dtype=dtype, null_test=null_test)
    return q, K, fac, moved


def rel_fro(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def project_out(v, V):
    if V is None or V.shape[1] == 0:
        return v
    return v - V @ np.linalg.lstsq(V, v, rcond=None)[0]
