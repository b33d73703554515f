"""Run the hybrid factorization once on a seeded synthetic system (for profilers).

    python -m paper_2208_01907_gb300.run_case --n 32 --phase schur

builds the 3D Stokes-like system (or with --workload elasticity the Q1 elasticity system
of the benchmark) at n^3 nodes, runs `factorize`
(twice with --warm, so that the delayed-row capacity has settled), then `schur` and
`solve` as requested by --phase, and prints one line.  --phase gram / update runs one
block-GCR product (hf_gram_fp64 / hf_update_fp64) on seeded L x m operands instead;
--phase iterate compares iterative refinement, GCR per column and block GCR on K11
X = B (hf_k11_iterate, seeded B with --cols columns) after the factorization.  Nothing is timed here; the
point is a fixed, short sequence of launches for a kernel profiler.
"""
import argparse
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=32)
    ap.add_argument("--phase", choices=["factorize", "schur", "solve", "gram", "update", "iterate"], default="schur")
    ap.add_argument("--cols", type=int, default=16, help="right-hand sides of --phase iterate")
    ap.add_argument("--m", type=int, default=388, help="columns of the gram / update operands")
    ap.add_argument("--warm", action="store_true", help="factorize twice before the measured phases")
    ap.add_argument("--fp64-gemm", type=int, default=0)
    ap.add_argument("--workload", choices=["stokes", "elasticity"], default="stokes",
                    help="Stokes-like saddle point (null-pivot test) or Q1 elasticity (ratio test alone)")
    args = ap.parse_args()
    import torch
    import paper_2208_01907_gb300 as hf
    from workloads import stokes3d, elasticity3d, consistent_rhs

    if args.phase in ("gram", "update"):
        # one product of the block GCR at the workload's shape (L of the n^3 Stokes-like
        # system, m columns), seeded operands, through the public entry points
        from workloads import diffusion2d
        s = stokes3d(args.n, seed=2)
        small = diffusion2d(12, 12, n_islands=0, seed=3)
        H = hf.HybridFactor(small.L, small.rowptr, small.col, small.coords, fp64_gemm=args.fp64_gemm)
        g = torch.Generator(device="cuda").manual_seed(1)
        A = torch.randn(s.L, args.m, device="cuda", dtype=torch.float64, generator=g)
        B = torch.randn(s.L, args.m, device="cuda", dtype=torch.float64, generator=g)
        if args.phase == "gram":
            G = torch.zeros(args.m, args.m, device="cuda", dtype=torch.float64)
            H.gram_fp64(A, B, G, 1.0)
        else:
            C = torch.randn(args.m, args.m, device="cuda", dtype=torch.float64, generator=g)
            Y = torch.zeros_like(A)
            H.update_fp64(A, C, Y, B, -1.0)
        torch.cuda.synchronize()
        print(f"run_case {args.phase} L={s.L} m={args.m}")
        return
    if args.workload == "elasticity":
        s = elasticity3d(args.n, seed=3, n_incl=min(8, args.n // 3), incl=4 if args.n >= 24 else 2)
        H = hf.HybridFactor(s.L, s.rowptr, s.col, s.coords, fp64_gemm=args.fp64_gemm)
    else:
        s = stokes3d(args.n, seed=2)
        H = hf.HybridFactor(s.L, s.rowptr, s.col, s.coords, fp64_gemm=args.fp64_gemm, null_test=1)
    vals = torch.tensor(s.val, device="cuda", dtype=torch.float64)
    if args.warm:
        H.factorize(vals, 1e-2)
    H.factorize(vals, 1e-2)
    if args.phase == "iterate":
        # Alg. 3 / Alg. 4 / Alg. 5 on K11 X = B (seeded B, Lambda_2 rows zero), Fig. 2 style
        _, lam2 = H.split()
        g = torch.Generator(device="cuda").manual_seed(7)
        B = torch.randn(s.L, args.cols, device="cuda", dtype=torch.float64, generator=g)
        B[torch.as_tensor(lam2, device="cuda", dtype=torch.long)] = 0
        for method, name in ((2, "IR (Alg. 3)"), (1, "GCR per column (Alg. 4)"), (0, "block GCR (Alg. 5)")):
            X = torch.zeros_like(B)
            H.k11_iterate(method, B, X, maxit=40)                  # warm-up
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            rc, it, hist = H.k11_iterate(method, B, X, maxit=40)
            e1.record()
            torch.cuda.synchronize()
            print(f"{name:26s} cols={args.cols} rc={rc} iterations={it} time={e0.elapsed_time(e1):.1f} ms "
                  f"history={' '.join(f'{v:.2e}' for v in hist)}", flush=True)
        return
    if args.phase in ("schur", "solve"):
        H.schur()
    if args.phase == "solve":
        b = consistent_rhs(s, 11, 1, "solution")
        bt = torch.tensor(np.ascontiguousarray(b.T), device="cuda")
        xt = torch.zeros_like(bt)
        H.solve(bt, xt)
    torch.cuda.synchronize()
    i = H.info()
    launches = {k: v[1] for k, v in H.get_profile().items() if v[1]}
    print(f"run_case n={args.n} L={i['L']} M={i['M']} gcr_iters={i['gcr_iters']} kernel_dim={i['kernel_dim']} "
          f"launches={launches}")


if __name__ == "__main__":
    main()
