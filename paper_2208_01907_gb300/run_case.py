"""Run the hybrid factorization once on a seeded synthetic system (for profilers).

    python -m paper_2208_01907_gb300.run_case --n 32 --phase schur

builds the 3D Stokes-like system of the benchmark at n^3 nodes, runs `factorize`
(twice with --warm, so that the delayed-row capacity has settled), then `schur` and
`solve` as requested by --phase, and prints one line.  Nothing is timed here; the
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
    ap.add_argument("--phase", choices=["factorize", "schur", "solve"], default="schur")
    ap.add_argument("--warm", action="store_true", help="factorize twice before the measured phases")
    ap.add_argument("--fp64-gemm", type=int, default=0)
    args = ap.parse_args()
    import torch
    import paper_2208_01907_gb300 as hf
    from workloads import stokes3d, consistent_rhs

    s = stokes3d(args.n, seed=2)
    H = hf.HybridFactor(s.L, s.rowptr, s.col, s.coords, fp64_gemm=args.fp64_gemm)
    vals = torch.tensor(s.val, device="cuda", dtype=torch.float64)
    if args.warm:
        H.factorize(vals, 1e-2)
    H.factorize(vals, 1e-2)
    if args.phase in ("schur", "solve"):
        H.schur()
    if args.phase == "solve":
        b = consistent_rhs(s, 11, 1, "solution")
        bt = torch.tensor(np.ascontiguousarray(b.T), device="cuda")
        xt = torch.zeros_like(bt)
        H.solve(bt, xt)
    torch.cuda.synchronize()
    i = H.info()
    print(f"run_case n={args.n} L={i['L']} M={i['M']} gcr_iters={i['gcr_iters']} kernel_dim={i['kernel_dim']}")


if __name__ == "__main__":
    main()
