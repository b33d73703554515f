"""Time the batched form against the same systems one at a time.

    python -m paper_2208_01907_gb300.run_batched --count 96

builds the seeded batch of independent 2D systems (diffusion with islands and mixed
Darcy, L uniform in [2k, 60k]), and times factorize + schur (+ solve with 8 right-hand
sides) for all of them (a) one context after another on one stream and (b) through
hf_factorize_batched / hf_schur_batched / hf_solve_batched.  Prints one JSON line.
"""
import argparse
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--count", type=int, default=96)
    ap.add_argument("--lmin", type=int, default=2000)
    ap.add_argument("--lmax", type=int, default=60000)
    ap.add_argument("--nrhs", type=int, default=8)
    ap.add_argument("--reps", type=int, default=2)
    args = ap.parse_args()
    import torch
    import paper_2208_01907_gb300 as hf
    from workloads import batched_systems, consistent_rhs

    systems = batched_systems(count=args.count, Lmin=args.lmin, Lmax=args.lmax, seed=4)
    vals = [torch.tensor(s.val, device="cuda", dtype=torch.float64) for s in systems]
    bs = [torch.tensor(np.ascontiguousarray(consistent_rhs(s, 100 + i, args.nrhs, "uniform").T), device="cuda")
          for i, s in enumerate(systems)]
    xs = [torch.zeros_like(b) for b in bs]
    # saddle-point systems (mixed Darcy) with the null-pivot test, the others with the ratio
    # test of Sec. 2.2 alone
    nt = [int(bool(s.meta.get("saddle_point"))) for s in systems]
    one = [hf.HybridFactor(s.L, s.rowptr, s.col, s.coords, null_test=n) for s, n in zip(systems, nt)]
    bat = [hf.HybridFactor(s.L, s.rowptr, s.col, s.coords, null_test=n) for s, n in zip(systems, nt)]

    def run_one():
        for H, v, b, x in zip(one, vals, bs, xs):
            H.factorize(v, 1e-2)
            H.schur()
            H.solve(b, x)

    def run_batched():
        hf.factorize_batched(bat, vals, 1e-2)
        hf.schur_batched(bat)
        hf.solve_batched(bat, bs, xs)

    world = int(os.environ.get("WORLD_SIZE", "1"))
    if world > 1:
        # one process per GPU (torchrun): LPT shares of the systems, no collective in the
        # data path, results gathered on rank 0 (paper_2208_01907_gb300.shard)
        import torch.distributed as dist
        from paper_2208_01907_gb300.shard import estimated_cost, run_sharded
        rank = int(os.environ["RANK"])
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        dist.init_process_group("nccl")
        costs = [estimated_cost(s.L) for s in systems]

        def share(idx):
            hs = [bat[i] for i in idx]
            hf.factorize_batched(hs, [vals[i] for i in idx], 1e-2)
            hf.schur_batched(hs)
            hf.solve_batched(hs, [bs[i] for i in idx], [xs[i] for i in idx])
            return {i: int(bat[i].info()["M"]) for i in idx}

        dist.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        Ms = run_sharded(len(systems), costs, share, rank, world)
        torch.cuda.synchronize()
        dist.barrier()
        dt = time.perf_counter() - t0
        if rank == 0:
            print(json.dumps({"workload": f"batched_{args.count}_2d_L{args.lmin}-{args.lmax}_nrhs{args.nrhs}",
                              "systems": args.count, "n_gpus": world, "ms": dt * 1e3,
                              "systems_per_s": args.count / dt, "M_total": int(sum(Ms))}))
        dist.destroy_process_group()
        return

    res = {}
    for name, fn in (("one_by_one", run_one), ("batched", run_batched)):
        fn()                                   # warm-up (allocations, delayed-row capacity)
        torch.cuda.synchronize()
        t = []
        for _ in range(args.reps):
            t0 = time.perf_counter()
            fn()
            torch.cuda.synchronize()
            t.append(time.perf_counter() - t0)
        res[name] = min(t) * 1e3
    Ls = [s.L for s in systems]
    print(json.dumps({"workload": f"batched_{args.count}_2d_L{args.lmin}-{args.lmax}_nrhs{args.nrhs}",
                      "systems": args.count, "sum_L": int(sum(Ls)), "ms_one_by_one": res["one_by_one"],
                      "ms_batched": res["batched"], "speedup": res["one_by_one"] / res["batched"],
                      "systems_per_s": args.count / (res["batched"] / 1e3),
                      "M_total": int(sum(H.info()["M"] for H in bat))}))


if __name__ == "__main__":
    main()
