#!/usr/bin/env python
"""Benchmark of the hybrid factorization (Alg. 1) on GB300.

Workload: the 3D Stokes-like saddle point, 32^3 velocity nodes plus cell
pressures (L = 128,095), per-cell viscosity 10^U(-3,3), zero pressure block,
tau = 1e-2, seeded synthetic values.  One step = one pass of the whole path:
hf_factorize (scaling, FP32 factorization with postponing, Lambda_0 stage) +
hf_schur (block GCR for X12, S22, dense LDL^T) + hf_solve (Alg. 2, one rhs).
The metric is the factor + Schur time; the plain FP64 GPU form (S22 from an
FP64 factorization) is timed beside it.

Usage:  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Multi-GPU: one independent system per rank (the path does not shard).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "hybrid_factor_schur_time"
UNIT = "ms"
CONFIG_NAME = "stokes3d_32^3_mu1e-3..1e3_tau1e-2"
SAMPLE_N = 10          # oracle sample: the same generator at 10^3 nodes


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=32, help="nodes per axis of the Stokes-like grid")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--profile-print", action="store_true")
    return ap.parse_args()


# ---------------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------- CPU oracle leg
def _oracle_sample_time(n, threads=1):
    """Time the CPU oracle (Alg. 1 with block GCR) on the n^3 Stokes-like sample, in a child process."""
    code = f"""
import os, sys, time, json
sys.path.insert(0, {ROOT!r})
import numpy as np
import oracle as O
from workloads import stokes3d
s = stokes3d({n}, seed=2)
Kb = s.to_scipy()
q, K = O.scale_matrix(Kb)
m = max(1, int(np.ceil(np.log2(s.L / 512))) + 1)
sets, order = O.nested_dissection(K, s.coords, m)
t = time.perf_counter()
r = O.run_hybrid(Kb, [sets[l] for l in order], 1e-2, use_gcr=True)
el = time.perf_counter() - t
print(json.dumps(dict(seconds=el, L=s.L, M=int(r['fac'].M), kdim=int(r['kdim']))))
"""
    env = dict(os.environ)
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "NUMEXPR_NUM_THREADS"):
        env[v] = str(threads)
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=900)
    if out.returncode != 0:
        raise RuntimeError(out.stderr[-2000:])
    return json.loads(out.stdout.strip().splitlines()[-1])


def _extrapolate(seconds, L_sample, L_full):
    # 3D nested dissection: work grows as L^2 (George 1973, the ordering of Sec. 2.2)
    return seconds * (L_full / L_sample) ** 2


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from workloads import stokes3d
    L_full = stokes3d(args.n, seed=2).L if args.n <= 12 else 3 * args.n ** 3 + (args.n - 1) ** 3
    times = []
    for i in range(args.warmup + args.steps):
        r = _oracle_sample_time(SAMPLE_N)
        if i >= args.warmup:
            times.append(r["seconds"])
    t = sum(times) / len(times)
    val = _extrapolate(t, r["L"], L_full) * 1e3
    line = {
        "impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": val, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": CONFIG_NAME, "L": L_full},
        "cpu_baseline": {"value": val, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"stokes3d {SAMPLE_N}^3 (L={r['L']}), {t:.2f} s per run, "
                                   f"extrapolated by (L/L_sample)^2"},
        "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------- GPU arm
def run_ours(args):
    import numpy as np
    import torch
    import paper_2208_01907_gb300 as hf
    import scipy.sparse as sp
    from workloads import stokes3d, consistent_rhs

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev) if "device_id" in dist.init_process_group.__code__.co_varnames \
            else dist.init_process_group("nccl")

    def barrier():
        if dist is not None:
            dist.barrier()

    s = stokes3d(args.n, seed=2)
    H = hf.HybridFactor(s.L, s.rowptr, s.col, s.coords)
    vals = torch.tensor(s.val, device=dev, dtype=torch.float64)
    b = consistent_rhs(s, 11, 1, "solution")
    bt = torch.tensor(np.ascontiguousarray(b.T), device=dev)
    xt = torch.zeros_like(bt)

    def step(ev=None):
        if ev:
            ev[0].record()
        H.factorize(vals, 1e-2)
        if ev:
            ev[1].record()
        H.schur()
        if ev:
            ev[2].record()
        H.solve(bt, xt)
        if ev:
            ev[3].record()

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()
    info = H.info()
    H.profile(False)                    # counters reset; launches are counted, no events
    clocks = ClockSampler(local)
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(args.steps)]
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record()
    for k in range(args.steps):
        step(evs[k])
    t1.record()
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    total_ms = t0.elapsed_time(t1)
    launches = sum(v[1] for v in H.get_profile().values())        # launches in the timed steps
    # per-class device times from one more step with the library's event profiling on
    # (kept out of the timed steps: two event records per launch slow the host enqueue)
    H.profile(True)
    step()
    torch.cuda.synchronize()
    prof = H.get_profile()
    H.profile(False)
    prof_steps = 1
    fac = [e[0].elapsed_time(e[1]) for e in evs]
    sch = [e[1].elapsed_time(e[2]) for e in evs]
    sol = [e[2].elapsed_time(e[3]) for e in evs]
    fs_ms = (sum(fac) + sum(sch)) / args.steps
    step_ms = total_ms / args.steps
    if dist is not None:
        tt = torch.tensor([fs_ms, step_ms], device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        fs_ms, step_ms = float(tt[0]), float(tt[1])
    info = H.info()

    # accuracy gate of the timed configuration
    x = xt.cpu().numpy().T
    Kb = s.to_scipy()
    r = Kb @ x - b
    bwd = float(np.abs(r).max() / (abs(Kb).sum(axis=1).max() * np.abs(x).max() + np.abs(b).max()))
    relres = float(np.linalg.norm(r) / np.linalg.norm(b))

    # roofline of the dominant kernel class (device time from the events of the timed region,
    # algorithmic work counted by the library for exactly those launches)
    dom = max(prof, key=lambda k: prof[k][0])
    dom_ms, dom_n, dom_flops, dom_bytes = prof[dom]
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peaks = json.load(f)
    except Exception:
        pass
    hbm = peaks.get("hbm_gbs", 6800.0)
    fp32_simt = 152 * 128 * 2 * 2.07e9 / 1e12          # derived: SMs x FP32 lanes x FMA x max clock
    fp64_peak = 1.25                                    # nominal GB300 FP64 (profiling recipe table)
    bf16_sus = peaks.get("bf16_tflops_sustained", 1700.0)
    kinds = {
        "panel": ("alu", fp32_simt, "k_panel_cl (pivoted left-looking panel, cluster/DSMEM resident)",
                  "derived: 152 SMs x 128 FP32 lanes x 2 x 2.07 GHz"),
        "trailing": ("alu", fp32_simt, "k_trailing (FP32 SIMT rank-nb Schur update)",
                     "derived: 152 SMs x 128 FP32 lanes x 2 x 2.07 GHz"),
        "gram": ("tensor", bf16_sus, "k_oz_mma (FP64 Gram Q^T Z emulated: 36 BF16 slice products)",
                 "MEASURED_PEAKS.json bf16_tflops_sustained"),
        "block_update": ("tensor", bf16_sus, "k_oz_mma (FP64 update P C emulated: 36 BF16 slice products)",
                         "MEASURED_PEAKS.json bf16_tflops_sustained"),
        # with M ~ 400 right-hand sides the sweeps do 2 M flops per factor entry read: FP32 ALU-bound
        "trsv_fwd": ("alu", fp32_simt, "k_sweep_df<1> (dataflow forward sweep of a tree level, FP32)",
                     "derived: 152 SMs x 128 FP32 lanes x 2 x 2.07 GHz"),
        "trsv_bwd": ("alu", fp32_simt, "k_sweep_df<0> (dataflow backward sweep of a tree level, FP32)",
                     "derived: 152 SMs x 128 FP32 lanes x 2 x 2.07 GHz"),
        "spmm": ("hbm", hbm, "k_spmm (FP64 CSR x block)", "MEASURED_PEAKS.json hbm_gbs"),
    }
    bound, peak, kname, psrc = kinds.get(dom, ("alu", None, dom, None))
    if dom in ("gram", "block_update") and not info.get("fp64_native", False):
        dom_flops = 36.0 * dom_flops      # tensor work: 36 slice products per FP64 multiply-add
    if bound == "hbm":
        achieved = dom_bytes / (dom_ms / 1e3) / 1e9
        unit = "GB/s"
    else:
        achieved = dom_flops / (dom_ms / 1e3) / 1e12 if dom_flops else None
        unit = "TFLOP/s"
    roof = {"bound": bound, "achieved": achieved, "peak": peak, "unit": unit,
            "frac": (achieved / peak) if (achieved and peak) else None,
            "traffic": measured_traffic(kname.split(" ")[0]),
            "kernel": kname, "peak_source": psrc, "launches_per_step": dom_n / prof_steps,
            "ms_per_step": dom_ms / prof_steps}

    # end to end through the C ABI with host buffers: H2D of the values, D2H of S22
    hv = torch.tensor(s.val, dtype=torch.float64).pin_memory()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    dvals = torch.empty_like(vals)
    M = info["M"]
    hs22 = torch.empty((max(M, 1), max(M, 1)), dtype=torch.float64).pin_memory()
    torch.cuda.synchronize()
    e0.record()
    for _ in range(args.steps):
        dvals.copy_(hv, non_blocking=True)
        H.factorize(dvals, 1e-2)
        H.schur()
        hs22[:M, :M].copy_(H.s22(torch), non_blocking=True)
    e1.record()
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1) / args.steps

    # plain FP64 GPU form (Table 1 "double"): factor in FP64, S22 from the factor
    fp64 = fp32 = None
    if not args.no_fp64:
        H64 = hf.HybridFactor(s.L, s.rowptr, s.col, s.coords, precision=hf.HF_PREC_FP64)
        H64.factorize(vals, 1e-2)
        H64.schur()
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        c_ = torch.cuda.Event(enable_timing=True)
        a.record()
        H64.factorize(vals, 1e-2)
        H64.schur()
        c_.record()
        torch.cuda.synchronize()
        x64 = torch.zeros_like(bt)
        H64.solve(bt, x64)
        xx = x64.cpu().numpy().T
        rr = Kb @ xx - b
        fp64 = {"factor_schur_ms": a.elapsed_time(c_),
                "backward_error": float(np.abs(rr).max() / (abs(Kb).sum(axis=1).max() * np.abs(xx).max() + np.abs(b).max())),
                "M": H64.info()["M"], "kernel_dim": H64.info()["kernel_dim"]}
        fp64["speedup_mixed_vs_fp64"] = fp64["factor_schur_ms"] / fs_ms
        H64.free()
        # FP32-only form (Table 1 "single"): factor and S22 in FP32, no iteration; its
        # backward error shows why the hybrid form iterates in FP64
        H32 = hf.HybridFactor(s.L, s.rowptr, s.col, s.coords, precision=hf.HF_PREC_FP32)
        H32.factorize(vals, 1e-2)
        H32.schur()
        torch.cuda.synchronize()
        a.record()
        H32.factorize(vals, 1e-2)
        H32.schur()
        c_.record()
        torch.cuda.synchronize()
        x32 = torch.zeros_like(bt)
        H32.solve(bt, x32)
        xx = x32.cpu().numpy().T
        rr = Kb @ xx - b
        be32 = float(np.abs(rr).max() / (abs(Kb).sum(axis=1).max() * np.abs(xx).max() + np.abs(b).max()))
        fp32 = {"factor_schur_ms": a.elapsed_time(c_), "backward_error": be32, "gate_1e-12": bool(be32 <= 1e-12)}
        H32.free()

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        try:
            rs = _oracle_sample_time(12)
            cpu_ms = _extrapolate(rs["seconds"], rs["L"], s.L) * 1e3
            cpu = {"value": cpu_ms, "unit": UNIT, "cores": 1, "kind": "oracle",
                   "sample": f"stokes3d 12^3 (L={rs['L']}) factor+Schur by the CPU oracle in "
                             f"{rs['seconds']:.1f} s on 1 core, extrapolated by (L/L_sample)^2"}
        except Exception as e:  # noqa: BLE001
            cpu = {"value": None, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": f"failed: {e}"[:300]}

    if rank == 0:
        factor_bytes = info["nnz_factor"] * 4
        line = {
            "metric": METRIC, "value": fs_ms, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": max(3, args.warmup), "ms_per_step": step_ms, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": CONFIG_NAME, "L": s.L, "nnz": s.nnz, "M": info["M"],
                       "n_lambda0": info["n_lambda0"], "kernel_dim": info["kernel_dim"],
                       "gcr_iters": info["gcr_iters"], "levels": info["levels"],
                       "l2": "working set (factor arena %.1f GB) larger than L2" % (info["front_bytes"] / 1e9),
                       "parallelism": f"replicas x{world}"},
            "phases_ms": {"factorize": sum(fac) / args.steps, "schur": sum(sch) / args.steps,
                          "solve": sum(sol) / args.steps},
            "factor_GBps": factor_bytes / (sum(fac) / args.steps / 1e3) / 1e9,
            "systems_per_s": world * 1e3 / step_ms,
            "rel_residual": relres, "backward_error": bwd, "gate_1e-12": bwd <= 1e-12,
            "roofline": roof,
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_ms, "unit": UNIT, "h2d_bytes_per_step": s.nnz * 8,
                    "d2h_bytes_per_step": M * M * 8},
            "fp64_form": fp64,
            "fp32_form": fp32,
            "gpu_launches": launches,
            "kernel_ms": {k: round(v[0] / prof_steps, 3) for k, v in prof.items()},
            "kernel_work": kernel_work(prof, prof_steps),
            "clocks": clk,
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def kernel_work(prof, steps):
    """Per kernel class: algorithmic GFLOP and GB per step and the rates they give over the
    class's measured time.  prof maps a class to (ms, launches, flops, bytes) summed over
    `steps` steps; classes with no counted work are left out."""
    out = {}
    for k, v in prof.items():
        ms, flops, nbytes = v[0], v[2], v[3]
        if not (flops or nbytes):
            continue
        out[k] = {"gflop": round(flops / steps / 1e9, 3), "gbytes": round(nbytes / steps / 1e9, 3),
                  "tflop_s": round(flops / ms * 1e-9, 3) if ms > 0 else None,
                  "gb_s": round(nbytes / ms * 1e-6, 1) if ms > 0 else None}
    return out


def measured_traffic(kernel):
    """DRAM bytes per launch of `kernel` (dram__bytes_read.sum + dram__bytes_write.sum) from
    a committed ncu summary under profiles/ that names the kernel, its source file and
    the SHA-256 of that source at capture time; None when there is none or the source
    changed since (the counters then describe another kernel).

    The hash covers the whole file, or with `source_from: <line>` / `source_until: <line>`
    the part of the file from the first line and before the second (the kernel, its helpers and its launches, when host code that
    cannot reach the kernel follows); `headers: a, b@line` with `headers_sha256` adds the
    concatenated headers the kernel is compiled with, `@line` cutting one before that
    line (where only host-side declarations follow)."""
    import glob
    import hashlib
    keys = ("kernel:", "source:", "source_from:", "source_until:", "source_sha256:", "headers:",
            "headers_sha256:", "dram_bytes_per_launch:")
    for path in sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md"))):
        fields = {}
        with open(path) as f:
            for line in f:
                if line.strip().startswith(keys):
                    k, v = line.strip().split(":", 1)
                    fields[k] = v.strip()
        if fields.get("kernel") != kernel or "dram_bytes_per_launch" not in fields:
            continue
        try:
            with open(os.path.join(ROOT, fields["source"]), "rb") as f:
                src = f.read()
            if "source_from" in fields:
                at = src.find(fields["source_from"].encode())
                if at < 0:
                    return None
                src = src[at:]
            if "source_until" in fields:
                at = src.find(fields["source_until"].encode())
                if at < 0:
                    return None
                src = src[:at]
            if hashlib.sha256(src).hexdigest() != fields.get("source_sha256"):
                return None
            if "headers" in fields:
                h = hashlib.sha256()
                for entry in fields["headers"].split(","):
                    name, _, until = entry.strip().partition("@")
                    with open(os.path.join(ROOT, name), "rb") as f:
                        text = f.read()
                    if until:
                        at = text.find(until.encode())
                        if at < 0:
                            return None
                        text = text[:at]
                    h.update(text)
                if h.hexdigest() != fields.get("headers_sha256"):
                    return None
            return float(fields["dram_bytes_per_launch"])
        except (OSError, KeyError, ValueError):
            return None
    return None


def main():
    args = _args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
