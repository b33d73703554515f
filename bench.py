#!/usr/bin/env python
"""Benchmark of the hybrid factorization (Alg. 1) on GB300.

Workload (default): 3D Q1 linear elasticity on a 40^3 node grid (L = 192,000, 3 dofs
per node), Young's modulus 1 with 8 seeded 4^3-element inclusions of modulus 1e6,
nu = 0.3, traction free (6 rigid-body modes), tau = 1e-2, the postponing rule of
Sec. 2.2 (ratio test alone), seeded synthetic values.  One step = one pass of the
whole path: hf_factorize (scaling, FP32 factorization with postponing, Lambda_0
stage) + hf_schur (block GCR for X12, S22, dense LDL^T) + hf_solve (Alg. 2, one rhs).
The metric is the factor + Schur time; the plain FP64 GPU form (S22 from an FP64
factorization) and the FP32-only form are timed beside it over the same steps, and
the thresholds tau = 1e-1 and 1e-4 are reported too.  --workload stokes32 runs the
3D Stokes-like saddle point (32^3 nodes, L = 128,095) with the null-pivot test.

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
# workload -> (generator call, tau, null-pivot test, name).  The Stokes-like saddle point
# needs the null-pivot test at tau = 1e-2: with the ratio test alone FP32 noise pivots of
# its singular zero block pass the test at 32^3 and stay in K11.
WORKLOADS = {
    "elasticity40": ("elasticity3d(40, seed=3)", 1e-2, 0, "elasticity3d_40^3_E1e6_incl8_tau1e-2"),
    "stokes32": ("stokes3d(32, seed=2)", 1e-2, 1, "stokes3d_32^3_mu1e-3..1e3_tau1e-2_nulltest"),
}
# oracle samples of the same generator (and rule): fit sizes, and the reference arm's step
SAMPLES = {
    "elasticity40": {"fit": (10, 12, 14), "step": 10,
                     "make": lambda n: f"elasticity3d({n}, seed=3, n_incl={n // 3}, incl={2 if n < 14 else 3})"},
    "stokes32": {"fit": (8, 10, 12), "step": 10, "make": lambda n: f"stokes3d({n}, seed=2)"},
}


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="elasticity40", choices=sorted(WORKLOADS))
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-extra", action="store_true", help="skip the other thresholds and forms")
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
def _oracle_sample_time(workload, n, threads=1):
    """Time the CPU oracle (Alg. 1 with block GCR) on the n^3 sample of the workload's
    generator, in a child process with `threads` BLAS threads."""
    _, tau, null_test, _ = WORKLOADS[workload]
    make = SAMPLES[workload]["make"](n)
    code = f"""
import os, sys, time, json
sys.path.insert(0, {ROOT!r})
import numpy as np
import oracle as O
from workloads import stokes3d, elasticity3d
s = {make}
Kb = s.to_scipy()
q, K = O.scale_matrix(Kb)
m = max(1, int(np.ceil(np.log2(s.L / 512))) + 1)
sets, order = O.nested_dissection(K, s.coords, m)
t = time.perf_counter()
r = O.run_hybrid(Kb, [sets[l] for l in order], {tau!r}, use_gcr=True, null_test={bool(null_test)!r})
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


def fit_exponent(samples):
    """Least-squares slope p of log(seconds) against log(L) over the oracle samples
    [(L, seconds), ...]: the oracle's time grows as L^p over the sampled range."""
    xs = [math.log(L) for L, _ in samples]
    ys = [math.log(t) for _, t in samples]
    mx, my = sum(xs) / len(xs), sum(ys) / len(ys)
    sxx = sum((x - mx) ** 2 for x in xs)
    return sum((x - mx) * (y - my) for x, y in zip(xs, ys)) / sxx if sxx > 0 else 2.0


def extrapolate(seconds, L_sample, L_full, p):
    return seconds * (L_full / L_sample) ** p


def cpu_model():
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "cpu part", "hardware")):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.processor() or platform.machine()


def full_size_L(workload):
    return {"elasticity40": 3 * 40 ** 3, "stokes32": 3 * 32 ** 3 + 31 ** 3}[workload]


def run_reference(args):
    """The CPU oracle as it stands, on the host cores: the warm-up steps time it on the
    three fit sizes (the exponent of its growth), the timed steps on the step sample; the
    value is the step sample's mean time carried to the full workload by that exponent."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    wl = args.workload
    smp = SAMPLES[wl]
    fit = []
    for i in range(max(args.warmup, len(smp["fit"]))):
        n = smp["fit"][i] if i < len(smp["fit"]) else smp["step"]
        r = _oracle_sample_time(wl, n)
        if i < len(smp["fit"]):
            fit.append((r["L"], r["seconds"]))
    p = fit_exponent(fit)
    times = []
    for _ in range(args.steps):
        r = _oracle_sample_time(wl, smp["step"])
        times.append(r["seconds"])
    t = sum(times) / len(times)
    L_full = full_size_L(wl)
    val = extrapolate(t, r["L"], L_full, p) * 1e3
    line = {
        "impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": val, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": WORKLOADS[wl][3], "L": L_full},
        "cpu_baseline": {"value": val, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"{smp['make'](smp['step'])} (L={r['L']}): {t:.2f} s per run on 1 core "
                                   f"({args.steps} runs), carried to L={L_full} by L^{p:.2f}, the exponent "
                                   f"fitted to the oracle's times at n = {smp['fit']} "
                                   f"({', '.join(f'L={a}: {b:.2f} s' for a, b in fit)})",
                         "measured": {"L": r["L"], "seconds_per_run": t, "fit": fit, "exponent": p},
                         "cpu": cpu_model()},
        "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def cpu_baseline_leg(workload):
    """The oracle timed on the host: one core on the three fit sizes (the growth exponent)
    and once with every core on the middle size; carried to the full workload."""
    smp = SAMPLES[workload]
    fit = [(r["L"], r["seconds"]) for r in (_oracle_sample_time(workload, n) for n in smp["fit"])]
    p = fit_exponent(fit)
    L_full = full_size_L(workload)
    L_big, t_big = fit[-1]
    ncores = os.cpu_count() or 1
    mid = _oracle_sample_time(workload, smp["fit"][1], threads=ncores)
    return {"value": extrapolate(t_big, L_big, L_full, p) * 1e3, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"oracle on {', '.join(smp['make'](n) for n in smp['fit'])} on 1 core "
                      f"({', '.join(f'L={a}: {b:.2f} s' for a, b in fit)}); value = the largest sample "
                      f"carried to L={L_full} by the fitted L^{p:.2f}",
            "measured": {"fit": fit, "exponent": p,
                         "all_cores": {"cores": ncores, "L": mid["L"], "seconds": mid["seconds"],
                                       "value_ms": extrapolate(mid["seconds"], mid["L"], L_full, p) * 1e3}},
            "cpu": cpu_model()}


# ---------------------------------------------------------------------------- GPU arm
def make_system(workload):
    from workloads import stokes3d, elasticity3d
    return eval(WORKLOADS[workload][0], {"__builtins__": {}, "stokes3d": stokes3d, "elasticity3d": elasticity3d})


def backward_error(Kb, x, b):
    import numpy as np
    r = Kb @ x - b
    return float(np.abs(r).max() / (abs(Kb).sum(axis=1).max() * np.abs(x).max() + np.abs(b).max()))


def time_steps(H, vals, tau, bt, xt, steps, warmup, solve=True):
    """W untimed then K timed steps of factorize + schur (+ solve); per-step device times
    (CUDA events on the current stream, which is the library's stream) of each phase."""
    import torch
    for _ in range(warmup):
        H.factorize(vals, tau)
        H.schur()
        if solve:
            H.solve(bt, xt)
    torch.cuda.synchronize()
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(steps)]
    for e in evs:
        e[0].record()
        H.factorize(vals, tau)
        e[1].record()
        H.schur()
        e[2].record()
        if solve:
            H.solve(bt, xt)
        e[3].record()
    torch.cuda.synchronize()
    fac = [e[0].elapsed_time(e[1]) for e in evs]
    sch = [e[1].elapsed_time(e[2]) for e in evs]
    sol = [e[2].elapsed_time(e[3]) for e in evs]
    tot = evs[0][0].elapsed_time(evs[-1][3])
    return fac, sch, sol, tot


def form_line(hf, s, vals, bt, b, tau, steps, warmup, **opts):
    """Another form or threshold on the same system, timed over the given steps."""
    import torch
    H = hf.HybridFactor(s.L, s.rowptr, s.col, s.coords, **opts)
    xt = torch.zeros_like(bt)
    try:
        fac, sch, _, _ = time_steps(H, vals, tau, bt, xt, steps, warmup, solve=False)
    except hf.HFError as e:                      # e.g. a threshold that postpones too much
        H.free()
        torch.cuda.empty_cache()
        return {"error": str(e), "code": e.code}
    H.solve(bt, xt)
    torch.cuda.synchronize()
    info = H.info()
    be = backward_error(s.to_scipy(), xt.cpu().numpy().T, b)
    out = {"factor_schur_ms": (sum(fac) + sum(sch)) / steps, "steps": steps, "warmup": warmup,
           "M": info["M"], "kernel_dim": info["kernel_dim"], "gcr_iters": info["gcr_iters"],
           "backward_error": be, "gate_1e-12": bool(be <= 1e-12)}
    H.free()
    torch.cuda.empty_cache()
    return out


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        src = "of measured (MEASURED_PEAKS.json)"
    except Exception:
        p, src = {}, "of fallback (profiling recipe)"
    return {"hbm": p.get("hbm_gbs", 6800.0), "bf16": p.get("bf16_tflops_sustained", 1700.0),
            "fp32_simt": 152 * 128 * 2 * 2.07e9 / 1e12, "src": src}


def kernel_rooflines(prof, steps, trailing_tc):
    """Per kernel: its device time per step, the algorithmic work the library counted for
    exactly those launches, and the fraction of the roof that binds it.  Each profile class
    is one kernel (the glue launches around them have classes of their own); the two block
    GCR products are one kernel, k_oz_mma, and are merged."""
    pk = peaks()
    simt = ("alu", pk["fp32_simt"], "TFLOP/s", "derived: 152 SMs x 128 FP32 lanes x 2 x 2.07 GHz")
    hbm = ("hbm", pk["hbm"], "GB/s", "hbm_gbs " + pk["src"])
    bf16 = ("tensor", pk["bf16"], "TFLOP/s", "bf16_tflops_sustained " + pk["src"])
    table = {
        "panel": ("k_panel_cl", "pivoted left-looking panel in cluster shared memory (latency chain)", simt, 1.0),
        "panel_global": ("k_panel", "pivoted left-looking panel in global memory, one CTA per front (levels of "
                                    "many small fronts)", simt, 1.0),
        "trailing": ("k_trailing_tc" if trailing_tc else "k_trailing",
                     "trailing Schur update" + (" (exact 3 x BF16 split of FP32, 6 products on tcgen05; "
                                                "levels of fronts < 256 rows on the FP32 SIMT kernel)"
                                                if trailing_tc else " (FP32 SIMT)"),
                     bf16 if trailing_tc else simt, 6.0 if trailing_tc else 1.0),
        "trsv_fwd": ("k_sweep_df<1>", "dataflow forward sweep of a tree level (FP32 factor streamed)", hbm, 1.0),
        "trsv_bwd": ("k_sweep_df<0>", "dataflow backward sweep of a tree level (FP32 factor streamed)", hbm, 1.0),
        "spmm": ("k_spmm", "FP64 CSR x block", hbm, 1.0),
        "oz": ("k_oz_mma", "FP64-accurate Grams and block updates: 36 BF16 slice products", bf16, 36.0),
    }
    merged = dict(prof)
    g, u = prof.get("gram", (0, 0, 0, 0)), prof.get("block_update", (0, 0, 0, 0))
    merged["oz"] = tuple(a + b for a, b in zip(g, u))
    out = {}
    for cls, (kname, what, (bound, peak, unit, psrc), mult) in table.items():
        ms, n, flops, nbytes = merged.get(cls, (0.0, 0, 0.0, 0.0))
        if ms <= 0 or n == 0:
            continue
        if bound == "hbm":
            achieved = nbytes / (ms / 1e3) / 1e9
        else:
            achieved = mult * flops / (ms / 1e3) / 1e12
        out[kname] = {"bound": bound, "achieved": achieved, "peak": peak, "unit": unit, "frac": achieved / peak,
                      "traffic": measured_traffic(kname), "kernel": kname, "what": what, "peak_source": psrc,
                      "ms_per_step": ms / steps, "launches_per_step": n / steps,
                      "algorithmic_per_launch": (nbytes if bound == "hbm" else mult * flops) / n,
                      "algorithmic_unit": "bytes" if bound == "hbm" else "flops"}
    return out


def run_ours(args):
    import numpy as np
    import torch
    import paper_2208_01907_gb300 as hf
    from workloads import consistent_rhs

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

    wl = args.workload
    _, tau, null_test, cfg_name = WORKLOADS[wl]
    s = make_system(wl)
    Kb = s.to_scipy()
    H = hf.HybridFactor(s.L, s.rowptr, s.col, s.coords, null_test=null_test)
    vals = torch.tensor(s.val, device=dev, dtype=torch.float64)
    b = consistent_rhs(s, 11, 1, "solution")
    bt = torch.tensor(np.ascontiguousarray(b.T), device=dev)
    xt = torch.zeros_like(bt)
    warm = max(3, args.warmup)
    time_steps(H, vals, tau, bt, xt, 1, warm - 1)          # warm-up (delay capacities settle)
    H.profile(False)                                       # counters reset; launches counted, no events
    H.get_profile()
    clocks = ClockSampler(local)
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    fac, sch, sol, total_ms = time_steps(H, vals, tau, bt, xt, args.steps, 0)
    barrier()
    clk = clocks.stop()
    launches = sum(v[1] for v in H.get_profile().values())        # launches in the timed steps
    # per-kernel device times from more steps with the library's event profiling on (kept out
    # of the timed steps: two event records per launch slow the host enqueue)
    prof_steps = min(3, args.steps)
    H.profile(True)
    time_steps(H, vals, tau, bt, xt, prof_steps, 0)
    prof = H.get_profile()
    H.profile(False)
    fs_ms = (sum(fac) + sum(sch)) / args.steps
    step_ms = total_ms / args.steps
    if dist is not None:
        tt = torch.tensor([fs_ms, step_ms], device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        fs_ms, step_ms = float(tt[0]), float(tt[1])
    info = H.info()
    x = xt.cpu().numpy().T
    bwd = backward_error(Kb, x, b)
    relres = float(np.linalg.norm(Kb @ x - b) / np.linalg.norm(b))

    trailing_tc = H.opts.trailing == 0
    roofs = kernel_rooflines(prof, prof_steps, trailing_tc)
    dom = max(roofs.values(), key=lambda r: r["ms_per_step"]) if roofs else None

    # end to end through the C ABI with host buffers: H2D of the values, D2H of S22
    hv = torch.tensor(s.val, dtype=torch.float64).pin_memory()
    dvals = torch.empty_like(vals)
    M = info["M"]
    hs22 = torch.empty((max(M, 1), max(M, 1)), dtype=torch.float64).pin_memory()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        dvals.copy_(hv, non_blocking=True)
        H.factorize(dvals, tau)
        H.schur()
        hs22[:M, :M].copy_(H.s22(torch), non_blocking=True)
    e1.record()
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1) / args.steps
    H.free()
    torch.cuda.empty_cache()

    # the forms of Table 1 beside the hybrid one, over the same warm-up and timed steps:
    # plain FP64 (factor in FP64, S22 from the factor) and FP32 only ("single")
    forms = {}
    if not args.no_fp64:
        forms["fp64_form"] = form_line(hf, s, vals, bt, b, tau, args.steps, warm, precision=hf.HF_PREC_FP64,
                                       null_test=null_test)
        if "factor_schur_ms" in forms["fp64_form"]:
            forms["fp64_form"]["speedup_mixed_vs_fp64"] = forms["fp64_form"]["factor_schur_ms"] / fs_ms
        forms["fp32_form"] = form_line(hf, s, vals, bt, b, tau, args.steps, warm, precision=hf.HF_PREC_FP32,
                                       null_test=null_test)
    extra = {}
    if not args.no_extra:
        ks, kw = min(args.steps, 5), 3
        other = 1 if trailing_tc else 0
        extra[f"trailing={'simt' if other else 'tensor_cores'}"] = form_line(
            hf, s, vals, bt, b, tau, ks, kw, null_test=null_test, trailing=other)
        for t2 in (1e-1, 1e-4):
            extra[f"tau={t2:g}"] = form_line(hf, s, vals, bt, b, t2, ks, kw, null_test=null_test)
        if not null_test:
            extra["tau=1e-4_nulltest"] = form_line(hf, s, vals, bt, b, 1e-4, ks, kw, null_test=1)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        try:
            cpu = cpu_baseline_leg(wl)
        except Exception as e:  # noqa: BLE001
            cpu = {"value": None, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": f"failed: {e}"[:300]}

    if rank == 0:
        roof = None
        if dom is not None:
            roof = {k: dom[k] for k in ("bound", "achieved", "peak", "unit", "frac", "traffic")}
            roof.update({k: dom[k] for k in ("kernel", "what", "peak_source", "ms_per_step", "launches_per_step",
                                             "algorithmic_per_launch", "algorithmic_unit")})
        line = {
            "metric": METRIC, "value": fs_ms, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": warm, "ms_per_step": step_ms, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": cfg_name, "L": s.L, "nnz": s.nnz, "tau": tau,
                       "postponing": "ratio test + null-pivot test" if null_test else "ratio test (Sec. 2.2)",
                       "M": info["M"], "n_lambda0": info["n_lambda0"], "kernel_dim": info["kernel_dim"],
                       "gcr_iters": info["gcr_iters"], "levels": info["levels"],
                       "l2": "working set (factor arena %.1f GB) larger than L2" % (info["front_bytes"] / 1e9),
                       "parallelism": f"replicas x{world}"},
            "phases_ms": {"factorize": sum(fac) / args.steps, "schur": sum(sch) / args.steps,
                          "solve": sum(sol) / args.steps},
            "systems_per_s": world * 1e3 / step_ms,
            "rel_residual": relres, "backward_error": bwd, "gate_1e-12": bwd <= 1e-12,
            "roofline": roof,
            "kernels": {k: {kk: (round(v, 4) if isinstance(v, float) else v) for kk, v in r.items()
                            if kk in ("ms_per_step", "achieved", "unit", "frac", "bound")}
                        for k, r in roofs.items()},
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_ms, "unit": UNIT, "h2d_bytes_per_step": s.nnz * 8,
                    "d2h_bytes_per_step": M * M * 8},
            **forms,
            "other_forms": extra,
            "gpu_launches": launches,
            "kernel_ms": {k: round(v[0] / prof_steps, 3) for k, v in prof.items()},
            "kernel_work": kernel_work(prof, prof_steps),
            "paths": {k: info[k] for k in ("panel_cluster", "panel_global", "sweep_blocks", "ldlt_kernel")},
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
                    continue
                src = src[at:]
            if "source_until" in fields:
                at = src.find(fields["source_until"].encode())
                if at < 0:
                    continue
                src = src[:at]
            if hashlib.sha256(src).hexdigest() != fields.get("source_sha256"):
                continue                      # a note on another version of the kernel
            if "headers" in fields:
                h = hashlib.sha256()
                for entry in fields["headers"].split(","):
                    name, _, until = entry.strip().partition("@")
                    with open(os.path.join(ROOT, name), "rb") as f:
                        text = f.read()
                    if until:
                        at = text.find(until.encode())
                        if at < 0:
                            break
                        text = text[:at]
                    h.update(text)
                if h.hexdigest() != fields.get("headers_sha256"):
                    continue
            return float(fields["dram_bytes_per_launch"])
        except (OSError, KeyError, ValueError):
            continue
    return None


def main():
    args = _args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
