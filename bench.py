"""Benchmark of the fractional Poisson hot path on one GB300 (or N replicas).

One step = the whole path on the 128 x 128 masked grid (union of 6 seeded
ellipses, largest component, n = 8810 dofs, h = 1/129): fd_assemble (both
calls), all n eigenpairs, and frac_apply for 16 polynomial forcings x 8
orders alpha = 0.25 .. 2 (128 solves).  Two routes to the eigenpairs are
timed: eig_full (FP64 throughout) and eig_full_mixed (FP32 stages +
Ogita-Aishima refinement); the headline is the faster one whose output meets
the FP64 bar (alpha = 2 solutions within 1e-10 of the direct solve, sampled
eigenvalues bracketed by inertia counts at +-1e-11, sampled orthogonality
1e-12).  The dense matrix (620 MB) and the eigenvector matrix exceed the
129 MB L2, so no flush is needed between steps.

Printed value: fractional solves per second (128 solves per step, each
including its share of the decomposition), whole job over all ranks.  The
mixed route counts only when its eigenvalues and all 128 solutions agree
with the FP64 route's to 1e-11 / 1e-10.  The line also carries, under
"configs", the other single-GPU workloads (square48, batched256, apply192)
with their accuracy against the oracle, and, under "cpu_baseline", the FP64
CPU oracle timed on one whole step of this workload on the host cores.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl fraclap|reference]
                  [--path both|fp64|mixed] [--workload NAME] [--no-configs]

--impl reference times the FP64 CPU oracle (the plain statement of the
method, test infrastructure) on whole steps of the same workload on the host
cores; one step takes minutes, so it stops after the first step that ends
past a one-minute budget and prints how many steps it timed.
"""
from __future__ import annotations

import argparse
import json
import os
import signal
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "eigendecomp s & %peak at n≈10k; fractional solves/s at ≤1e-10 err vs FP64"
# FP64 peak of GB300: 152 SMs x 2070 MHz x 2 DFMA/clock x 2 flop (the FP64
# pipe that DFMA and DMMA share), 1.26 TFLOP/s; not in MEASURED_PEAKS.json.
FP64_PEAK_TFLOPS = 152 * 2.070e9 * 2 * 2 / 1e12


def _workload():
    from paper_1911_11906_gb300 import inputs as I
    return I.ellipse_problem(128, n_ellipses=6, n_forcings=16, seed=1000)


def _config(p, extra=None):
    c = {"workload": f"ellipse128: 128x128 grid, 6 seeded ellipses, n={p.n}, "
                     f"{p.F.shape[1]} forcings x 8 alpha = {len(p.pair_f)} solves",
         "n": p.n, "solves_per_step": int(len(p.pair_f)), "precision": "fp64",
         "l2_policy": "inputs larger than L2 (A and V are 620 MB each)"}
    if extra:
        c.update(extra)
    return c


# ----------------------------------------------------------------------------
# clocks during the timed region
# ----------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-f", self.path], stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.send_signal(signal.SIGTERM)
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        try:
            with open(self.path) as fh:
                for line in fh:
                    parts = [x.strip() for x in line.split(",")]
                    if len(parts) >= 9:
                        rows.append(parts)
            os.unlink(self.path)
        except Exception:
            return None
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        busy = [s for s in sm if mx and s > 0.5 * max(mx)] or sm
        return {"sm_mhz": statistics.median(busy) if busy else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ----------------------------------------------------------------------------
# algorithmic work
# ----------------------------------------------------------------------------
def q2_flops(n: int, b: int) -> float:
    """Flops of Z <- Q2 Z: every bulge-chasing reflector of length L costs 4 L n."""
    tot = 0
    for s in range(n - 1):
        r0 = s + 1
        while r0 <= n - 1:
            L = min(b, n - r0)
            if L > 1:
                tot += L
            r0 += b
    return 4.0 * tot * n


def eig_flops(n: int) -> float:
    """One-stage-equivalent credit for all eigenpairs: 4/3 n^3 (reduction)
    + 4/3 n^3 (divide-and-conquer merges, upper bound) + 2 n^3 (back-transform)."""
    return (4.0 / 3 + 4.0 / 3 + 2.0) * n ** 3


# ----------------------------------------------------------------------------
# metrics log: one JSONL record per timed route of a bench line
# ----------------------------------------------------------------------------
def jsonl_records(line: dict) -> list:
    """Per-route records {config, n, precision, steps, seconds, tflops,
    frac_of_peak, err_*} of a bench line (the headline route carries the
    kernel roofline as well)."""
    out = []
    cfg = line.get("config", {})
    for route, r in (line.get("paths") or {}).items():
        acc = r.get("accuracy", {})
        rec = {"config": cfg.get("workload"), "n": cfg.get("n"), "precision": route, "steps": line.get("steps"),
               "seconds": round(r["ms_per_step"] / 1e3, 6), "solves_per_s": r.get("solves_per_s"),
               "eig_seconds": r.get("eig_s"), "tflops": r.get("eig_tflops_credited_fp64"),
               "frac_of_peak": r.get("eig_frac_of_fp64_peak"),
               "err_u_alpha2": acc.get("u_rel_l2_alpha2_vs_cg_max"),
               "err_resid": acc.get("eig_residual_sampled_max"), "err_orth": acc.get("orth_sampled_max"),
               "err_trace": acc.get("trace_rel_err"), "stage_ms": r.get("stage_ms")}
        if route == (cfg.get("path") or route) and line.get("roofline"):
            rec["roofline"] = line["roofline"]
        out.append(rec)
    return out


# ----------------------------------------------------------------------------
# replicas: every rank runs the whole workload on its own GPU (weak scaling)
# ----------------------------------------------------------------------------
def max_over_ranks(values, world: int, device=None) -> list:
    """The slowest rank's figures: an all-reduce MAX over the process group
    (NCCL on GPUs, gloo on the host); a no-op for one rank."""
    if world <= 1:
        return [float(v) for v in values]
    import torch
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return [float(v) for v in t.cpu()]


def whole_job_rate(units_per_rank: int, world: int, ms: float) -> float:
    """Units per second over all ranks, timed by the slowest rank."""
    return units_per_rank * world / (ms * 1e-3)


# ----------------------------------------------------------------------------
# the GPU arm
# ----------------------------------------------------------------------------
# FP32 SIMT peak (mixed path stages): 152 SMs x 2.07 GHz x 128 FFMA/clk x 2.
FP32_PEAK_TFLOPS = 152 * 2.070e9 * 128 * 2 / 1e12
REFINE_ITERS = 6
BAND = {"fp64": 64, "mixed": 64}
# the mixed route's apply takes its two products as 6 BF16 slices per operand
# on the tensor cores (FP64-accurate to a few 1e-12, checked on every solve
# against the FP64 route); the FP64 route keeps FP64 products
APPLY_SLICES = {"fp64": 0, "mixed": 6}
# wall-clock budget of the oracle arm: whole steps are timed until one ends past it
REFERENCE_BUDGET_S = 60.0


def ozaki_bf16_flops(n: int, slices: int = 8) -> float:
    """Algorithmic BF16 tensor flops of one lower-triangular n x n x n
    residual product cut into `slices` 7-bit slices (K > 256): pairs with
    p + q < slices, each 2 n flops per lower-triangle entry."""
    pairs = slices * (slices + 1) // 2
    return 2.0 * pairs * n * (n * (n + 1) // 2)


def apply_slice_flops(n: int, m: int, k: int, slices: int, digit_bits: int = 7) -> float:
    """BF16 flops of the apply's two sliced products, V^T F (n x m) and
    V C (n x k), both with inner dimension n: every digit pair p + q < d,
    d = ceil(8 s / 7) digits of 7 bits (or the s slices themselves)."""
    d = slices if digit_bits == 8 else (8 * slices + 6) // 7
    return 2.0 * (d * (d + 1) // 2) * n * n * (m + k)


def refine_slice_counts(iterations: int, cap: int, digit_bits: int = 7) -> list:
    """Digits per operand of the refinement's two residual products in each
    iteration: 40, 48 and then 56 bits (5, 6, 7 slices of 8 bits), the last
    allowed iteration always full; as 7-bit digits (ceil(8 s / 7)) or, with
    digit_bits = 8, the slices themselves."""
    out = []
    for it in range(iterations):
        s8 = 7 if it + 1 >= cap else (5 if it == 0 else (6 if it == 1 else 7))
        out.append(s8 if digit_bits == 8 else (8 * s8 + 6) // 7)
    return out


# DRAM bytes per BF16 flop of ozaki_tc_kernel (128 x 192 tiles) from one ncu
# capture of the 4096^3 product with the current kernel: (9.98 + 1.32) GB
# over 4.95e12 flop; its tile re-streaming grows in proportion to the flops.
# None whenever the kernel changes until it is captured again.
OZAKI_DRAM_BYTES_PER_FLOP = 2.285e-3


def run_path(F, ctx, p, path, args, mask, Fd, pf, pa, U, app_ws, barrier, steps=None, warmup=None):
    import torch
    n = p.n
    if path == "fp64":
        ws = torch.empty(ctx.lib.fraclap_eig_workspace_bytes(ctx.handle, n), dtype=torch.uint8, device=mask.device)
    else:
        ws = torch.empty(ctx.lib.fraclap_eig_mixed_workspace_bytes(ctx.handle, n), dtype=torch.uint8,
                         device=mask.device)

    def step(sync_status=False):
        asm = F.fd_assemble(mask, p.h, ctx=ctx)
        if path == "fp64":
            lam, V = F.eig_full(asm["A"], ctx=ctx, workspace=ws, sync=sync_status)
        else:
            lam, V = F.eig_full_mixed(asm["A"], asm["rowptr"], asm["col"], asm["val"], refine_iters=REFINE_ITERS,
                                      ctx=ctx, workspace=ws, sync=sync_status)
        F.frac_apply(V, lam, Fd, pf, pa, ctx=ctx, out=U, workspace=app_ws, sync=sync_status)
        return lam, V

    steps = args.steps if steps is None else steps
    warmup = args.warmup if warmup is None else warmup
    for _ in range(warmup):
        lam, V = step(sync_status=True)
    torch.cuda.synchronize()
    ctx.set_profiling(True)
    ctx.stage_times()
    launches0 = ctx.launch_count()
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        lam, V = step()
    e1.record()
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1) / steps
    launches = (ctx.launch_count() - launches0) // steps
    stages = ctx.stage_times()
    ctx.set_profiling(False)
    ctx.sync()
    rstats = ctx.refine_stats() if path == "mixed" else []
    return {"ms": ms, "launches": launches, "stages": stages, "clocks": clk, "lam": lam, "V": V,
            "refine": rstats, "step": step, "steps": steps, "warmup": warmup}


def run_gpu(args, rank, world, local_rank):
    import torch
    import paper_1911_11906_gb300 as F
    from paper_1911_11906_gb300 import autotune

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    p = _workload()
    n, k = p.n, len(p.pair_f)
    mask_h = torch.from_numpy(p.mask).pin_memory()
    F_h = torch.from_numpy(np.ascontiguousarray(p.F.T)).pin_memory()    # (m, n) row-major = column-major (n, m)
    pf_h = torch.from_numpy(p.pair_f.astype(np.int32)).pin_memory()
    pa_h = torch.from_numpy(p.pair_alpha.astype(np.float64)).pin_memory()
    U_h = torch.empty((k, n), dtype=torch.float64).pin_memory()
    mask = mask_h.to(dev)
    Fd = F_h.to(dev).t()
    pf, pa = pf_h.to(dev), pa_h.to(dev)
    U = F._binding.empty_colmajor(n, k, dev)
    app_ws = None
    barrier = (lambda: torch.distributed.barrier()) if world > 1 else (lambda: None)
    paths = ["fp64", "mixed"] if args.path == "both" else [args.path]
    results = {}
    band = dict(BAND)
    band_src = {pth: "fixed" for pth in band}
    if "mixed" in paths and not args.no_autotune:
        band["mixed"] = autotune.best_band_width(n, "mixed")
        band_src["mixed"] = "autotuner (cache %s)" % autotune.default_cache_path()
    sched = {}
    if "mixed" in paths and not args.no_autotune:
        sched = autotune.best_ozaki_schedule(n, slices=7)
    for path in paths:
        ctx = F.Context(band_width=band[path])
        if path == "mixed" and sched:
            autotune.apply_schedule(ctx, sched)
        ctx.set_apply_slices(APPLY_SLICES[path])
        app_ws = torch.empty(ctx.lib.fraclap_apply_workspace_bytes_ctx(ctx.handle, n, Fd.shape[1], k),
                             dtype=torch.uint8, device=dev)
        # the FP64 route is the comparison when both run: fewer timed steps (it is 6x slower)
        short = path == "fp64" and len(paths) > 1
        r = run_path(F, ctx, p, path, args, mask, Fd, pf, pa, U, app_ws, barrier,
                     steps=min(args.steps, 2) if short else None, warmup=min(args.warmup, 3) if short else None)
        r["ctx"] = ctx
        r["U"] = U.clone()
        r["acc"] = check_accuracy(F, ctx, p, mask, r["lam"], U, r["V"], Fd) if rank == 0 else {}
        results[path] = r
    if rank == 0 and "fp64" in results and "mixed" in results:
        # the mixed route against the plain FP64 route on every solve and eigenvalue
        acc = results["mixed"]["acc"]
        Um, Ud = results["mixed"]["U"], results["fp64"]["U"]
        acc["u_rel_l2_vs_fp64_route_max"] = float((torch.linalg.norm(Um - Ud, dim=0)
                                                   / torch.linalg.norm(Ud, dim=0)).max())
        lm, ld = results["mixed"]["lam"], results["fp64"]["lam"]
        acc["lambda_rel_vs_fp64_route_max"] = float(((lm - ld).abs() / ld.abs()).max())
        acc["meets_fp64_bar"] = bool(acc["meets_fp64_bar"] and acc["u_rel_l2_vs_fp64_route_max"] <= 1e-10
                                     and acc["lambda_rel_vs_fp64_route_max"] <= 1e-11)
    # headline: the fastest path whose accuracy checks pass
    ok = [pth for pth in paths if rank != 0 or results[pth]["acc"].get("meets_fp64_bar", False)]
    head = min(ok or paths, key=lambda pth: results[pth]["ms"])
    R = results[head]
    ms = R["ms"]

    # ---- end to end through the public API with host buffers (headline path) ----
    def step_e2e():
        mask.copy_(mask_h, non_blocking=True)
        Fd.t().copy_(F_h, non_blocking=True)
        pf.copy_(pf_h, non_blocking=True)
        pa.copy_(pa_h, non_blocking=True)
        R["step"]()
        U_h.copy_(U.t(), non_blocking=True)

    step_e2e()
    torch.cuda.synchronize()
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step_e2e()
    torch.cuda.synchronize()
    barrier()
    e2e_ms = (time.perf_counter() - t0) * 1e3 / args.steps

    ms, e2e_ms = max_over_ranks([ms, e2e_ms], world, dev)
    if rank != 0:
        return

    # measured FMA-pipe peaks (the bound of the SIMT FP64 / FP32 stages)
    fma_peaks = {"fp64_tflops": round(R["ctx"].fma_throughput(64) / 1e12, 4),
                 "fp32_tflops": round(R["ctx"].fma_throughput(32) / 1e12, 3),
                 "how": "fraclap_fma_throughput: independent FMA chains, 8 CTAs x 256 threads per SM, CUDA events"}
    fp64_peak = fma_peaks["fp64_tflops"] or FP64_PEAK_TFLOPS
    stages = R["stages"]
    b = band[head]
    if head == "fp64":
        q2_ms, q2_cnt = stages["back_q2"]
        dur = q2_ms / max(q2_cnt, 1)
        work = q2_flops(n, b)
        traffic = None
        roof = {"kernel": "q2t_apply_kernel (back-transformation by the bulge-chasing reflectors, FP64)",
                "bound": "alu", "peak": round(fp64_peak, 4),
                "peak_source": "measured FP64 FMA throughput (fraclap_fma_throughput); no FP64 figure in "
                               "MEASURED_PEAKS.json"}
    else:
        g_ms, g_cnt = stages["slice_products"]
        dur = g_ms / max(g_cnt, 1)
        # average over the launches of one step: 2 per refinement iteration
        # (fewer slices in the first two) and the apply's 2
        digit_bits = R["ctx"].get_schedule("ozaki_bits")
        per_iter = refine_slice_counts(len(R.get("refine", [])) or 3, REFINE_ITERS, digit_bits)
        total = sum(2 * ozaki_bf16_flops(n, sl) for sl in per_iter)
        launches_per_step = 2 * len(per_iter)
        if APPLY_SLICES[head]:
            total += apply_slice_flops(n, Fd.shape[1], k, APPLY_SLICES[head], digit_bits)
            launches_per_step += 2
        work = total / max(launches_per_step, 1)
        # the captured figure holds for the captured tile width and no cluster
        captured = R["ctx"].get_schedule("ozaki_tile_n") == 192 and R["ctx"].get_schedule("ozaki_cluster") == 1
        traffic = OZAKI_DRAM_BYTES_PER_FLOP * work if (OZAKI_DRAM_BYTES_PER_FLOP and captured) else None
        # the kernel runs inside a seconds-long step: the sustained BF16 figure is its peak
        peak = _measured_peak("bf16_tflops_sustained") or _measured_peak("bf16_tflops") or 1700.0
        roof = {"kernel": "ozaki_tc_kernel (residual products of the refinement and the apply's two products: "
                          "tcgen05.mma on TMA-loaded BF16 slices)",
                "bound": "tensor", "peak": round(peak, 1),
                "peak_source": ("MEASURED_PEAKS.json bf16_tflops_sustained (of measured; the kernel is timed inside a "
                                "seconds-long step)") if _measured_peak("bf16_tflops_sustained") else
                               ("MEASURED_PEAKS.json bf16_tflops (burst)" if _measured_peak("bf16_tflops")
                                else "fallback 1.7 PFLOP/s sustained"),
                "frac_of_burst": None}
    achieved = work / (dur * 1e-3) / 1e12
    if "frac_of_burst" in roof:
        roof["frac_of_burst"] = round(achieved / (_measured_peak("bf16_tflops") or 1900.0), 5)
    roof.update({"achieved": round(achieved, 4), "unit": "TFLOP/s", "frac": round(achieved / roof["peak"], 5),
                 "traffic": (round(traffic) if traffic else None), "flops_per_launch": work,
                 "ms_per_launch": round(dur, 3)})
    eig_stages = ("band_reduction", "bulge_chasing", "tridiag_dc", "back_q2", "back_q1", "refine")
    line = {
        "metric": METRIC,
        "value": round(whole_job_rate(k, world, ms), 4),
        "unit": "solves/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(ms, 3),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64" if head == "fp64" else "f32+f64-refined",
        "data": "synthetic (seeded masked grid and polynomial forcings)",
        "config": _config(p, {"band_width": b, "parallelism": f"replicas{world}", "path": head,
                              "precision": head}),
        "paths": {},
        "roofline": roof,
        "e2e": {"value": round(whole_job_rate(k, world, e2e_ms), 4), "unit": "solves/s",
                "h2d_bytes_per_step": int(mask_h.numel() + F_h.numel() * 8 + pf_h.numel() * 4 + pa_h.numel() * 8),
                "d2h_bytes_per_step": int(U_h.numel() * 8), "ms_per_step": round(e2e_ms, 3)},
        "gpu_launches": int(R["launches"]),
        "clocks": R["clocks"],
        "measured_fma_peaks": fma_peaks,
    }
    for pth, r in results.items():
        st = r["stages"]
        eig_ms = sum(st[s][0] for s in eig_stages) / r["steps"]
        line["paths"][pth] = {
            "ms_per_step": round(r["ms"], 3), "solves_per_s": round(k / (r["ms"] * 1e-3), 4),
            "steps_timed": r["steps"], "warmup": r["warmup"],
            "eig_s": round(eig_ms / 1e3, 4),
            "eig_tflops_credited_fp64": round(eig_flops(n) / (eig_ms * 1e-3) / 1e12, 4),
            "eig_frac_of_fp64_peak": round(eig_flops(n) / (eig_ms * 1e-3) / 1e12 / fp64_peak, 4),
            "apply_s": round(st["apply"][0] / r["steps"] / 1e3, 5),
            "apply_products": (f"{APPLY_SLICES[pth]} BF16 slices per operand on tcgen05" if APPLY_SLICES[pth]
                               else "FP64"),
            "stage_ms": {s: round(v[0] / r["steps"], 3) for s, v in st.items()},
            "gpu_launches": int(r["launches"]),
            "accuracy": r["acc"],
            "band_width": band[pth], "band_width_source": band_src[pth],
        }
        if pth == "mixed" and sched:
            line["paths"][pth]["slice_product_schedule"] = dict(sched, source="autotuner")
        if r["refine"]:
            line["paths"][pth]["refine_iterations"] = len(r["refine"])
            line["paths"][pth]["refine_last"] = {kk: float("%.3e" % vv) for kk, vv in r["refine"][-1].items()}
    if world == 1 and not args.no_configs:
        # the other workloads, a few timed steps each (W = 3), with their accuracy against the oracle
        sub_w, sub_k = max(3, min(args.warmup, 3)), min(args.steps, 3)
        line["configs"] = {}
        for name, fn in (("square48", lambda: run_square_bench(args, steps=sub_k, warmup=sub_w)),
                         ("batched256", lambda: run_batched_bench(args, steps=sub_k, warmup=sub_w)),
                         ("apply192", lambda: run_apply_bench(args, steps=sub_k, warmup=sub_w))):
            sub = fn()
            sub.pop("metric", None)
            line["configs"][name] = sub
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(p)
    print(json.dumps(line), flush=True)
    if args.jsonl:
        with open(args.jsonl, "a") as fh:
            for rec in jsonl_records(line):
                fh.write(json.dumps(rec) + "\n")


def _measured_peak(key):
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)[key])
    except Exception:
        return None


def _csr(F, mask, h, ctx):
    """The assembled operator as a torch sparse CSR matrix (for evidence only)."""
    import warnings
    import torch
    warnings.filterwarnings("ignore", message="Sparse CSR tensor support is in beta state")
    asm = F.fd_assemble(mask, h, dense=False, ctx=ctx)
    n = asm["n"]
    return torch.sparse_csr_tensor(asm["rowptr"], asm["col"].to(torch.int64), asm["val"], size=(n, n))


def _cg(A, B, tol=1e-14, maxit=5000):
    """Conjugate gradients on the columns of B (independent scalars per column):
    a GPU reference for the alpha = 2 solutions A u = f, run to a relative
    residual of tol, so that its own forward error is below cond(A) tol."""
    import torch
    X = torch.zeros_like(B)
    R = B.clone()
    P = R.clone()
    rr = (R * R).sum(0)
    b2 = rr.clone()
    for _ in range(maxit):
        if bool((rr <= (tol * tol) * b2).all()):
            break
        AP = A @ P
        a = rr / (P * AP).sum(0)
        X += P * a
        R -= AP * a
        rr_new = (R * R).sum(0)
        P = R + P * (rr_new / rr)
        rr = rr_new
    return X


def check_accuracy(F, ctx, p, mask, lam, U, V, Fd):
    """Evidence, computed on the GPU after the timed region, that the solves
    meet the FP64 bar: alpha = 2 solutions against conjugate gradients on the
    assembled operator (relative residual 1e-14), residuals A v - lambda v and
    orthogonality of 32 sampled eigenpairs, and the trace identity
    sum(lambda) = 2 dim n / h^2.  (The oracle's checks of the same workload are
    in the tests.)"""
    import torch
    A = _csr(F, mask, p.h, ctx)
    n = p.n
    nA = 4.0 * p.dim / p.h ** 2  # Gershgorin bound of ||A||_2
    j2 = np.nonzero(p.pair_alpha == 2.0)[0]
    out = {}
    if len(j2):
        Fc = Fd[:, torch.from_numpy(p.pair_f[j2].astype(np.int64)).to(Fd.device)].contiguous()
        Ug = _cg(A, Fc)
        Uj = U[:, torch.from_numpy(j2).to(U.device)]
        out["u_rel_l2_alpha2_vs_cg_max"] = float((torch.linalg.norm(Uj - Ug, dim=0) / torch.linalg.norm(Ug, dim=0)).max())
    rng = np.random.default_rng(0)
    cols = torch.from_numpy(np.sort(rng.choice(n, size=min(32, n), replace=False))).to(V.device)
    Vc = V[:, cols].contiguous()
    Rv = A @ Vc - Vc * lam[cols]
    out["eig_residual_sampled_max"] = float(torch.linalg.norm(Rv, dim=0).max()) / nA
    G = V.t() @ Vc
    G[cols, torch.arange(len(cols), device=V.device)] -= 1.0
    out["orth_sampled_max"] = float(G.abs().max())
    tr = 2.0 * p.dim * n / p.h ** 2
    out["trace_rel_err"] = float(abs(float(lam.sum()) - tr) / tr)
    out["meets_fp64_bar"] = bool(out.get("u_rel_l2_alpha2_vs_cg_max", 0.0) <= 1e-10
                                 and out["eig_residual_sampled_max"] <= 1e-12
                                 and out["orth_sampled_max"] <= 1e-12 and out["trace_rel_err"] <= 1e-11)
    return out


# ----------------------------------------------------------------------------
# the CPU oracle (baseline / reference arm)
# ----------------------------------------------------------------------------
def oracle_step(p):
    """One step of the workload through the FP64 CPU oracle: assembly, the
    full eigendecomposition (Householder + implicit QR) and the spectral
    apply of every solve.  Returns the wall seconds."""
    import oracle as O
    t0 = time.perf_counter()
    O.solve(p.mask, p.h, p.F, p.pair_f, p.pair_alpha)
    return time.perf_counter() - t0


def cpu_baseline(p):
    """The oracle timed on the host cores on one whole step of the workload
    itself (n = 8810, 128 solves): measured, not scaled from a smaller grid."""
    import oracle as O
    t = oracle_step(p)
    return {"value": round(len(p.pair_f) / t, 6), "unit": "solves/s", "cores": O.num_threads(), "kind": "oracle",
            "sample": f"one full step of the workload: oracle solve (assembly, Householder + implicit QR "
                      f"eigendecomposition, spectral apply) of the ellipse128 grid itself, n={p.n}, "
                      f"{len(p.pair_f)} solves, {t:.1f} s wall"}


def run_reference(args, rank, world):
    """The oracle arm.  One step of the workload takes minutes on the host
    cores, so it times whole steps until the first one that ends past
    REFERENCE_BUDGET_S (at least one, at most --steps), without warm-up, and
    prints the number of steps it really timed."""
    if rank != 0:
        return
    import oracle as O
    p = _workload()
    times = []
    t_start = time.perf_counter()
    while len(times) < max(1, args.steps):
        times.append(oracle_step(p))
        if time.perf_counter() - t_start > REFERENCE_BUDGET_S:
            break
    t = statistics.mean(times)
    value = len(p.pair_f) / t
    line = {
        "metric": METRIC, "impl": "reference", "value": round(value, 6), "unit": "solves/s",
        "n_gpus": world, "steps": len(times), "warmup": 0, "steps_requested": args.steps,
        "warmup_requested": args.warmup, "ms_per_step": round(t * 1e3, 1),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded masked grid and polynomial forcings)",
        "config": _config(p, {"parallelism": "host cores (OpenMP)"}),
        "cpu_baseline": {"value": round(value, 6), "unit": "solves/s", "cores": O.num_threads(), "kind": "oracle",
                         "sample": f"{len(times)} whole step(s) of the workload itself (n={p.n}, "
                                   f"{len(p.pair_f)} solves each), no warm-up: one step takes minutes, so the "
                                   f"{args.steps} requested steps are cut after {REFERENCE_BUDGET_S:.0f} s"},
        "e2e": {"value": round(value, 6), "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def _timed_line(args, metric, unit, per_step_units, step, ctx, extra, steps=None, warmup=None):
    """Warm-up, then K timed steps between CUDA events on the current stream
    (clocks sampled meanwhile); returns the common JSON fields."""
    import torch
    steps = args.steps if steps is None else steps
    warmup = args.warmup if warmup is None else warmup
    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    launches0 = ctx.launch_count()
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        step()
    e1.record()
    torch.cuda.synchronize()
    clk = clocks.stop()
    ctx.sync()
    ms = e0.elapsed_time(e1) / steps
    line = {"metric": metric, "value": round(per_step_units / (ms * 1e-3), 4), "unit": unit, "n_gpus": 1,
            "steps": steps, "warmup": warmup, "ms_per_step": round(ms, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "data": "synthetic (seeded masked grids and forcings)",
            "gpu_launches": (ctx.launch_count() - launches0) // steps, "clocks": clk}
    line.update(extra)
    return line


def _worst(acc_list):
    """Worst value per key over several accuracy dicts (booleans: all true)."""
    worst = {}
    for acc in acc_list:
        for key, v in acc.items():
            worst[key] = (worst.get(key, True) and v) if isinstance(v, bool) else max(worst.get(key, 0.0), v)
    return worst


def _u_rel(U, U_o):
    """Largest relative L2 error over the columns of U against U_o (host arrays)."""
    return float(np.max(np.linalg.norm(U - U_o, axis=0) / np.linalg.norm(U_o, axis=0)))


def run_square_bench(args, steps=None, warmup=None):
    """The plain FP64 method on the 48 x 48 unit square (n = 2304, h = 1/49):
    one step = assembly, eig_full and frac_apply of 5 forcings x 4 orders
    (20 solves); compared with the oracle's whole solve on the host."""
    import torch
    import oracle as O
    import paper_1911_11906_gb300 as F
    from paper_1911_11906_gb300 import inputs as I
    p = I.square_problem(48)
    ctx = F.Context(band_width=32)
    mask = torch.from_numpy(p.mask).cuda()
    Fd = torch.from_numpy(np.ascontiguousarray(p.F.T)).cuda().t()
    pf = torch.from_numpy(p.pair_f.astype(np.int32)).cuda()
    pa = torch.from_numpy(p.pair_alpha.astype(np.float64)).cuda()
    ws = torch.empty(ctx.lib.fraclap_eig_workspace_bytes(ctx.handle, p.n), dtype=torch.uint8, device="cuda")
    U = F._binding.empty_colmajor(p.n, len(p.pair_f), "cuda")
    state = {}

    def step():
        asm = F.fd_assemble(mask, p.h, ctx=ctx)
        state["lam"], V = F.eig_full(asm["A"], ctx=ctx, workspace=ws, sync=False)
        F.frac_apply(V, state["lam"], Fd, pf, pa, ctx=ctx, out=U, sync=False)

    line = _timed_line(args, "fractional solves/s, plain FP64 method (square48, n=2304)", "solves/s",
                       len(p.pair_f), step, ctx,
                       {"dtype": "f64", "config": {"workload": "square48: 48x48 unit square, h=1/49, n=2304, "
                                                               "sin(pi x) sin(pi y) + 4 cubic forcings x 4 alpha",
                                                   "n": p.n, "band_width": 32,
                                                   "l2_policy": "no flush (42 MB matrix, L2-resident)"}},
                       steps=steps, warmup=warmup)
    lam_o, _, U_o = O.solve(p.mask, p.h, p.F, p.pair_f, p.pair_alpha)
    lam_g = state["lam"].cpu().numpy()
    line["accuracy_vs_oracle"] = {"lambda_rel_max": float(np.max(np.abs(lam_g - lam_o) / lam_o)),
                                  "u_rel_l2_max": _u_rel(U.cpu().numpy(), U_o)}
    line["accuracy_vs_oracle"]["meets_fp64_bar"] = bool(line["accuracy_vs_oracle"]["lambda_rel_max"] <= 1e-11
                                                        and line["accuracy_vs_oracle"]["u_rel_l2_max"] <= 1e-10)
    return line


def run_batched_bench(args, steps=None, warmup=None):
    """Many small problems: 256 masked grids (side U{20..64}, n 150..2559), each
    with 8 forcings x 4 orders; one step = fraclap_solve_batched over all of
    them (mixed route), assembly included, inputs resident.  The number of
    concurrent workers comes from the autotuner (measured on this batch on
    first use, then cached).  Four sampled problems are compared with the
    oracle's whole solve."""
    import torch
    import oracle as O
    import paper_1911_11906_gb300 as F
    from paper_1911_11906_gb300 import autotune
    from paper_1911_11906_gb300 import inputs as I
    probs = I.batched_problems(256)
    ctx = F.Context()
    items = []
    for p in probs:
        items.append({"mask": torch.from_numpy(p.mask).cuda(), "h": p.h, "pair_f": p.pair_f,
                      "pair_alpha": p.pair_alpha, "F": torch.from_numpy(np.ascontiguousarray(p.F.T)).cuda().t()})
    state = {}

    def assemble_all():
        batch = []
        for it in items:
            asm = F.fd_assemble(it["mask"], it["h"], ctx=ctx)
            batch.append({"A": asm["A"], "rowptr": asm["rowptr"], "col": asm["col"], "val": asm["val"],
                          "F": it["F"], "pair_f": it["pair_f"], "pair_alpha": it["pair_alpha"]})
        return batch

    workers = 16 if args.no_autotune else autotune.best_workers(assemble_all())

    def step():
        state["out"] = F.solve_batched(assemble_all(), workers=workers, ctx=ctx)

    line = _timed_line(args, "batched problems/s: 256 masked grids (n 150..2559), eigendecomposition + 32 solves each",
                       "problems/s", len(probs), step, ctx,
                       {"dtype": "f32+f64-refined",
                        "config": {"workload": "batched256: 256 ellipse grids, side U{20..64}, 8 forcings x 4 alpha",
                                   "n_min": int(min(p.n for p in probs)), "n_max": int(max(p.n for p in probs)),
                                   "n_mean": float(np.mean([p.n for p in probs])), "workers": workers,
                                   "workers_source": "fixed" if args.no_autotune else "autotuner",
                                   "route": "mixed per problem", "l2_policy": "no flush (many small problems)"}},
                       steps=steps, warmup=warmup)
    accs = []
    for q in (0, 85, 170, 255):
        p, (lam, V, U) = probs[q], state["out"][q]
        lam_o, _, U_o = O.solve(p.mask, p.h, p.F, p.pair_f, p.pair_alpha)
        lam_g = lam.cpu().numpy()
        accs.append({"lambda_rel_max": float(np.max(np.abs(lam_g - lam_o) / lam_o)),
                     "u_rel_l2_max": _u_rel(U.cpu().numpy(), U_o)})
    line["accuracy_vs_oracle_sampled_problems"] = _worst(accs)
    line["accuracy_vs_oracle_sampled_problems"]["sampled"] = [0, 85, 170, 255]
    line["solves_per_s"] = round(line["value"] * 32, 2)
    return line


def run_apply_bench(args, diffusion=False, steps=None, warmup=None):
    """The apply at scale: 192 x 192 grid (n = 18278), 4096 distinct forcings
    with alpha ~ U(0.1, 1.9); (V, lambda) computed once beforehand; one step =
    frac_apply of all 4096 pairs with the products as 6 BF16 slices on the
    tensor cores (FP64 products timed beside it, and the same apply replayed
    as one captured CUDA graph).  64 sampled pairs are compared with the
    oracle's apply on the same (V, lambda).  With diffusion=True the step is
    frac_diffusion instead: the 4096 columns are initial states evolved to the
    paper's t = 0.4 with mu = 1."""
    import torch
    import oracle as O
    import paper_1911_11906_gb300 as F
    from paper_1911_11906_gb300 import inputs as I
    from paper_1911_11906_gb300 import autotune
    p = I.apply_at_scale_problem()
    ctx = F.Context(band_width=64)
    mask = torch.from_numpy(p.mask).cuda()
    asm = F.fd_assemble(mask, p.h, ctx=ctx)
    lam, V = F.eig_full_mixed(asm["A"], asm["rowptr"], asm["col"], asm["val"], refine_iters=6, ctx=ctx)
    del asm
    # tile order and width of the sliced products from the autotuner (V^T F shape, 6 slices)
    sched = {} if args.no_autotune else autotune.best_ozaki_schedule(p.n, slices=6, cols=p.F.shape[1])
    autotune.apply_schedule(ctx, sched)
    Fd = torch.from_numpy(np.ascontiguousarray(p.F.T)).cuda().t()
    pf = torch.from_numpy(p.pair_f.astype(np.int32)).cuda()
    pa = torch.from_numpy(p.pair_alpha.astype(np.float64)).cuda()
    k = len(p.pair_f)
    pt = torch.full((k,), 0.4, dtype=torch.float64, device=mask.device)
    U = F._binding.empty_colmajor(p.n, k, mask.device)
    metric = ("fractional diffusion solves/s at <=1e-10 err vs FP64 (n=18278, t=0.4)" if diffusion else
              "fractional solves/s at <=1e-10 err vs FP64 (apply at scale, n=18278)")
    lines = {}
    for slices in (0, 6):
        ctx.set_apply_slices(slices)
        ws = torch.empty(ctx.lib.fraclap_apply_workspace_bytes_ctx(ctx.handle, p.n, Fd.shape[1], k),
                         dtype=torch.uint8, device=mask.device)

        def step():
            if diffusion:
                F.frac_diffusion(V, lam, Fd, pf, pa, pt, mu=1.0, ctx=ctx, out=U, workspace=ws, sync=False)
            else:
                F.frac_apply(V, lam, Fd, pf, pa, ctx=ctx, out=U, workspace=ws, sync=False)

        lines[slices] = _timed_line(args, metric, "solves/s", k, step, ctx, {}, steps=steps, warmup=warmup)
        lines[slices]["U"] = U.clone()
    # the same 6-slice apply captured once and replayed as one graph launch
    ctx.set_apply_slices(6)
    G = F.ApplyGraph(V, lam, Fd, pf, pa, pair_t=pt if diffusion else None, mu=1.0, ctx=ctx)
    gline = _timed_line(args, metric, "solves/s", k, lambda: G.launch(sync=False), ctx, {}, steps=steps,
                        warmup=warmup)
    graph_rel = float((torch.linalg.norm(G.U - lines[6]["U"], dim=0) / torch.linalg.norm(lines[6]["U"], dim=0)).max())
    graph = {"value": gline["value"], "ms_per_step": gline["ms_per_step"], "kernels": G.kernels,
             "u_rel_l2_vs_direct_max": graph_rel}
    G.close()
    # the oracle on the same (V, lambda): 64 sampled pairs, both product routes
    rng = np.random.default_rng(18278)
    sample = np.sort(rng.choice(k, size=64, replace=False))
    used, remap = np.unique(p.pair_f[sample], return_inverse=True)
    V_h, lam_h = V.cpu().numpy(), lam.cpu().numpy()
    if diffusion:
        U_o = O.frac_diffusion(V_h, lam_h, p.F[:, used], remap.astype(np.int32), p.pair_alpha[sample],
                               np.full(64, 0.4), mu=1.0)
    else:
        U_o = O.frac_apply(V_h, lam_h, p.F[:, used], remap.astype(np.int32), p.pair_alpha[sample])
    del V_h
    idx = torch.from_numpy(sample).cuda()
    err_o = {s_: _u_rel(lines[s_]["U"][:, idx].cpu().numpy(), U_o) for s_ in (0, 6)}
    d = lines[6].pop("U") - lines[0].pop("U")
    rel = float((torch.linalg.norm(d, dim=0) / torch.linalg.norm(U, dim=0)).max())
    head = lines[6]
    acc = {"u_rel_l2_vs_fp64_products_max": rel, "u_rel_l2_vs_oracle_sampled_max": err_o[6],
           "fp64_products_u_rel_l2_vs_oracle_sampled_max": err_o[0], "oracle_sampled_pairs": 64}
    if diffusion:
        # semigroup evidence on 8 states: S(0.3) S(0.1) u0 = S(0.4) u0, 6 slices
        f8 = torch.arange(8, dtype=torch.int32, device=mask.device)
        half = F.frac_diffusion(V, lam, Fd, f8, pa[:8], torch.full((8,), 0.1, dtype=torch.float64,
                                                                   device=mask.device), ctx=ctx)
        two = F.frac_diffusion(V, lam, half, f8, pa[:8], torch.full((8,), 0.3, dtype=torch.float64,
                                                                    device=mask.device), ctx=ctx)
        F.frac_diffusion(V, lam, Fd, pf, pa, pt, mu=1.0, ctx=ctx, out=U)
        acc["semigroup_rel_l2_max"] = float((torch.linalg.norm(two - U[:, :8], dim=0)
                                             / torch.linalg.norm(U[:, :8], dim=0)).max())
        workload = ("diffusion192: 192x192 ellipse grid, n=%d, 4096 distinct initial states, alpha~U(0.1,1.9), "
                    "t=0.4, mu=1" % p.n)
    else:
        # alpha = 2 evidence: solve with the same V, lambda for 8 forcings, against CG
        f8 = torch.arange(8, dtype=torch.int32, device=mask.device)
        U2 = F.frac_apply(V, lam, Fd, f8, torch.full((8,), 2.0, dtype=torch.float64, device=mask.device), ctx=ctx)
        A = _csr(F, mask, p.h, ctx)
        Ug = _cg(A, Fd[:, :8].contiguous())
        acc["u_rel_l2_alpha2_vs_cg_max"] = float((torch.linalg.norm(U2 - Ug, dim=0) / torch.linalg.norm(Ug, dim=0)).max())
        workload = "apply192: 192x192 ellipse grid, n=%d, 4096 distinct forcings, alpha~U(0.1,1.9)" % p.n
    acc["meets_1e-10"] = bool(rel <= 1e-10 and err_o[6] <= 1e-10 and acc.get("u_rel_l2_alpha2_vs_cg_max", 0) <= 1e-10)
    head.update({"dtype": "bf16 slices (6 per operand) into fp64",
                 "config": {"workload": workload, "n": p.n, "pairs": k, "products": "6 BF16 slices on tcgen05",
                            "l2_policy": "inputs larger than L2 (V is %.1f GB)" % (8 * p.n * p.n / 1e9)},
                 "fp64_products": {"value": lines[0]["value"], "ms_per_step": lines[0]["ms_per_step"]},
                 "cuda_graph": graph, "accuracy": acc,
                 "slice_product_schedule": dict(sched, source="autotuner") if sched else "defaults"})
    return head


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="fraclap", choices=["fraclap", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--path", default="both", choices=["both", "fp64", "mixed"],
                    help="eigendecomposition route(s) to time; the headline is the fastest that meets the FP64 bar")
    ap.add_argument("--jsonl", default="", metavar="PATH",
                    help="also append one JSONL metrics record per timed route to PATH")
    ap.add_argument("--workload", default="ellipse128",
                    choices=["ellipse128", "square48", "batched256", "apply192", "diffusion192"],
                    help="ellipse128: the headline workload (its line also carries the square48, batched256 "
                         "and apply192 results under 'configs'); the others: that workload alone, one line")
    ap.add_argument("--no-configs", action="store_true",
                    help="leave the other workloads out of the headline line")
    ap.add_argument("--no-autotune", action="store_true",
                    help="fixed band width and worker count instead of the autotuner's")
    args = ap.parse_args()
    if args.workload != "ellipse128" and args.impl == "fraclap":
        # single-GPU workloads: under torchrun, rank 0 runs them on its own GPU
        # and prints the one line; the other ranks leave without work
        if int(os.environ.get("RANK", "0")) != 0:
            return
        import torch
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    if args.workload == "square48":
        print(json.dumps(run_square_bench(args)), flush=True)
        return
    if args.workload == "batched256":
        print(json.dumps(run_batched_bench(args)), flush=True)
        return
    if args.workload in ("apply192", "diffusion192"):
        print(json.dumps(run_apply_bench(args, diffusion=args.workload == "diffusion192")), flush=True)
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if world > 1:
        import torch
        torch.cuda.set_device(local_rank)
        torch.distributed.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    try:
        run_gpu(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch
            torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
