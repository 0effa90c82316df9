"""Benchmark: Poisson solves of the 32^3-element, p=7 deformed box (FP64 method).

One step = one whole solve (x0 = 0) of the pressure-Poisson problem with flexible PCG to a
relative residual of 1e-8, preconditioned by the p-multigrid V-cycle 7->5->3->1 with a
Chebyshev-accelerated RAS or Jacobi smoother of order 1..3 (chosen during set-up by the paper's
run-time preconditioner search, Sec. 5; --smoother fixes it) and a p=1 Jacobi-PCG coarse solve,
all in FP64.
value = gridpoints solved per second, n = E p^3 per solve (the paper's work-rate measure),
summed over ranks.  Inputs (mesh, geometry, FDM factors, right-hand side) are resident in HBM
before the timed region; every step works on ~12 GB of state, far larger than L2.

--impl reference runs the FP64 CPU oracle (test infrastructure) on a bounded sample of the same
workload instead.  N > 1: independent replicas, one problem per rank (weak scaling).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    "box32_p7": dict(nel=(32, 32, 32), p=7, perturb=0.05, seed=0, schedule=(7, 5, 3, 1)),
    "box24_p7": dict(nel=(24, 24, 24), p=7, perturb=0.05, seed=0, schedule=(7, 5, 3, 1)),
    "box16_p7": dict(nel=(16, 16, 16), p=7, perturb=0.05, seed=0, schedule=(7, 5, 3, 1)),
    "box4_p7": dict(nel=(4, 4, 4), p=7, perturb=0.0, seed=0, schedule=(7, 3, 1)),
}
SAMPLE = dict(nel=(10, 10, 10), p=7, perturb=0.05, seed=0, schedule=(7, 5, 3, 1))
METRIC = "Poisson solve time & Ax/smoother GDOF/s (%HBM roof); served solves/s, p99"
FP64_FMA_PER_CLK_PER_SM = 2      # GB300: 1.25 TFLOP/s FP64 nominal at 152 SMs x 2.07 GHz
N_SMS_NOMINAL = 152              # used only when no device is there to ask (host-side tests)


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), \
        int(os.environ.get("LOCAL_RANK", 0))


def max_over_ranks(value, world):
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64,
                     device="cuda" if dist.get_backend() == "nccl" else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value, world):
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64,
                     device="cuda" if dist.get_backend() == "nccl" else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [ln for ln in out.splitlines() if ln.strip()]

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


VARIANT_KIND = ("f64", "f32", "df64")
DF64_INSTR_PER_FLOP = 7.5   # a df64 FMA (2 flops) is 15 FP32 instructions (see csrc/df64.h)


def alu_peak_tflops(kind, sm_max_mhz, sms=N_SMS_NOMINAL):
    """Derived ALU peak: SMs x (128 FP32 | 2 FP64) FMA lanes per clock x 2 flop x clock;
    df64: the FP32 instruction rate (SMs x 128 x clock) / 7.5 FP32 instructions per df64 flop.
    The SM count is the device's (cudaDevAttrMultiProcessorCount) when a device is present."""
    if kind == "df64":
        return sms * 128 * sm_max_mhz * 1e6 / DF64_INSTR_PER_FLOP / 1e12
    return sms * (128 if kind == "f32" else FP64_FMA_PER_CLK_PER_SM) * 2 * sm_max_mhz * 1e6 / 1e12


def _profile_entry(kernel, variant):
    try:
        with open(os.path.join(ROOT, "profiles", "dram_traffic.json")) as f:
            tab = json.load(f)
    except OSError:
        return None
    return tab.get(f"{kernel}:{variant}")


def dram_traffic(kernel, variant):
    """DRAM bytes per launch from the committed ncu capture summary, if one matches."""
    e = _profile_entry(kernel, variant)
    if not e:
        return None, None
    return e["bytes_per_launch_bench_workload"], e["source"]


def pipe_busy(kernel, variant):
    """Executed-instruction pipe utilisation of the kernel from its committed ncu capture."""
    e = _profile_entry(kernel, variant)
    return e.get("pipe_busy_ncu") if e else None


def roofline(kernel, variant, d, pk, pk_kind):
    """Bound = the roof that takes longer for this kernel's algorithmic bytes and flops."""
    kind = VARIANT_KIND[variant // 32]
    fp32 = kind == "f32"
    sm_max = pk.get("sm_max_mhz", 2070.0)
    sms = pk.get("sms", N_SMS_NOMINAL)
    alu = alu_peak_tflops(kind, sm_max, sms)
    hbm = pk["hbm_gbs"]
    n = max(d["launches"], 1)
    avg_s = d["ms"] / n * 1e-3
    t_alu = d["flops"] / (alu * 1e12)
    t_hbm = d["bytes"] / (hbm * 1e9)
    traffic, src = dram_traffic(kernel, variant)
    name = f"{kernel} p={variant % 32} {kind}"
    if t_alu >= t_hbm:
        achieved = d["flops"] / n / avg_s / 1e12
        return {"bound": "alu", "kernel": name, "achieved": round(achieved, 4), "peak": round(alu, 4),
                "unit": "TFLOP/s", "frac": round(achieved / alu, 4), "traffic": traffic,
                "algorithmic_bytes_per_launch": d["bytes"] / n, "flops_per_launch": d["flops"] / n,
                "avg_launch_ms": round(avg_s * 1e3, 4), "traffic_source": src,
                "pipe_busy_ncu": pipe_busy(kernel, variant),
                "peak_source": (f"derived: {sms} SMs x 128 FP32 instr/clk x {sm_max:.0f} MHz / "
                                f"{DF64_INSTR_PER_FLOP} FP32 instr per df64 flop") if kind == "df64" else
                               (f"derived: {sms} SMs x {128 if fp32 else 2} {'FP32' if fp32 else 'FP64'} "
                                f"FMA/clk x 2 flop x {sm_max:.0f} MHz"),
                "measured_alu_tflops": pk.get("measured_alu_tflops")}
    achieved = d["bytes"] / n / avg_s / 1e9
    return {"bound": "hbm", "kernel": name, "achieved": round(achieved, 1), "peak": hbm,
            "unit": "GB/s", "frac": round(achieved / hbm, 4), "traffic": traffic,
            "algorithmic_bytes_per_launch": d["bytes"] / n, "flops_per_launch": d["flops"] / n,
            "avg_launch_ms": round(avg_s * 1e3, 4), "traffic_source": src,
            "peak_source": f"{pk_kind} (MEASURED_PEAKS.json hbm_gbs)" if pk_kind == "measured"
            else "fallback 6.8 TB/s"}


def profiled_variants(se, solve, steps, stream, label="profiled_pass"):
    """Runs `solve` (host-driven) `steps` times with every library launch bracketed by CUDA events
    on its stream; returns (ms per solve of the pass, per-class totals, per-variant totals).  The
    pass is an NVTX range named `label` (the headline's: "profiled_pass"), so that a profiler can
    select exactly these launches."""
    import torch
    se.se_prof_reset()
    se.se_prof_enable(True)
    p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.nvtx.range_push(label)
    p0.record(stream)
    for _ in range(steps):
        solve()
    p1.record(stream)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    se.se_prof_enable(False)
    prof = {se.KERNEL_NAMES[k]: se.se_prof_query(k) for k in range(se.SE_K_COUNT)}
    variants = {}
    for k in range(se.SE_K_COUNT):
        for v in range(96):
            q = se.se_prof_query_variant(k, v)
            if q["launches"]:
                variants[(se.KERNEL_NAMES[k], v)] = q
    return p0.elapsed_time(p1) / steps, prof, variants


def kernel_table(variants, steps, pk, pk_kind):
    """Per kernel class x level order x precision: time per step, launches, share, and the
    fraction of its own binding roof (algorithmic bytes or flops per launch)."""
    tot_ms = max(sum(v["ms"] for v in variants.values()), 1e-9)
    kernels = {}
    for (k, v), q in sorted(variants.items(), key=lambda kv: -kv[1]["ms"]):
        r = roofline(k, v, q, pk, pk_kind) if q["ms"] > 0 and (q["bytes"] > 0 or q["flops"] > 0) else None
        kernels[f"{k} p={v % 32} {VARIANT_KIND[v // 32]}"] = {
            "ms_per_step": round(q["ms"] / steps, 3),
            "launches_per_step": q["launches"] / steps, "share": round(q["ms"] / tot_ms, 4),
            "bound": r["bound"] if r else None, "roof_frac": r["frac"] if r else None}
    return kernels


def measured_alu(se, stream):
    """FMA throughput measured on this device (se_prof_fma_peak) and its SM count."""
    out, sms = {}, None
    for kind, name in ((0, "f64"), (1, "f32"), (2, "f32x2")):
        t, sms = se.se_prof_fma_peak(kind, stream)
        out[name] = round(t, 3)
    return out, sms


def schwarz_record(se, m, b, x, stream, wk, pk, pk_kind, op_df, steps):
    """The paper's own smoother on the same mesh and right-hand side: Cheby-RAS(2) on the
    workload's schedule, with the FP64 V-cycle and with the FP32 V-cycle (FP64 Krylov), each
    timed as graph solves, then profiled host-driven for its FDM kernels' roof fractions."""
    import torch
    rec = {}
    for name, prec in (("fp64", se.SE_FP64), ("fp32_vcycle", se.SE_FP32)):
        t0 = time.perf_counter()
        P = se.se_pmg_setup(m, se.pmg_desc(wk["schedule"], se.SE_SMOOTH_RAS, 2, precision=prec))
        torch.cuda.synchronize()
        setup_ms = (time.perf_counter() - t0) * 1e3
        try:
            def solve(graph=1):
                x.zero_()
                return se.se_solve(m, P, b, x, tol=1e-8, maxit=500, stream=stream,
                                   graph_capture=graph, operator_df64=op_df)
            for _ in range(2):
                st = solve()
            k = max(2, min(steps, 5))
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(k):
                st = solve()
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / k
            solve(graph=0)
            torch.cuda.synchronize()
            _, _, variants = profiled_variants(se, lambda: solve(graph=0), 1, stream,
                                               label="profiled_pass_schwarz")
            table = kernel_table(variants, 1, pk, pk_kind)
            fdm = {}
            for (kk, v), q in variants.items():
                if kk == "fdm":
                    r = roofline(kk, v, q, pk, pk_kind)
                    fdm[r["kernel"]] = {"ms_per_launch": r["avg_launch_ms"],
                                        "launches_per_solve": q["launches"], "bound": r["bound"],
                                        "achieved": r["achieved"], "unit": r["unit"],
                                        "peak": r["peak"], "roof_frac": r["frac"],
                                        "algorithmic_bytes_per_launch": r["algorithmic_bytes_per_launch"],
                                        "flops_per_launch": r["flops_per_launch"]}
            rec[name] = {"preconditioner": "Cheby-RAS(2)", "schedule": list(wk["schedule"]),
                         "precision": "FP64 V-cycle" if prec == se.SE_FP64
                         else "FP32 V-cycle, FP64 Krylov/coarse/Arnoldi",
                         "ms_per_solve": round(ms, 3), "timed_solves": k,
                         "iterations": st.iterations, "rel_residual": st.rel_residual,
                         "setup_ms": round(setup_ms, 1), "fdm": fdm,
                         "kernels": dict(list(table.items())[:6])}
        finally:
            se.se_pmg_destroy(P)
    return rec


def run_peaks(args):
    """ALU roofs of this GPU (FMA throughput, se_prof_fma_peak) next to the derived peaks the
    roofline divides by, with the clocks sampled while the probes ran."""
    import torch
    from paper_2110_07663_gb300 import se
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    se.se_prof_fma_peak(1, stream)  # warm-up: clocks ramp, module load
    with ClockSampler(0) as clk:
        meas, sms = {}, None
        for _ in range(3):
            for kind, name in ((0, "f64"), (1, "f32"), (2, "f32x2"), (3, "tf32_mma_sync")):
                t, sms = se.se_prof_fma_peak(kind, stream)
                meas[name] = max(meas.get(name, 0.0), round(t, 3))
    pk, _ = peaks()
    sm_max = pk.get("sm_max_mhz", 2070.0)
    derived = {k: round(alu_peak_tflops(k, sm_max, sms), 4) for k in ("f64", "f32", "df64")}
    print(json.dumps({"measured_fma_tflops": meas, "sms": sms, "derived_tflops": derived,
                      "derived_from": f"{sms} SMs x FMA lanes/clk (FP64 2, FP32 128) x 2 flop x "
                                      f"{sm_max:.0f} MHz",
                      "tf32_mma_sync_over_f32x2": round(meas["tf32_mma_sync"] / meas["f32x2"], 3),
                      "frac_of_derived": {"f64": round(meas["f64"] / derived["f64"], 4),
                                          "f32": round(meas["f32"] / derived["f32"], 4),
                                          "f32x2": round(meas["f32x2"] / derived["f32"], 4)},
                      "clocks": clk.summary(),
                      "gpu": torch.cuda.get_device_name(0)}))


def run_gpu(args):
    import numpy as np
    import torch

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_2110_07663_gb300 import se
    import workloads as wl

    wk = WORKLOADS[args.workload]
    nel, p = wk["nel"], wk["p"]
    m = se.se_mesh_create(nel, p, perturb_frac=wk["perturb"], seed=wk["seed"] + rank,
                          deform_amp=wl.DEFORM_AMP, flags=se.SE_MESH_GS_MAP if args.gs_map else 0)
    info = se.se_mesh_get_info(m)
    L = info.L
    xyz = torch.empty(3 * L, dtype=torch.float64, device=dev)
    se.se_mesh_nodes(m, xyz)
    X = xyz.view(3, L)
    f = 3.0 * math.pi ** 2 * torch.sin(math.pi * X[0]) * torch.sin(math.pi * X[1]) * torch.sin(math.pi * X[2])
    b = torch.empty(L, dtype=torch.float64, device=dev)
    se.se_mesh_rhs(m, f.contiguous(), b)
    del xyz, X, f
    prec = se.SE_FP32 if args.precond_fp32 else (se.SE_DF64 if args.df64 else se.SE_FP64)
    op_df = 1 if (args.df64 or args.operator_df64) else 0
    sm_names = {se.SE_SMOOTH_RAS: "RAS", se.SE_SMOOTH_JACOBI: "Jac", se.SE_SMOOTH_ASM: "ASM"}
    t_setup0 = time.perf_counter()
    tiles = None
    if args.tune_tiles:
        # the project's launch-tile autotuner for every order of the schedule (set-up, untimed)
        prec_t = se.SE_FP32 if args.precond_fp32 else se.SE_FP64
        tiles = {}
        for pp in sorted(q for q in set(wk["schedule"]) if q >= 2):
            t64 = se.se_tune(pp, se.SE_FP64)
            tiles[f"p={pp} f64"] = [t64.ax_elems_per_block, t64.fdm_elems_per_block]
            if prec_t == se.SE_FP32:
                t32 = se.se_tune(pp, se.SE_FP32)
                tiles[f"p={pp} f32"] = [t32.ax_elems_per_block, t32.fdm_elems_per_block]
    search = None
    if args.smoother == "auto":
        # the method's run-time preconditioner selection (Sec. 5) over the workload's smoother set,
        # Cheby-RAS(k) and Cheby-Jac(k), k = 1..3: each set up and timed on the first solves
        # (untimed here, part of the set-up); the fastest is kept for the timed steps
        cands = []
        for sm in (se.SE_SMOOTH_RAS, se.SE_SMOOTH_JACOBI):
            for k in (1, 2, 3):
                c = se.se_tune_candidate()
                c.pmg = se.pmg_desc(wk["schedule"], sm, k, precision=prec)
                cands.append(c)
        best, timed, P = se.se_pmg_autotune(m, b, cands, repeats=2, tol=1e-8, maxit=500,
                                            operator_df64=op_df)
        search = [{"preconditioner": f"Cheby-{sm_names[c.pmg.smoother]}({c.pmg.cheb_order[0]})",
                   "solve_ms": round(c.ms, 2), "iterations": c.iterations} for c in timed]
        smoother, cheb_order = timed[best].pmg.smoother, timed[best].pmg.cheb_order[0]
    else:
        smoother = {"ras": se.SE_SMOOTH_RAS, "jacobi": se.SE_SMOOTH_JACOBI, "asm": se.SE_SMOOTH_ASM}[args.smoother]
        cheb_order = args.cheb_order
        P = se.se_pmg_setup(m, se.pmg_desc(wk["schedule"], smoother, cheb_order, precision=prec,
                                           cycle=se.SE_CYCLE_ADDITIVE if args.cycle == "additive"
                                           else se.SE_CYCLE_MULTIPLICATIVE))
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t_setup0
    x = torch.zeros(L, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream()

    # One step = one whole solve through the public API, device-driven: se_solve with
    # graph_capture=1 runs the FPCG loop as one CUDA graph (WHILE/IF conditional nodes, no host
    # round trip per iteration); the graph is captured on the first call and replayed after.
    def step(graph=1):
        x.zero_()
        return se.se_solve(m, P, b, x, tol=1e-8, maxit=500, stream=stream, graph_capture=graph,
                           operator_df64=op_df)

    for _ in range(args.warmup):
        st = step()
    iters = st.iterations
    # ---- timed region (device-resident inputs, no per-kernel events)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        e0.record(stream)
        for _ in range(args.steps):
            st = step()
        e1.record(stream)
        torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    ms_max = max_over_ranks(ms, world)
    assert st.iterations == iters
    # ---- profiled pass: the same solve host-driven (same kernels, same result), every launch
    # bracketed by CUDA events on its stream; gives the per-kernel times and the roofline
    step(graph=0)
    torch.cuda.synchronize()
    se.se_pmg_coarse_stats(P, reset=True)
    host_loop_ms, prof, variants = profiled_variants(se, lambda: step(graph=0), args.steps, stream)
    coarse_solves, coarse_iters = se.se_pmg_coarse_stats(P)
    # our kernels per timed step: those of the profiled pass plus the graph's own control
    # kernels (one at the start, one convergence test per iteration)
    launches = sum(v["launches"] for v in prof.values()) + args.steps * (1 + iters)
    # ---- end to end through the public API with host buffers (copies inside the timed region)
    # (se_solve_host: b copied in, x from zero, x copied out, all inside the library call)
    b_host = b.cpu().pin_memory()
    x_host = torch.empty(L, dtype=torch.float64).pin_memory()
    torch.cuda.synchronize()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e2e_steps = max(1, min(args.steps, 5))
    se.se_solve_host(m, P, b_host, x_host, tol=1e-8, maxit=500, stream=stream, graph_capture=1,
                     operator_df64=op_df)  # captures
    torch.cuda.synchronize()
    f0.record(stream)
    for _ in range(e2e_steps):
        se.se_solve_host(m, P, b_host, x_host, tol=1e-8, maxit=500, stream=stream, graph_capture=1,
                         operator_df64=op_df)
    f1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks(f0.elapsed_time(f1) / e2e_steps, world)
    n_dof = info.n_dof
    total_dof = sum_over_ranks(float(n_dof), world)
    value = total_dof / (ms_max * 1e-3) / 1e9
    e2e_value = total_dof / (e2e_ms * 1e-3) / 1e9
    prec_name = {se.SE_FP64: "FP64", se.SE_FP32: "FP32", se.SE_DF64: "df64"}[prec]
    op_name = "df64" if op_df else "FP64"
    dtype = {se.SE_FP64: "f64", se.SE_FP32: "f64+f32", se.SE_DF64: "f64+df64"}[prec]
    if prec == se.SE_FP64 and op_df:
        dtype = "f64+df64"
    # ---- roofline of the dominant kernel (kernel class x level order x precision)
    pk, pk_kind = peaks()
    pk["measured_alu_tflops"], pk["sms"] = measured_alu(se, stream)
    (dom, dvar), d = max(variants.items(), key=lambda kv: kv[1]["ms"])
    roof = roofline(dom, dvar, d, pk, pk_kind)
    kernels = kernel_table(variants, args.steps, pk, pk_kind)
    coarse = None
    if coarse_solves and "coarse_pcg" in prof and prof["coarse_pcg"]["launches"]:
        # the coarse Jacobi-PCG: latency-bound (one grid synchronisation per iteration); its FP64
        # work per iteration and node: 27-point product 54 flops, preconditioner 1, six vector
        # updates 12, three inner products 6, direction updates 4 -> 77 flops
        n_c = se.se_pmg_level_info(P, len(wk["schedule"]) - 1).n_global
        ms_c = prof["coarse_pcg"]["ms"]
        us_it = ms_c * 1e3 / max(coarse_iters, 1)
        tf = 77.0 * n_c * coarse_iters / (ms_c * 1e-3) / 1e12
        fp64_peak = alu_peak_tflops("f64", pk.get("sm_max_mhz", 2070.0), pk["sms"])
        coarse = {"solves_per_step": coarse_solves / args.steps,
                  "iterations_per_solve": round(coarse_iters / coarse_solves, 2),
                  "us_per_iteration": round(us_it, 2), "nodes": n_c,
                  "fp64_tflops": round(tf, 4), "fp64_peak_tflops": round(fp64_peak, 4),
                  "roof_frac": round(tf / fp64_peak, 4),
                  "bound": "latency (one grid synchronisation per iteration)"}
        kernels["coarse_pcg p=0 f64"]["roof_frac"] = coarse["roof_frac"]
        kernels["coarse_pcg p=0 f64"]["bound"] = "alu"
    schwarz = None
    if not args.no_schwarz:
        schwarz = schwarz_record(se, m, b, x, stream, wk, pk, pk_kind, op_df, args.steps)
    out = {
        "metric": METRIC, "value": round(value, 4), "unit": "GDOF/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_max, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": dtype,
        "data": "synthetic",
        "config": {"workload": f"{args.workload}: deformed box {nel[0]}x{nel[1]}x{nel[2]} hex, p={p}, "
                               f"n={n_dof} (E p^3), pMG {'-'.join(map(str, wk['schedule']))} "
                               + (f"{sm_names[smoother]}, additive V-cycle (no Chebyshev), " if args.cycle == "additive"
                                  else f"Cheby-{sm_names[smoother]}({cheb_order}), ")
                               + f"FPCG tol 1e-8, {prec_name} preconditioner, {op_name} outer operator",
                   "iterations": iters, "setup_s": round(setup_s, 2), "tuned_tiles": tiles,
                   "time_to_solution_cold_s": round(setup_s + ms_max * 1e-3, 3),
                   "e2e_scope": ("per step: one se_solve_host call (b host->device, the graph solve from "
                                 "x = 0, x device->host, pinned host buffers); mesh and preconditioner "
                                 "set-up (setup_s, incl. the search) are outside it"),
                   "preconditioner_choice": ("run-time search (Sec. 5) over Cheby-RAS(k), Cheby-Jac(k), "
                                             "k = 1..3, inside set-up" if search else "fixed by --smoother"),
                   "preconditioner_search": search,
                   "solve_path": "se_solve graph_capture=1 (device-driven CUDA graph)",
                   "qqt": ("sorted index map (SE_MESH_GS_MAP)" if args.gs_map
                           else "direction sweeps over the box lattice"),
                   "profiled_pass_ms_per_step": round(host_loop_ms, 3),
                   "profiled_pass": "same solve host-driven, per-kernel CUDA events (kernels, roofline)",
                   "l2": "inputs larger than L2 (about 12 GB of resident state per solve)",
                   "parallelism": f"replicas x{world}"},
        "e2e": {"value": round(e2e_value, 4), "unit": "GDOF/s", "h2d_bytes_per_step": int(8 * L),
                "d2h_bytes_per_step": int(8 * L)},
        "gpu_launches": int(launches),
        "roofline": roof,
        "kernels": kernels,
        "clocks": clk.summary(),
        "coarse": coarse,
        "schwarz": schwarz,
    }
    if rank == 0 and not args.no_cpu_baseline and world == 1:
        out["cpu_baseline"] = cpu_baseline_subprocess(args.cpu_timeout, sm_names[smoother], cheb_order)
    se.se_pmg_destroy(P)
    se.se_mesh_destroy(m)
    del x, b
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    if world == 1 and not args.no_extras:
        # the batched and served modes, measured in the same run after the headline's mesh is
        # freed (outside its timed region)
        bm = batch_measure(64, 3, 3)
        out["batch"] = {"workload": bm["config"]["workload"], "ms_per_batch": bm["ms_per_step"],
                        "value": bm["value"], "unit": bm["unit"], "groups": bm["config"]["groups"],
                        "grouped_problems": bm["config"]["grouped_problems"],
                        "iterations_min_max": bm["config"]["iterations_min_max"],
                        "worst_rel_residual": bm["config"]["worst_rel_residual"],
                        "serial_fp64_ms": bm["serial_fp64"]["ms"],
                        "speedup_over_serial_fp64": bm["serial_fp64"]["speedup_of_batch"],
                        "profiled_pass_ms": bm["profiled_pass_ms"], "roofline": bm["roofline"],
                        "top_kernels": dict(list(bm["kernels"].items())[:6])}
        torch.cuda.empty_cache()
        import workloads as wl_
        free, _ = torch.cuda.mem_get_info()
        reqs = wl_.serve_requests(n=300, rate=200.0, seed=0)
        served = serve_stream(se, reqs, int(0.8 * free), 8, se.SE_FP32)
        serial = serve_stream(se, reqs[:30], int(0.8 * free), 1, se.SE_FP64)
        out["serve"] = {"workload": "first 300 requests of the Poisson-arrival stream at 200/s (E log-uniform "
                                    "in [512, 65536], p in {5,7,9}, 30% resident-mesh reuse), tol 1e-8, "
                                    "8 slots, FP32 V-cycle / FP64 Krylov",
                        "served": served,
                        "one_slot_fp64_first_30": {k: serial[k] for k in ("solves_per_s", "p50_ms", "p99_ms",
                                                                          "completed")}}
    if rank == 0:
        print(json.dumps(out))
    if world > 1:
        torch.distributed.destroy_process_group()


# --------------------------------------------------------------------------------- CPU oracle
ORACLE_SMOOTHERS = {"ras": "ras", "jacobi": "jacobi", "asm": "asm", "RAS": "ras", "Jac": "jacobi",
                    "ASM": "asm"}


def oracle_sample(timeout_s, smoother="ras", order=2):
    """Oracle solve of the bounded sample (same method and tolerance, 10^3 elements)."""
    import numpy as np
    import oracle as o
    import workloads as wl
    V = wl.vertex_lattice(SAMPLE["nel"], SAMPLE["perturb"], SAMPLE["seed"])
    lv, b = o.problem(V, SAMPLE["nel"], SAMPLE["p"], amp=wl.DEFORM_AMP)
    pmg = o.pmg_setup(V, SAMPLE["nel"], SAMPLE["schedule"], smoother=ORACLE_SMOOTHERS[smoother],
                      order=order, amp=wl.DEFORM_AMP)
    t0 = time.perf_counter()
    x, it, rel = o.solve(lv, b, pmg, tol=1e-8)
    t = time.perf_counter() - t0
    n = int(np.prod(SAMPLE["nel"])) * SAMPLE["p"] ** 3
    return n / t / 1e9, t, it


def cpu_baseline_subprocess(timeout_s, smoother="ras", order=2):
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    code = ("import sys, json; sys.path.insert(0, %r); import bench; "
            "v, t, it = bench.oracle_sample(0, %r, %d); print(json.dumps([v, t, it]))"
            % (ROOT, smoother, order))
    try:
        r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True,
                           timeout=timeout_s, env=env)
        v, t, it = json.loads(r.stdout.strip().splitlines()[-1])
    except Exception as e:  # noqa: BLE001
        return {"value": None, "unit": "GDOF/s", "cores": 1, "nproc": os.cpu_count(),
                "kind": "oracle", "sample": f"failed: {type(e).__name__}"}
    return {"value": round(v, 6), "unit": "GDOF/s", "cores": 1, "nproc": os.cpu_count(),
            "kind": "oracle",
            "sample": f"one full solve of a 10x10x10-element p=7 piece of the same workload "
                      f"(same map, schedule, smoother Cheby-{smoother}({order}), tolerance): {it} "
                      f"iterations in {t:.1f} s, single thread"}


def batch_measure(nprob, steps, warmup, op_df=0):
    """64 independent problems (E from {8^3..24^3}, p from {3,5,7,9}, seeded maps and right-hand
    sides), FP32 V-cycle / FP64 Krylov, all solved by ONE graph launch per step, tiles tuned per
    p first; compared with the same 64 problems solved one after another with the plain FP64
    method (FP64 V-cycle, host-driven loop)."""
    import numpy as np
    import torch
    from paper_2110_07663_gb300 import se
    import workloads as wl
    torch.cuda.set_device(0)
    specs = wl.batch_problems(nprob)
    t0 = time.perf_counter()
    tuned = {p: se.se_tune(p, se.SE_FP32) for p in sorted({sp["p"] for sp in specs})}
    tune_s = time.perf_counter() - t0
    probs, total_dof = [], 0
    for sp in specs:
        m = se.se_mesh_create(sp["nel"], sp["p"], perturb_frac=sp["perturb_frac"], seed=sp["seed"],
                              deform_amp=wl.DEFORM_AMP)
        info = se.se_mesh_get_info(m)
        xyz = torch.empty(3 * info.L, dtype=torch.float64, device="cuda")
        se.se_mesh_nodes(m, xyz)
        X = xyz.view(3, -1)
        (k1, k2, k3), a = sp["modes"]
        u = a * torch.sin(k1 * math.pi * X[0]) * torch.sin(k2 * math.pi * X[1]) * torch.sin(k3 * math.pi * X[2])
        f = (math.pi ** 2) * (k1 * k1 + k2 * k2 + k3 * k3) * u
        b = torch.empty(info.L, dtype=torch.float64, device="cuda")
        se.se_mesh_rhs(m, f.contiguous(), b)
        del xyz, X, u, f
        P32 = se.se_pmg_setup(m, se.pmg_desc(sp["schedule"], se.SE_SMOOTH_RAS, 2, precision=se.SE_FP32))
        P64 = se.se_pmg_setup(m, se.pmg_desc(sp["schedule"], se.SE_SMOOTH_RAS, 2, precision=se.SE_FP64))
        probs.append((m, P32, P64, b, torch.zeros_like(b), info))
        total_dof += info.n_dof
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0
    B = se.se_batch_create([(m, P32, b, x) for (m, P32, P64, b, x, info) in probs], tol=1e-8, maxit=500,
                           operator_df64=op_df)
    groups, grouped = se.se_batch_info(B)
    stream = torch.cuda.current_stream()

    def batch_step():
        for pr in probs:
            pr[4].zero_()
        se.se_batch_run(B, stream)

    for _ in range(warmup):
        batch_step()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(0) as clk:
        e0.record(stream)
        for _ in range(steps):
            batch_step()
        e1.record(stream)
        torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    stats = se.se_batch_stats(B, len(probs), stream)
    its = [s_.iterations for s_ in stats]
    worst = max(s_.rel_residual for s_ in stats)
    # profiled pass: the same batch with host-driven loops (same launches), each launch timed
    Bh = se.se_batch_create([(m, P32, b, x) for (m, P32, P64, b, x, info) in probs], tol=1e-8, maxit=500,
                            operator_df64=op_df, graph_capture=0)

    def host_batch():
        for pr in probs:
            pr[4].zero_()
        se.se_batch_run(Bh, stream)

    host_batch()
    torch.cuda.synchronize()
    prof_ms, _, variants = profiled_variants(se, host_batch, 1, stream, label="profiled_pass_batch")
    se.se_batch_destroy(Bh)
    pk, pk_kind = peaks()
    pk["sms"] = torch.cuda.get_device_properties(0).multi_processor_count
    ktable = kernel_table(variants, 1, pk, pk_kind)
    (dom, dvar), dq = max(variants.items(), key=lambda kv: kv[1]["ms"])
    roof = roofline(dom, dvar, dq, pk, pk_kind)
    # plain FP64 serial: each problem alone, FP64 V-cycle, host-driven FPCG
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    its64 = []
    for (m, P32, P64, b, x, info) in probs:
        x.zero_()
        its64.append(se.se_solve(m, P64, b, x, tol=1e-8, maxit=500, stream=stream).iterations)
    f1.record(stream)
    torch.cuda.synchronize()
    ms64 = f0.elapsed_time(f1)
    se.se_batch_destroy(B)
    for (m, P32, P64, b, x, info) in probs:
        se.se_pmg_destroy(P32)
        se.se_pmg_destroy(P64)
        se.se_mesh_destroy(m)
    out = {
        "metric": "batched Poisson solves: total time & aggregate GDOF/s", "value": round(total_dof / (ms * 1e-3) / 1e9, 4),
        "unit": "GDOF/s", "n_gpus": 1, "steps": steps, "warmup": warmup,
        "ms_per_step": round(ms, 2), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32 V-cycle / f64 Krylov" + (" (df64 operator)" if op_df else ""), "data": "synthetic",
        "config": {"workload": f"{len(probs)} problems, E in {{8^3..24^3}}, p in {{3,5,7,9}}, "
                               f"n total {total_dof}, Cheby-RAS(2) pMG, FPCG tol 1e-8, one graph launch",
                   "groups": groups, "grouped_problems": grouped,
                   "batch_path": "problems sharing a preconditioner configuration solved as one union "
                                 "problem per group: one launch per phase for all members",
                   "iterations_min_max": [min(its), max(its)], "worst_rel_residual": worst,
                   "setup_s": round(setup_s, 1), "tune_s": round(tune_s, 1),
                   "tiles": {p: [t.ax_elems_per_block, t.fdm_elems_per_block] for p, t in tuned.items()}},
        "serial_fp64": {"ms": round(ms64, 2), "value": round(total_dof / (ms64 * 1e-3) / 1e9, 4),
                        "iterations_min_max": [min(its64), max(its64)],
                        "speedup_of_batch": round(ms64 / ms, 2)},
        "clocks": clk.summary(),
        "profiled_pass_ms": round(prof_ms, 2),
        "profiled_pass": "same batch with host-driven loops (same launches), per-kernel CUDA events",
        "roofline": roof,
        "kernels": ktable,
    }
    return out


def run_batch(args):
    print(json.dumps(batch_measure(args.batch, args.steps, args.warmup,
                                   1 if args.operator_df64 else 0)))


SERVE_SCHEDULES = {5: (5, 3, 1), 7: (7, 3, 1), 9: (9, 5, 1)}


def serve_stream(se, reqs, budget, slots, precision, t_scale=1.0, proj=0, op_df=0):
    """Submit `reqs` at their (scaled) arrival times, wait for all, return the server summary."""
    import workloads as wl
    S = se.se_serve_create(budget, slots, proj_vectors=proj, operator_df64=op_df)
    tickets, keep = [], []
    refused = 0
    t0 = time.perf_counter()
    for r in reqs:
        delay = t0 + r["t"] * t_scale - time.perf_counter()
        if delay > 0:
            time.sleep(delay)
        m = r["mesh"]
        md = se.mesh_desc(m["nel"], m["p"], perturb_frac=m["perturb_frac"], seed=m["seed"],
                          deform_amp=wl.DEFORM_AMP)
        pd = se.pmg_desc(SERVE_SCHEDULES[m["p"]], se.SE_SMOOTH_RAS, 2, precision=precision,
                         arnoldi_df64=op_df)
        modes, amp = wl.request_modes(r["rhs_seed"])
        key = hash((tuple(m["nel"]), m["p"], m["seed"])) & ((1 << 63) - 1)
        q = se.make_request(md, key, pd, modes=modes, amplitude=amp, tol=1e-8)
        keep.append(q)
        try:
            tickets.append(se.se_serve_submit(S, q))
        except se.SeError:
            refused += 1
    results = [se.se_serve_wait(S, t, 3.6e6, allow=(se.SE_ENOTCONV, se.SE_ETIMEOUT)) for t in tickets]
    wall = time.perf_counter() - t0
    st = se.se_serve_stats(S)
    se.se_serve_destroy(S)
    ok = [r for r in results if r.status == se.SE_OK]
    its = [r.iterations for r in ok]
    worst = max(r.rel_residual for r in ok) if ok else None
    setups = [r.setup_ms for r in results if r.new_mesh]
    solves = [r.solve_ms for r in ok]
    failures = []  # every failed request, with what identifies its mesh
    for i, r in enumerate(results):
        if r.status != se.SE_OK:
            m = reqs[i]["mesh"]
            failures.append({"index": i, "status": r.status, "iterations": r.iterations,
                             "rel_residual": r.rel_residual, "new_mesh": r.new_mesh,
                             "nel": list(m["nel"]), "p": m["p"], "seed": m["seed"],
                             "perturb_frac": m["perturb_frac"], "rhs_seed": reqs[i]["rhs_seed"],
                             "setup_ms": round(r.setup_ms, 1), "solve_ms": round(r.solve_ms, 1)})
    return {"requests": len(reqs), "completed": st.completed, "refused": st.refused + refused,
            "failed": st.failed, "solves_per_s": round(st.solves_per_s, 2),
            "p50_ms": round(st.p50_ms, 1), "p99_ms": round(st.p99_ms, 1), "mean_ms": round(st.mean_ms, 1),
            "max_concurrent": st.max_concurrent, "meshes_created": st.meshes_created,
            "mesh_reuses": st.mesh_reuses, "evictions": st.evictions, "wall_s": round(wall, 1),
            "iterations_min_max": [min(its), max(its)] if its else None, "worst_rel_residual": worst,
            "mean_setup_ms_new_mesh": round(statistics.mean(setups), 1) if setups else None,
            "mean_solve_ms": round(statistics.mean(solves), 1) if solves else None,
            "proj_vectors": proj, "projected": st.projected,
            "mean_iterations": round(statistics.mean(its), 2) if its else None,
            "failures": failures[:20]}


def run_serve(args):
    """Poisson-arrival stream of solve requests (E log-uniform in [512, 65536], p in {5,7,9},
    30% on a resident mesh with a new right-hand side) through the continuous-batching server
    (FP32 V-cycle / FP64 Krylov, admission by HBM footprint), against the same stream through a
    one-slot server with the plain FP64 method."""
    import torch
    from paper_2110_07663_gb300 import se
    import workloads as wl
    torch.cuda.set_device(0)
    free, total = torch.cuda.mem_get_info()
    budget = int(0.8 * free)
    reqs = wl.serve_requests(n=args.serve, rate=args.rate, seed=0)
    with ClockSampler(0) as clk:
        served = serve_stream(se, reqs, budget, args.slots, se.SE_FP32, proj=args.proj,
                              op_df=1 if args.operator_df64 else 0)
    low = None
    if args.low_rate > 0:  # the same kind of stream at a rate below capacity: latency unqueued
        low_reqs = wl.serve_requests(n=args.low_n, rate=args.low_rate, seed=1)
        low = serve_stream(se, low_reqs, budget, args.slots, se.SE_FP32, proj=args.proj,
                           op_df=1 if args.operator_df64 else 0)
        low["rate"] = args.low_rate
    base_reqs = reqs[:args.serve_baseline] if args.serve_baseline else reqs
    serial = serve_stream(se, base_reqs, budget, 1, se.SE_FP64)
    out = {"metric": "served Poisson solves: solves/s, p50/p99 latency", "value": served["solves_per_s"],
           "unit": "solves/s", "n_gpus": 1, "higher_is_better": True,
           "dtype": "f32 V-cycle / f64 Krylov" + (" (df64 operator)" if args.operator_df64 else ""),
           "data": "synthetic",
           "config": {"workload": f"{len(reqs)} requests, Poisson arrivals at {args.rate}/s, E log-uniform "
                                  f"[512, 65536], p in {{5,7,9}}, 30% resident-mesh reuse, tol 1e-8",
                      "slots": args.slots, "hbm_budget_GB": round(budget / 2 ** 30, 1)},
           "served": served, "serial_fp64": serial, "clocks": clk.summary()}
    if low is not None:
        out["served_below_capacity"] = low
    print(json.dumps(out))


def run_setup_profile(args):
    """Set-up cost of a new served mesh (the part of serving that does not overlap with solves):
    mesh creation, the FP32-V-cycle Cheby-RAS(2) preconditioner set-up with FP64 and with df64
    Arnoldi rounds (per-kernel-class times of the set-up from the library's event profiler), the
    first graph solve (capture included) and a steady graph solve, for meshes of the served size
    range."""
    import torch
    from paper_2110_07663_gb300 import se
    import workloads as wl
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    cases = [((8, 8, 8), 5), ((24, 24, 24), 7), ((40, 40, 40), 9)]
    out = []
    for nel, p in cases:
        rec = {"nel": list(nel), "p": p}
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        m = se.se_mesh_create(nel, p, perturb_frac=0.05, seed=1, deform_amp=wl.DEFORM_AMP)
        torch.cuda.synchronize()
        rec["mesh_ms"] = round((time.perf_counter() - t0) * 1e3, 2)
        info = se.se_mesh_get_info(m)
        rec["n_dof"] = info.n_dof
        b = torch.empty(info.L, dtype=torch.float64, device="cuda")
        for arn in (0, 1):
            desc = se.pmg_desc(SERVE_SCHEDULES[p], se.SE_SMOOTH_RAS, 2, precision=se.SE_FP32, arnoldi_df64=arn)
            se.se_prof_reset()
            se.se_prof_enable(True)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            P = se.se_pmg_setup(m, desc)
            torch.cuda.synchronize()
            wall = (time.perf_counter() - t0) * 1e3
            se.se_prof_enable(False)
            prof = {se.KERNEL_NAMES[k]: round(se.se_prof_query(k)["ms"], 2) for k in range(se.SE_K_COUNT)
                    if se.se_prof_query(k)["launches"]}
            key = "pmg_df64_arnoldi" if arn else "pmg_fp64_arnoldi"
            rec[key] = {"wall_ms": round(wall, 2), "kernels_ms": prof}
            if arn:
                xyz = torch.empty(3 * info.L, dtype=torch.float64, device="cuda")
                se.se_mesh_nodes(m, xyz)
                X = xyz.view(3, -1)
                f = 3 * math.pi ** 2 * torch.sin(math.pi * X[0]) * torch.sin(math.pi * X[1]) * torch.sin(math.pi * X[2])
                se.se_mesh_rhs(m, f.contiguous(), b)
                del xyz, X, f
                x = torch.zeros_like(b)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                st = se.se_solve(m, P, b, x, tol=1e-8, graph_capture=1, stream=stream)
                rec["first_solve_ms"] = round((time.perf_counter() - t0) * 1e3, 2)
                x.zero_()
                st = se.se_solve(m, P, b, x, tol=1e-8, graph_capture=1, stream=stream)
                rec["steady_solve_ms"] = round(st.ms_total, 2)
                rec["iterations"] = st.iterations
            se.se_pmg_destroy(P)
        se.se_mesh_destroy(m)
        out.append(rec)
    print(json.dumps({"metric": "new-mesh set-up of served requests (ms)", "cases": out}))


def run_precision_study(args):
    """FP32 V-cycle / FP64 Krylov against the all-FP64 method on the 4^3-element box at p = 7 and
    p = 9: iterations, solve time, and the error of each solution against the FP64 oracle
    solution and against the manufactured solution."""
    import numpy as np
    import torch
    import oracle as o
    from paper_2110_07663_gb300 import se
    import workloads as wl
    torch.cuda.set_device(0)
    nel = (4, 4, 4)
    V = wl.vertex_lattice(nel)
    rows = []
    for p, sched in [(7, (7, 3, 1)), (9, (9, 5, 1)), (9, (9, 7, 5, 1))]:
        m = se.se_mesh_create(nel, p, vertex_xyz=V, deform_amp=wl.DEFORM_AMP)
        info = se.se_mesh_get_info(m)
        xyz = torch.empty(3 * info.L, dtype=torch.float64, device="cuda")
        se.se_mesh_nodes(m, xyz)
        X = xyz.view(3, -1).cpu().numpy()
        b = torch.empty(info.L, dtype=torch.float64, device="cuda")
        se.se_mesh_rhs(m, torch.from_numpy(wl.f_rhs(X[0], X[1], X[2])).cuda(), b)
        lv, bo = o.problem(V, nel, p, amp=wl.DEFORM_AMP)
        pmg = o.pmg_setup(V, nel, sched, smoother="ras", order=2, amp=wl.DEFORM_AMP)
        xo, it_o, _ = o.solve(lv, bo, pmg, tol=1e-8)
        ustar = wl.u_exact(*lv.X).reshape(-1)
        row = {"p": p, "schedule": list(sched), "oracle_iterations": it_o}
        for name, prec in (("fp64", se.SE_FP64), ("fp32_vcycle", se.SE_FP32)):
            P = se.se_pmg_setup(m, se.pmg_desc(sched, se.SE_SMOOTH_RAS, 2, precision=prec))
            x = torch.zeros_like(b)
            for _ in range(3):
                x.zero_()
                st = se.se_solve(m, P, b, x, tol=1e-8, graph_capture=1)
            xg = x.cpu().numpy()
            r = bo.reshape(-1) - o.ax(lv, xg.reshape(lv.gid.shape)).reshape(-1)
            row[name] = {"iterations": st.iterations, "ms": round(st.ms_total, 3),
                         "rel_residual": st.rel_residual,
                         "true_rel_residual": float(np.sqrt(o.dot(lv, r.reshape(lv.gid.shape), r.reshape(lv.gid.shape)) / o.dot(lv, bo, bo))),
                         "max_err_vs_oracle_solution": float(np.max(np.abs(xg - xo.reshape(-1))) / np.max(np.abs(xo))),
                         "max_err_vs_exact": float(np.max(np.abs(xg - ustar)))}
            se.se_pmg_destroy(P)
        rows.append(row)
        se.se_mesh_destroy(m)
    print(json.dumps({"metric": "mixed-precision preconditioner: iterations and error vs FP64 oracle",
                      "config": {"workload": "4x4x4-element box, smooth map, Cheby-RAS(2) pMG, FPCG tol 1e-8"},
                      "rows": rows}))


def run_autotune(args):
    """Run-time preconditioner selection (Sec. 5, Table 5 without SEMFEM) on the bench workload:
    every candidate of the default space (and, with --autotune-orders, Cheby-RAS(k) and
    Cheby-Jac(k) for k = 1..3 on the same schedules) set up and timed on the first solve, for the
    FP64 V-cycle, the df64 one (with the df64 outer operator) and the FP32 one; prints the timed
    table and the choice."""
    import torch
    from paper_2110_07663_gb300 import se
    import workloads as wl
    torch.cuda.set_device(0)
    wk = WORKLOADS[args.workload]
    nel, p = wk["nel"], wk["p"]
    m = se.se_mesh_create(nel, p, perturb_frac=wk["perturb"], seed=wk["seed"], deform_amp=wl.DEFORM_AMP)
    info = se.se_mesh_get_info(m)
    xyz = torch.empty(3 * info.L, dtype=torch.float64, device="cuda")
    se.se_mesh_nodes(m, xyz)
    X = xyz.view(3, -1)
    f = 3.0 * math.pi ** 2 * torch.sin(math.pi * X[0]) * torch.sin(math.pi * X[1]) * torch.sin(math.pi * X[2])
    b = torch.empty(info.L, dtype=torch.float64, device="cuda")
    se.se_mesh_rhs(m, f.contiguous(), b)
    del xyz, X, f
    names = {se.SE_SMOOTH_ASM: "Cheby-ASM", se.SE_SMOOTH_RAS: "Cheby-RAS", se.SE_SMOOTH_JACOBI: "Cheby-Jac"}
    out = []
    for prec_name, prec in (("fp64", se.SE_FP64), ("df64", se.SE_DF64), ("fp32_vcycle", se.SE_FP32)):
        cands = se.se_pmg_autotune_space(p, prec)
        if args.autotune_orders:
            for base in (cands[1], cands[2]):
                for k in (1, 2, 3):
                    if k == 2:
                        continue
                    c = se.se_tune_candidate()
                    c.pmg = se.pmg_desc(list(base.pmg.schedule[:base.pmg.nlev]), base.pmg.smoother, k,
                                        precision=prec)
                    cands.append(c)
        t0 = time.perf_counter()
        best, timed, P = se.se_pmg_autotune(m, b, cands, repeats=args.steps, tol=1e-8, maxit=500,
                                            keep=False, operator_df64=1 if prec == se.SE_DF64 else 0)
        wall = time.perf_counter() - t0
        rows = [{"preconditioner": f"{names[c.pmg.smoother]}({c.pmg.cheb_order[0]})",
                 "schedule": list(c.pmg.schedule[:c.pmg.nlev]),
                 "setup_ms": round(c.setup_ms, 1), "solve_ms": round(c.ms, 2),
                 "iterations": c.iterations, "status": c.status} for c in timed]
        out.append({"precision": prec_name, "chosen": rows[best], "search_wall_s": round(wall, 2),
                    "candidates": rows})
    se.se_mesh_destroy(m)
    print(json.dumps({"metric": "run-time preconditioner selection: time to solution per candidate",
                      "config": {"workload": f"{args.workload}: {nel[0]}x{nel[1]}x{nel[2]} elements, "
                                             f"p={p}, FPCG to 1e-8, graph solve, "
                                             f"{args.steps} timed solves per candidate"},
                      "searches": out}))


def run_smoother_sweep(args):
    """The bench workload's full smoother set: Cheby-RAS(k) and Cheby-Jac(k), k = 1, 2, 3, on the
    pMG schedule 7-5-3-1, FPCG to 1e-8 (graph solves, mean of --steps timed solves after one
    untimed), in FP64, df64 (with the df64 outer operator) and the FP32 V-cycle."""
    import torch
    from paper_2110_07663_gb300 import se
    import workloads as wl
    torch.cuda.set_device(0)
    wk = WORKLOADS[args.workload]
    nel, p, sched = wk["nel"], wk["p"], wk["schedule"]
    m = se.se_mesh_create(nel, p, perturb_frac=wk["perturb"], seed=wk["seed"], deform_amp=wl.DEFORM_AMP)
    info = se.se_mesh_get_info(m)
    xyz = torch.empty(3 * info.L, dtype=torch.float64, device="cuda")
    se.se_mesh_nodes(m, xyz)
    X = xyz.view(3, -1)
    f = 3.0 * math.pi ** 2 * torch.sin(math.pi * X[0]) * torch.sin(math.pi * X[1]) * torch.sin(math.pi * X[2])
    b = torch.empty(info.L, dtype=torch.float64, device="cuda")
    se.se_mesh_rhs(m, f.contiguous(), b)
    del xyz, X, f
    rows = []
    for prec_name, prec in (("fp64", se.SE_FP64), ("df64", se.SE_DF64), ("fp32_vcycle", se.SE_FP32)):
        cands = []
        for sm in (se.SE_SMOOTH_RAS, se.SE_SMOOTH_JACOBI):
            for k in (1, 2, 3):
                c = se.se_tune_candidate()
                c.pmg = se.pmg_desc(sched, sm, k, precision=prec)
                cands.append(c)
        best, timed, _ = se.se_pmg_autotune(m, b, cands, repeats=args.steps, tol=1e-8, maxit=500,
                                            keep=False, operator_df64=1 if prec == se.SE_DF64 else 0)
        for c in timed:
            rows.append({"arithmetic": prec_name,
                         "preconditioner": f"Cheby-{'RAS' if c.pmg.smoother == se.SE_SMOOTH_RAS else 'Jac'}"
                                           f"({c.pmg.cheb_order[0]})",
                         "iterations": c.iterations, "solve_ms": round(c.ms, 2),
                         "gdof_per_s": round(info.n_dof / (c.ms * 1e-3) / 1e9, 4),
                         "setup_ms": round(c.setup_ms, 1), "status": c.status})
    se.se_mesh_destroy(m)
    print(json.dumps({"metric": "Poisson solve time per smoother (Cheby-RAS(k), Cheby-Jac(k), k = 1..3)",
                      "config": {"workload": f"{args.workload}: {nel[0]}x{nel[1]}x{nel[2]} elements, p={p}, "
                                             f"n={info.n_dof}, pMG {'-'.join(map(str, sched))}, FPCG to 1e-8, "
                                             f"graph solves, {args.steps} timed per entry"},
                      "rows": rows}))


def skewed_problem(se, torch, nel, p, eps, segments=2):
    """Mesh on the skewed lattice (workloads.skewed_lattice, no smooth map) and b for
    f = 3 pi^2 sin(pi x) sin(pi y) sin(pi z)."""
    import workloads as wl
    m = se.se_mesh_create(nel, p, vertex_xyz=wl.skewed_lattice(nel, eps, segments), deform_amp=0.0)
    info = se.se_mesh_get_info(m)
    xyz = torch.empty(3 * info.L, dtype=torch.float64, device="cuda")
    se.se_mesh_nodes(m, xyz)
    X = xyz.view(3, -1)
    f = 3.0 * math.pi ** 2 * torch.sin(math.pi * X[0]) * torch.sin(math.pi * X[1]) * torch.sin(math.pi * X[2])
    b = torch.empty(info.L, dtype=torch.float64, device="cuda")
    se.se_mesh_rhs(m, f.contiguous(), b)
    return m, info, b


def study_solve(se, torch, m, b, desc, method, maxit):
    """Set up, solve from x = 0 to 1e-8 (not converging within maxit is a result, not an error)."""
    P = se.se_pmg_setup(m, desc)
    x = torch.zeros_like(b)
    st = se.se_solve(m, P, b, x, method=method, tol=1e-8, maxit=maxit, restart=20,
                     allow_notconv=True)
    se.se_pmg_destroy(P)
    ok = st.status == se.SE_OK and st.rel_residual <= 1e-8
    return ok, st


def run_lambda_study(args):
    """Synthetic analogue of Table 1: iterations to 1e-8 of GMRES(20) with the pMG (7,3,1)
    Cheby-ASM(2) preconditioner for Chebyshev bounds (lo, hi) x lambda-tilde, on the skewed
    lattice (eps = 0.3, 24^3 elements, p = 7 by default); '-' = not converged within maxit."""
    import torch
    from paper_2110_07663_gb300 import se
    torch.cuda.set_device(0)
    nel = (args.study_nel,) * 3
    m, info, b = skewed_problem(se, torch, nel, 7, args.study_eps, args.study_segments)
    prec = se.SE_FP32 if args.study_fp32 else se.SE_FP64
    lows = [0.0, 0.025, 0.05, 0.1, 0.2, 0.25]
    highs = [0.9, 0.95, 1.0, 1.1, 1.2, 1.3]
    grid, times = [], []
    t0 = time.perf_counter()
    for lo in lows:
        row, trow = [], []
        for hi in highs:
            d = se.pmg_desc((7, 3, 1), se.SE_SMOOTH_ASM, 2, eig_lo=lo, eig_hi=hi, precision=prec)
            ok, st = study_solve(se, torch, m, b, d, se.SE_FGMRES, args.study_maxit)
            row.append(st.iterations if ok else "-")
            trow.append(round(st.ms_total, 1))
        grid.append(row)
        times.append(trow)
    se.se_mesh_destroy(m)
    print(json.dumps({
        "metric": "iterations to 1e-8 vs Chebyshev bounds (synthetic analogue of Table 1)",
        "config": {"workload": f"skewed lattice eps={args.study_eps} segments={args.study_segments}, "
                               f"{nel[0]}^3 elements, p=7, "
                               f"pMG (7,3,1) Cheby-ASM(2), FGMRES(20), maxit {args.study_maxit}",
                   "precision": "fp32_vcycle" if args.study_fp32 else "fp64"},
        "lambda_min_multipliers": lows, "lambda_max_multipliers": highs,
        "iterations": grid, "solve_ms": times, "wall_s": round(time.perf_counter() - t0, 1)}))


def run_order_study(args):
    """Synthetic analogue of the paper's order study (Sec. 4.1): fixed n = E p^3, p = 3..10, on
    the skewed lattice for eps in {1, 0.3, 0.05}, with the three pMG preconditioners of the
    autotuner space; iterations of GMRES(20) to 1e-8 and time per solve."""
    import torch
    from paper_2110_07663_gb300 import se
    torch.cuda.set_device(0)
    prec = se.SE_FP32 if args.study_fp32 else se.SE_FP64
    names = {se.SE_SMOOTH_ASM: "Cheby-ASM(2)", se.SE_SMOOTH_RAS: "Cheby-RAS(2)",
             se.SE_SMOOTH_JACOBI: "Cheby-Jac(2)"}
    rows = []
    t0 = time.perf_counter()
    for eps in args.study_eps_list:
        for p in range(3, 11):
            ne = max(2, round((args.study_n / p ** 3) ** (1.0 / 3.0)))
            nel = (ne, ne, ne)
            m, info, b = skewed_problem(se, torch, nel, p, eps, args.study_segments)
            for c in se.se_pmg_autotune_space(p, prec):
                ok, st = study_solve(se, torch, m, b, c.pmg, se.SE_FGMRES, args.study_maxit)
                rows.append({"eps": eps, "p": p, "E": ne ** 3, "n": ne ** 3 * p ** 3,
                             "preconditioner": names[c.pmg.smoother],
                             "schedule": list(c.pmg.schedule[:c.pmg.nlev]),
                             "iterations": st.iterations if ok else "-",
                             "solve_ms": round(st.ms_total, 2),
                             "gdof_per_s": round(ne ** 3 * p ** 3 / st.ms_total * 1e-6, 4) if ok else None})
            se.se_mesh_destroy(m)
    print(json.dumps({
        "metric": "iterations and time per solve vs polynomial order (synthetic analogue of the order study)",
        "config": {"workload": f"skewed lattice segments={args.study_segments}, n = E p^3 ~ "
                               f"{args.study_n:.3g}, FGMRES(20) to 1e-8, "
                               f"maxit {args.study_maxit}",
                   "precision": "fp32_vcycle" if args.study_fp32 else "fp64"},
        "rows": rows, "wall_s": round(time.perf_counter() - t0, 1)}))


def oracle_full(args):
    """The oracle once on the whole workload (not a sample): set-up and one solve, timed."""
    import numpy as np
    import oracle as o
    import workloads as wl
    wk = WORKLOADS[args.workload]
    sm = ORACLE_SMOOTHERS[args.smoother if args.smoother != "auto" else "jacobi"]
    order = args.cheb_order if args.smoother != "auto" else 1
    t0 = time.perf_counter()
    V = wl.vertex_lattice(wk["nel"], wk["perturb"], wk["seed"])
    lv, b = o.problem(V, wk["nel"], wk["p"], amp=wl.DEFORM_AMP)
    pmg = o.pmg_setup(V, wk["nel"], wk["schedule"], smoother=sm, order=order, amp=wl.DEFORM_AMP)
    t1 = time.perf_counter()
    x, it, rel = o.solve(lv, b, pmg, tol=1e-8)
    t2 = time.perf_counter()
    n = int(np.prod(wk["nel"])) * wk["p"] ** 3
    print(json.dumps({"impl": "reference", "oracle_full": {
        "workload": args.workload, "preconditioner": f"Cheby-{sm}({order})",
        "schedule": list(wk["schedule"]), "n_dof": n, "setup_s": round(t1 - t0, 1),
        "solve_s": round(t2 - t1, 1), "iterations": it, "rel_residual": rel,
        "gdof_per_s": round(n / (t2 - t1) / 1e9, 7), "cores": 1, "nproc": os.cpu_count()}}))


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    env_threads = 1
    if args.oracle_full:
        oracle_full(args)
        return
    search = None
    if args.smoother == "auto":
        # the same run-time search as the GPU arm, on the oracle: each candidate solves the
        # sample once (untimed set-up), the fastest is then timed
        search = []
        for sm in ("ras", "jacobi"):
            for k in (1, 2, 3):
                v, t, it = oracle_sample(0, sm, k)
                search.append({"preconditioner": f"Cheby-{sm}({k})", "solve_s": round(t, 2),
                               "iterations": it, "sm": sm, "k": k})
        bestc = min(search, key=lambda r: r["solve_s"])
        smoother, order = bestc["sm"], bestc["k"]
        for r in search:
            del r["sm"], r["k"]
    else:
        smoother, order = args.smoother, args.cheb_order
    vals = []
    t_total = 0.0
    for _ in range(args.steps):
        v, t, it = oracle_sample(0, smoother, order)
        vals.append(v)
        t_total += t
    value = statistics.median(vals)
    ms = t_total / args.steps * 1e3
    out = {
        "impl": "reference", "metric": METRIC, "value": round(value, 6), "unit": "GDOF/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 1),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": f"{args.workload} (oracle on a bounded 10x10x10-element p=7 sample), "
                               f"Cheby-{smoother}({order})",
                   "preconditioner_search": search, "parallelism": "cpu"},
        "cpu_baseline": {"value": round(value, 6), "unit": "GDOF/s", "cores": env_threads,
                         "nproc": os.cpu_count(), "kind": "oracle",
                         "sample": f"each step one full oracle solve of a 10x10x10-element p=7 piece "
                                   f"of the workload with Cheby-{smoother}({order})"},
        "e2e": {"value": round(value, 6), "unit": "GDOF/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="box32_p7", choices=sorted(WORKLOADS))
    ap.add_argument("--smoother", default="auto", choices=["auto", "ras", "jacobi", "asm"],
                    help="auto: the run-time preconditioner search over Cheby-RAS(k), Cheby-Jac(k)")
    ap.add_argument("--cheb-order", type=int, default=2)
    ap.add_argument("--cycle", default="mult", choices=["mult", "additive"],
                    help="additive: the additive V-cycle of Schwarz smoothers without Chebyshev "
                         "(needs --smoother ras or asm)")
    ap.add_argument("--precond-fp32", action="store_true")
    ap.add_argument("--gs-map", action="store_true",
                    help="QQ^T of every level from the sorted index map instead of the sweeps")
    ap.add_argument("--df64", action="store_true",
                    help="SE_DF64 preconditioner and df64 outer operator (FP64 vectors)")
    ap.add_argument("--operator-df64", action="store_true",
                    help="df64 outer operator (solve, batch, serve); serve: also df64 Arnoldi set-up")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--tune-tiles", action="store_true",
                    help="run the launch-tile autotuner for the schedule's orders during set-up")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the batch and serve records of the headline line")
    ap.add_argument("--no-schwarz", action="store_true",
                    help="skip the Cheby-RAS(2) FP64 / FP32-V-cycle record of the headline line")
    ap.add_argument("--oracle-full", action="store_true",
                    help="with --impl reference: time the oracle once on the whole workload")
    ap.add_argument("--setup-profile", action="store_true",
                    help="time the set-up of new served meshes (mesh, preconditioner, first solve)")
    ap.add_argument("--peaks", action="store_true",
                    help="measure the FP64 / FP32 / packed-FP32 FMA roofs of this GPU and exit")
    ap.add_argument("--cpu-timeout", type=float, default=240.0)
    ap.add_argument("--batch", type=int, default=0, help="run the batched workload of N problems")
    ap.add_argument("--serve", type=int, default=0, help="run the serving workload of N requests")
    ap.add_argument("--rate", type=float, default=200.0)
    ap.add_argument("--slots", type=int, default=8)
    ap.add_argument("--serve-baseline", type=int, default=0)
    ap.add_argument("--low-rate", type=float, default=0.0,
                    help="serving: also run a stream at this (below-capacity) rate")
    ap.add_argument("--low-n", type=int, default=100)
    ap.add_argument("--proj", type=int, default=0,
                    help="serving: prior solutions kept per resident mesh for the initial guess")
    ap.add_argument("--precision-study", action="store_true")
    ap.add_argument("--autotune", action="store_true",
                    help="time the preconditioner candidates of Table 5 on the workload")
    ap.add_argument("--autotune-orders", action="store_true",
                    help="autotune: add Chebyshev orders 1 and 3 for RAS and Jacobi")
    ap.add_argument("--smoother-sweep", action="store_true",
                    help="Cheby-RAS(k) and Cheby-Jac(k), k = 1..3, on the workload's schedule")
    ap.add_argument("--lambda-study", action="store_true",
                    help="iterations vs Chebyshev bounds on the skewed lattice (Table 1 analogue)")
    ap.add_argument("--order-study", action="store_true",
                    help="iterations and time vs p at fixed n on the skewed lattice")
    ap.add_argument("--study-nel", type=int, default=24)
    ap.add_argument("--study-eps", type=float, default=0.3)
    ap.add_argument("--study-segments", type=int, default=2)
    ap.add_argument("--study-n", type=float, default=2.88e6)
    ap.add_argument("--study-eps-list", type=float, nargs="+", default=[1.0, 0.3, 0.05])
    ap.add_argument("--study-maxit", type=int, default=1000)
    ap.add_argument("--study-fp32", action="store_true", help="studies: FP32 V-cycle")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "gb300":
        ap.error("--warmup must be >= 3")
    if args.cycle == "additive" and args.smoother not in ("ras", "asm"):
        ap.error("--cycle additive needs --smoother ras or asm (the additive V-cycle has no Chebyshev)")
    if args.impl == "reference":
        # the oracle is timed on one host thread (numpy's BLAS included)
        for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
            os.environ[var] = "1"
        run_reference(args)
    elif args.peaks:
        run_peaks(args)
    elif args.setup_profile:
        run_setup_profile(args)
    elif args.batch:
        run_batch(args)
    elif args.serve:
        run_serve(args)
    elif args.precision_study:
        run_precision_study(args)
    elif args.autotune:
        run_autotune(args)
    elif args.smoother_sweep:
        run_smoother_sweep(args)
    elif args.lambda_study:
        run_lambda_study(args)
    elif args.order_study:
        run_order_study(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
