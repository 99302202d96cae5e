"""Benchmark: full FP64 Newton solve of the ghost-gluon DSE system plus the gluon
Schwinger function (arXiv:1206.1779 Sec. 3 Newton iteration, Sec. 2.2 / 5
Schwinger function) on GB300, through the C ABI of include/dse.h.

One step = one solve from the seeded starting guess to a dimensionless residual
below 1e-10 (N = 64 coefficients per dressing function, 256 radial x 128 angular
Gauss-Legendre nodes, every Newton matrix assembled on the device, LU on the
device) followed by Delta(t) at 4096 seeded times with 8192 nodes.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl {gb300,reference}]

Under torchrun each rank runs an independent replica (the path does not shard):
rank 0 prints one JSON line with the whole-job throughput.  --impl reference
times the FP64 CPU oracle on this host's cores instead (rank 0 only).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1206_1779_gb300 import inputs  # noqa: E402

METRIC = "Newton-matrix entries*quad-nodes/s and Newton solves/s at 1e-8 accuracy, % FP64 peak"
UNIT = "entries*nodes/s"
WORKLOAD = "full_solve_n64"
N_T = 4096
N_NODES = 8192
TOL = 1e-10
L2_FLUSH_BYTES = 256 << 20
# Nominal unit counts (context only; the roofline divides by the rates that
# dse_alu_peak measures on this GPU): 152 SMs, 2 FP64 FMA lanes and 128 FP32
# lanes per SM per clock, 4 schedulers per SM issuing one warp instruction per clock.
N_SM = 152
FP64_FLOP_PER_CLK_SM = 4.0
FP32_INST_PER_CLK_SM = 128.0
WARP_ISSUE_PER_CLK_SM = 4.0


SERIES_TABLE_N = (24, 256)  # the kernel reads Z(z), G(z), W(z) from the series table for these N
SERIES_TABLE_DEGREE = 15    # degree of the table's local polynomials
SERIES_TABLE_DF_STEPS = 7   # Horner steps in double-float per polynomial (the rest in FP32; 7 at N = 64)


def work_per_triple(N: int):
    """Algorithmic work of the hot kernel per (x, y, theta) triple in the Newton-matrix
    mode: (FP64 operations, FP64 flops, FP32 operations, double-float multiply-adds).

    FP64 operations are the instructions of the FP64 pipe, each of which takes one
    slot of it whether it is an FMA, an add or a multiply; flops count an FMA as 2.
    On the table path (43 operations, 53 flops): z (1); ln z and 1/z (9: the FMAs
    of r and of e ln2_hi, the leading sums, the product by inv_j); s and u (4); the
    widened table values (3); T_2 .. T_5 for the anchors (7); the integrands (13);
    the angular sums (6).  Without the table (N < 24) the two series and the
    recurrence add 3N FMAs and the exponentials replace the table lookup.
    FP32 (double-float, on the FP32 pipe), in operations (a paired f32x2 instruction
    performs two): the derivative sums weight * T_j (3N double-float multiply-adds,
    12 operations each), the T_j recurrences (N multiply-subtracts, 15 each: the
    stride-4 anchors and the steps to T_4i+2, T_4i+3), the three table polynomials
    (3 x SERIES_TABLE_DF_STEPS double-float steps of 15, the others one FMA each) and
    the small terms of ln z and 1/z (40)."""
    if SERIES_TABLE_N[0] <= N <= SERIES_TABLE_N[1]:
        f64_ops, f64 = 43.0, 53.0
        horner = 3.0 * (SERIES_TABLE_DF_STEPS * 15.0 + (SERIES_TABLE_DEGREE - SERIES_TABLE_DF_STEPS))
        df_ops = 3.0 * N + N + 3.0 * SERIES_TABLE_DF_STEPS
    else:
        f64_ops, f64 = 43.0 + 3.0 * N, 53.0 + 6.0 * N
        horner = 0.0
        df_ops = 3.0 * N + N
    f32 = 12.0 * 3 * N + 15.0 * N + horner + 40.0
    return f64_ops, f64, f32, df_ops


def roofline_model(N: int, triples: int, fp64_ops_per_s: float, fp32_ops_per_s: float):
    """Lower bound on one launch's duration (s): the FP64 and FP32 pipes issue
    independently, so the bound is the larger of the two pipes' times at their
    measured rates (FP64 operations at the measured FP64 FMA instruction rate, FP32
    operations at the faster of the measured scalar and paired FP32 FMA rates); and
    the FP64-equivalent flops of the launch (a double-float multiply-add or
    -subtract counted as one FP64 FMA, 2 flops)."""
    f64_ops, f64, f32, df_ops = work_per_triple(N)
    t_fp64 = triples * f64_ops / fp64_ops_per_s
    t_fp32 = triples * f32 / fp32_ops_per_s
    flops = triples * (f64 + 2.0 * df_ops)
    return max(t_fp64, t_fp32), flops, t_fp64, t_fp32


def measure_alu_peaks(dse, local: int):
    """FP64 FMA, FP32 FMA and special-function (exp2, log2) rates of this GPU by
    the library's microbenchmark, with the SM clock sampled meanwhile."""
    clocks = ClockSampler(local)
    clocks.start()
    out = {}
    for name, kind in (("fp64_fma", dse.DSE_PEAK_FP64_FMA), ("fp32_fma", dse.DSE_PEAK_FP32_FMA),
                       ("mufu_ex2", dse.DSE_PEAK_MUFU_EX2), ("mufu_lg2", dse.DSE_PEAK_MUFU_LG2),
                       ("fp64_dmma", dse.DSE_PEAK_FP64_DMMA), ("fp32x2_fma", dse.DSE_PEAK_FP32X2_FMA)):
        best = 0.0
        for _ in range(2):
            rate, _ms = dse.alu_peak(kind, 150.0)
            best = max(best, rate)
        out[name + "_per_s"] = best
    clk = clocks.stop()
    out["fp64_tflops"] = 2.0 * out["fp64_fma_per_s"] / 1e12
    out["fp32_tflops"] = 2.0 * out["fp32_fma_per_s"] / 1e12
    # the paired f32x2 FMA, both lanes counted: the FP32 bound takes the faster form
    out["fp32x2_tflops"] = 2.0 * out["fp32x2_fma_per_s"] / 1e12
    # the FP64 tensor cores (mma.sync m8n8k4) against the FP64 FMA pipe: the y-only
    # contraction would move to them only if they were faster
    out["fp64_dmma_tflops"] = 2.0 * out["fp64_dmma_per_s"] / 1e12
    out["clocks"] = clk
    out["how"] = ("dse_alu_peak: eight independent FMA (or exp2/log2) chains per thread, SM count x resident "
                  "blocks of 256 threads, ~150 ms per launch, CUDA events, best of 2")
    return out


class ClockSampler:
    """nvidia-smi clocks and throttle reasons during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines: list[str] = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (FileNotFoundError, OSError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(max(smax)) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# the sources the hot kernel is compiled from (its translation unit and the headers it includes)
HOT_KERNEL_SOURCES = [os.path.join(ROOT, "paper_1206_1779_gb300", "csrc", f) for f in
                      ("dse_triple.cu", "dse_df.cuh", "dse_lnrcp.cuh", "dse_lntab.cuh", "dse_internal.cuh")] + \
                     [os.path.join(ROOT, "include", "dse.h")]


def hot_kernel_hash() -> str:
    h = hashlib.sha256()
    for f in HOT_KERNEL_SOURCES:
        h.update(open(f, "rb").read())
    return h.hexdigest()


def traffic_record():
    """ncu record of the hot kernel (DRAM bytes and warp instructions per launch at
    the benchmark's size), if it was taken on the current kernel sources (else None)."""
    path = os.path.join(ROOT, "profiles", "triple_kernel_traffic.json")
    try:
        rec = json.load(open(path))
    except (OSError, ValueError):
        return None
    if rec.get("kernel_sources_sha256") != hot_kernel_hash():
        return None
    return rec


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
    return world, rank, local, dist


def max_over_ranks(dist, v: float) -> float:
    if dist is None:
        return v
    import torch
    t = torch.tensor([v], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(dist):
    if dist is not None:
        dist.barrier()


def run_gb300(args):
    import torch

    import paper_1206_1779_gb300 as dse

    world, rank, local, dist = dist_setup(args)
    torch.cuda.set_device(local)
    dse.load()
    p = inputs.workload_problem(WORKLOAD)
    N, nr, na = p["n_cheb"], p["n_radial"], p["n_angular"]
    c0 = inputs.starting_guess(p, seed=0)
    tt = inputs.schwinger_times(N_T, seed=0)
    stream = torch.cuda.current_stream()
    peaks = measure_alu_peaks(dse, local)

    t_plan0 = time.perf_counter()
    plan = dse.Plan(p)
    t_plan = time.perf_counter() - t_plan0
    c0_dev = torch.from_numpy(c0).cuda()
    t_dev = torch.from_numpy(tt).cuda()
    coef = torch.empty_like(c0_dev)
    delta = torch.empty_like(t_dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")

    def step():
        coef.copy_(c0_dev)
        it, st = plan.solve(coef, tol=TOL, max_iter=50)
        plan.schwinger(coef, t_dev, N_NODES, out=delta)
        return it, st

    for _ in range(max(args.warmup, 3) if args.warmup > 0 else 0):
        step()
    torch.cuda.synchronize()

    def timed_steps():
        times, iters = [], []
        for _ in range(args.steps):
            flush.fill_(1.0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            it, st = step()
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
            iters.append(it)
        return times, iters

    # timed region: each step bracketed by CUDA events, L2 flushed between steps;
    # the Newton iteration of a solve runs as one CUDA graph (device-side loop)
    clocks = ClockSampler(local)
    launches0 = plan.counters()[0]
    barrier(dist)
    torch.cuda.synchronize()
    clocks.start()
    times, iters = timed_steps()
    torch.cuda.synchronize()
    launches1 = plan.counters()[0]
    # the hot kernel's launch times: the same steps once more with CUDA events around
    # every quadrature-kernel launch on the plan's stream (an instrumented plan drives
    # its Newton steps from the host, since a graph's loop body cannot hold events)
    plan.profile(True)
    times_prof, _ = timed_steps()
    torch.cuda.synchronize()
    clk = clocks.stop()
    _, n_timed, timed_ms = plan.counters()
    plan.profile(False)
    barrier(dist)
    total_ms = max_over_ranks(dist, float(np.sum(times)))
    host_loop_ms = max_over_ranks(dist, float(np.sum(times_prof))) / args.steps

    matrices_per_step = float(np.mean(iters))
    entries_nodes = 4.0 * N * N * nr * na
    units = world * args.steps * matrices_per_step * entries_nodes
    value = units / (total_ms * 1e-3)
    solves_per_s = world * args.steps / (total_ms * 1e-3)

    # roofline of the hot kernel: FP64-equivalent algorithmic flops per launch /
    # event time, against the rate at the lower bound on the duration that the
    # measured FP64 and FP32 pipe rates give (the pipes overlapped)
    Rt = N + 1 + (1 if p["x_G"] > 0 else 0)
    triples = Rt * nr * na
    avg_launch_ms = timed_ms / max(n_timed, 1)
    sm_mhz = clk.get("sm_mhz") or 2070.0
    t_min, flops_launch, t_fp64, t_fp32 = roofline_model(N, triples, peaks["fp64_fma_per_s"],
                                                         max(peaks["fp32_fma_per_s"], peaks["fp32x2_fma_per_s"]))
    achieved = flops_launch / (avg_launch_ms * 1e-3) / 1e12
    peak = flops_launch / t_min / 1e12
    f64ops_pt, f64_pt, f32_pt, dfops_pt = work_per_triple(N)
    rec = traffic_record()
    traffic = rec.get("dram_bytes_per_launch_full_size") if rec else None
    issue = None
    if rec and rec.get("warp_instructions_per_launch"):
        # every scheduler issues at most one warp instruction per clock
        t_issue = rec["warp_instructions_per_launch"] / (N_SM * WARP_ISSUE_PER_CLK_SM * sm_mhz * 1e6)
        issue = {"warp_instructions_per_launch": rec["warp_instructions_per_launch"],
                 "t_issue_bound_ms": t_issue * 1e3, "frac_of_issue_bound": t_issue / (avg_launch_ms * 1e-3)}

    # mixed precision (FP32 integrands for the Newton matrix, FP64 residual)
    mixed = None
    if not args.no_mixed:
        mixed = measure_mixed(dse, p, c0_dev, t_dev, coef, args, total_ms / args.steps)

    diff = None
    if rank == 0 and not args.no_grad:
        diff = measure_differentiation(dse, args)
    n16 = None
    if rank == 0 and not args.no_n16:
        n16 = measure_newton_matrix_n16(dse, args)
    n128 = None
    if rank == 0 and not args.no_n128:
        n128 = measure_mixed_n128(dse, args)
    sweep = None
    if rank == 0 and not args.no_batch:
        sweep = measure_batch(dse, args)
    paper = None
    if rank == 0 and not args.no_paper:
        paper = measure_paper_algorithm(dse, args)

    # end to end through the public API with host buffers (pinned), copies timed
    c0_host = torch.from_numpy(c0).pin_memory()
    t_host = torch.from_numpy(tt).pin_memory()
    out_c = torch.empty_like(c0_host).pin_memory()
    out_d = torch.empty_like(t_host).pin_memory()
    e2e_steps = max(1, min(args.steps, 10))
    torch.cuda.synchronize()
    barrier(dist)
    w0 = time.perf_counter()
    for _ in range(e2e_steps):
        coef.copy_(c0_host, non_blocking=True)
        t_dev.copy_(t_host, non_blocking=True)
        plan.solve(coef, tol=TOL, max_iter=50)
        plan.schwinger(coef, t_dev, N_NODES, out=delta)
        out_c.copy_(coef, non_blocking=True)
        out_d.copy_(delta, non_blocking=True)
        torch.cuda.synchronize()
    e2e_s = max_over_ranks(dist, time.perf_counter() - w0)
    e2e_value = world * e2e_steps * matrices_per_step * entries_nodes / e2e_s
    # one Newton matrix (dse_newton_matrix: tables, series table, quadrature kernel,
    # row contraction, assembly) at the seeded guess, 20 calls, CUDA events
    Jm = torch.empty(2 * N, 2 * N, dtype=torch.float64, device="cuda")
    Fm = torch.empty(2 * N, dtype=torch.float64, device="cuda")
    cm = torch.from_numpy(c0).cuda()
    plan.newton_matrix(cm, Jm, Fm)
    em = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    torch.cuda.synchronize()
    em[0].record(stream)
    for _ in range(20):
        plan.newton_matrix(cm, Jm, Fm)
    em[1].record(stream)
    em[1].synchronize()
    newton_matrix_ms = em[0].elapsed_time(em[1]) / 20
    plan.close()

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline_sample(p, c0)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n_cheb": N, "n_radial": nr, "n_angular": na,
                       "newton_tol_scaled": TOL, "schwinger": {"n_t": N_T, "n_nodes": N_NODES},
                       "newton_matrices_per_step": matrices_per_step, "parallelism": "replicas%d" % world,
                       "l2": "flushed between steps (256 MiB write); working set < 2 MiB"},
            "solves_per_s": solves_per_s,
            "ms_per_step_host_loop": host_loop_ms,
            "newton_matrix_ms": newton_matrix_ms,
            "plan_create_s": t_plan,
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "kernel": "k_triple (radial x angular quadrature: FP64 integrands, double-float derivative sums)",
                         "peak_source": ("measured (dse_alu_peak on this GPU): FP64-equivalent flops of a launch over "
                                         "max(t_fp64, t_fp32), the FP64 operations at the measured FP64 FMA "
                                         "instruction rate and the FP32 operations at the faster of the measured "
                                         "scalar and paired (f32x2) FP32 FMA rates, the two pipes overlapped; "
                                         "the hot kernel is timed in a second pass of the same steps with CUDA "
                                         "events around each of its launches"),
                         "timed_launches": n_timed, "avg_launch_ms": avg_launch_ms, "triples_per_launch": triples,
                         "fp64_operations_per_triple": f64ops_pt,
                         "fp64_flops_per_triple": f64_pt, "fp32_operations_per_triple": f32_pt,
                         "double_float_ops_per_triple": dfops_pt,
                         "t_fp64_bound_ms": t_fp64 * 1e3, "t_fp32_bound_ms": t_fp32 * 1e3,
                         "fp64_achieved_tflops": triples * f64_pt / (avg_launch_ms * 1e-3) / 1e12,
                         "fp64_measured_peak_tflops": peaks["fp64_tflops"],
                         "fp32_measured_peak_tflops": peaks["fp32_tflops"],
                         "fp32x2_measured_peak_tflops": peaks["fp32x2_tflops"],
                         "issue": issue},
            "alu_peaks": peaks,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(c0.nbytes + tt.nbytes),
                    "d2h_bytes_per_step": int(c0.nbytes + tt.nbytes)},
            "gpu_launches": int(launches1 - launches0),
            "clocks": clk,
        }
        if cpu is not None:
            line["cpu_baseline"] = cpu
        if mixed is not None:
            line["mixed_precision"] = mixed
        if n128 is not None:
            line["mixed_precision_n128"] = n128
        if n16 is not None:
            line["newton_matrix_n16"] = n16
        if diff is not None:
            line["differentiation"] = diff
        if sweep is not None:
            line["batched_sweep"] = sweep
        if paper is not None:
            line["paper_algorithm"] = paper
        print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()


def measure_mixed(dse, p, c0_dev, t_dev, coef_fp64, args, fp64_ms_per_step):
    """The same step with precision = 1, and its accuracy against the FP64 solve."""
    import torch
    N, nr, na = p["n_cheb"], p["n_radial"], p["n_angular"]
    plan = dse.Plan(dict(p, precision=1))
    coef = torch.empty_like(c0_dev)
    delta = torch.empty_like(t_dev)
    stream = torch.cuda.current_stream()

    def step():
        coef.copy_(c0_dev)
        it, st = plan.solve(coef, tol=TOL, max_iter=50)
        plan.schwinger(coef, t_dev, N_NODES, out=delta)
        return it

    for _ in range(max(args.warmup, 1)):
        step()
    torch.cuda.synchronize()
    times, iters = [], []
    for _ in range(args.steps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        iters.append(step())
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    ms = float(np.mean(times))
    x = torch.from_numpy(np.exp(np.linspace(np.log(p["eps2"]), np.log(p["lambda2"]), 257))).cuda()
    lg_m, lz_m = plan.dressing(coef, x)
    lg_d, lz_d = plan.dressing(coef_fp64, x)
    torch.cuda.synchronize()
    dG = float((lg_m - lg_d).abs().max())
    dZ = float((lz_m - lz_d).abs().max())
    plan.close()
    mats = float(np.mean(iters))
    return {"ms_per_step": ms, "solves_per_s": 1e3 / ms, "newton_matrices_per_step": mats,
            "value": mats * 4.0 * N * N * nr * na / (ms * 1e-3), "unit": UNIT,
            "speedup_vs_fp64_step": fp64_ms_per_step / ms,
            "max_abs_dlnG_vs_fp64_solve": dG, "max_abs_dlnZ_vs_fp64_solve": dZ,
            "note": "Newton matrix from FP32 integrands with FP64 block sums; FP64 residual near convergence"}


def measure_differentiation(dse, args):
    """Loss gradient through the converged solve (N = 64, 256 x 128 nodes,
    G(x_G)^{-1} = 0.01): forward = solve from the seeded guess (rho = 1/2 for six
    steps) + ln Z at 64 seeded momenta; backward = dressing VJP, adjoint solve
    J^T lambda = dL/dc and lambda^T dF/dtheta."""
    import torch
    from paper_1206_1779_gb300 import autograd as ad
    p = inputs.workload_problem(WORKLOAD, ginv_G=0.01)
    c0 = torch.from_numpy(inputs.starting_guess(p, seed=0)).cuda()
    x = torch.from_numpy(inputs.loss_momenta(64)).cuda()
    fac = torch.from_numpy(inputs.target_factors(64)).cuda()
    plan = dse.Plan(p)
    stream = torch.cuda.current_stream()

    def run():
        theta = torch.tensor([p["g2nc"], p["ginv_G"]], dtype=torch.float64, requires_grad=True)
        e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        e[0].record(stream)
        cs = ad.solve(plan, theta, c0, tol=TOL, max_iter=60, rho_relax=0.5, n_relax=6)
        _, lZ = ad.dressing(plan, cs, theta, x)
        Z = torch.exp(lZ)
        L = ((Z - Z.detach() * fac) ** 2).sum()
        e[1].record(stream)
        L.backward()
        e[2].record(stream)
        e[2].synchronize()
        return e[0].elapsed_time(e[1]), e[1].elapsed_time(e[2]), theta.grad.numpy().copy()

    for _ in range(2):
        run()
    fw, bw = [], []
    for _ in range(max(1, min(args.steps, 5))):
        f, b, g = run()
        fw.append(f)
        bw.append(b)
    plan.close()
    return {"workload": "full_solve_n64 with G(x_G)^-1 = 0.01, loss over 64 momenta",
            "forward_ms": float(np.mean(fw)), "backward_ms": float(np.mean(bw)),
            "dL_dg2nc": float(g[0]), "dL_dginv_G": float(g[1]),
            "note": "backward: dressing VJP + FP64 Newton matrix + adjoint solve + parameter derivatives"}


def measure_mixed_n128(dse, args):
    """Mixed precision at N = 128 with 512 x 256 nodes (matrix_n128): a solve from
    the seeded guess in mixed precision and in FP64, their Newton-matrix times,
    and the largest difference of the converged ln G, ln Z."""
    import torch
    p = inputs.workload_problem("matrix_n128")
    N, nr, na = p["n_cheb"], p["n_radial"], p["n_angular"]
    c0 = torch.from_numpy(inputs.starting_guess(p, seed=0)).cuda()
    stream = torch.cuda.current_stream()
    out = {"workload": "matrix_n128", "n_cheb": N, "n_radial": nr, "n_angular": na}
    coefs = {}
    for name, prec in (("fp64", 0), ("mixed", 1)):
        plan = dse.Plan(dict(p, precision=prec))
        coef = c0.clone()
        J = torch.empty(2 * N, 2 * N, dtype=torch.float64, device="cuda")
        F = torch.empty(2 * N, dtype=torch.float64, device="cuda")
        plan.newton_matrix(coef, J, F)
        e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        e[0].record(stream)
        for _ in range(3):
            plan.newton_matrix(coef, J, F)
        e[1].record(stream)
        e[2].record(stream)
        it, _ = plan.solve(coef, tol=TOL, max_iter=50)
        e[3].record(stream)
        e[3].synchronize()
        out[name] = {"newton_matrix_ms": e[0].elapsed_time(e[1]) / 3, "solve_ms": e[2].elapsed_time(e[3]),
                     "newton_steps": it}
        coefs[name] = coef
        plan.close()
    xg = torch.from_numpy(np.exp(np.linspace(np.log(p["eps2"]), np.log(p["lambda2"]), 257))).cuda()
    with dse.Plan(p) as plan:
        lg_d, lz_d = plan.dressing(coefs["fp64"], xg)
        lg_m, lz_m = plan.dressing(coefs["mixed"], xg)
        torch.cuda.synchronize()
    out["max_abs_dlnG_mixed_vs_fp64"] = float((lg_m - lg_d).abs().max())
    out["max_abs_dlnZ_mixed_vs_fp64"] = float((lz_m - lz_d).abs().max())
    out["solve_speedup"] = out["fp64"]["solve_ms"] / out["mixed"]["solve_ms"]
    return out


def measure_batch(dse, args):
    """The parameter sweep: 256 problems with N_Z, N_G in {24, 32, 48, 64},
    quadrature 128 x 64 or 256 x 128 and G(x_G)^{-1} log-uniform in [1e-3, 1e-1],
    solved together (rho = 1/2 for six steps) to a dimensionless residual below
    1e-10; one CUDA graph (one persistent quadrature launch) per Newton step."""
    import torch
    probs = inputs.batch_problems(256)
    c0 = torch.from_numpy(np.concatenate([inputs.starting_guess(p, seed=b) for b, p in enumerate(probs)])).cuda()
    stream = torch.cuda.current_stream()
    batch = dse.Batch(probs)
    t0 = time.perf_counter()
    units, tune_ms = batch.tune(c0)
    tune_s = time.perf_counter() - t0
    coef = torch.empty_like(c0)
    res = None
    times = []
    for rep in range(1 + max(1, min(args.steps, 3))):
        coef.copy_(c0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        its, status, stats = batch.solve(coef, tol=TOL, max_iter=40, rho_relax=0.5, n_relax=6, check=False)
        e1.record(stream)
        e1.synchronize()
        if rep > 0:
            times.append(e0.elapsed_time(e1))
        res = (its, status, stats)
    launches, graphs, _ = batch.counters()
    batch.close()
    its, status, stats = res
    ms = float(np.mean(times))
    entries_nodes = 0.0
    for b, p in enumerate(probs):
        nz = p["n_cheb"]
        ng = p["n_cheb_G"] or nz
        entries_nodes += its[b] * float(nz + ng) ** 2 * p["n_radial"] * p["n_angular"]
    return {"workload": "sweep of 256 problems: N_Z, N_G in {24,32,48,64}, 128x64 or 256x128 nodes, "
                        "G(x_G)^-1 log-uniform in [1e-3, 1e-1]",
            "ms_per_sweep": ms, "solves_per_s": 256 / (ms * 1e-3),
            "value": entries_nodes / (ms * 1e-3), "unit": UNIT,
            "converged": int(sum(1 for v in status if v == 0)), "newton_steps_max": int(max(its)),
            "newton_steps_total": int(sum(its)), "max_scaled_residual": float(max(s[1] for s in stats)),
            "units_per_item": units, "tune_ms_per_candidate": tune_ms, "tune_s": tune_s,
            "graph_launches_per_sweep": int(max(its))}


def measure_newton_matrix_n16(dse, args):
    """The small configuration (newton_step_n16: N = 16 per function, 64 x 32 nodes):
    time per dse_newton_matrix call, launched one by one and replayed from a CUDA
    graph that captured one call (the launch overhead of the six kernels is what
    the graph removes), over 200 calls each."""
    import torch
    p = inputs.workload_problem("newton_step_n16")
    N, nr, na = p["n_cheb"], p["n_radial"], p["n_angular"]
    reps = 200
    with dse.Plan(p) as plan:
        coef = torch.from_numpy(inputs.starting_guess(p, seed=0)).cuda()
        J = torch.empty(2 * N, 2 * N, dtype=torch.float64, device="cuda")
        F = torch.empty(2 * N, dtype=torch.float64, device="cuda")
        for _ in range(5):
            plan.newton_matrix(coef, J, F)
        stream = torch.cuda.current_stream()
        e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        torch.cuda.synchronize()
        e[0].record(stream)
        for _ in range(reps):
            plan.newton_matrix(coef, J, F)
        e[1].record(stream)
        e[1].synchronize()
        J1 = J.clone()
        per_call_us = e[0].elapsed_time(e[1]) * 1e3 / reps
        units = 4.0 * N * N * nr * na
        out = {"workload": "newton_step_n16", "n_cheb": N, "n_radial": nr, "n_angular": na,
               "per_call_us": per_call_us, "per_call_value": units / (per_call_us * 1e-6), "unit": UNIT}
        try:
            g = torch.cuda.CUDAGraph()
            # (relaxed: the launchers set kernel attributes, a host call, while capturing)
            with torch.cuda.graph(g, capture_error_mode="relaxed"):
                plan.newton_matrix(coef, J, F)
            for _ in range(3):
                g.replay()
            torch.cuda.synchronize()
            e[2].record(stream)
            for _ in range(reps):
                g.replay()
            e[3].record(stream)
            e[3].synchronize()
            graph_us = e[2].elapsed_time(e[3]) * 1e3 / reps
            out.update({"graph_replay_us": graph_us, "graph_replay_value": units / (graph_us * 1e-6),
                        "graph_matches_calls": bool(torch.equal(J, J1))})
        except Exception as exc:  # noqa: BLE001 (reported, not fatal)
            out["graph_replay_us"] = None
            out["graph_error"] = str(exc)[:200]
    return out


def measure_paper_algorithm(dse, args):
    """The paper's own discretisation and Jacobian at the benchmark's size: N = 64,
    the radial split [0, eps2] + [eps2, x] + [x, lambda2] with 85 nodes per piece
    (255 per external momentum) and 128 tanh-sinh angular nodes.  Times the
    paper's central-difference Newton matrix (2n = 256 perturbed residuals, one
    batched launch) against the analytic one, and a full solve."""
    import torch
    p = inputs.problem(64, 85, 128, radial_mode=1, angular_mode=1)
    c0 = torch.from_numpy(inputs.starting_guess(p, seed=0)).cuda()
    stream = torch.cuda.current_stream()
    n = 128
    out = {"workload": "N=64, radial split 3x85 nodes, tanh-sinh 128 nodes"}
    with dse.Plan(p) as plan:
        J = torch.empty(n, n, dtype=torch.float64, device="cuda")
        F = torch.empty(n, dtype=torch.float64, device="cuda")
        Jf = torch.empty(n, n, dtype=torch.float64, device="cuda")
        plan.newton_matrix(c0, J, F)
        plan.newton_matrix_fd(c0, 1e-5, J=Jf)
        reps = max(1, min(args.steps, 3))
        e = [torch.cuda.Event(enable_timing=True) for _ in range(6)]
        e[0].record(stream)
        for _ in range(reps):
            plan.newton_matrix(c0, J, F)
        e[1].record(stream)
        e[2].record(stream)
        for _ in range(reps):
            plan.newton_matrix_fd(c0, 1e-5, J=Jf)
        e[3].record(stream)
        coef = c0.clone()
        e[4].record(stream)
        it, st = plan.solve(coef, tol=TOL, max_iter=50)
        e[5].record(stream)
        e[5].synchronize()
        an = e[0].elapsed_time(e[1]) / reps
        fd = e[2].elapsed_time(e[3]) / reps
        rowmax = J.abs().max(dim=1, keepdim=True).values
        out.update({"newton_matrix_ms": an, "fd_newton_matrix_ms": fd, "fd_over_analytic": fd / an,
                    "max_abs_fd_minus_analytic_over_rowmax": float(((Jf - J).abs() / rowmax).max()),
                    "solve_ms": e[4].elapsed_time(e[5]), "newton_steps": it, "scaled_residual": st[1]})
    return out


def cpu_baseline_sample(p, c0, budget_s: float = 12.0):
    """The oracle as it stands, on this host's cores: Newton matrices of the
    same workload until about budget_s seconds of CPU work."""
    from oracle import oracle as O
    O.build()
    N, nr, na = p["n_cheb"], p["n_radial"], p["n_angular"]
    n = 0
    t0 = time.perf_counter()
    while True:
        O.newton_matrix(p, c0)
        n += 1
        if time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    return {"value": n * 4.0 * N * N * nr * na / dt, "unit": UNIT, "cores": O.num_threads(), "kind": "oracle",
            "sample": "%d Newton matrices (residual + analytic Jacobian) of %s, N=%d, %dx%d nodes, %.1f s"
                      % (n, WORKLOAD, N, nr, na, dt)}


def run_reference(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from oracle import oracle as O
    O.build()
    p = inputs.workload_problem(WORKLOAD)
    N, nr, na = p["n_cheb"], p["n_radial"], p["n_angular"]
    c0 = inputs.starting_guess(p, seed=0)
    tt = inputs.schwinger_times(N_T, seed=0)

    def step():
        c, it, _ = O.solve(p, c0, tol=TOL, max_iter=50)
        O.schwinger(p, c, tt, N_NODES)
        return it + 1

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    mats = 0
    for _ in range(args.steps):
        mats += step()
    dt = time.perf_counter() - t0
    value = mats * 4.0 * N * N * nr * na / dt
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": WORKLOAD, "n_cheb": N, "n_radial": nr, "n_angular": na,
                       "newton_tol_scaled": TOL, "schwinger": {"n_t": N_T, "n_nodes": N_NODES}},
            "solves_per_s": args.steps / dt,
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": O.num_threads(), "kind": "oracle",
                             "sample": "%d full solves + Schwinger of %s on host cores" % (args.steps, WORKLOAD)},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["gb300", "reference"], default="gb300")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-mixed", action="store_true")
    ap.add_argument("--no-grad", action="store_true")
    ap.add_argument("--no-n128", action="store_true")
    ap.add_argument("--no-n16", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-paper", action="store_true")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gb300(args)


if __name__ == "__main__":
    main()
