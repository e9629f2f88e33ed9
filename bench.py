"""Benchmark: multigrid-preconditioned CG (one V(1,1)-cycle per iteration, tau=0.25,
sigma=5h^-2) solved from x0 = 0 to relative residual 1e-8 through the C ABI.  One step =
one complete solve.  Prints ONE JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--precision fp64|fp32|bf16] [--workload KEY]

Default: FP64 on the 2D multi-patch workload grid2d_K16_p4_m256 (1,073,296 dofs).  Other
modes: --batch (512 independent problems), --serve (Poisson arrivals, p50/p99 latency),
--fichera (the Table II runs), --micro fd|fp64 (the finest smoother alone, the DGEMM rate).

The default run also reports the FP32 and BF16 variants of the same solve, the cycle of
each precision as the solve replays it, the tensor-core FD kernel's and the stiffness
apply's rooflines, and the oracle on the host cores (median of 3 solves with one thread
and with every logical CPU allowed).

--impl reference times the CPU oracle (FP64 NumPy/SciPy restatement of the method) on
the host cores, one thread, on a bounded sample of the same workload family."""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MDOF/s to rel. residual 1e-8 (FP64 vs mixed), V-cycle HBM frac; p50/p99 lat"
WORKLOAD = "grid2d_K16_p4_m256"
WORKLOAD_DESC = ("2D Poisson, K=16 bilinear patches of a 5x5 vertex grid on [0,4]^2 with interior "
                 "vertices perturbed by U(-0.1,0.1) (seed 2), p=4, 256 intervals per patch direction, "
                 "9 levels (coarsest 1 interval/patch), Dirichlet x=0,y=0, Neumann x=4,y=4, "
                 "rhs = mass matrix times U(-1,1) spline coefficients (seed 2), FP64 PCG + V(1,1), tol 1e-8")
ORACLE_SAMPLE = dict(nper=4, p=4, m=64, levels=7, seed=2)
TOL = 1e-8
# FP64 FMA pipe of one GB300, nominal: 152 SMs x 2 FMA/clk/SM x 2 flop x 2.07 GHz (1.26 TFLOP/s);
# the GPU runs measure it (fp64_peaks) and use the measured rate
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12


# FP32 FMA pipes of one GB300: 152 SMs x 128 FMA/clk/SM x 2 flop x 2.07 GHz
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12


# profile entries that are sub-accounts of the kernel classes (never summed with them)
SUB_ACCOUNTS = ("tensor_exec", "tc_kernel")


def combined_roofline(prof, ms_step, precision, pk, fp64_peak=None):
    """Roofline time of one solve: t_roof = sum over the kernel classes of
    max(algorithmic bytes / HBM bandwidth, flops / pipe peak).  The interior FD counts its
    issued tensor-core MMA FLOPs at the BF16 peak (its FMA-run levels are left out), every
    other class its flops on the FP64 pipe (FP32 pipes in the FP32/BF16 variants), so
    t_roof is a lower bound and frac = t_roof / measured time an upper bound on the
    fraction of the combined roofline the solve reaches."""
    alu = (fp64_peak or FP64_PEAK_TFLOPS) if precision == "fp64" else FP32_PEAK_TFLOPS
    tx = prof.get("tensor_exec", {}).get("flops", 0.0)
    per, t = {}, 0.0
    for k, v in prof.items():
        if k in SUB_ACCOUNTS:
            continue
        tb = v["bytes"] / (pk["hbm_gbs"] * 1e9)
        tf = tx / (pk["bf16_tflops"] * 1e12) if (k == "interior_fd" and tx > 0) else v["flops"] / (alu * 1e12)
        per[k] = round(max(tb, tf) * 1e3, 4)
        t += max(tb, tf)
    return {"t_roof_ms": round(t * 1e3, 3), "frac": round(t * 1e3 / ms_step, 4), "per_class_ms": per,
            "alu_peak_tflops": round(alu, 2)}


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


# ---------------------------------------------------------------- clocks

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.path = tempfile.mktemp(suffix=".csv")
        self.proc = None
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(gpu_index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        self.proc.wait(timeout=10)
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- oracle (CPU)

def oracle_sample_json():
    """Runs in a subprocess with one BLAS/OpenMP thread: oracle setup (untimed), then one
    full PCG solve to 1e-8 of the sample problem (timed)."""
    import numpy as np  # noqa: F401
    import workloads
    from oracle import multipatch, solver
    s = ORACLE_SAMPLE
    pr = workloads.perturbed_grid_2d(s["nper"], s["p"], s["m"], s["levels"], s["seed"])
    t0 = time.perf_counter()
    H = solver.build_hierarchy(pr)
    sp = H.levels[-1].space
    _, Mg = multipatch.stiffness(pr, sp, want_mass=True)
    b = Mg @ workloads.rhs_coefficients(sp.N, 2)
    t_setup = time.perf_counter() - t0
    steps = int(os.environ.get("IGAMG_ORACLE_STEPS", "1"))
    warm = int(os.environ.get("IGAMG_ORACLE_WARMUP", "0"))
    for _ in range(warm):
        solver.pcg(H, b, tol=TOL)
    times, cpu, its = [], [], []
    for _ in range(steps):
        r0, t0 = os.times(), time.perf_counter()
        its.append(solver.pcg(H, b, tol=TOL).iters)
        r1, t1 = os.times(), time.perf_counter()
        times.append(t1 - t0)
        cpu.append((r1.user - r0.user) + (r1.system - r0.system))
    t = statistics.median(times)
    return {"N": sp.N, "t_solve_s": t, "t_runs_s": [round(x, 4) for x in times], "iters": its[-1],
            "t_setup_s": t_setup, "steps": steps, "cores_used": round(sum(cpu) / max(sum(times), 1e-9), 2)}


def host_cpu():
    """(logical CPUs of this host, CPU model name)."""
    n = os.cpu_count() or 1
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    if model is None:
        try:
            for line in open("/proc/cpuinfo"):
                if line.lower().startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
        except OSError:
            pass
    return n, model or "unknown"


def run_oracle(steps=1, warmup=0, threads=1):
    t = str(threads)
    env = dict(os.environ, OMP_NUM_THREADS=t, OPENBLAS_NUM_THREADS=t, MKL_NUM_THREADS=t,
               IGAMG_ORACLE_STEPS=str(steps), IGAMG_ORACLE_WARMUP=str(warmup))
    out = subprocess.run([sys.executable, os.path.abspath(__file__), "--_oracle"], env=env,
                         stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True, timeout=1800)
    if out.returncode != 0:
        raise RuntimeError(out.stderr[-2000:])
    return json.loads(out.stdout.strip().splitlines()[-1])


def sample_desc(runs=1):
    s = ORACLE_SAMPLE
    return (f"same workload family at {s['m']} intervals per patch direction ({s['levels']} levels): "
            f"full PCG+V(1,1) solves to 1e-8, setup excluded, median of {runs}")


def cpu_baseline_json(runs=3):
    """The oracle on the host cores: `runs` solves with one thread and `runs` with every
    logical CPU allowed (BLAS/OpenMP threads); value = the better median.  `cores` is the
    CPU time over the wall time of the solves (SciPy's sparse kernels run on one thread, so
    allowing more threads changes little)."""
    n, model = host_cpu()
    one = run_oracle(runs, 0, 1)
    allc = run_oracle(runs, 0, n)
    best = one if one["t_solve_s"] <= allc["t_solve_s"] else allc
    return {"value": round(best["N"] / best["t_solve_s"] / 1e6, 6), "unit": "MDOF/s",
            "cores": max(1, round(best["cores_used"])), "kind": "oracle", "sample": sample_desc(runs),
            "sample_dofs": best["N"], "sample_iters": best["iters"], "nproc": n, "cpu_model": model,
            "one_thread": {"value": round(one["N"] / one["t_solve_s"] / 1e6, 6), "runs_s": one["t_runs_s"],
                           "cores_used": one["cores_used"]},
            "all_threads": {"threads": n, "value": round(allc["N"] / allc["t_solve_s"] / 1e6, 6),
                            "runs_s": allc["t_runs_s"], "cores_used": allc["cores_used"]}}


# ---------------------------------------------------------------- replicas over ranks

def combine_over_ranks(ms_total, dofs, tdist=None, device="cpu"):
    """Replicas: every rank solves its own copy.  The job time is the slowest rank's; the
    work is the sum of the ranks' dofs.  Returns (max ms, total dofs)."""
    if tdist is None:
        return ms_total, dofs
    import torch
    t = torch.tensor([ms_total], dtype=torch.float64, device=device)
    tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
    n = torch.tensor([dofs], dtype=torch.float64, device=device)
    tdist.all_reduce(n, op=tdist.ReduceOp.SUM)
    return float(t.item()), int(n.item())


# ---------------------------------------------------------------- GPU arm

def fp64_peaks():
    """Measured FP64 rates of this GPU (the library's FMA-chain and m8n8k4 MMA probes) and
    its SM count; the FMA rate is the FP64-pipe peak of the roofline fractions."""
    from paper_1804_02539_gb300 import igamg
    fma, sms = igamg.igamg_micro_fp64(0, 1 << 16)
    mma, _ = igamg.igamg_micro_fp64(1, 1 << 14)
    return {"fma_tflops": round(fma, 4), "mma_tflops": round(mma, 4), "sm_count": sms}


def tensor_roofline(prof, pk, src):
    """Roofline of the tensor-core FD kernel (class 7, all its launches): the BF16 MMA FLOPs
    its tiles execute (class 6) over its event-timed launches, against the measured BF16
    peak (sustained: the kernel is timed inside a long solve)."""
    tc, tx = prof.get("tc_kernel", {}), prof.get("tensor_exec", {})
    if not tc.get("launches") or not tc.get("ms"):
        return None
    ach = tx["flops"] / (tc["ms"] * 1e-3) / 1e12
    peak = pk.get("bf16_tflops_sustained", pk["bf16_tflops"])
    return {"bound": "tensor", "achieved": round(ach, 2), "peak": peak, "unit": "TFLOP/s",
            "frac": round(ach / peak, 4), "peak_source": src + " (bf16_tflops_sustained)",
            "kernel": "k_gemm_tc<7> (tensor-core FD contractions, every level and face it runs)",
            "launches": tc["launches"], "avg_launch_ms": round(tc["ms"] / tc["launches"], 5),
            "fp64_equiv_tflops": round(tc["flops"] / (tc["ms"] * 1e-3) / 1e12, 3),
            "traffic": None, "traffic_finest_launch": TC_TRAFFIC_FINEST_LAUNCH}


# DRAM bytes (read + write) from ncu captures of the unchanged kernels, summarised in
# profiles/: one finest-level launch of the tensor-core FD on the 2D benchmark (the average
# over all its launches is not captured, so `traffic` stays null), and the average over the
# band-apply launches of one timed FP64 solve of the 2D benchmark.
TC_TRAFFIC_FINEST_LAUNCH = 22.81e6
BAND_TRAFFIC_PER_LAUNCH = {("grid2d_K16_p4_m256", "fp64"): 158.82e6}


def run_precision_variant(pr, prec_name, b, xr, dev, stream, steps, warmup):
    """The FP32 or BF16 variant of the same solve (FP64 iterative refinement around the
    low-precision PCG): MDOF/s, iterations, error against the FP64 GPU solution xr, and the
    graph-replayed low-precision cycle against its algorithmic bytes."""
    import torch
    from paper_1804_02539_gb300 import igamg
    opts = igamg.igamg_default_options()
    opts.precision = {"fp32": igamg.IGAMG_FP32, "bf16": igamg.IGAMG_BF16}[prec_name]
    ctx = igamg.Context(pr, opts, stream=stream)
    N = ctx.num_dofs()
    x = torch.zeros(N, dtype=torch.float64, device=dev)
    for _ in range(warmup):
        x.zero_()
        ctx.solve(b, x, TOL)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        x.zero_()
        res, st = ctx.solve(b, x, TOL)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    err = float(torch.linalg.norm(x - xr) / torch.linalg.norm(xr))
    ms_v, by_v = ctx.cycle_time(b, 10)
    # per-class breakdown of one solve (every launch bracketed by events; untimed)
    ctx.profile_enable(0xFF)
    x.zero_()
    ctx.solve(b, x, TOL)
    prof = ctx.profile_read()
    ctx.profile_enable(0)
    out = {"value": round(N / (ms * 1e-3) / 1e6, 4), "ms_per_step": round(ms, 3), "iters": res.iters,
           "outer_iters": res.outer_iters, "relres": res.relres, "status": st, "rel_err_vs_fp64_solution": err,
           "vcycle": {"ms": round(ms_v, 4), "algorithmic_gb": round(by_v / 1e9, 4)},
           "kernel_breakdown": {k: {"ms_per_step": round(v["ms"], 3), "launches_per_step": v["launches"],
                                    "gbyte_per_step": round(v["bytes"] / 1e9, 4)}
                                for k, v in prof.items() if k not in SUB_ACCOUNTS}}
    ctx.free()
    return out


def run_ours(args, rank, world, local_rank):
    import numpy as np
    import torch
    import workloads
    from paper_1804_02539_gb300 import igamg

    dist = world > 1
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    if dist:
        import torch.distributed as tdist
        tdist.init_process_group("nccl")
    stream = torch.cuda.Stream(device=dev)
    pk, src = peaks()
    f64 = fp64_peaks()
    pr = workloads.CONFIGS[args.workload]()
    prec = {"fp64": igamg.IGAMG_FP64, "fp32": igamg.IGAMG_FP32, "bf16": igamg.IGAMG_BF16}[args.precision]
    opts = igamg.igamg_default_options()
    opts.precision = prec
    opts.autotune = 0 if args.no_autotune else 1
    with torch.cuda.stream(stream):
        ctx = igamg.Context(pr, opts, stream=stream)
        N = ctx.num_dofs()
        coef = torch.tensor(workloads.rhs_coefficients(N, 2), device=dev)
        b = torch.empty(N, dtype=torch.float64, device=dev)
        ctx.rhs_from_coefs(coef, b)
        x = torch.zeros(N, dtype=torch.float64, device=dev)
        for _ in range(args.warmup):
            x.zero_()
            res, st = ctx.solve(b, x, TOL)
        iters = res.iters if args.warmup else None
        # pass 1 (untimed): per-class breakdown of one solve, every class timed with events
        ctx.profile_enable(0xFF)
        x.zero_()
        ctx.solve(b, x, TOL)
        prof1 = ctx.profile_read()
        main = {k: v for k, v in prof1.items() if k not in SUB_ACCOUNTS}
        dom = max(main, key=lambda k: main[k]["ms"])
        # the timed solve's first step carries timing nodes around the dominant class and
        # around the tensor-core kernel's launches
        tbits = (1 << igamg.Context.PROFILE_CLASSES.index(dom)) | (1 << igamg.Context.TC_KERNEL_CLASS)
        ctx.profile_enable(0)
        # both graph variants of the PCG iteration (plain, and with timing nodes) are
        # captured before the timed region
        ctx.profile_enable(tbits)
        x.zero_()
        ctx.solve(b, x, TOL)
        ctx.profile_enable(0)
        # timed region: the solves as a user runs them (graph-replayed PCG iterations)
        sampler = ClockSampler(local_rank)
        if dist:
            tdist.barrier()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        torch.cuda.nvtx.range_push("timed")  # lets a profiler capture exactly these launches
        prof = None
        for step in range(args.steps):
            if step == 0:
                ctx.profile_enable(tbits)
            x.zero_()
            res, st = ctx.solve(b, x, TOL)
            if step == 0:
                prof = ctx.profile_read()
                ctx.profile_enable(0)
        torch.cuda.nvtx.range_pop()
        e1.record(stream)
        torch.cuda.synchronize()
        if dist:
            tdist.barrier()
        ms_total = e0.elapsed_time(e1)
        clocks = sampler.stop()
        iters = res.iters
        outer = res.outer_iters
        relres = res.relres
        # the FP64 GPU solution to 1e-12: reference of the precision variants' errors
        if prec == igamg.IGAMG_FP64:
            xr = torch.zeros_like(x)
            ctx.solve(b, xr, 1e-12)
        else:
            ref = igamg.Context(pr, stream=stream)
            xr = torch.zeros_like(x)
            ref.solve(b, xr, 1e-12)
            ref.free()
        err_vs_fp64 = None if prec == igamg.IGAMG_FP64 else float(torch.linalg.norm(x - xr) / torch.linalg.norm(xr))
        ms_total, dofs_all = combine_over_ranks(ms_total, N, tdist if dist else None, dev)
        # end to end: host vectors, H2D + D2H inside the timed region
        e2e_s = float("nan")
        if not args.no_e2e:
            # pinned host vectors (page-locked, so the copies run at full PCIe/C2C rate)
            bh = b.cpu().pin_memory().numpy()
            xh = torch.zeros(N, dtype=torch.float64).pin_memory().numpy()
            ctx.solve_host(bh, xh, TOL)
            t0 = time.perf_counter()
            for _ in range(args.steps):
                xh[:] = 0.0
                r2, _ = ctx.solve_host(bh, xh, TOL)
            e2e_s = (time.perf_counter() - t0) / args.steps
        setup_ms = res.t_setup_ms
        assemble_ms = res.t_assemble_ms
        dev_bytes = ctx.device_bytes()
        # one cycle of the working precision as the solve runs it (graph replay), against its
        # algorithmic bytes: the V-cycle's HBM roofline fraction
        ms_v, by_v = ctx.cycle_time(b, 10)
        gb_v = by_v / 1e9
        variants = {}
        if rank == 0 and world == 1 and prec == igamg.IGAMG_FP64 and not args.no_variants:
            for pn in ("fp32", "bf16"):
                v = run_precision_variant(pr, pn, b, xr, dev, stream, max(2, min(args.steps, 5)), 2)
                v["vcycle"]["achieved_gbs"] = round(v["vcycle"]["algorithmic_gb"] / (v["vcycle"]["ms"] * 1e-3), 1)
                v["vcycle"]["hbm_frac"] = round(v["vcycle"]["achieved_gbs"] / pk["hbm_gbs"], 4)
                variants[pn] = v
    ms_step = ms_total / args.steps
    value = dofs_all / (ms_step * 1e-3) / 1e6
    # rooflines: the tensor-core FD kernel (tensor pipe) and the stiffness apply (FP64 pipe,
    # or HBM for FP32/BF16 bands); the top-level one is the kernel class with the larger time
    troof = tensor_roofline(prof, pk, src)
    ap = prof1["apply"]
    if args.precision == "fp64":
        ach = ap["flops"] / (ap["ms"] * 1e-3) / 1e12
        aroof = {"bound": "alu", "achieved": round(ach, 4), "peak": f64["fma_tflops"], "unit": "TFLOP/s",
                 "frac": round(ach / f64["fma_tflops"], 4),
                 "peak_source": "measured in this run: FP64 FMA chains (igamg_micro_fp64 kind 0)",
                 "kernel": "k_band_apply (stiffness apply / residual, every level)",
                 "traffic": BAND_TRAFFIC_PER_LAUNCH.get((args.workload, args.precision))}
    else:
        ach = ap["bytes"] / (ap["ms"] * 1e-3) / 1e9
        aroof = {"bound": "hbm", "achieved": round(ach, 1), "peak": pk["hbm_gbs"], "unit": "GB/s",
                 "frac": round(ach / pk["hbm_gbs"], 4), "peak_source": src,
                 "kernel": "k_band_apply (stiffness apply / residual, every level)", "traffic": None}
    aroof["launches"] = ap["launches"]
    aroof["avg_launch_ms"] = round(ap["ms"] / max(ap["launches"], 1), 5)
    tc_ms = prof1.get("tc_kernel", {}).get("ms", 0.0)
    if troof is not None and tc_ms >= ap["ms"]:
        roof, other = troof, aroof
    else:
        roof, other = aroof, troof
    roof["timing"] = ("CUDA-event nodes around each launch in the first timed solve, on the stream each launch "
                      "runs on; the interface pieces run on a second stream concurrently with the interiors")
    breakdown = {k: {"ms_per_step": round(v["ms"], 3), "launches_per_step": v["launches"],
                     "gflop_per_step": round(v["flops"] / 1e9, 4),
                     "gbyte_per_step": round(v["bytes"] / 1e9, 4)} for k, v in prof1.items() if k not in SUB_ACCOUNTS}
    breakdown["tc_kernel (within interior_fd + interface)"] = {
        "ms_per_step": round(prof1["tc_kernel"]["ms"], 3), "launches_per_step": prof1["tc_kernel"]["launches"],
        "mma_tflop_per_step": round(prof1["tensor_exec"]["flops"] / 1e12, 4)}
    launches = sum(v["launches"] for k, v in prof.items() if k not in SUB_ACCOUNTS) * args.steps
    # whole-solve HBM view: algorithmic bytes of every class (bands, vectors, bases) per solve
    gb = sum(v["bytes"] for k, v in prof1.items() if k not in SUB_ACCOUNTS) / 1e9
    hbm = {"algorithmic_gb_per_step": round(gb, 3), "achieved_gbs": round(gb / (ms_step * 1e-3), 1),
           "peak": pk["hbm_gbs"], "frac": round(gb / (ms_step * 1e-3) / pk["hbm_gbs"], 4)}
    out = {
        "metric": METRIC, "value": round(value, 4), "unit": "MDOF/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_step, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp64": "f64", "fp32": "f32 (f64 refinement)", "bf16": "bf16 bands, f32 (f64 refinement)"}[args.precision],
        "data": "synthetic",
        "config": {"workload": args.workload, "description": WORKLOAD_DESC if args.workload == WORKLOAD
                   else args.workload, "dofs": N, "iters": iters, "outer_iters": outer,
                   "precision": args.precision, "rel_err_vs_fp64_solution": err_vs_fp64,
                   "relres": relres, "tol": TOL, "l2": "inputs larger than L2 (operator bands 0.94 GB)",
                   "parallelism": f"replicas x{world}", "setup_ms": round(setup_ms, 1),
                   "device_gb": round(dev_bytes / 1e9, 3),
                   "assemble_ms": round(assemble_ms, 1), "sm_count": f64["sm_count"]},
        "e2e": {"value": None if e2e_s != e2e_s else round(N * world / e2e_s / 1e6, 4), "unit": "MDOF/s",
                "h2d_bytes_per_step": 16 * N, "d2h_bytes_per_step": 8 * N},
        "gpu_launches": int(launches),
        "roofline": roof,
        "roofline_other_kernel": other,
        "fp64_peaks_measured": f64,
        "hbm_whole_solve": hbm,
        "vcycle": {"ms": round(ms_v, 4), "algorithmic_gb": round(gb_v, 4),
                   "achieved_gbs": round(gb_v / (ms_v * 1e-3), 1), "peak_gbs": pk["hbm_gbs"],
                   "hbm_frac": round(gb_v / (ms_v * 1e-3) / pk["hbm_gbs"], 4),
                   "note": f"one {args.precision} cycle (igamg_cycle_time), graph-replayed as inside the solve"},
        "clocks": clocks,
        "kernel_breakdown": breakdown,
    }
    if variants:
        out["precision_variants"] = variants
    try:  # the combined roofline of the whole solve (per-class bounds of the breakdown above)
        out["roofline_whole_solve"] = combined_roofline(prof1, ms_step, args.precision, pk, f64["fma_tflops"])
    except Exception as e:  # an optional field: never lose the bench line over it
        out["roofline_whole_solve"] = {"error": repr(e)}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline_json(3)
    if rank == 0:
        print(json.dumps(out), flush=True)
    ctx.free()
    if dist:
        tdist.destroy_process_group()


def run_reference(args, rank):
    if rank != 0:
        return
    o = run_oracle(max(args.steps, 1), args.warmup)
    value = o["N"] / o["t_solve_s"] / 1e6
    out = {"metric": METRIC, "value": round(value, 6), "unit": "MDOF/s", "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(o["t_solve_s"] * 1e3, 1),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp64": "f64", "fp32": "f32 (f64 refinement)", "bf16": "bf16 bands, f32 (f64 refinement)"}[args.precision],
           "data": "synthetic", "impl": "reference",
           "config": {"workload": WORKLOAD, "description": WORKLOAD_DESC, "sample": sample_desc(),
                      "sample_dofs": o["N"], "iters": o["iters"]},
           "cpu_baseline": {"value": round(value, 6), "unit": "MDOF/s", "cores": max(1, round(o["cores_used"])),
                            "kind": "oracle", "sample": sample_desc(max(args.steps, 1)) + ", 1 thread",
                            "nproc": host_cpu()[0], "cpu_model": host_cpu()[1]},
           "e2e": {"value": round(value, 6), "unit": "MDOF/s", "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


# Table II (iteration counts to 1e-8, PCG + V(1,1), Fichera corner, K = 448): rows l, columns p
TABLE_II_IT = {1: {2: 30, 3: 31, 4: 31, 5: 26, 6: 22}, 2: {2: 33, 3: 32, 4: 33, 5: 31, 6: 28},
               3: {2: 39, 3: 38, 4: 37, 5: 33, 6: 30}, 4: {2: 44, 3: 44, 4: 42, 5: 37, 6: 35}}


def fichera_table(cases):
    """Sec. 5.2 experiment: -Laplace u = 75 pi^2 sin(5 pi x) sin(5 pi y) sin(5 pi z) on the
    Fichera corner, Dirichlet on xyz = 0, PCG + V(1,1) to 1e-8; the source enters as its
    quasi-interpolant at the Greville points.  Prints one JSON line per case."""
    import numpy as np
    import torch
    import workloads
    from paper_1804_02539_gb300 import igamg
    for split, lev, p, mu in cases:
        pr = workloads.fichera_corner(split, p, 2 ** lev, lev + 1)
        opts = igamg.igamg_default_options()
        opts.mu = mu
        t0 = time.perf_counter()
        ctx = igamg.Context(pr, opts)
        t_setup = time.perf_counter() - t0
        X = ctx.greville_points()
        f = 75 * np.pi ** 2 * np.sin(5 * np.pi * X[:, 0]) * np.sin(5 * np.pi * X[:, 1]) * np.sin(5 * np.pi * X[:, 2])
        coef = torch.tensor(f, device="cuda")
        b = torch.empty_like(coef)
        ctx.rhs_from_coefs(coef, b)
        x = torch.zeros_like(b)
        res, st = ctx.solve(b, x, TOL)
        paper = TABLE_II_IT.get(lev, {}).get(p) if split == 4 and mu == 1 else None
        print(json.dumps({"K": pr.num_patches, "l": lev, "p": p, "cycle": "V" if mu == 1 else "W",
                          "dofs": ctx.num_dofs(), "coarse_dofs": ctx.num_dofs(0), "iters": res.iters,
                          "paper_iters": paper, "relres": res.relres, "setup_s": round(t_setup, 2),
                          "solve_ms": round(res.t_solve_ms, 1)}), flush=True)
        ctx.free()


# ---------------------------------------------------------------- batched workload

BATCH_COUNT, BATCH_SEED = 512, 4
BATCH_DESC = ("512 independent 2D Poisson problems (seed 4): sqrt(K) x sqrt(K) rectangle patches on [0,1]^2, "
              "K in {4,9,16,25,36}, p in {2..6}, m in {16,32,64,128} intervals per patch direction, iid uniform; "
              "all Dirichlet, f = 2 pi^2 sin(pi x) sin(pi y) through its Greville interpolant; FP64 PCG + V(1,1) "
              "to 1e-8 each, all resident, solved together (lockstep engine: one launch per cycle step over "
              "all problems)")
BATCH_ORACLE_SAMPLE = 6   # the oracle solves the first problems of the batch with m <= 32


def sin_rhs_coefs(X):
    import numpy as np
    return 2 * np.pi ** 2 * np.sin(np.pi * X[:, 0]) * np.sin(np.pi * X[:, 1])


def oracle_greville(pr, sp):
    """Greville points of the oracle's dofs (oracle numbering): Greville abscissae of the
    owning patch's finest knot vectors through its bilinear map."""
    import numpy as np
    from oracle import patch as opatch
    X = np.zeros((sp.N, 2))
    for k in range(pr.num_patches):
        ids = sp.l2g[k].ravel()
        keep = ids >= 0
        g = []
        for j in range(2):
            t = sp.knots[k][j]
            p = int(sp.p[k, j])
            g.append(np.array([t[i + 1:i + p + 1].mean() for i in range(len(t) - p - 1)]))
        grid = np.stack([a.ravel() for a in np.meshgrid(g[0], g[1], indexing="ij")], 1)
        Xk, _ = opatch.geometry(np.asarray(pr.corners[k]), grid)
        X[ids[keep]] = Xk[keep]
    return X


def oracle_batch_json():
    """Subprocess, one thread: oracle setup (untimed) and one PCG solve each (timed) of the
    first BATCH_ORACLE_SAMPLE problems of the batch with at most 32 intervals."""
    import workloads
    from oracle import multipatch, solver
    probs = [p for p in workloads.batch_problems(BATCH_COUNT, BATCH_SEED) if int(p.name.split("_m")[-1]) <= 32]
    probs = probs[:BATCH_ORACLE_SAMPLE]
    N = 0
    t = 0.0
    its = []
    for pr in probs:
        H = solver.build_hierarchy(pr)
        sp = H.levels[-1].space
        _, Mg = multipatch.stiffness(pr, sp, want_mass=True)
        b = Mg @ sin_rhs_coefs(oracle_greville(pr, sp))
        t0 = time.perf_counter()
        its.append(solver.pcg(H, b, tol=TOL).iters)
        t += time.perf_counter() - t0
        N += sp.N
    return {"N": N, "t_solve_s": t, "iters": its, "problems": [p.name for p in probs]}


def run_batch(args):
    import numpy as np
    import torch
    import workloads
    from paper_1804_02539_gb300 import igamg
    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    probs = workloads.batch_problems(BATCH_COUNT, BATCH_SEED)
    opts = igamg.igamg_default_options()
    opts.precision = {"fp64": igamg.IGAMG_FP64, "fp32": igamg.IGAMG_FP32, "bf16": igamg.IGAMG_BF16}[args.precision]
    with torch.cuda.stream(stream):
        t0 = time.perf_counter()
        B = igamg.Batch(probs, opts, workers=args.workers, stream=stream)
        t_setup = time.perf_counter() - t0
        Ns = [c.num_dofs() for c in B.contexts]
        rhs, xs = [], []
        for c in B.contexts:
            coef = torch.tensor(sin_rhs_coefs(c.greville_points()), device="cuda")
            b = torch.empty_like(coef)
            c.rhs_from_coefs(coef, b)
            rhs.append(b)
            xs.append(torch.zeros_like(b))
        torch.cuda.synchronize()
        for _ in range(args.warmup):
            for x in xs:
                x.zero_()
            B.solve(rhs, xs, TOL)
        sampler = ClockSampler(0)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            for x in xs:
                x.zero_()
            st, res, sts = B.solve(rhs, xs, TOL)
        e1.record(stream)
        torch.cuda.synchronize()
        ms_total = e0.elapsed_time(e1)
        clocks = sampler.stop()
        assert st == 0, sts
        # profiled pass (untimed, worker streams: the contexts' own accounting; the lockstep
        # engine counts its launches and FLOPs itself)
        prof = {}
        if B.engine() == "streams":
            for c in B.contexts:
                c.profile_enable(0x3F)
            for x in xs:
                x.zero_()
            B.solve(rhs, xs, TOL)
            for c in B.contexts:
                for k, v in c.profile_read().items():
                    acc = prof.setdefault(k, {"launches": 0, "ms": 0.0, "flops": 0.0, "bytes": 0.0})
                    for f in acc:
                        acc[f] += v[f]
                c.profile_enable(0)
        # end to end: pinned host rhs in, solutions out, inside the timed region
        e2e = None
        if not args.no_e2e:
            hb = [r.cpu().pin_memory() for r in rhs]
            hx = [torch.empty(n, dtype=torch.float64).pin_memory() for n in Ns]
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for _ in range(args.steps):
                for h, r in zip(hb, rhs):
                    r.copy_(h, non_blocking=True)
                for x in xs:
                    x.zero_()
                B.solve(rhs, xs, TOL)
                for h, x in zip(hx, xs):
                    h.copy_(x, non_blocking=True)
                torch.cuda.synchronize()
            e2e = (time.perf_counter() - t0) / args.steps
    ms_step = ms_total / args.steps
    Ntot = sum(Ns)
    value = Ntot / (ms_step * 1e-3) / 1e6
    for k in SUB_ACCOUNTS:
        prof.pop(k, None)
    f64 = fp64_peaks()
    engine = B.engine()
    lk = B.stats() if engine == "lockstep" else None
    flops = lk["flops"] if lk else sum(v["flops"] for v in prof.values())
    byts = sum(v["bytes"] for v in prof.values())
    ach = flops / (ms_step * 1e-3) / 1e12
    pk, src = peaks()
    out = {
        "metric": METRIC, "value": round(value, 4), "unit": "MDOF/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms_step, 3), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": {"fp64": "f64", "fp32": "f32 (f64 refinement)",
                                       "bf16": "bf16 bands, f32 (f64 refinement)"}[args.precision],
        "data": "synthetic",
        "config": {"workload": "batch512_2d_rect", "description": BATCH_DESC, "problems": len(probs),
                   "engine": engine, "launches_per_solve": lk["launches"] if lk else None,
                   "dofs_total": Ntot, "dofs_min": min(Ns), "dofs_max": max(Ns), "workers": min(args.workers or 16, len(probs)),
                   "iters_min": min(r.iters for r in res), "iters_max": max(r.iters for r in res),
                   "setup_s": round(t_setup, 1), "l2": "inputs larger than L2 (vectors of 5.3e7 dofs)",
                   "device_gb": round(sum(c.device_bytes() for c in B.contexts) / 1e9, 3)},
        "e2e": {"value": None if e2e is None else round(Ntot / e2e / 1e6, 4), "unit": "MDOF/s",
                "h2d_bytes_per_step": 8 * Ntot, "d2h_bytes_per_step": 8 * Ntot},
        "gpu_launches": int((lk["launches"] if lk else sum(v["launches"] for v in prof.values())) * args.steps),
        "roofline": {"bound": "alu", "achieved": round(ach, 4), "peak": f64["fma_tflops"],
                     "unit": "TFLOP/s", "frac": round(ach / f64["fma_tflops"], 4),
                     "peak_source": "measured in this run: FP64 FMA chains (igamg_micro_fp64 kind 0)",
                     "kernel": "whole batch step (all classes, " + ("lockstep launches over all problems"
                               if lk else "concurrent streams") + ")",
                     "hbm_gbs": round(byts / (ms_step * 1e-3) / 1e9, 1) if not lk else None,
                     "hbm_peak": pk["hbm_gbs"], "traffic": None,
                     "tensor_tflops": round(lk["mma_flops"] / (ms_step * 1e-3) / 1e12, 2) if lk else None},
        "clocks": clocks,
        "kernel_breakdown": {k: {"launches_per_step": v["launches"], "gflop_per_step": round(v["flops"] / 1e9, 3),
                                 "gbyte_per_step": round(v["bytes"] / 1e9, 3)} for k, v in prof.items()} if not lk
                            else {"all": {"launches_per_step": lk["launches"], "gflop_per_step": round(lk["flops"] / 1e9, 3),
                                          "mma_tflop_per_step": round(lk["mma_flops"] / 1e12, 3)}},
    }
    if not args.no_cpu_baseline:
        env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
        o = subprocess.run([sys.executable, os.path.abspath(__file__), "--_oracle_batch"], env=env,
                           stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True, timeout=1800)
        if o.returncode == 0:
            d = json.loads(o.stdout.strip().splitlines()[-1])
            out["cpu_baseline"] = {"value": round(d["N"] / d["t_solve_s"] / 1e6, 6), "unit": "MDOF/s", "cores": 1,
                                   "kind": "oracle", "sample": f"the first {BATCH_ORACLE_SAMPLE} problems of the "
                                   "batch with m <= 32, one PCG solve each, setup excluded, 1 thread",
                                   "sample_dofs": d["N"], "sample_iters": d["iters"]}
    print(json.dumps(out), flush=True)
    B.free()


# ---------------------------------------------------------------- served workload

SERVE_DESC = ("Poisson arrivals of single-rhs requests over a catalog of 110 models: the 100 2D problems of the "
              "batched family (K in {4,9,16,25,36}, p in {2..6}, m in {16,32,64,128}) drawn with 80% probability "
              "and 10 perturbed 2x2x2 cubes (p in {2,3}, m in {16,24,32,40,48}) with 20%; rhs = U(-1,1) load "
              "vectors; PCG + V(1,1) to relative residual 1e-8 (mixed precision: FP64 iterative refinement); "
              "hierarchies resident under the device-memory budget (one untimed warm-up request per model "
              "builds them); waiting requests of one 2D model taken together (up to 16) and solved as "
              "several right-hand sides in lockstep (FP64 numerics)")


def run_serve(args):
    import threading
    import numpy as np
    import workloads
    from paper_1804_02539_gb300 import igamg
    probs, is3d = workloads.serving_models()
    opts = igamg.igamg_default_options()
    opts.precision = {"fp64": igamg.IGAMG_FP64, "fp32": igamg.IGAMG_FP32, "bf16": igamg.IGAMG_BF16}[args.precision]
    srv = igamg.Server(opts, workers=args.workers, hbm_budget_bytes=int(args.budget_gb * (1 << 30)))
    ids = [srv.add_model(p) for p in probs]
    rng = np.random.default_rng(5)
    rhs = [[rng.uniform(-1, 1, n) for _ in range(2)] for _, n, _ in ids]
    t0 = time.perf_counter()
    warm = [srv.submit(ids[m][0], rhs[m][0], TOL)[0] for m in range(len(ids))]
    for r in warm:
        assert srv.wait(r)["status"] == 0
    t_warm = time.perf_counter() - t0
    lines = []
    for rate in args.rates:
        reqs = workloads.serving_requests(is3d, rate, args.serve_requests)
        rids = []
        infos = [None] * len(reqs)
        ready = threading.Semaphore(0)

        def waiter():
            for i in range(len(reqs)):
                ready.acquire()
                infos[i] = srv.wait(rids[i])

        th = threading.Thread(target=waiter)
        th.start()
        sampler = ClockSampler(0)
        start = time.perf_counter()
        for (ta, m, seed) in reqs:
            delay = start + ta - time.perf_counter()
            if delay > 0:
                time.sleep(delay)
            rids.append(srv.submit(ids[m][0], rhs[m][seed % 2], TOL)[0])
            ready.release()
        th.join()
        clocks = sampler.stop()
        lat = np.array([i["t_done_ms"] - i["t_submit_ms"] for i in infos])
        svc = np.array([i["t_done_ms"] - i["t_start_ms"] for i in infos])
        span = max(i["t_done_ms"] for i in infos) - min(i["t_submit_ms"] for i in infos)
        dofs = sum(ids[m][1] for _, m, _ in reqs)
        assert all(i["status"] == 0 for i in infos)
        lines.append({"rate_per_s": rate, "requests": len(reqs), "p50_ms": round(float(np.percentile(lat, 50)), 2),
                      "p99_ms": round(float(np.percentile(lat, 99)), 2),
                      "mean_service_ms": round(float(svc.mean()), 2),
                      "mdof_per_s": round(dofs / (span * 1e-3) / 1e6, 3),
                      "mean_group": round(float(np.mean([i["group"] for i in infos])), 2),
                      "max_group": int(max(i["group"] for i in infos)),
                      "served_per_s": round(len(reqs) / (span * 1e-3), 1), "clocks": clocks})
    st = srv.stats()
    srv.free()
    best = max(lines, key=lambda l: l["mdof_per_s"])
    out = {"metric": METRIC, "value": best["mdof_per_s"], "unit": "MDOF/s", "n_gpus": 1,
           "steps": len(args.rates), "warmup": 1, "ms_per_step": None, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None,
           "dtype": {"fp64": "f64", "fp32": "f32 (f64 refinement)", "bf16": "bf16 bands, f32 (f64 refinement)"}[args.precision],
           "data": "synthetic",
           "config": {"workload": "serve_110_models", "description": SERVE_DESC, "workers": args.workers,
                      "precision": args.precision,
                      "budget_gb": args.budget_gb, "warmup_s": round(t_warm, 1), "models": len(probs),
                      "resident": st["resident"], "setups": st["setups"], "evictions": st["evictions"],
                      "groups": st["groups"], "grouped_requests": st["grouped"],
                      "device_gb": round(st["device_bytes"] / 1e9, 3),
                      "l2": "inputs larger than L2 (resident hierarchies of GBs)"},
           "serving": lines}
    print(json.dumps(out), flush=True)


# ---------------------------------------------------------------- smoother micro-benchmark

def run_micro_fd(args):
    """The finest-level smoother of the workload (patch-interior FD contractions plus the
    interface pieces) applied `steps` times after `warmup`, timed with CUDA events; with
    --no-autotune the static engine rule applies (tensor cores on the 2D interiors)."""
    import numpy as np
    import torch
    import workloads
    from paper_1804_02539_gb300 import igamg
    torch.cuda.set_device(0)
    pr = workloads.CONFIGS[args.workload]()
    o = igamg.igamg_default_options()
    o.autotune = 0 if args.no_autotune else 1
    o.fd_engine = args.fd_engine
    ctx = igamg.Context(pr, o)
    L = pr.num_levels - 1
    r = torch.tensor(np.random.default_rng(1).normal(size=ctx.num_dofs()), device="cuda")
    z = torch.empty_like(r)
    for _ in range(args.warmup):
        ctx.smooth(L, r, z)
    ctx.profile_enable(0xFF)
    ctx.smooth(L, r, z)
    prof = ctx.profile_read()
    ctx.profile_enable(0)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    torch.cuda.nvtx.range_push("timed")  # lets a profiler capture exactly these launches
    for _ in range(args.steps):
        ctx.smooth(L, r, z)
    torch.cuda.nvtx.range_pop()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    fd, tc = prof["interior_fd"], prof["tc_kernel"]
    print(json.dumps({"micro": "finest smoother", "workload": args.workload, "fd_engine": args.fd_engine,
                      "autotune": o.autotune, "ms_per_smoother": round(ms, 4),
                      "fd_ms_profiled": round(fd["ms"], 4), "fd_launches": fd["launches"],
                      "tc_gemm_ms_profiled": round(tc["ms"], 4), "tc_gemm_launches": tc["launches"],
                      "interface_ms_profiled": round(prof["interface"]["ms"], 4),
                      "tc_mma_tflops": round(prof["tensor_exec"]["flops"] / max(tc["ms"], 1e-9) / 1e9, 1),
                      "fd_fp64_tflops": round(fd["flops"] / (fd["ms"] * 1e-3) / 1e12, 3)}), flush=True)
    ctx.free()


def run_micro_fp64():
    """FP64 reference rate of this GPU: cuBLAS DGEMM (torch.matmul in float64, 8192^3),
    best of 5 after warm-up; the denominator the FP64 roofline fractions are compared with."""
    import torch
    n = 8192
    a = torch.randn(n, n, dtype=torch.float64, device="cuda")
    b = torch.randn(n, n, dtype=torch.float64, device="cuda")
    for _ in range(2):
        torch.matmul(a, b)
    torch.cuda.synchronize()
    best = 1e30
    for _ in range(5):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        torch.matmul(a, b)
        e1.record()
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1))
    f64 = fp64_peaks()
    print(json.dumps({"micro": "fp64", "dgemm_n": n, "dgemm_ms": round(best, 3),
                      "dgemm_tflops": round(2 * n ** 3 / (best * 1e-3) / 1e12, 4),
                      "fma_chain_tflops": f64["fma_tflops"], "mma_m8n8k4_tflops": f64["mma_tflops"],
                      "sm_count": f64["sm_count"],
                      "nominal_fma_peak_tflops": round(f64["sm_count"] * 2 * 2 * 2.07e9 / 1e12, 4)}), flush=True)


def main():
    if "--_oracle_batch" in sys.argv:
        print(json.dumps(oracle_batch_json()))
        return
    if "--fichera" in sys.argv:
        cases = [(4, l, 2, 1) for l in (1, 2, 3, 4)] + [(4, l, 2, 2) for l in (1, 2, 3)]
        cases += [(2, l, p, 1) for p in (3, 4) for l in (1, 2, 3, 4)]
        fichera_table(cases)
        return
    if "--_oracle" in sys.argv:
        print(json.dumps(oracle_sample_json()))
        return
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-variants", action="store_true", help="skip the FP32/BF16 lines of the default run")
    ap.add_argument("--workload", default=WORKLOAD, help="key of workloads.CONFIGS")
    ap.add_argument("--precision", default="fp64", choices=["fp64", "fp32", "bf16"])
    ap.add_argument("--batch", action="store_true", help="the 512-problem batched workload")
    ap.add_argument("--workers", type=int, default=16, help="host worker threads of the batch")
    ap.add_argument("--micro", choices=["fd", "fp64"], help="micro-benchmark instead of the solve")
    ap.add_argument("--serve", action="store_true", help="the served workload (Poisson arrivals)")
    ap.add_argument("--rates", type=float, nargs="+", default=[200.0, 500.0, 2000.0])
    ap.add_argument("--serve-requests", type=int, default=4000)
    ap.add_argument("--budget-gb", type=float, default=96.0)
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--fd-engine", type=int, default=0)
    args = ap.parse_args()
    if args.micro == "fp64":
        run_micro_fp64()
        return
    if args.micro:
        run_micro_fd(args)
        return
    if args.serve:
        if args.workers == 16:
            args.workers = 8
        run_serve(args)
        return
    if args.batch:
        run_batch(args)
        return
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
    else:
        run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
