"""Benchmark of the matrix-free hybrid multigrid solve on GB300.

One step = one complete solve of the variable-coefficient diffusion workload
(log-normal K per cell, Q4 on a 32^3 hex mesh, 4,096,000 dofs): outer FP64 CG
to a 1e-8 relative residual, preconditioned by one hybrid V-cycle (block-Jacobi
with per-cell inner PCG to eps = 1e-2, Q1 coarse space with aggregation AMG).
Every step of the hot path runs: operator apply, fused smoother, residual,
restriction, AMG cycle, prolongation, Krylov vector kernels.

  value      dofs solved per second (GDOF/s), inputs resident in HBM, L2
             flushed between steps (a 256 MiB write outside the timed events)
  e2e        the same through the C ABI with host buffers: f copied in from
             pinned memory and u copied back, inside the timed region
  roofline   the dominant kernel (the fused smoother, FP64): the FP64
             operations it issues per launch / its CUDA-event duration in the
             timed steps, against the FP64 pipe peak (4 flop/clk/SM x 152 SMs
             x 2070 MHz); the generic operation count (32 n^4 + 120 n^3 per
             cell and apply) beside it
  extra      apply GDOF/s (FP64 and FP32), the mixed-precision solve time

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl dgmg|reference]
Under torchrun (N > 1) each rank solves its own replica (weak scaling, no
collective on the data path); rank 0 prints one JSON line.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "DG apply GDOF/s; solve s to 1e-8 residual (FP64 vs mixed); serve p99 latency"
WORKLOAD = dict(kind="lognormal", n=32, p=4)
SM_COUNT = 152
FP64_FLOP_PER_CLK_SM = 4          # 1.25 TFLOP/s nominal / (152 SMs x 2.07 GHz)
SM_MAX_MHZ = 2070.0
CPU_SAMPLE = dict(n=8, p=4)        # oracle sample: same workload family, 8^3 cells
# DRAM bytes (read + write) of one k_smooth_pcg<double> launch on this mesh, from
# the ncu capture summarised in profiles/k_smooth_pcg_fp64_lognormal_32cubed_q4.txt;
# None while no capture of the current kernel exists.
SMOOTHER_TRAFFIC_BYTES = 102.546176e6 + 14.194944e6


def fp64_peak_tflops():
    mhz = SM_MAX_MHZ
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            mhz = float(json.load(fh).get("sm_max_mhz", mhz))
    except (OSError, ValueError):
        pass
    return SM_COUNT * FP64_FLOP_PER_CLK_SM * mhz * 1e6 / 1e12


# ---------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as fh:
            for line in fh:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------- ranks
def max_over_ranks(value, world, device="cpu"):
    """Largest value over all ranks (the job's time is its slowest rank)."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(ndof, steps, world, total_ms):
    """Whole-job GDOF/s: dofs solved by all ranks over the slowest rank's time."""
    return ndof * steps * world / (total_ms / 1e3) / 1e9


# ---------------------------------------------------------------- workload
def make_workload():
    from paper_1805_11930_gb300 import inputs
    return inputs.lognormal(WORKLOAD["n"], WORKLOAD["p"])


def setup_context(w, device):
    import torch
    from paper_1805_11930_gb300 import dgmg, inputs
    ctx = dgmg.Context(device)
    ctx.set_mesh(*w["nc"], *w["L"], w["p"], w["bc"])
    ctx.set_coefficients(w["K"], b_vertex=w["b"], c_cell=w["c"])
    vol, face = ctx.quadrature_points()
    s = ctx.sizes()
    f = torch.empty(s["ndof"], dtype=torch.float64, device=f"cuda:{device}")
    ctx.assemble_rhs(inputs.evaluate(w["f"], vol), f, g_qp=inputs.evaluate(w["g"], face),
                     j_qp=inputs.evaluate(w["j"], face))
    return ctx, f, s


def run_dgmg(args, rank, world, local_rank):
    import torch
    import torch.distributed as dist
    from paper_1805_11930_gb300 import dgmg, flops

    torch.cuda.set_device(local_rank)
    dev = f"cuda:{local_rank}"
    w = make_workload()
    ctx, f, s = setup_context(w, local_rank)
    ndof, ncell, n = s["ndof"], s["ncell"], w["p"] + 1
    stream = torch.cuda.current_stream(local_rank)
    u = torch.zeros_like(f)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    opts = dgmg.default_opts(timing=1)
    # launch shapes (warps per block) and work layouts (line / factored /
    # plane) of the operator and smoother kernels, timed on this mesh for each
    # arithmetic before anything is measured
    shapes, layouts = {}, {}
    for name, prec in (("fp64", dgmg.FP64), ("fp32", dgmg.FP32), ("df64", dgmg.DF64)):
        shapes[name] = ctx.autotune(prec)
        layouts[name] = [dgmg.LAYOUT_NAMES[x] for x in ctx.get_layout(prec)]

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        u.zero_()
        ctx.solve(f, u, opts)
    barrier()
    clocks = ClockSampler(local_rank)
    clocks.start()
    stats = []
    step_ms = []
    torch.cuda.nvtx.range_push("timed_steps")   # lets a profiler select the timed region
    for _ in range(args.steps):
        flush.fill_(1.0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        u.zero_()
        st = ctx.solve(f, u, opts)
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        stats.append(st)
    torch.cuda.nvtx.range_pop()
    barrier()
    clk = clocks.stop()
    total_ms = max_over_ranks(sum(step_ms), world, dev)
    value = job_throughput(ndof, args.steps, world, total_ms)

    # dominant kernel: the fused smoother (CUDA events around each launch)
    sm_ms = sum(x["ms_smooth"] for x in stats)
    ap_ms = sum(x["ms_apply"] for x in stats)
    sweeps = sum(x["sweeps"] for x in stats)
    zero = sum(x["zero_sweeps"] for x in stats)
    its = sum(x["inner_its_total"] for x in stats)
    sm_gflops = flops.algorithmic_smoother(n, ncell, sweeps, zero, its)
    sm_kflops = flops.kernel_smoother(n, ncell, sweeps, zero, its)
    nap = sum(x["applies"] for x in stats)
    ap_gflops = flops.algorithmic_apply(n) * ncell * nap
    ap_kflops = flops.kernel_apply_full(n) * ncell * nap
    peak = fp64_peak_tflops()
    dominant = "smoother" if sm_ms >= ap_ms else "apply"
    if dominant == "smoother":
        k_flops, g_flops, k_ms, launches = sm_kflops, sm_gflops, sm_ms, max(sweeps, 1)
    else:
        k_flops, g_flops, k_ms, launches = ap_kflops, ap_gflops, ap_ms, max(nap, 1)
    achieved = k_flops / (k_ms / 1e3) / 1e12
    achieved_generic = g_flops / (k_ms / 1e3) / 1e12
    roofline = {"bound": "alu", "kernel": "k_smooth_pcg<double>" if dominant == "smoother" else "k_apply<double>",
                "achieved": round(achieved, 4), "peak": round(peak, 4), "unit": "TFLOP/s",
                "frac": round(achieved / peak, 4),
                "traffic": SMOOTHER_TRAFFIC_BYTES if dominant == "smoother" else None,
                "traffic_note": "ncu dram__bytes_read.sum + dram__bytes_write.sum of one sweep with defect on this "
                                "mesh (profiles/k_smooth_pcg_fp64_lognormal_32cubed_q4.txt); algorithmic bytes "
                                "4 x 8 B x ndof = 131 MB, part of it served from L2",
                "flops_per_launch": k_flops / launches, "launch_ms": round(k_ms / launches, 4),
                "launches": launches,
                "flops_note": "FP64 flops the kernel issues, an FMA counted as 2 (flops.kernel_smoother / "
                              "kernel_apply_full): per inner iteration the factored block apply and the PCG vector "
                              "work, per defect the factored full operator; timed by CUDA events around every "
                              "launch on the solve's stream inside the timed steps",
                "achieved_generic_count": round(achieved_generic, 4),
                "frac_generic_count": round(achieved_generic / peak, 4),
                "generic_count_note": "the generic count (32 n^4 + 120 n^3 per cell per apply, one apply "
                                      "per defect and per inner iteration) over the same time; above 1 because the "
                                      "kernels do the same operator with fewer operations",
                "peak_note": "FP64 pipe: 4 flop/clk/SM x 152 SMs x sm_max_mhz (derived from the nominal "
                             "1.25 TFLOP/s; no measured FP64 peak in MEASURED_PEAKS.json)",
                "time_share": {k: (round(sum(x[key] for x in stats) / total_ms, 3) if world == 1 else None)
                               for k, key in (("smoother", "ms_smooth"), ("apply", "ms_apply"),
                                              ("transfer", "ms_transfer"), ("coarse", "ms_coarse"),
                                              ("krylov", "ms_krylov"))}}

    # apply throughput, FP64 and FP32 (separate timed loop, inputs resident)
    def time_apply(dtype, reps=20, df64=False):
        x = torch.rand(ndof, dtype=dtype, device=dev)
        y = torch.empty_like(x)
        for _ in range(3):
            ctx.apply(x, y, df64=df64)
        torch.cuda.synchronize()
        ms = []
        for _ in range(reps):
            flush.fill_(1.0)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            ctx.apply(x, y, df64=df64)
            b.record(stream)
            b.synchronize()
            ms.append(a.elapsed_time(b))
        return ndof / (statistics.median(ms) / 1e3) / 1e9, statistics.median(ms)

    apply64, apply64_ms = time_apply(torch.float64)
    apply32, apply32_ms = time_apply(torch.float32)
    applydf, applydf_ms = time_apply(torch.float64, df64=True)

    def time_solve(opts, reps=3):
        for _ in range(2):
            u.zero_()
            ctx.solve(f, u, opts)
        ms, st = [], None
        for _ in range(reps):
            flush.fill_(1.0)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            u.zero_()
            st = ctx.solve(f, u, opts)
            b.record(stream)
            b.synchronize()
            ms.append(a.elapsed_time(b))
        return statistics.median(ms), st

    # mixed precision (FP32 smoother and V-cycle, FP64 flexible CG) and the
    # double-float variants (FP64 vectors, FP32-pair arithmetic)
    mixed_ms, mst = time_solve(dgmg.default_opts(smoother_prec=dgmg.FP32, krylov=dgmg.KRYLOV_FCG))
    mdf_ms, mdfst = time_solve(dgmg.default_opts(smoother_prec=dgmg.FP32, krylov=dgmg.KRYLOV_FCG,
                                                 apply_prec=dgmg.DF64))
    df_ms, dfst = time_solve(dgmg.default_opts(smoother_prec=dgmg.DF64, krylov=dgmg.KRYLOV_FCG,
                                               apply_prec=dgmg.DF64))
    # exact block solves by stored inverses (partially matrix-free smoother)
    t_inv = time.perf_counter()
    ctx.block_inverse(dgmg.FP64)
    ctx.block_inverse(dgmg.FP32)
    inv_setup_s = time.perf_counter() - t_inv
    pmf_ms, pmfst = time_solve(dgmg.default_opts(inner=dgmg.INNER_DIRECT))
    pmf32_ms, pmf32st = time_solve(dgmg.default_opts(inner=dgmg.INNER_DIRECT, smoother_prec=dgmg.FP32,
                                                     krylov=dgmg.KRYLOV_FCG))

    # end to end through the C ABI with host buffers: the same solve options as
    # the timed steps, the same L2 flush before each step (outside its timer),
    # f copied in from pinned memory and u copied back inside it
    f_host = f.cpu().pin_memory()
    u_host = torch.empty(ndof, dtype=torch.float64).pin_memory()
    f_dev = torch.empty_like(f)
    barrier()
    e2e_s = 0.0
    for _ in range(args.steps):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        f_dev.copy_(f_host, non_blocking=True)
        u.zero_()
        ctx.solve(f_dev, u, opts)
        u_host.copy_(u, non_blocking=True)
        torch.cuda.synchronize()
        e2e_s += time.perf_counter() - t0
    barrier()
    e2e_s = max_over_ranks(e2e_s, world, dev)
    e2e = {"value": round(job_throughput(ndof, args.steps, world, e2e_s * 1e3), 9), "unit": "GDOF/s",
           "h2d_bytes_per_step": ndof * 8, "d2h_bytes_per_step": ndof * 8}

    last = stats[-1]
    out = {
        "metric": METRIC, "value": round(value, 9), "unit": "GDOF/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(total_ms / args.steps, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {**workload_config(), "l2": "flushed between steps (256 MiB write)",
                   "parallelism": f"replicas x{world}",
                   "warps_per_block": {k: {"apply": a, "smoother": b} for k, (a, b) in shapes.items()},
                   "layouts": {k: {"apply": a, "smoother": b} for k, (a, b) in layouts.items()}},
        "e2e": e2e,
        "gpu_launches": int(sum(x["kernel_launches"] for x in stats)),
        "roofline": roofline,
        "clocks": clk,
        "solve": {"iterations": last["iterations"], "rel_residual": last["rel_residual"],
                  "inner_mean": round(last["inner_mean"], 3), "inner_std": round(last["inner_std"], 3),
                  "inner_max": last["inner_max"],
                  "solve_s_fp64": round(total_ms / args.steps / 1e3, 5),
                  "solve_s_mixed": round(mixed_ms / 1e3, 5),
                  "mixed_iterations": mst["iterations"], "mixed_rel_residual": mst["rel_residual"],
                  "solve_s_mixed_df64_outer": round(mdf_ms / 1e3, 5), "mixed_df64_rel_residual": mdfst["rel_residual"],
                  "solve_s_df64": round(df_ms / 1e3, 5), "df64_iterations": dfst["iterations"],
                  "df64_rel_residual": dfst["rel_residual"],
                  "block_inverse_setup_s": round(inv_setup_s, 4),
                  "solve_s_fp64_direct": round(pmf_ms / 1e3, 5), "fp64_direct_iterations": pmfst["iterations"],
                  "fp64_direct_rel_residual": pmfst["rel_residual"],
                  "solve_s_mixed_direct": round(pmf32_ms / 1e3, 5), "mixed_direct_iterations": pmf32st["iterations"],
                  "mixed_direct_rel_residual": pmf32st["rel_residual"]},
        "apply": {"gdofs_fp64": round(apply64, 4), "ms_fp64": round(apply64_ms, 4),
                  "gdofs_fp32": round(apply32, 4), "ms_fp32": round(apply32_ms, 4),
                  "gdofs_df64": round(applydf, 4), "ms_df64": round(applydf_ms, 4)},
    }
    return out


def workload_config():
    """The config of the benchmark line (both arms): the workload one step solves."""
    n, p = WORKLOAD["n"], WORKLOAD["p"]
    ndof = n ** 3 * (p + 1) ** 3
    return {"workload": f"variable-coefficient diffusion, log-normal K per cell (sigma 1, seed 1805), "
                        f"SIPG Q{p} on {n}^3 hexes, {ndof} dofs, FP64 CG + hybrid V-cycle "
                        f"(block-Jacobi omega 0.8, inner PCG eps 1e-2, Q1 + AMG), rtol 1e-8",
            "ndof": ndof, "p": p, "mesh": [n, n, n]}


# ---------------------------------------------------------------- oracle (CPU)
def oracle_solve_sample(repeats=1, n=CPU_SAMPLE["n"]):
    """The CPU oracle (MX design: assembled block-CSR A, PCG on dense blocks,
    P^T A P + AMG, CG) on a bounded sample of the same workload family, with
    the benchmark's solver settings (block-Jacobi damping 0.8, the library's
    default).  Set-up once, then `repeats` solves from u = 0.  Also times the
    oracle's block-CSR apply A u and one dense-LU block-Jacobi sweep (LU
    factors computed before the timer).  Returns ([(dofs per second of the
    solve phase, seconds)] per solve, description, {apply_gdofs,
    lu_sweep_gdofs})."""
    import numpy as np
    from oracle import amg, dg, solvers, transfer
    from paper_1805_11930_gb300 import inputs
    w = inputs.lognormal(n, CPU_SAMPLE["p"])
    t0 = time.perf_counter()
    P = dg.Problem(*w["nc"], *w["L"], w["p"], w["bc"], w["K"])
    A = P.assemble()
    X = P.volume_points()
    pts = np.concatenate([xyz.reshape(-1, 3) for _, xyz in P.boundary_points()])
    F = P.rhs(inputs.evaluate(w["f"], X), g_qp=inputs.evaluate(w["g"], pts))
    Pm = transfer.prolongation(P)
    am = amg.AggregationAMG(transfer.q1_matrix(P), P.nv)
    S = solvers.BlockJacobi(A, P.N, inner="pcg", eps=1e-2)
    V = solvers.HybridVCycle(A, Pm, S, am.vcycle, omega=0.8)
    t1 = time.perf_counter()
    out = []
    for _ in range(repeats):
        ta = time.perf_counter()
        x, it, hist = solvers.cg(lambda v: A @ v, F, V, rtol=1e-8)
        tb = time.perf_counter()
        out.append((P.ndof / (tb - ta), tb - ta))
    desc = (f"oracle solve of lognormal {n}^3 Q{CPU_SAMPLE['p']} ({P.ndof} dofs), "
            f"CG {it} its to {hist[-1]:.1e}, setup {t1 - t0:.1f} s excluded, solve {out[-1][1]:.1f} s, 1 thread")
    u = np.random.default_rng(0).uniform(-1, 1, P.ndof)
    ta = time.perf_counter()
    for _ in range(10):
        A @ u
    t_apply = (time.perf_counter() - ta) / 10
    lu = solvers.BlockJacobi(A, P.N, inner="lu")
    lu(F, u, 1, 0.8)                                  # factors the blocks
    ta = time.perf_counter()
    lu(F, u, 1, 0.8)
    t_sweep = time.perf_counter() - ta
    parts = {"apply_gdofs": round(P.ndof / t_apply / 1e9, 6), "lu_sweep_gdofs": round(P.ndof / t_sweep / 1e9, 6)}
    return out, desc, parts


def oracle_subprocess(repeats=1, n=CPU_SAMPLE["n"]):
    """Run the oracle sample (n^3 cells) in a fresh single-threaded process;
    returns ([(dofs/s, seconds)] per solve, description, oracle apply and
    LU-sweep rates) or (None, error text, {})."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--cpu-baseline-worker",
                        "--worker-repeats", str(repeats), "--oracle-cells", str(n)], env=env,
                       capture_output=True, text=True,
                       timeout=600 + 120 * repeats)
    if r.returncode != 0:
        return None, "failed: " + r.stderr[-300:], {}
    d = json.loads(r.stdout.strip().splitlines()[-1])
    return d["samples"], d["desc"], d["parts"]


def host_cpu():
    """CPU model and logical core count of this host (lscpu, else /proc/cpuinfo)."""
    model = None
    try:
        r = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10)
        for line in r.stdout.splitlines():
            if line.strip().startswith("Model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    if model is None:
        try:
            with open("/proc/cpuinfo") as fh:
                for line in fh:
                    if line.lower().startswith(("model name", "cpu model")):
                        model = line.split(":", 1)[1].strip()
                        break
        except OSError:
            pass
    import platform
    return {"cpu_model": model or platform.machine(), "nproc": os.cpu_count()}


CORES_NOTE = ("the oracle runs on one core: its block-CSR product (scipy.sparse) and its per-cell dense solves "
              "(numpy) are single-threaded, and it is timed as it stands, with BLAS threads pinned to 1")


def cpu_baseline_subprocess(n=CPU_SAMPLE["n"]):
    """The cpu_baseline object of the GPU line: one oracle solve."""
    samples, desc, parts = oracle_subprocess(1, n)
    host = host_cpu()
    if samples is None:
        return {"value": None, "unit": "GDOF/s", "cores": 1, "kind": "oracle", "sample": desc, **host,
                "cores_note": CORES_NOTE}
    return {"value": round(samples[0][0] / 1e9, 9), "unit": "GDOF/s", "cores": 1, "kind": "oracle",
            "sample": desc, "seconds": round(samples[0][1], 2), **parts, **host, "cores_note": CORES_NOTE}


def run_reference(args):
    """The oracle as the reference arm: one process sets the sample up once,
    then runs W untimed and K timed solves of it; each step is one solve."""
    steps = max(1, args.steps)
    warm = max(0, args.warmup)
    samples, desc, parts = oracle_subprocess(warm + steps, args.oracle_cells)
    if samples is None:
        return {"impl": "reference", "unavailable": desc}
    timed = samples[warm:]
    secs = sum(t for _, t in timed)
    sample_dofs = args.oracle_cells ** 3 * (CPU_SAMPLE["p"] + 1) ** 3
    v = round(sample_dofs * len(timed) / secs / 1e9, 9)       # dofs solved / solve time
    return {"impl": "reference", "metric": METRIC, "value": v, "unit": "GDOF/s", "n_gpus": 1,
            "steps": steps, "warmup": warm, "ms_per_step": round(secs / steps * 1e3, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(),
            "cpu_baseline": {"value": v, "unit": "GDOF/s", "cores": 1, "kind": "oracle", "sample": desc, **parts,
                             **host_cpu(), "cores_note": CORES_NOTE},
            "e2e": {"value": v, "unit": "GDOF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="dgmg", choices=["dgmg", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-baseline-worker", action="store_true")
    ap.add_argument("--worker-repeats", type=int, default=1)
    ap.add_argument("--oracle-cells", type=int, default=CPU_SAMPLE["n"],
                    help="cells per direction of the oracle sample (reference arm and cpu_baseline)")
    args = ap.parse_args()

    if args.cpu_baseline_worker:
        samples, desc, parts = oracle_solve_sample(args.worker_repeats, args.oracle_cells)
        print(json.dumps({"samples": samples, "desc": desc, "parts": parts}))
        return

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(run_reference(args)), flush=True)
        return
    if args.warmup < 3:
        args.warmup = 3
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    out = run_dgmg(args, rank, world, local_rank)
    if rank == 0:
        if world == 1 and not args.no_cpu_baseline:
            out["cpu_baseline"] = cpu_baseline_subprocess(args.oracle_cells)
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
