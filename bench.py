"""Benchmark: Newton linearise-and-solve steps per second of the in-situ-combustion
model on the 60x60x20 field workload (72,000 cells, 8 unknowns per cell).

One step = the whole hot path on one batch: restore the iterate, property
evaluation + residual/Jacobian assembly, convergence norms, Gauss-Jordan
decoupling, block ILU(0) factorisation, GMRES(30) to the relative tolerance,
safeguarded update. Inputs are resident in HBM for ``value``; ``e2e`` goes
through the C ABI with host buffers (state in, state out) every step. The
line also carries the same step with the FP32 preconditioner (``mixed``), with
an FP32 inner GMRES inside the flexible FP64 GMRES (``mixed_fgmres``, with the
FP32 SpMV's roofline), the discrete adjoint of a 40x40x10 time loop
(``adjoint``) and the step with the CPR-PF preconditioner (``cpr``, FP64 and
mixed).

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl isc|reference]
Under torchrun each rank runs an independent replica (the path has no
data-path exchange on one GPU per problem); value sums all ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Newton steps/s"
UNIT = "Newton steps/s"
FIELD = dict(nx=60, ny=60, nz=20)
# algorithmic bytes per unit: one FP64 8x8 block = 512 B + 4 B column index
BLOCK_BYTES = 516


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="isc", choices=["isc", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true", help="skip the discrete-adjoint measurement")
    ap.add_argument("--no-extras", action="store_true",
                    help="time only the headline step (no mixed, CPR-PF, adjoint or end-to-end legs); for profiling")
    ap.add_argument("--grid", default=None,
                    help="NXxNYxNZ: run the same field recipe on a smaller grid (profiling captures)")
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed", "mixed_fgmres"],
                    help="precision of the timed step's linear solve (the headline is fp64)")
    ap.add_argument("--workload", default="field", choices=["field", "mixed", "large"],
                    help="field: 60x60x20 (the headline); mixed: 100x100x30; large: 200x200x50, 3 facies, 5-spot")
    return ap.parse_args()


def max_over_ranks(x, device="cpu"):
    """Largest value of x over the ranks of the default process group (x itself
    without one): the whole job is as slow as its slowest replica."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world, steps, ms_max):
    """Whole-job Newton steps per second: every rank ran `steps` steps."""
    return world * steps / (ms_max / 1e3)


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.t.join(timeout=2)
        sm, mx, reasons = [], None, set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def field_case(grid=None, workload="field"):
    import isc_inputs as inp
    if grid:
        nx, ny, nz = (int(v) for v in grid.lower().split("x"))
        return inp.field_case(nx, ny, nz, 0, 1, f"field {nx}x{ny}x{nz}", 30 * inp.DAY, 40)
    return inp.config({"field": 2, "mixed": 3, "large": 5}[workload])


def l2_bytes():
    try:
        import torch
        return int(torch.cuda.get_device_properties(torch.cuda.current_device()).L2_cache_size)
    except Exception:
        return 126 * 2**20


def workload_config(case, dt, extra, nnzb=None):
    nnzb = nnzb if nnzb is not None else case.n * 7
    c = {"workload": f"{case.name} ({case.n} cells, 8 unknowns/cell), first Newton step of "
                     f"the first time step (dt {dt:.0f} s) from the ignited initial state",
         "solver": "GMRES(30), block ILU(0), Gauss-Jordan decoupling, FP64, tol_lin 1e-6",
         "l2": f"inputs larger than L2: the FP64 Jacobian ({nnzb * 512 / 1e6:.0f} MB) and staged properties "
               f"({case.n * 16 * 9 * 8 / 1e6:.0f} MB) exceed the {l2_bytes() / 2**20:.0f} MiB L2"}
    c.update(extra)
    return c


def run_isc(args):
    import numpy as np
    import torch

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    from paper_1811_11992_gb300 import build, isc
    build.build()
    case = field_case(args.grid, args.workload)
    dt = case.dt0
    g = isc.Simulator(case, profile=1, precision=args.precision, inner_its=INNER_ITS)
    g.init_equilibrium()
    n = case.n
    # resident snapshot of the starting iterate (torch owns the buffers)
    u0 = torch.empty(8 * n, dtype=torch.float64, device="cuda")
    c0 = torch.empty(n, dtype=torch.float64, device="cuda")
    g.get_state_device(u0.data_ptr(), c0.data_ptr())
    torch.cuda.synchronize()

    def step():
        g.set_state_device(u0.data_ptr(), c0.data_ptr())
        return g.newton_step(dt)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    g.reset_stats()
    infos = []
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    t0 = time.perf_counter()
    ev0.record()
    for _ in range(args.steps):
        infos.append(step())
    ev1.record()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    wall = time.perf_counter() - t0
    ms_dev = ev0.elapsed_time(ev1)
    stats = g.stats()
    clocks = sampler.stop()
    ms_total = max_over_ranks(max(ms_dev, wall * 1e3), "cuda")
    value = job_throughput(world, args.steps, ms_total)
    kry = [i.krylov_iterations for i in infos]
    e2e = mixed = mixed_fgmres = cpr_block = None
    mst = fst = None
    if not args.no_extras:
        # end-to-end through the C ABI with host buffers
        uh, ch = g.get_state()
        u_host = torch.from_numpy(uh.reshape(-1).copy()).pin_memory().numpy()
        c_host = torch.from_numpy(ch.copy()).pin_memory().numpy()
        g.set_state_device(u0.data_ptr(), c0.data_ptr())
        u_start, c_start = g.get_state()
        u_start_p = torch.from_numpy(u_start.reshape(-1).copy()).pin_memory().numpy()
        c_start_p = torch.from_numpy(c_start.copy()).pin_memory().numpy()
        for _ in range(max(1, args.warmup // 2)):
            g.set_state(u_start_p.reshape(8, n), c_start_p)
            g.newton_step(dt)
            g.get_state()
        e2e_steps = max(3, args.steps // 2)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            g.set_state(u_start_p.reshape(8, n), c_start_p)
            g.newton_step(dt)
            u_out, c_out = g.get_state()
        torch.cuda.synchronize()
        e2e_s = time.perf_counter() - t0
        e2e_val = job_throughput(world, e2e_steps, max_over_ranks(e2e_s * 1e3, "cuda"))
        io_bytes = 9 * n * 8
        e2e = {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": io_bytes, "d2h_bytes_per_step": io_bytes}
        solve_fp64 = sum(stats[k]["ms"] for k in SOLVE_CLASSES) / args.steps

        def precision_leg(precision, **extra):
            """The headline step again under another precision of the linear solve."""
            g.set_options(precision=precision, **extra)
            for _ in range(max(1, args.warmup)):
                step()
            torch.cuda.synchronize()
            g.reset_stats()
            ev0.record()
            minfo = [step() for _ in range(args.steps)]
            ev1.record()
            torch.cuda.synchronize()
            ms_leg = ev0.elapsed_time(ev1) / args.steps
            mstats = g.stats()
            g.set_options(precision="fp64")
            solve_leg = sum(mstats[k]["ms"] for k in SOLVE_CLASSES) / args.steps
            return mstats, {
                "value": 1e3 / ms_leg, "unit": UNIT, "ms_per_step": ms_leg,
                "krylov_iterations_per_step": statistics.median([i.krylov_iterations for i in minfo]),
                "rel_residual": max(i.krylov_rel_residual for i in minfo),
                "prec_apply_ms_per_call": mstats["prec_apply"]["ms"] / max(1, mstats["prec_apply"]["calls"]),
                "solve_ms_fp64": solve_fp64, "solve_ms": solve_leg,
                "solve_speedup_vs_fp64": solve_fp64 / solve_leg if solve_leg > 0 else None}

        # mixed precision on the same step: FP32 ILU(0) factors and sweeps inside the FP64 GMRES
        mst, mixed = precision_leg("mixed")
        # FP32 inner GMRES (FP32 SpMV, Gram-Schmidt and ILU(0)) inside the flexible FP64 GMRES
        fst, mixed_fgmres = precision_leg("mixed_fgmres", inner_its=INNER_ITS)
        mixed_fgmres["inner_its"] = INNER_ITS
        mixed_fgmres["inner_iterations_per_step"] = mixed_fgmres["krylov_iterations_per_step"] * INNER_ITS
        mixed_fgmres["roofline_spmv32"] = spmv32_roofline(fst, case, g.nnzb)
        # CPR-PF (the paper's Example-2 preconditioner) on the same step, FP64 and mixed
        cpr_block = {}
        for precision in ("fp64", "mixed"):
            g.set_options(prec="cpr", precision=precision)
            for _ in range(max(1, args.warmup)):
                step()
            torch.cuda.synchronize()
            g.reset_stats()
            ev0.record()
            cinfo = [step() for _ in range(args.steps)]
            ev1.record()
            torch.cuda.synchronize()
            ms_c = ev0.elapsed_time(ev1) / args.steps
            cst = g.stats()
            cpr_block[precision] = {
                "value": 1e3 / ms_c, "unit": UNIT, "ms_per_step": ms_c,
                "krylov_iterations_per_step": statistics.median([i.krylov_iterations for i in cinfo]),
                "rel_residual": max(i.krylov_rel_residual for i in cinfo),
                "pressure_stage_ms_per_step": cst["cpr"]["ms"] / args.steps,
                "ilu_stage_ms_per_step": cst["prec_apply"]["ms"] / args.steps,
                "speedup_vs_ilu0_fp64": ms_total / args.steps / ms_c}
        g.set_options(prec="bilu0", precision="fp64")
    # roofline of the dominant kernel class
    launches = sum(v["launches"] for v in stats.values())
    dom = max(stats, key=lambda k: stats[k]["ms"])
    roof = roofline(dom, stats, g, case, kry, args.precision)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_total / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f64+f32",
        "data": "synthetic",
        "config": workload_config(case, dt, {"parallelism": f"replicas x{world}",
                                             "krylov_iterations_per_step": statistics.median(kry) if kry else None,
                                             "precision": args.precision},
                                  g.nnzb),
        "e2e": e2e,
        "gpu_launches": launches,
        "kernel_ms": {k: round(v["ms"], 3) for k, v in stats.items()},
        "kernel_launches": {k: v["launches"] for k, v in stats.items()},
        "roofline": roof,
        "hbm": hbm_table(stats, mst, fst, case, g.nnzb),
        "clocks": clocks,
        "mixed": mixed,
        "mixed_fgmres": mixed_fgmres,
        "cpr": cpr_block,
    }
    if not args.no_adjoint and not args.no_extras and args.grid is None and args.workload == "field":
        line["adjoint"] = adjoint_block()
    if rank == 0 and world == 1 and not args.no_cpu_baseline and args.workload == "field" and args.grid is None:
        line["cpu_baseline"] = cpu_baseline(max_seconds=30.0)
    g.close()
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()


def adjoint_block():
    """The discrete adjoint on the 40x40x10 workload (20 frozen steps, states
    checkpointed every 5): wall time of the loss alone and of loss + gradient
    (forward sweep, recomputation, 20 transposed solves), CUDA-event time of
    the adjoint kernels."""
    import isc_inputs as inp
    from paper_1811_11992_gb300 import isc
    case = inp.config(4)
    dts = inp.adjoint_steps(case)
    g = isc.Simulator(case, tol_newton=1e-9, tol_lin=1e-6, maxit_newton=40, maxit_lin=3000, profile=1)
    g.init_equilibrium()
    g.adjoint(dts, checkpoint_every=5, tol_adjoint=1e-10)      # warm-up (allocates the checkpoint store)
    g.init_equilibrium()
    t0 = time.perf_counter()
    L_only = g.adjoint(dts, checkpoint_every=5, gradient=False)[0]
    t_fwd = time.perf_counter() - t0
    g.init_equilibrium()
    g.reset_stats()
    t0 = time.perf_counter()
    L, gk, ge, ga, info = g.adjoint(dts, checkpoint_every=5, tol_adjoint=1e-10)
    t_grad = time.perf_counter() - t0
    st = g.stats()
    g.close()
    return {"workload": f"adjoint {case.nx}x{case.ny}x{case.nz} ({case.n} cells), {len(dts)} frozen steps "
                        f"({sum(dts) / inp.DAY:.1f} d), checkpoints every 5, gradient w.r.t. {case.n} ln k + "
                        f"{2 * int(case.reactions['nr'])} reaction parameters",
            "loss_kg": L, "loss_only_s": t_fwd, "loss_and_gradient_s": t_grad,
            "gradient_cost_ratio": t_grad / t_fwd, "same_loss": L == L_only,
            "newton_iterations": info["newton_iterations"], "recomputed_steps": info["recomputed_steps"],
            "krylov_iterations_forward": info["krylov_iterations_forward"],
            "krylov_iterations_adjoint": info["krylov_iterations_adjoint"],
            "adjoint_rel_residual": info["adjoint_rel_residual"],
            "kernel_ms": {k: round(v["ms"], 3) for k, v in st.items()}}


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


FP64_PEAK_GFLOPS = 1200.0   # measured DFMA throughput on this GB300
# dram__bytes_read.sum + dram__bytes_write.sum per call (forward + backward FP64 sweep)
MEASURED_TRAFFIC = {("prec_apply", 60, 60, 20): (313.40e6, "profiles/k_ilu_sweeps_field_60x60x20.md")}


SOLVE_CLASSES = ("spmv", "spmv32", "prec_apply", "blas1", "ilu_factor")
INNER_ITS = 10


def spmv32_roofline(stats, case, nnzb):
    """The inner solve's FP32 SpMV: FP32 off-diagonal blocks and their column
    indices, x read twice (neighbours and the unit diagonal) and y written."""
    peaks = measured_peaks()
    hbm = peaks.get("hbm_gbs", 6800.0)
    s = stats["spmv32"]
    calls = max(1, s["calls"])
    ms = s["ms"] / calls
    byts = (nnzb - case.n) * (256 + 4) + 3 * case.n * 32
    ach = byts / (ms * 1e-3) / 1e9 if ms > 0 else 0.0
    return {"kernel": "k_spmv<float>", "bound": "hbm", "calls": calls, "ms_per_call": ms, "bytes_per_call": byts,
            "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm, "peak_source": "MEASURED_PEAKS.json hbm_gbs"}


def class_gbs(stats, cls, byts):
    """Algorithmic bytes per call of one kernel class over its mean CUDA-event time."""
    hbm = measured_peaks().get("hbm_gbs", 6800.0)
    s = stats.get(cls, {"calls": 0, "ms": 0.0})
    if not s["calls"] or s["ms"] <= 0:
        return None
    ms = s["ms"] / s["calls"]
    gbs = byts / (ms * 1e-3) / 1e9
    return {"ms_per_call": ms, "bytes_per_call": byts, "gbs": gbs, "hbm_frac": gbs / hbm}


def hbm_table(stats64, stats_mixed, stats_fg, case, nnzb):
    """SpMV and preconditioner-apply GB/s against the measured HBM bandwidth (the
    metric's second part): FP64 from the headline step, the FP32 sweeps from the
    `mixed` leg, the FP32 SpMV from the `mixed_fgmres` leg."""
    n, off = case.n, nnzb - case.n
    out = {"spmv_fp64": class_gbs(stats64, "spmv", off * BLOCK_BYTES + 3 * n * 64),
           "ilu_apply_fp64": class_gbs(stats64, "prec_apply", off * BLOCK_BYTES + 2 * n * 512 + 4 * n * 64)}
    if stats_mixed is not None:
        out["ilu_apply_fp32"] = class_gbs(stats_mixed, "prec_apply", off * 260 + 2 * n * 256 + 2 * n * 64 + 2 * n * 32)
    if stats_fg is not None:
        out["spmv_fp32"] = class_gbs(stats_fg, "spmv32", off * 260 + 3 * n * 32)
    return out


def roofline(dom, stats, g, case, kry, precision="fp64"):
    """Algorithmic bytes (or flops) per call of the dominant kernel class over its
    average CUDA-event duration."""
    n, nnzb = case.n, g.nnzb
    peaks = measured_peaks()
    hbm = peaks.get("hbm_gbs", 6800.0)
    s = stats[dom]
    calls = max(1, s["calls"])
    ms = s["ms"] / calls
    nlev = case.nx + case.ny + case.nz - 2
    nlow = nnzb - n  # off-diagonal blocks (both triangles)
    if dom == "spmv":
        byts = (nnzb - n) * BLOCK_BYTES + 3 * n * 64
        flops = 2 * 64 * (nnzb - n)
    elif dom == "prec_apply":
        byts = nlow * BLOCK_BYTES + 2 * n * 512 + 4 * n * 64
        flops = 2 * 64 * (nlow + 2 * n)
    elif dom == "ilu_factor":
        byts = (nlow // 2) * 2 * BLOCK_BYTES + 2 * n * 512
        flops = (nlow // 2) * 2 * 2 * 512 + n * 2 * 512 * 2
    elif dom == "gj":
        byts = 2 * (nnzb * BLOCK_BYTES + n * 64)
        flops = n * 8 * 7 * 2 * 57
    elif dom in ("props", "flux"):
        byts = nnzb * 512 + n * (8 + 8 + 7 + 3) * 8
        flops = None
    else:
        byts = 0
        flops = None
    ach_gbs = byts / (ms * 1e-3) / 1e9 if ms > 0 else 0.0
    out = {"kernel": dom, "calls": calls, "ms_per_call": ms, "bytes_per_call": byts}
    if flops is not None and ms > 0:
        ach_tf = flops / (ms * 1e-3) / 1e9
        # FP64 kernels on GB300 sit above the FP64 ridge (1.2 TFLOP/s / 6.8 TB/s = 0.18 flop/B)
        if flops / max(byts, 1) > FP64_PEAK_GFLOPS / hbm:
            out.update(bound="alu", achieved=ach_tf, peak=FP64_PEAK_GFLOPS, unit="GFLOP/s",
                       frac=ach_tf / FP64_PEAK_GFLOPS, peak_source="measured FP64 DFMA probe",
                       hbm_achieved_gbs=ach_gbs, hbm_frac=ach_gbs / hbm)
        else:
            out.update(bound="hbm", achieved=ach_gbs, peak=hbm, unit="GB/s", frac=ach_gbs / hbm,
                       peak_source="MEASURED_PEAKS.json hbm_gbs")
    else:
        out.update(bound="hbm", achieved=ach_gbs, peak=hbm, unit="GB/s", frac=ach_gbs / hbm if hbm else None,
                   peak_source="MEASURED_PEAKS.json hbm_gbs")
    # DRAM bytes per call from one ncu capture of the current kernels on this grid (FP64 solve)
    measured = MEASURED_TRAFFIC.get((dom, case.nx, case.ny, case.nz)) if precision == "fp64" else None
    out["traffic"] = measured[0] if measured else None
    if precision != "fp64":
        out["note"] = "bytes and flops of the FP64 operands; this step ran its preconditioner in FP32"
    if measured:
        out["traffic_source"] = measured[1]
    return out


# ------------------------------------------------------------------ oracle
SAMPLE = dict(nx=30, ny=30, nz=10)


def oracle_sample_step():
    """One oracle Newton step on a 30x30x10 block cut to the field workload's
    recipe (same generator, 1/8 of the cells)."""
    import isc_inputs as inp
    from oracle import model, sim
    case = inp.field_case(SAMPLE["nx"], SAMPLE["ny"], SAMPLE["nz"], 0, 1, "field sample 30x30x10", 30 * inp.DAY, 40)
    u, c = sim.initial_state(case)
    acc_old = model.old_accumulation(case, u, c)
    opts = sim.NewtonOptions(tol=0.0)
    opts.solve.rtol = 1e-6
    t0 = time.perf_counter()
    r = sim.newton_step(case, u, c, acc_old, case.dt0, opts)
    return time.perf_counter() - t0, case.n, r


def cpu_baseline(max_seconds=30.0):
    full = FIELD["nx"] * FIELD["ny"] * FIELD["nz"]
    secs = []
    t_start = time.perf_counter()
    while True:
        dt, ncell, _ = oracle_sample_step()
        secs.append(dt)
        if time.perf_counter() - t_start + dt > max_seconds or len(secs) >= 3:
            break
    per = statistics.median(secs)
    scale = ncell / full
    return {"value": scale / per, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{len(secs)} oracle Newton step(s) on a 30x30x10 block of the field recipe "
                      f"({ncell} cells, {per:.2f} s each), scaled by cell count to the 72,000-cell workload"}


def run_reference(args):
    rank, world, local = dist_env()
    if rank != 0:
        return
    for _ in range(args.warmup):
        oracle_sample_step()
    full = FIELD["nx"] * FIELD["ny"] * FIELD["nz"]
    t0 = time.perf_counter()
    ncell = None
    for _ in range(args.steps):
        _, ncell, _ = oracle_sample_step()
    wall = time.perf_counter() - t0
    per = wall / args.steps
    value = (ncell / full) / per
    case = field_case()
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": per * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f64+f32",
        "data": "synthetic",
        "config": workload_config(case, case.dt0, {"parallelism": "host oracle, 1 thread"}),
        "cpu_baseline": {"value": value, "unit": UNIT, "kind": "oracle", "cores": 1,
                         "sample": f"one oracle Newton step per timed step on a 30x30x10 block ({ncell} cells), "
                                   f"scaled by cell count to the 72,000-cell workload"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


if __name__ == "__main__":
    a = parse()
    if a.impl == "reference":
        run_reference(a)
    else:
        run_isc(a)
