"""Benchmark: Newton linearise-and-solve steps per second of the in-situ-combustion
model on the large workload (200x200x50 = 2,000,000 cells, 16M unknowns, 3-facies
permeability, 5-spot wells), with the SpMV and ILU(0)-apply bandwidth against the
HBM roof and the FP64 against the mixed-precision time to a 1e-6 relative linear
residual.

One step = the whole hot path on one batch: restore the iterate, property
evaluation + residual/Jacobian assembly, convergence norms, Gauss-Jordan
decoupling, block ILU(0) factorisation, GMRES(30) to the relative tolerance,
safeguarded update. Inputs are resident in HBM for ``value``; ``e2e`` goes
through the C ABI with host buffers (state in, state out) every step. The line
also carries the same step with the FP32 preconditioner (``mixed``), with an
FP32 inner GMRES inside the flexible FP64 GMRES (``mixed_fgmres``), with the
CPR-PF preconditioner (``cpr``), the 100x100x30 and 60x60x20 workloads
(``workloads``), the discrete adjoint of a 40x40x10 time loop (``adjoint``) and
the oracle's timing on the host (``cpu_baseline``).

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
WORKLOADS = {"field": 2, "mixed": 3, "large": 5}
# algorithmic bytes: one FP64 8x8 block = 512 B + its 4-byte column index; FP32 256 + 4
BLOCK_BYTES = 516
BLOCK_BYTES32 = 260
SOLVE_CLASSES = ("spmv", "spmv32", "prec_apply", "blas1", "ilu_factor")
INNER_ITS = 10


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="isc", choices=["isc", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-fullsize", action="store_true",
                    help="also time the oracle's SpMV and ILU(0) apply on the full-size matrix (about 2 min and "
                         "40 GB of host memory at 200x200x50; skipped with a note when less memory is free)")
    ap.add_argument("--no-adjoint", action="store_true", help="skip the discrete-adjoint measurement")
    ap.add_argument("--no-extras", action="store_true",
                    help="time only the headline step (no other legs or workloads); for profiling")
    ap.add_argument("--grid", default=None,
                    help="NXxNYxNZ: run the workload's recipe on another grid (profiling captures)")
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed", "mixed_fgmres"],
                    help="precision of the timed step's linear solve (the headline is fp64)")
    ap.add_argument("--prec", default="bilu0", choices=["bilu0", "cpr"],
                    help="preconditioner of the timed step (the headline is block ILU(0))")
    ap.add_argument("--orth", default="cgs1", choices=["cgs2", "cgs1"],
                    help="orthogonalisation of the FP64 GMRES (the headline: classical Gram-Schmidt once)")
    ap.add_argument("--workload", default="large", choices=sorted(WORKLOADS),
                    help="large: 200x200x50 (the headline); mixed: 100x100x30; field: 60x60x20")
    return ap.parse_args(argv)


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


def workload_case(workload="large", grid=None):
    import isc_inputs as inp
    if grid:
        nx, ny, nz = (int(v) for v in grid.lower().split("x"))
        if workload == "large":
            return inp.large_case(nx, ny, nz)
        return inp.field_case(nx, ny, nz, 0, 1, f"field {nx}x{ny}x{nz}", 30 * inp.DAY, 40)
    return inp.config(WORKLOADS[workload])


def l2_bytes():
    try:
        import torch
        return int(torch.cuda.get_device_properties(torch.cuda.current_device()).L2_cache_size)
    except Exception:
        return 126 * 2**20


def workload_config(case, world, precision="fp64", prec="bilu0", orth="cgs1"):
    """The `config` object of the line: the workload and solver only (measured
    numbers go elsewhere), identical for the library and the reference arm."""
    nnzb = case.n + 2 * ((case.nx - 1) * case.ny * case.nz + case.nx * (case.ny - 1) * case.nz
                         + case.nx * case.ny * (case.nz - 1))
    pname = {"bilu0": "block ILU(0)", "cpr": "CPR-PF"}[prec]
    oname = {"cgs2": "classical Gram-Schmidt twice", "cgs1": "classical Gram-Schmidt once"}[orth]
    return {"workload": f"{case.name} ({case.n} cells, 8 unknowns/cell), first Newton step of the first time step "
                        f"(dt {case.dt0:.0f} s) from the ignited initial state",
            "solver": f"GMRES(30) ({oname}), {pname}, Gauss-Jordan decoupling, tol_lin 1e-6",
            "precision": precision,
            "l2": f"inputs larger than L2, no flush: the FP64 Jacobian ({nnzb * 512 / 1e6:.0f} MB) and staged "
                  f"properties ({case.n * 16 * 9 * 8 / 1e6:.0f} MB) exceed the {l2_bytes() / 2**20:.0f} MiB L2",
            "parallelism": f"replicas x{world}"}


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


def hbm_peak():
    return measured_peaks().get("hbm_gbs", 6800.0)


# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one call of a kernel
# class, per cell, from one ncu capture of the current kernels on a smaller grid
# of the same recipe; a call's traffic grows with the cells it sweeps, so the
# full-size figure is this times the workload's cells. Keyed by (class, precision,
# sweep layout): grids with few pencils run the one-pencil-per-warp sweeps.
MEASURED_TRAFFIC = {
    ("prec_apply", "fp64", "pair"): (1245.53e6 / 320000, "large 40x160x50",
                                     "profiles/k_sweep_fwd_bwd_large_40x160x50.md"),
    ("prec_apply", "mixed", "pair"): (648.48e6 / 320000, "large 40x160x50",
                                      "profiles/k_sweep_fwd_bwd_large_40x160x50.md"),
    ("prec_apply", "fp64", "single"): (313.37e6 / 72000, "field 60x60x20",
                                       "profiles/k_sweep1_fwd_bwd_field_60x60x20.md"),
    ("prec_apply", "mixed", "single"): (157.89e6 / 72000, "field 60x60x20",
                                        "profiles/k_sweep1_fwd_bwd_field_60x60x20.md"),
    # the SpMV has one layout (its figure holds for either sweep layout)
    ("spmv", "fp64", None): ((222.2e6 + 5.7e6) / 72000, "field 60x60x20", "profiles/k_spmv8_field_60x60x20.md"),
    ("spmv32", "mixed", None): ((112.09e6 + 3.26e6) / 72000, "field 60x60x20",
                                "profiles/k_spmv_f32_field_60x60x20.md"),
}


def measured_traffic(cls, precision, case):
    """(bytes per cell, workload, source) of the class's ncu DRAM traffic, or None."""
    p = "fp64" if precision == "fp64" else "mixed"
    return MEASURED_TRAFFIC.get((cls, p, sweep_layout(case, precision))) or MEASURED_TRAFFIC.get((cls, p, None))
# the largest ny * nz that runs the one-pencil-per-warp sweeps (SWEEP1_MAX_PENCILS64 /
# SWEEP1_MAX_PENCILS32 of the library's ILU(0) sweeps)
SWEEP1_MAX_PENCILS = {"fp64": 3000, "mixed": 3600}


def sweep_layout(case, precision):
    key = "fp64" if precision == "fp64" else "mixed"
    return "single" if case.ny * case.nz <= SWEEP1_MAX_PENCILS[key] else "pair"


def class_gbs(stats, cls, byts):
    """Algorithmic bytes per call of one kernel class over its mean CUDA-event time."""
    hbm = hbm_peak()
    s = stats.get(cls, {"calls": 0, "ms": 0.0})
    if not s["calls"] or s["ms"] <= 0:
        return None
    ms = s["ms"] / s["calls"]
    gbs = byts / (ms * 1e-3) / 1e9
    return {"ms_per_call": ms, "bytes_per_call": byts, "gbs": gbs, "hbm_frac": gbs / hbm}


def spmv_bytes(n, nnzb, fp32=False):
    """Off-diagonal blocks with their column indices (the decoupled diagonal is
    the identity and is not read), x for the neighbours and the diagonal, y."""
    if fp32:
        return (nnzb - n) * BLOCK_BYTES32 + 3 * n * 32
    return (nnzb - n) * BLOCK_BYTES + 3 * n * 64


def ilu_apply_bytes(n, nnzb, fp32=False):
    """Block ILU(0) apply, forward then backward substitution: every off-diagonal
    block with its column index once, the N inverted diagonal blocks once, and
    four vector passes (r in, the intermediate written and read back, z out;
    FP32 vectors inside the FP32 sweeps, FP64 r and z at the boundary)."""
    if fp32:
        return (nnzb - n) * BLOCK_BYTES32 + n * 256 + 2 * n * 64 + 2 * n * 32
    return (nnzb - n) * BLOCK_BYTES + n * 512 + 4 * n * 64


def ilu_apply_flops(n, nnzb):
    """Two flops per multiply-add of every off-diagonal block and one diagonal
    inverse per cell."""
    return 2 * 64 * (nnzb - n) + 2 * 64 * n


def hbm_table(stats64, stats_mixed, stats_fg, case, nnzb):
    """SpMV and preconditioner-apply GB/s against the measured HBM bandwidth (the
    metric's second part): FP64 from the headline step, the FP32 sweeps from the
    `mixed` leg, the FP32 SpMV from the `mixed_fgmres` leg."""
    n = case.n
    out = {"spmv_fp64": class_gbs(stats64, "spmv", spmv_bytes(n, nnzb)),
           "ilu_apply_fp64": class_gbs(stats64, "prec_apply", ilu_apply_bytes(n, nnzb))}
    if stats_mixed is not None:
        out["ilu_apply_fp32"] = class_gbs(stats_mixed, "prec_apply", ilu_apply_bytes(n, nnzb, fp32=True))
    if stats_fg is not None:
        out["spmv_fp32"] = class_gbs(stats_fg, "spmv32", spmv_bytes(n, nnzb, fp32=True))
    return out


def gmres_blas1_work(n, its, restart=30, orth="cgs1"):
    """Algorithmic bytes and flops of the Gram-Schmidt passes of `its` GMRES(m)
    iterations on vectors of 8n doubles. Classical Gram-Schmidt applied twice:
    iteration j of a cycle orthogonalises w against k = j + 1 basis vectors in
    three passes (V^T w; w -= V h0 with V^T w; w -= V h1 with ||w||^2), each
    reading the k vectors and w (the last two writing w), then scales w into the
    next basis vector: 8 * len * (3k + 7) bytes and len * (8k + 2) flops. Once:
    two passes (V^T w; w -= V h0 with ||w||^2) and the scaling, 8 * len *
    (2k + 5) bytes and len * (4k + 2) flops."""
    ln = 8 * n
    byts = flops = 0
    for it in range(int(its)):
        k = it % restart + 1
        if orth == "cgs1":
            byts += 8 * ln * (2 * k + 5)
            flops += ln * (4 * k + 2)
        else:
            byts += 8 * ln * (3 * k + 7)
            flops += ln * (8 * k + 2)
    return byts, flops


# Executed FP64 flops per cell of the assembly kernels (2 DFMA + DADD + DMUL from an
# ncu count of the dual-number tangent code, which has no closed-form flop count),
# profiles/fp64_instruction_counts_large_100x100x30.md
ASSEMBLY_FLOPS_PER_CELL = {"props": 5810.0, "flux": 3742.0 + 434.0}  # flux: face pass + gather


def class_model(cls, n, nnzb, fp32=False, its=None, orth="cgs1"):
    """(algorithmic bytes, flops) per call of a kernel class (None when unmodelled)."""
    if cls == "props":
        # reads u (64 B), the old accumulation (56 B), C_c^n and phi_ref (16 B); writes R (64 B),
        # the diagonal block (512 B) and the staged face quantities (16 x 9 doubles)
        return n * (64 + 56 + 16 + 64 + 512 + 16 * 9 * 8), n * ASSEMBLY_FLOPS_PER_CELL["props"]
    if cls == "flux":
        # face pass: reads the staged quantities (each cell's once from DRAM) and the
        # transmissibilities, writes the off-diagonal blocks, parks the face fluxes (3 x 7
        # doubles per cell); gather: reads the fluxes and rows 0..6 of the off-diagonal blocks
        # back, adds to R and the diagonal block
        return (n * (16 * 9 * 8 + 3 * 8) + (nnzb - n) * (512 + 448) + 2 * n * 3 * 7 * 8 + n * (64 + 512) * 2,
                n * ASSEMBLY_FLOPS_PER_CELL["flux"])
    if cls == "spmv":
        return spmv_bytes(n, nnzb), 2 * 64 * (nnzb - n)
    if cls == "prec_apply":
        return ilu_apply_bytes(n, nnzb, fp32), ilu_apply_flops(n, nnzb)
    if cls == "ilu_factor":
        # per cell three lower and three upper blocks read, D^-1 and the three
        # pre-scaled upper blocks written; three products D_k^-1 A_ki and A_ik (.),
        # one 8x8 inversion
        return (nnzb - n) * BLOCK_BYTES + n * 512 + (nnzb - n) // 2 * 512, n * (3 * 2 * 2 * 512 + 2 * 512)
    if cls == "gj":
        return 2 * (nnzb * BLOCK_BYTES + n * 64), n * 8 * 7 * 2 * 57
    if cls == "blas1" and its:
        return gmres_blas1_work(n, its, orth=orth)
    return None, None


def roofline(dom, stats, case, nnzb, fp64_gflops, precision="fp64", its=None, orth="cgs1"):
    """Algorithmic bytes (or flops) per call of a kernel class over its average
    CUDA-event duration, against the measured HBM copy bandwidth or the FP64 FMA
    rate measured at start-up (whichever bounds the class: FP64 work above the
    ridge fp64_gflops / hbm flop per byte is bound by the FP64 pipe). For the
    Gram-Schmidt class (blas1) the per-call figures are the step's totals over
    its calls (its: Krylov iterations of the timed steps)."""
    n = case.n
    hbm = hbm_peak()
    s = stats[dom]
    calls = max(1, s["calls"])
    ms = s["ms"] / calls
    fp32 = precision != "fp64"
    byts, flops = class_model(dom, n, nnzb, fp32, its, orth)
    if dom == "blas1" and byts:
        byts, flops = byts / calls, flops / calls
    out = {"kernel": dom, "calls": calls, "ms_per_call": ms, "bytes_per_call": byts, "flops_per_call": flops}
    if byts is None:
        out.update(bound=None, achieved=None, peak=None, unit=None, frac=None, traffic=None)
        return out
    ach_gbs = byts / (ms * 1e-3) / 1e9 if ms > 0 else 0.0
    if flops is not None and ms > 0 and not fp32 and flops / max(byts, 1) > fp64_gflops / hbm:
        ach = flops / (ms * 1e-3) / 1e9
        out.update(bound="alu", achieved=ach, peak=fp64_gflops, unit="GFLOP/s", frac=ach / fp64_gflops,
                   peak_source="FP64 FMA rate measured at start-up (isc_measure_fma_rates)",
                   hbm_achieved_gbs=ach_gbs, hbm_frac=ach_gbs / hbm)
    else:
        out.update(bound="hbm", achieved=ach_gbs, peak=hbm, unit="GB/s", frac=ach_gbs / hbm,
                   peak_source="MEASURED_PEAKS.json hbm_gbs")
    m = measured_traffic(dom, precision, case)
    out["traffic"] = m[0] * n if m else None
    if m:
        out["traffic_source"] = f"{m[2]} (captured on {m[1]}, scaled per cell to {case.n} cells)"
    return out


def spmv32_roofline(stats, case, nnzb):
    """The inner solve's FP32 SpMV against the HBM roof."""
    hbm = hbm_peak()
    s = stats["spmv32"]
    calls = max(1, s["calls"])
    ms = s["ms"] / calls
    byts = spmv_bytes(case.n, nnzb, fp32=True)
    ach = byts / (ms * 1e-3) / 1e9 if ms > 0 else 0.0
    m = measured_traffic("spmv32", "mixed", case)
    return {"kernel": "k_spmv<float>", "bound": "hbm", "calls": calls, "ms_per_call": ms, "bytes_per_call": byts,
            "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
            "peak_source": "MEASURED_PEAKS.json hbm_gbs", "traffic": m[0] * case.n,
            "traffic_source": f"{m[2]} (captured on {m[1]}, scaled per cell to {case.n} cells)"}


class Bench:
    """One libisc handle on one workload, its resident starting iterate and the
    timed Newton step."""

    def __init__(self, case, **opt):
        import torch
        from paper_1811_11992_gb300 import isc
        self.case = case
        self.g = isc.Simulator(case, profile=1, inner_its=INNER_ITS, **opt)
        self.g.init_equilibrium()
        n = case.n
        self.u0 = torch.empty(8 * n, dtype=torch.float64, device="cuda")
        self.c0 = torch.empty(n, dtype=torch.float64, device="cuda")
        self.g.get_state_device(self.u0.data_ptr(), self.c0.data_ptr())
        torch.cuda.synchronize()

    def step(self):
        self.g.set_state_device(self.u0.data_ptr(), self.c0.data_ptr())
        return self.g.newton_step(self.case.dt0)

    def leg(self, steps, warmup, **opt):
        """Time `steps` Newton steps with the options changed (restored after)."""
        import torch
        saved = {k: getattr(self.g.options, k) for k in opt}
        if opt:
            self.g.set_options(**opt)
        for _ in range(warmup):
            self.step()
        torch.cuda.synchronize()
        self.g.reset_stats()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        infos = [self.step() for _ in range(steps)]
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        st = self.g.stats()
        if opt:
            self.g.set_options(**saved)
        return ms, st, infos

    def close(self):
        self.g.close()


def leg_summary(ms, st, infos, steps, solve_ref_ms=None):
    solve = sum(st[k]["ms"] for k in SOLVE_CLASSES) / steps
    out = {"value": 1e3 / ms, "unit": UNIT, "ms_per_step": ms,
           "krylov_iterations_per_step": statistics.median([i.krylov_iterations for i in infos]),
           "rel_residual": max(i.krylov_rel_residual for i in infos),
           "solve_ms": solve,
           "prec_apply_ms_per_call": st["prec_apply"]["ms"] / max(1, st["prec_apply"]["calls"]),
           "kernel_ms_per_step": {k: round(v["ms"] / steps, 3) for k, v in st.items() if v["ms"] > 0}}
    if solve_ref_ms is not None:
        out["solve_ms_fp64"] = solve_ref_ms
        out["solve_speedup_vs_fp64"] = solve_ref_ms / solve if solve > 0 else None
    return out


def workload_block(cfg, steps, warmup, legs):
    """Another workload: FP64 and the listed precision legs of its Newton step."""
    import isc_inputs as inp
    b = Bench(inp.config(cfg))
    ms, st, infos = b.leg(steps, warmup)
    out = {"workload": f"{b.case.name} ({b.case.n} cells)", "fp64": leg_summary(ms, st, infos, steps)}
    ref = out["fp64"]["solve_ms"]
    for p in legs:
        ms, stp, infos = b.leg(steps, warmup, precision=p)
        out[p] = leg_summary(ms, stp, infos, steps, ref)
    out["hbm"] = hbm_table(st, None, None, b.case, b.g.nnzb)
    b.close()
    return out


def run_isc(args):
    import torch

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    from paper_1811_11992_gb300 import build, isc
    build.build()
    fp64_gflops, fp32_gflops = isc.measure_fma_rates()
    case = workload_case(args.workload, args.grid)
    b = Bench(case, precision=args.precision, prec=args.prec, orth=args.orth)
    g = b.g
    n = case.n
    for _ in range(args.warmup):
        b.step()
    torch.cuda.synchronize()
    g.reset_stats()
    infos = []
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    t0 = time.perf_counter()
    evs[0].record()
    for k in range(args.steps):
        infos.append(b.step())
        evs[k + 1].record()           # per-step times on the same stream (best and median)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    wall = time.perf_counter() - t0
    ms_dev = evs[0].elapsed_time(evs[-1])
    ms_steps = [evs[k].elapsed_time(evs[k + 1]) for k in range(args.steps)]
    stats = g.stats()
    clocks = sampler.stop()
    ms_total = max_over_ranks(max(ms_dev, wall * 1e3), "cuda")
    value = job_throughput(world, args.steps, ms_total)
    kry = [i.krylov_iterations for i in infos]
    headline = leg_summary(ms_total / args.steps, stats, infos, args.steps)
    dev_bytes = g.device_bytes()    # the handle's arrays for the timed configuration
    e2e = mixed = mixed_fgmres = cpr_block = orth_leg = None
    mst = fst = None
    leg_steps = max(3, args.steps // 4)
    leg_warm = max(1, min(2, args.warmup))
    if not args.no_extras:
        # end-to-end through the C ABI with host buffers: the state in from pinned
        # host memory, the Newton step, the state out into pinned host memory
        g.set_state_device(b.u0.data_ptr(), b.c0.data_ptr())
        u_start, c_start = g.get_state()
        u_start_p = torch.from_numpy(u_start.reshape(-1).copy()).pin_memory().numpy()
        c_start_p = torch.from_numpy(c_start.copy()).pin_memory().numpy()
        u_out_p = torch.empty(8 * n, dtype=torch.float64).pin_memory().numpy().reshape(8, n)
        c_out_p = torch.empty(n, dtype=torch.float64).pin_memory().numpy()
        for _ in range(leg_warm):
            g.set_state(u_start_p.reshape(8, n), c_start_p)
            g.newton_step(case.dt0)
            g.get_state(u_out_p, c_out_p)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(leg_steps):
            g.set_state(u_start_p.reshape(8, n), c_start_p)
            g.newton_step(case.dt0)
            g.get_state(u_out_p, c_out_p)
        torch.cuda.synchronize()
        e2e_s = time.perf_counter() - t0
        e2e_val = job_throughput(world, leg_steps, max_over_ranks(e2e_s * 1e3, "cuda"))
        io_bytes = 9 * n * 8
        e2e = {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": io_bytes, "d2h_bytes_per_step": io_bytes,
               "steps": leg_steps}
        if args.precision == "fp64" and args.prec == "bilu0":
            solve_fp64 = headline["solve_ms"]
            # FP32 ILU(0) factors and sweeps inside the FP64 GMRES
            ms, mst, mi = b.leg(leg_steps, leg_warm, precision="mixed")
            mixed = leg_summary(ms, mst, mi, leg_steps, solve_fp64)
            # FP32 inner GMRES (FP32 SpMV, Gram-Schmidt and ILU(0)) inside the flexible FP64 GMRES
            ms, fst, fi = b.leg(leg_steps, leg_warm, precision="mixed_fgmres")
            mixed_fgmres = leg_summary(ms, fst, fi, leg_steps, solve_fp64)
            mixed_fgmres["inner_its"] = INNER_ITS
            mixed_fgmres["roofline_spmv32"] = spmv32_roofline(fst, case, g.nnzb)
            # the same step with the other orthogonalisation (Gram-Schmidt twice or once)
            other = "cgs2" if args.orth == "cgs1" else "cgs1"
            ms, gst, gi = b.leg(leg_steps, leg_warm, orth=other)
            orth_leg = leg_summary(ms, gst, gi, leg_steps, solve_fp64)
            orth_leg["orth"] = other
            orth_leg["blas1_ms_per_step"] = gst["blas1"]["ms"] / leg_steps
            # CPR-PF (the paper's Example-2 preconditioner) on the same step
            cpr_block = {}
            for p in ("fp64", "mixed", "mixed_fgmres"):
                ms, cst, ci = b.leg(leg_steps, leg_warm, prec="cpr", precision=p)
                cpr_block[p] = leg_summary(ms, cst, ci, leg_steps, solve_fp64)
                cpr_block[p]["pressure_stage_ms_per_step"] = cst["cpr"]["ms"] / leg_steps
                cpr_block[p]["speedup_vs_ilu0_fp64"] = (ms_total / args.steps) / ms
    its_total = sum(kry)
    modelled = [k for k in stats if k not in ASSEMBLY_FLOPS_PER_CELL
                and class_model(k, n, g.nnzb, its=its_total)[0] is not None]
    dom = max(modelled, key=lambda k: stats[k]["ms"])
    roof = roofline(dom, stats, case, g.nnzb, fp64_gflops, args.precision, its_total, args.orth)
    rooflines = {k: roofline(k, stats, case, g.nnzb, fp64_gflops, args.precision, its_total, args.orth)
                 for k in ("prec_apply", "spmv", "blas1", "gj", "ilu_factor", "props", "flux") if stats[k]["calls"]}
    hbm = hbm_table(stats, mst, fst, case, g.nnzb)
    device_memory = {"bytes": dev_bytes, "bytes_per_cell": dev_bytes / n,
                     "bytes_with_all_legs": g.device_bytes()}   # + FP32 copies, inner basis, CPR levels
    launches = sum(v["launches"] for v in stats.values())
    nnzb = g.nnzb
    b.close()
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_total / args.steps,
        "ms_per_step_best": min(ms_steps), "ms_per_step_median": statistics.median(ms_steps),
        "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f64+f32",
        "data": "synthetic",
        "config": workload_config(case, world, args.precision, args.prec, args.orth),
        "krylov_iterations_per_step": statistics.median(kry) if kry else None,
        "rel_residual": headline["rel_residual"],
        "e2e": e2e,
        "gpu_launches": launches,
        "kernel_ms": {k: round(v["ms"], 3) for k, v in stats.items()},
        "kernel_launches": {k: v["launches"] for k, v in stats.items()},
        "roofline": roof,
        "rooflines": rooflines,
        "alu_peaks_gflops": {"fp64": fp64_gflops, "fp32": fp32_gflops,
                             "how": "isc_measure_fma_rates: register FMA chains on every SM, best of 5"},
        "hbm": hbm,
        "device_memory": device_memory,
        "clocks": clocks,
        "mixed": mixed,
        "mixed_fgmres": mixed_fgmres,
        "cpr": cpr_block,
        "orth_alternative": orth_leg,
        "blas1_ms_per_step": stats["blas1"]["ms"] / args.steps,
        "time_to_1e-6": None if mixed is None else {
            "fp64_solve_ms": headline["solve_ms"], "mixed_solve_ms": mixed["solve_ms"],
            "mixed_fgmres_solve_ms": mixed_fgmres["solve_ms"],
            "fp64_step_ms": headline["ms_per_step"], "mixed_step_ms": mixed["ms_per_step"],
            "mixed_fgmres_step_ms": mixed_fgmres["ms_per_step"],
            "rel_residuals": [headline["rel_residual"], mixed["rel_residual"], mixed_fgmres["rel_residual"]]},
    }
    if not args.no_extras and args.grid is None and args.workload == "large":
        line["workloads"] = {
            "mixed_100x100x30": workload_block(3, leg_steps, leg_warm, ("mixed", "mixed_fgmres")),
            "field_60x60x20": workload_block(2, leg_steps, leg_warm, ()),
        }
    if not args.no_adjoint and not args.no_extras and args.grid is None:
        line["adjoint"] = adjoint_block()
    if rank == 0 and world == 1 and not args.no_cpu_baseline and args.grid is None:
        line["cpu_baseline"] = cpu_baseline(case, statistics.median(kry) if kry else 0, nnzb)
        if args.cpu_fullsize:
            line["cpu_baseline"]["fullsize_kernels"] = oracle_fullsize_kernels(case)
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


# ------------------------------------------------------------------ oracle
# Bounded samples of the large workload's recipe (3 facies, 5-spot, same
# generator): the cpu_baseline breakdown (about 15 s of host work) and the
# reference arm's per-step sample (about 5 s, so that 25 steps end within a few
# minutes).
SAMPLE = (30, 30, 10)
REF_SAMPLE = (20, 20, 10)


def oracle_sample_case(dims=SAMPLE):
    import isc_inputs as inp
    return inp.large_case(*dims)


def oracle_sample_step(dims=REF_SAMPLE):
    """One oracle Newton step (as it stands) on a sample. Returns (s, cells, its)."""
    from oracle import model, sim
    case = oracle_sample_case(dims)
    u, c = sim.initial_state(case)
    acc_old = model.old_accumulation(case, u, c)
    opts = sim.NewtonOptions(tol=0.0)
    opts.solve.rtol = 1e-6
    t0 = time.perf_counter()
    r = sim.newton_step(case, u, c, acc_old, case.dt0, opts)
    return time.perf_counter() - t0, case.n, r["its"]


def oracle_breakdown():
    """The oracle's Newton step on the sample, part by part: residual and
    Jacobian, Gauss-Jordan, ILU(0) set-up, GMRES(30) to 1e-6 (and its
    iterations), plus 10 SpMVs and 10 ILU(0) applies on the decoupled matrix."""
    import numpy as np
    from oracle import linalg, model, sim
    case = oracle_sample_case()
    u, c = sim.initial_state(case)
    acc_old = model.old_accumulation(case, u, c)
    dt = case.dt0
    geom = model.faces(case)
    t = {}
    t0 = time.perf_counter()
    F = model.residual(case, u, c, acc_old, dt, geom)
    rp, col, J = model.jacobian(case, u, c, acc_old, dt, geom=geom)
    t["assembly"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    val, rhs = linalg.gauss_jordan_decouple(rp, col, J, -F.T.copy())
    t["gauss_jordan"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    M = linalg.ILU0Preconditioner(rp, col, val)
    A = linalg.bsr_to_scipy(rp, col, val)
    t["ilu_setup"] = time.perf_counter() - t0
    mv = lambda v: (A @ v.reshape(-1)).reshape(v.shape)
    t0 = time.perf_counter()
    _, its, rel = linalg.gmres(mv, rhs, M, 30, 1e-6, 1000)
    t["gmres"] = time.perf_counter() - t0
    x = np.random.default_rng(1).standard_normal(rhs.shape)
    t0 = time.perf_counter()
    for _ in range(10):
        mv(x)
    t["spmv"] = (time.perf_counter() - t0) / 10
    t0 = time.perf_counter()
    for _ in range(10):
        M.apply(x)
    t["ilu_apply"] = (time.perf_counter() - t0) / 10
    return t, case.n, its, rel


def cpu_baseline(case, kry_full, nnzb):
    """The oracle as it stands (numpy/scipy, one thread: its sparse products and
    triangular solves are single-threaded) on the host cores, on the bounded
    sample; every part of the Newton step costs O(cells), so the full-size
    figures are per-cell costs times the workload's cells, with the GMRES part
    taken at the full-size Krylov iteration count the GPU measured on the same
    matrix recipe (an estimate: the oracle itself never runs 2M cells here)."""
    t, ns, its, rel = oracle_breakdown()
    scale = case.n / ns
    setup = t["assembly"] + t["gauss_jordan"] + t["ilu_setup"]
    per_it = t["gmres"] / max(its, 1)
    est = scale * (setup + kry_full * per_it)
    spmv_full_ms = t["spmv"] * scale * 1e3
    ilu_full_ms = t["ilu_apply"] * scale * 1e3
    return {"value": 1.0 / est, "unit": UNIT, "cores": 1, "kind": "oracle", "host_cores": os.cpu_count(),
            "sample": f"one oracle Newton step on a {SAMPLE[0]}x{SAMPLE[1]}x{SAMPLE[2]} block of the large "
                      f"workload's recipe ({ns} cells; assembly {t['assembly']:.2f} s, Gauss-Jordan "
                      f"{t['gauss_jordan']:.2f} s, ILU(0) set-up {t['ilu_setup']:.2f} s, GMRES {t['gmres']:.2f} s "
                      f"for {its} iterations to {rel:.1e}); estimate = cells x (per-cell set-up + "
                      f"{kry_full:.0f} full-size iterations x per-cell iteration cost)",
            "estimate_s_per_step": est,
            "spmv_s_per_call_sample": t["spmv"], "ilu_apply_s_per_call_sample": t["ilu_apply"],
            "spmv_gbs_sample": spmv_bytes(ns, 7 * ns) / t["spmv"] / 1e9,
            "spmv_ms_full_estimate": spmv_full_ms, "ilu_apply_ms_full_estimate": ilu_full_ms}


def host_mem_available_gb():
    try:
        with open("/proc/meminfo") as f:
            for ln in f:
                if ln.startswith("MemAvailable:"):
                    return int(ln.split()[1]) / 1e6
    except OSError:
        pass
    return 0.0


def oracle_fullsize_kernels(case, need_gb=96.0):
    """The oracle's SpMV (scipy CSR product) and block ILU(0) apply (two scipy
    sparse triangular solves and the D^-1 products) timed on the workload's
    full-size pattern, as they stand, on one host thread. The matrix and factor
    values are synthetic (identity diagonal blocks, constant off-diagonal
    entries): neither routine's cost depends on the values, and the oracle's
    own factorisation (a Python loop over the cells) is not part of the apply."""
    import numpy as np
    from oracle import linalg, model
    avail = host_mem_available_gb()
    if avail < need_gb:
        return {"skipped": f"{avail:.0f} GB of host memory available, {need_gb:.0f} GB needed"}
    t0 = time.perf_counter()
    rp, col = model.bsr_pattern(case)
    n, nnzb = case.n, len(col)
    val = np.full((nnzb, 8, 8), 1.0e-3)
    rows = np.repeat(np.arange(n), np.diff(rp))
    val[col == rows] = np.eye(8)
    del rows
    prep = time.perf_counter() - t0
    A = linalg.bsr_to_scipy(rp, col, val)
    x = np.ones(8 * n)
    A @ x
    t0 = time.perf_counter()
    for _ in range(3):
        A @ x
    spmv = (time.perf_counter() - t0) / 3
    del A
    t0 = time.perf_counter()
    M = linalg.ILU0Preconditioner(rp, col, val, factors=val)
    setup = time.perf_counter() - t0
    r = np.ones((n, 8))
    t0 = time.perf_counter()
    for _ in range(2):
        M.apply(r)
    ilu = (time.perf_counter() - t0) / 2
    return {"cells": n, "nnzb": nnzb, "cores": 1, "spmv_s_per_call": spmv, "ilu_apply_s_per_call": ilu,
            "spmv_gbs_at_algorithmic_bytes": spmv_bytes(n, nnzb) / spmv / 1e9, "csr_setup_s": setup, "pattern_and_values_s": prep,
            "host_mem_available_gb": avail,
            "note": "synthetic values on the full-size pattern; CSR conversion and triangular-factor set-up "
                    "are outside the timed calls"}


def run_reference(args):
    rank, world, local = dist_env()
    if rank != 0:
        return
    case = workload_case(args.workload, args.grid)
    for _ in range(args.warmup):
        oracle_sample_step()
    t0 = time.perf_counter()
    ncell = its = None
    for _ in range(args.steps):
        _, ncell, its = oracle_sample_step()
    wall = time.perf_counter() - t0
    per = wall / args.steps
    value = (ncell / case.n) / per
    sample = (f"one oracle Newton step per timed step on a {REF_SAMPLE[0]}x{REF_SAMPLE[1]}x{REF_SAMPLE[2]} block of the "
              f"workload's recipe ({ncell} cells, {its} GMRES iterations), scaled by cell count to {case.n} cells")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": per * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(case, world, args.precision, args.prec, args.orth),
        "cpu_baseline": {"value": value, "unit": UNIT, "kind": "oracle", "cores": 1, "host_cores": os.cpu_count(),
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


if __name__ == "__main__":
    a = parse()
    if a.impl == "reference":
        run_reference(a)
    else:
        run_isc(a)
