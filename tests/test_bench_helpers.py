"""The bench line's derived numbers (CPU): per-class GB/s from kernel-class times,
the algorithmic bytes of the SpMV and ILU(0) apply, the roofline's bound
(FP64 pipe or HBM) and the traffic figure's scaling rule."""
import importlib.util
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


class _Case:
    def __init__(self, nx, ny, nz):
        self.nx, self.ny, self.nz, self.n = nx, ny, nz, nx * ny * nz
        self.name = f"box {nx}x{ny}x{nz}"
        self.dt0 = 100.0


def _nnzb(nx, ny, nz):
    return nx * ny * nz + 2 * ((nx - 1) * ny * nz + nx * (ny - 1) * nz + nx * ny * (nz - 1))


def test_class_gbs(bench):
    st = {"spmv": {"calls": 4, "ms": 2.0, "launches": 4}}
    out = bench.class_gbs(st, "spmv", 1_000_000)
    assert out["ms_per_call"] == pytest.approx(0.5)
    assert out["gbs"] == pytest.approx(1e6 / 0.5e-3 / 1e9)
    assert bench.class_gbs(st, "blas1", 10) is None          # class never ran
    assert bench.class_gbs({"x": {"calls": 0, "ms": 0.0}}, "x", 10) is None


def test_hbm_table_bytes(bench):
    case = _Case(60, 60, 20)
    nnzb = _nnzb(60, 60, 20)
    assert nnzb == 492_000
    st = {k: {"calls": 1, "ms": 1.0, "launches": 1} for k in ("spmv", "prec_apply", "spmv32")}
    t = bench.hbm_table(st, st, st, case, nnzb)
    off = nnzb - case.n
    assert t["spmv_fp64"]["bytes_per_call"] == off * 516 + 3 * case.n * 64
    assert t["spmv_fp32"]["bytes_per_call"] == off * 260 + 3 * case.n * 32
    # ILU(0) apply: every off-diagonal block once, one inverted diagonal block per cell, four vector passes
    assert t["ilu_apply_fp64"]["bytes_per_call"] == off * 516 + case.n * 512 + 4 * case.n * 64
    assert t["ilu_apply_fp32"]["bytes_per_call"] < t["ilu_apply_fp64"]["bytes_per_call"]
    assert set(bench.hbm_table(st, None, None, case, nnzb)) == {"spmv_fp64", "ilu_apply_fp64"}


def test_roofline_bound_follows_the_measured_ridge(bench):
    case = _Case(200, 200, 50)
    nnzb = _nnzb(200, 200, 50)
    assert nnzb == 13_880_000
    st = {"prec_apply": {"calls": 114, "ms": 114 * 3.8, "launches": 228}}
    # FP64 at 1.2 TFLOP/s: 0.25 flop/B is above the ridge (0.18), so the FP64 pipe bounds the apply
    r = bench.roofline("prec_apply", st, case, nnzb, 1200.0, "fp64")
    assert r["bound"] == "alu" and r["unit"] == "GFLOP/s"
    assert r["achieved"] == pytest.approx(bench.ilu_apply_flops(case.n, nnzb) / 3.8e-3 / 1e9)
    assert r["hbm_achieved_gbs"] == pytest.approx(r["bytes_per_call"] / 3.8e-3 / 1e9)
    # the same apply on a GPU with a fast FP64 pipe is bound by HBM
    r2 = bench.roofline("prec_apply", st, case, nnzb, 60000.0, "fp64")
    assert r2["bound"] == "hbm" and r2["frac"] == pytest.approx(r2["achieved"] / r2["peak"])
    # FP32 sweeps are never FP64-bound
    r3 = bench.roofline("prec_apply", st, case, nnzb, 1200.0, "mixed")
    assert r3["bound"] == "hbm"


def test_traffic_is_scaled_per_cell(bench):
    case = _Case(200, 200, 50)
    nnzb = _nnzb(200, 200, 50)
    st = {"prec_apply": {"calls": 10, "ms": 38.0, "launches": 20}}
    r = bench.roofline("prec_apply", st, case, nnzb, 1200.0, "fp64")
    per_cell = bench.MEASURED_TRAFFIC[("prec_apply", "fp64", "pair")][0]
    assert r["traffic"] == pytest.approx(per_cell * case.n)
    assert "scaled per cell" in r["traffic_source"]
    # the measured DRAM traffic is within a few per cent of the algorithmic bytes
    assert abs(r["traffic"] / r["bytes_per_call"] - 1) < 0.05
    r32 = bench.roofline("prec_apply", st, case, nnzb, 1200.0, "mixed")
    assert abs(r32["traffic"] / r32["bytes_per_call"] - 1) < 0.05
    # the SpMVs' figures (one layout) within a few per cent of their algorithmic bytes too
    rs = bench.roofline("spmv", {"spmv": {"calls": 1, "ms": 1.0, "launches": 1}}, case, nnzb, 1200.0, "fp64")
    assert abs(rs["traffic"] / rs["bytes_per_call"] - 1) < 0.05
    r32s = bench.spmv32_roofline({"spmv32": {"calls": 1, "ms": 0.6, "launches": 1}}, case, nnzb)
    assert abs(r32s["traffic"] / r32s["bytes_per_call"] - 1) < 0.05
    # a class without a capture has no traffic figure
    assert bench.roofline("gj", {"gj": {"calls": 1, "ms": 25.0, "launches": 1}}, case, nnzb, 1200.0,
                          "fp64")["traffic"] is None


def test_reference_and_library_arms_share_the_config(bench):
    case = _Case(200, 200, 50)
    a = bench.workload_config(case, 1)
    b = bench.workload_config(case, 1)
    assert a == b and "200x200x50" in a["workload"] and a["precision"] == "fp64"
    assert bench.parse([]).workload == "large"


def test_gram_schmidt_model(bench):
    # one iteration against one basis vector: 3 passes of (1 vector + w), 2 writes of w,
    # the scaling pass: (3*1 + 7) vector passes; 8*1 + 2 flops per element
    b, f = bench.gmres_blas1_work(10, 1, orth="cgs2")
    assert b == 8 * 80 * 10 and f == 80 * 10
    # once: two passes of (1 vector + w), one write of w, the scaling: (2*1 + 5) passes; 4*1 + 2 flops
    b1, f1 = bench.gmres_blas1_work(10, 1, orth="cgs1")
    assert b1 == 8 * 80 * 7 and f1 == 80 * 6
    # restart cycles: iteration 31 of GMRES(30) works on one vector again
    b31, _ = bench.gmres_blas1_work(10, 31, orth="cgs2")
    b30, _ = bench.gmres_blas1_work(10, 30, orth="cgs2")
    assert b31 - b30 == b
    case = _Case(200, 200, 50)
    nnzb = _nnzb(200, 200, 50)
    st = {"blas1": {"calls": 1140, "ms": 2800.0, "launches": 5700}}
    r = bench.roofline("blas1", st, case, nnzb, 1057.0, "fp64", its=1140, orth="cgs2")
    assert r["bound"] == "alu" and 0.5 < r["frac"] < 1.0


def test_fullsize_oracle_kernel_timing_runs_and_skips_without_memory(bench):
    """The opt-in full-size timing of the oracle's SpMV and ILU(0) apply, on a
    tiny grid of the same recipe: it runs the oracle's routines on the
    workload's own pattern, and declines with a note when the host lacks the
    memory the full-size matrix needs."""
    import isc_inputs as inp
    case = inp.large_case(6, 5, 4)
    r = bench.oracle_fullsize_kernels(case, need_gb=0.0)
    assert r["cells"] == case.n and r["nnzb"] == 7 * case.n - 2 * (case.ny * case.nz + case.nx * case.nz
                                                                     + case.nx * case.ny)
    assert r["spmv_s_per_call"] > 0 and r["ilu_apply_s_per_call"] > 0 and r["cores"] == 1
    skipped = bench.oracle_fullsize_kernels(case, need_gb=1.0e9)
    assert set(skipped) == {"skipped"}


def test_sweep_layout_thresholds_match_the_library(bench):
    """The bench picks the traffic figure of the sweep layout the library runs:
    its thresholds are the library's constants."""
    import re
    src = open(os.path.join(ROOT, "paper_1811_11992_gb300", "csrc", "isc_ilu_pipe.cu")).read()
    lib = {k: int(v) for k, v in re.findall(r"constexpr int (SWEEP1_MAX_PENCILS\d\d) = (\d+);", src)}
    assert bench.SWEEP1_MAX_PENCILS == {"fp64": lib["SWEEP1_MAX_PENCILS64"], "mixed": lib["SWEEP1_MAX_PENCILS32"]}
    small, large = _Case(60, 60, 20), _Case(200, 200, 50)
    assert bench.sweep_layout(small, "fp64") == "single" and bench.sweep_layout(large, "fp64") == "pair"
    nnzb = _nnzb(60, 60, 20)
    st = {"prec_apply": {"calls": 10, "ms": 3.2, "launches": 20}}
    r = bench.roofline("prec_apply", st, small, nnzb, 1200.0, "fp64")
    assert r["traffic"] == pytest.approx(bench.MEASURED_TRAFFIC[("prec_apply", "fp64", "single")][0] * small.n)
