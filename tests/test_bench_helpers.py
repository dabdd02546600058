"""The bench line's derived numbers (CPU): per-class GB/s from kernel-class times,
the FP32 SpMV roofline and the traffic-figure rule for non-FP64 runs."""
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


def test_class_gbs(bench):
    st = {"spmv": {"calls": 4, "ms": 2.0, "launches": 4}}
    out = bench.class_gbs(st, "spmv", 1_000_000)
    assert out["ms_per_call"] == pytest.approx(0.5)
    assert out["gbs"] == pytest.approx(1e6 / 0.5e-3 / 1e9)
    assert bench.class_gbs(st, "blas1", 10) is None          # class never ran
    assert bench.class_gbs({"x": {"calls": 0, "ms": 0.0}}, "x", 10) is None


def test_hbm_table_bytes(bench):
    case = _Case(60, 60, 20)
    nnzb = 492_000
    st = {k: {"calls": 1, "ms": 1.0, "launches": 1} for k in ("spmv", "prec_apply", "spmv32")}
    t = bench.hbm_table(st, st, st, case, nnzb)
    off = nnzb - case.n
    assert t["spmv_fp64"]["bytes_per_call"] == off * 516 + 3 * case.n * 64
    assert t["spmv_fp32"]["bytes_per_call"] == off * 260 + 3 * case.n * 32
    assert t["ilu_apply_fp32"]["bytes_per_call"] < t["ilu_apply_fp64"]["bytes_per_call"]
    assert set(bench.hbm_table(st, None, None, case, nnzb)) == {"spmv_fp64", "ilu_apply_fp64"}


def test_fp64_traffic_only_for_fp64_runs(bench):
    case = _Case(60, 60, 20)
    st = {"prec_apply": {"calls": 80, "ms": 26.0, "launches": 160}}

    class G:
        nnzb = 492_000
    r64 = bench.roofline("prec_apply", st, G(), case, [80], "fp64")
    r32 = bench.roofline("prec_apply", st, G(), case, [80], "mixed")
    assert r64["traffic"] == bench.MEASURED_TRAFFIC[("prec_apply", 60, 60, 20)][0]
    assert r32["traffic"] is None and "note" in r32
    # algorithmic bytes per call against the measured HBM copy bandwidth
    assert r64["hbm_achieved_gbs"] == pytest.approx(r64["bytes_per_call"] / (26.0 / 80 * 1e-3) / 1e9)
