"""Both layouts of the ILU(0) sweeps on either side of their dispatch: grids with
at most 3,000 x-pencils (ny*nz; 3,600 for the FP32 sweeps) run one pencil per
warp, larger ones pencil pairs. On grids at and just past the FP64 threshold,
including one-cell pencils (nx = 1), the GPU's apply of a seeded block
matrix on the 7-point pattern (unit diagonal, as after decoupling) is compared
element by element with the oracle's textbook block ILU(0) (IKJ form) at 1e-11;
the FP32 factors and sweeps (precision "mixed") on both sides of their own
threshold at the FP32 level."""
import numpy as np
import pytest

import isc_inputs as inp
from oracle import linalg, model

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def Simulator():
    from paper_1811_11992_gb300 import build
    build.build()
    from paper_1811_11992_gb300 import Simulator as S
    return S


# (nx, ny, nz): 3,000 pencils (one per warp), 3,001 and 3,050 (pairs), 1,200 with nx = 3
GRIDS = [(1, 60, 50), (1, 3001, 1), (2, 50, 61), (3, 40, 30)]
# the FP32 sweeps' threshold: 3,600 pencils (one per warp) and 3,660 (pairs)
GRIDS32 = [(1, 60, 60), (2, 60, 61)]


def _apply_against_oracle(Simulator, dims, **opt):
    nx, ny, nz = dims
    case = inp.field_case(nx, ny, nz, 0, 13, f"field {nx}x{ny}x{nz}", inp.DAY, 4)
    rp, col = model.bsr_pattern(case)
    n = case.n
    rng = np.random.default_rng(nx * 100003 + ny * 101 + nz)
    val = rng.standard_normal((len(col), 8, 8)) * 0.04
    rows = np.repeat(np.arange(n), np.diff(rp))
    val[col == rows] = np.eye(8)
    g = Simulator(case, **opt)
    g.set_system(val, np.zeros((8, n)), decoupled=True)
    g.build_preconditioner()
    r = rng.standard_normal((8, n))
    z = g.precond_apply(r)
    zo = linalg.ILU0Preconditioner(rp, col, val).apply(r.T.copy()).T
    g.close()
    return np.max(np.abs(z - zo)) / np.abs(zo).max()


@pytest.mark.parametrize("dims", GRIDS, ids=lambda d: "x".join(map(str, d)))
def test_ilu0_apply_matches_oracle_on_both_sides_of_the_layout_threshold(Simulator, dims):
    assert _apply_against_oracle(Simulator, dims) <= 1e-11


@pytest.mark.parametrize("dims", GRIDS32, ids=lambda d: "x".join(map(str, d)))
def test_fp32_ilu0_apply_on_both_sides_of_its_layout_threshold(Simulator, dims):
    err = _apply_against_oracle(Simulator, dims, precision="mixed")
    assert err < 2e-5, err          # FP32 factors and sweeps against the FP64 oracle
    assert err > 1e-12              # really FP32
