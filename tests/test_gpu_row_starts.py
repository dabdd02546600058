"""The ILU(0) sweeps and factorisation compute each cell's BSR row start in
closed form instead of loading rowptr. isc_check_row_starts compares both of
their closed forms with a rowptr built here from the pattern's definition
(one block for the cell and one per existing neighbour, rows in cell order:
a cumulative sum), itself checked against the oracle's pattern on the small
grids, for edge shapes and for the grids the bench and the capacity run use
(up to 16M cells)."""
import numpy as np
import pytest

import isc_inputs as inp
from oracle import model



def _rowptr(nx, ny, nz):
    """rowptr of the 7-point pattern from its definition."""
    x = np.arange(nx)
    y = np.arange(ny)
    z = np.arange(nz)
    cx = 1 + (x > 0) + (x < nx - 1)
    cy = (y > 0).astype(np.int64) + (y < ny - 1)
    cz = (z > 0).astype(np.int64) + (z < nz - 1)
    per = (cx[None, None, :] + cy[None, :, None] + cz[:, None, None]).reshape(-1)
    return np.concatenate([[0], np.cumsum(per)]).astype(np.int64)


SMALL = [(1, 1, 1), (2, 1, 1), (1, 2, 1), (1, 1, 2), (5, 1, 4), (1, 4, 3), (5, 3, 1), (4, 3, 2), (7, 5, 5)]
LARGE = [(60, 60, 20), (100, 100, 30), (1, 3001, 1), (3001, 1, 1), (2, 160, 100), (200, 200, 50), (400, 400, 100)]


@pytest.mark.parametrize("dims", SMALL, ids=lambda d: "x".join(map(str, d)))
def test_definition_is_the_oracle_pattern(dims):
    case = inp.small_box(*dims)
    rp, _ = model.bsr_pattern(case)
    assert np.array_equal(_rowptr(*dims), rp)


@pytest.mark.gpu
@pytest.mark.parametrize("dims", SMALL + LARGE, ids=lambda d: "x".join(map(str, d)))
def test_closed_form_row_starts_match(dims):
    from paper_1811_11992_gb300 import build, isc
    build.build()
    rp = _rowptr(*dims)
    assert rp[-1] < 2**31
    assert isc.check_row_starts(*dims, rp) == (0, -1)
    # a planted error is found (the row after the middle cell starts one block later)
    bad = rp.copy()
    mid = len(rp) // 2
    bad[mid] += 1
    cnt, first = isc.check_row_starts(*dims, bad)
    assert cnt == 1 and first == mid
