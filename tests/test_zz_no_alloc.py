"""The allocation-free ILU(0) apply (isc_bilu0_apply_noalloc) serves callers
that cannot allocate GPU memory themselves: it must give the same result as
the library's own preconditioner apply (isc_precond_apply) and as the oracle's
textbook block ILU(0) on the same matrix, on two calls in a row (the shared
static scratch keeps the previous call's contents), and reject grids larger
than its fixed scratch."""
import numpy as np
import pytest

import isc_inputs as inp
from oracle import linalg
from oracle_system import decoupled

pytestmark = pytest.mark.gpu


def test_noalloc_ilu_apply_matches_precond_apply_twice():
    torch = pytest.importorskip("torch")
    from paper_1811_11992_gb300 import build
    build.build()
    from paper_1811_11992_gb300 import Simulator, isc

    case = inp.small_box(7, 5, 5)
    # the oracle's decoupled system (assembly, Gauss-Jordan) and its textbook block ILU(0)
    rp, col, _, _, Jd, Fd = decoupled(case, 909, 910)
    g = Simulator(case)
    g.set_system(Jd, Fd, decoupled=True)
    g.build_preconditioner()
    F = linalg.block_ilu0(rp, col, Jd)
    M = linalg.ILU0Preconditioner(rp, col, Jd)
    rows = np.repeat(np.arange(case.n), np.diff(rp))
    Dinv = np.linalg.inv(F[col == rows])
    rp = rp.astype(np.int32)
    dev = torch.device("cuda")
    d_rp = torch.from_numpy(rp).to(dev)
    d_A = torch.from_numpy(np.ascontiguousarray(Jd).reshape(-1)).to(dev)
    d_D = torch.from_numpy(np.ascontiguousarray(Dinv).reshape(-1)).to(dev)
    rng = np.random.default_rng(3)
    for _ in range(2):
        r = rng.standard_normal((8, case.n))
        z_ref = g.precond_apply(r)
        d_r = torch.from_numpy(np.ascontiguousarray(r.T).reshape(-1)).to(dev)
        d_z = torch.empty_like(d_r)
        torch.cuda.synchronize()
        isc.bilu0_apply_noalloc(case.nx, case.ny, case.nz, d_rp.data_ptr(), d_A.data_ptr(), d_D.data_ptr(),
                                d_r.data_ptr(), d_z.data_ptr())
        z = d_z.cpu().numpy().reshape(case.n, 8).T
        assert np.max(np.abs(z - z_ref)) <= 1e-11 * np.abs(z_ref).max()
        z_or = M.apply(r.T.copy()).T
        assert np.max(np.abs(z - z_or)) <= 1e-11 * np.abs(z_or).max()
    # a grid beyond the static scratch is rejected before any GPU work
    too_big = isc.NOALLOC_MAX_CELLS + 1
    with pytest.raises(isc.IscError) as err:
        isc.bilu0_apply_noalloc(too_big, 1, 1, d_rp.data_ptr(), d_A.data_ptr(), d_D.data_ptr(),
                                d_r.data_ptr(), d_z.data_ptr())
    assert err.value.status == -1
    g.close()
