"""Failures injected on the host (nothing faults or hangs the GPU): a NaN in
the state, a singular diagonal block in a caller's system, a Krylov iteration
cap too small for the tolerance. Each call returns its status (non-finite or
coke failure; singular block; Krylov non-convergence) and the handle stays
usable: the next call on valid data gives the oracle's result."""
import numpy as np
import pytest

import isc_inputs as inp
from oracle import linalg
from oracle_system import assembled

pytestmark = pytest.mark.gpu

ISC_ERR_SINGULAR_BLOCK, ISC_ERR_KRYLOV_NOCONV, ISC_ERR_NONFINITE, ISC_ERR_COKE = -4, -5, -7, -8


@pytest.fixture(scope="module")
def Simulator():
    from paper_1811_11992_gb300 import build
    build.build()
    from paper_1811_11992_gb300 import Simulator as S
    return S


def test_nan_in_the_state_is_reported_and_the_handle_recovers(Simulator):
    from paper_1811_11992_gb300 import isc
    case = inp.small_box(4, 3, 2)
    g = Simulator(case)
    g.init_equilibrium()
    u0, c0 = g.get_state()
    ref = g.newton_step(60.0)            # the step from the valid state
    u_ref, _ = g.get_state()
    bad = u0.copy()
    bad[5, 7] = np.nan                   # temperature of one cell
    g.set_state(bad, c0)
    with pytest.raises(isc.IscError) as err:
        g.newton_step(60.0)
    assert err.value.status in (ISC_ERR_NONFINITE, ISC_ERR_COKE)
    # the same handle, back on the valid state: the same step, bit for bit
    g.set_state(u0, c0)
    info = g.newton_step(60.0)
    u1, _ = g.get_state()
    assert info.krylov_iterations == ref.krylov_iterations
    assert np.array_equal(u1, u_ref)
    g.close()


def test_singular_diagonal_block_is_reported_and_the_handle_recovers(Simulator):
    from paper_1811_11992_gb300 import isc
    case = inp.small_box(4, 3, 2)
    rp, col, J, F = assembled(case, 505, 606)
    rows = np.repeat(np.arange(case.n), np.diff(rp))
    diag = np.flatnonzero(col == rows)
    Js = J.copy()
    Js[diag[5]] = 0.0                    # cell 5's diagonal block
    g = Simulator(case)
    g.set_system(Js, F)
    with pytest.raises(isc.IscError) as err:
        g.decouple()
    assert err.value.status == ISC_ERR_SINGULAR_BLOCK
    # a valid system on the same handle: the oracle's decoupling
    g.set_system(J, F)
    g.decouple()
    _, _, Jd = g.jacobian()
    vo, _ = linalg.gauss_jordan_decouple(rp, col, J, F.T.copy())
    assert np.max(np.abs(Jd - vo)) <= 1e-11 * np.abs(vo).max()
    g.close()


def test_krylov_cap_is_reported_and_the_handle_recovers(Simulator):
    from paper_1811_11992_gb300 import isc
    case = inp.small_box(4, 3, 2)
    rp, col, J, F = assembled(case, 707, 808)
    g = Simulator(case, tol_lin=1e-10, maxit_lin=1)
    g.set_system(J, F)
    g.decouple()
    with pytest.raises(isc.IscError) as err:
        g.solve()
    assert err.value.status == ISC_ERR_KRYLOV_NOCONV
    g.set_options(maxit_lin=400)
    g.set_system(J, F)
    g.decouple()
    info = g.solve()
    assert info.krylov_rel_residual <= 1e-10
    du = g.newton_update()
    A = linalg.bsr_to_dense(rp, col, J)
    x = np.linalg.solve(A, -F.T.reshape(-1)).reshape(case.n, 8).T
    assert np.max(np.abs(du - x)) <= 1e-6 * np.abs(x).max()
    g.close()
