"""GPU discrete adjoint with coupled wells (bottom-hole pressure unknown, Sec. 2.2
Well Modeling) against the oracle's tangent-linear model of the bordered time
loop (an independent, forward-mode algorithm): the loss (oil produced at the
coupled producer at its converged bottom-hole pressures) and the gradient
along random directions in ln k and in the reaction parameters, for a
rate-controlled and a BHP-controlled coupled producer and a BHP-controlled
coupled injector."""
import numpy as np
import pytest

import isc_inputs as inp
from oracle import adjoint

pytestmark = pytest.mark.gpu

DTS = [10.0, 40.0]
CASES = {
    "producer_total_rate": lambda: inp.with_coupled_producer(inp.small_box(3, 2, 2), inp.CTRL_TOTAL_RATE, 8.0, 4.6e6),
    "producer_bhp": lambda: inp.with_coupled_producer(inp.small_box(3, 2, 2), inp.CTRL_BHP, 4.55e6, 4.6e6),
    "injector_bhp": lambda: inp.with_coupled_injector(inp.small_box(3, 2, 2), inp.CTRL_BHP, 5.3e6, 5.3e6),
}


@pytest.mark.parametrize("name", list(CASES))
def test_coupled_well_gradient_matches_oracle_tangent(name):
    pytest.importorskip("torch")
    from paper_1811_11992_gb300 import build
    build.build()
    from paper_1811_11992_gb300 import Simulator

    case = CASES[name]()
    us, bs, cs = adjoint.trajectory_coupled(case, DTS, tol=1e-11)
    L0 = adjoint.loss_coupled(case, DTS, us, bs)
    assert L0 > 0
    g = Simulator(case, tol_newton=1e-10, tol_lin=1e-10, maxit_newton=40)
    g.init_equilibrium()
    L, gk, ge, ga, info = g.adjoint(DTS, checkpoint_every=1, tol_adjoint=1e-12)
    assert L == pytest.approx(L0, rel=1e-8)
    n, nr = case.n, int(case.reactions["nr"])
    rng = np.random.default_rng(sum(map(ord, name)))
    for _ in range(2):
        v = rng.standard_normal(n)
        ref = adjoint.tangent_coupled(case, DTS, us, bs, cs, v, np.zeros(nr), np.zeros(nr))
        assert float(gk @ v) == pytest.approx(ref, rel=1e-6, abs=1e-9 * abs(L0))
    vE, vA = rng.standard_normal(nr) * 1e3, rng.standard_normal(nr)
    ref = adjoint.tangent_coupled(case, DTS, us, bs, cs, np.zeros(n), vE, vA)
    assert float(ge @ vE + ga @ vA) == pytest.approx(ref, rel=1e-6, abs=1e-9 * abs(L0))
    # the bottom-hole pressures at the end of the loop are the oracle's
    assert np.allclose(g.well_bhp(), bs[-1], rtol=1e-8)
    g.close()
