"""The library's time loop (isc_run: halving of failed steps and the step
controller of the implicit-Euler scheme, Sec. 3.1) against the oracle's
(sim.run, the same rule) on the 50-cell combustion tube: the same accepted
step lengths, the same number of halvings and the same final state. The GPU
solves each Newton system to 1e-12 (the oracle solves it densely), so both
sides take the same convergence decisions and the controller sees the same
changes of T and S."""
import numpy as np
import pytest

import isc_inputs as inp
from oracle import sim

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def Simulator():
    from paper_1811_11992_gb300 import build
    build.build()
    from paper_1811_11992_gb300 import Simulator as S
    return S


def _oracle(case, t_end, dt0, dt_max):
    opts = sim.NewtonOptions(tol=1e-6, maxit=25)
    opts.solve.solver = "dense"
    return sim.run(case, t_end, dt0, dt_max, opts)


def _assert_same_state(u_g, c_g, u_o, c_o):
    rel_p = np.max(np.abs(u_g[0] - u_o[0]) / u_o[0])
    rel_T = np.max(np.abs(u_g[5] - u_o[5]) / u_o[5])
    d_S = max(np.max(np.abs(u_g[6] - u_o[6])), np.max(np.abs(u_g[7] - u_o[7])))
    assert rel_p < 1e-7 and rel_T < 1e-7 and d_S < 1e-7, (rel_p, rel_T, d_S)
    assert np.allclose(c_g, c_o, rtol=1e-6, atol=1e-12 * max(c_o.max(), 1.0))


@pytest.mark.parametrize("dt0,cuts", [(5.0, 0), (160.0, 2)])
def test_time_loop_matches_the_oracle_controller(Simulator, dt0, cuts):
    case = inp.tube_case()
    t_end, dt_max = 600.0, 150.0
    u_o, c_o, dts_o, st_o = _oracle(case, t_end, dt0, dt_max)
    assert st_o["cuts"] == cuts        # 160 s and 80 s fail at the ignition, 40 s converges
    g = Simulator(case, tol_newton=1e-6, maxit_newton=25, tol_lin=1e-12, maxit_lin=400)
    g.init_equilibrium()
    info, dts = g.run(t_end, dt0, dt_max)
    assert info.status == 0 and info.cuts == cuts
    assert info.steps == len(dts_o)
    assert np.allclose(dts, dts_o, rtol=1e-6, atol=0.0), (dts, dts_o)
    assert info.t == pytest.approx(t_end, rel=1e-12)
    u_g, c_g = g.get_state()
    _assert_same_state(u_g, c_g, u_o, c_o)
    # the run leaves an accepted state: a second call continues from it
    info2, _ = g.run(60.0, info.dt_next, dt_max)
    assert info2.status == 0 and info2.t == pytest.approx(60.0, rel=1e-12)
    g.close()


def test_time_loop_gives_up_after_max_cuts_and_restores_the_state(Simulator):
    from paper_1811_11992_gb300 import isc
    case = inp.tube_case()
    g = Simulator(case, tol_newton=1e-6, maxit_newton=25, tol_lin=1e-12, maxit_lin=400)
    g.init_equilibrium()
    u0, c0 = g.get_state()
    info, dts = g.run(600.0, 160.0, 150.0, max_cuts=1, check=False)
    assert info.status < 0 and info.cuts == 1 and info.steps == 0 and info.t == 0.0
    assert info.dt_next == 80.0
    u1, c1 = g.get_state()
    assert np.array_equal(u0, u1) and np.array_equal(c0, c1)
    # invalid arguments are rejected before any work
    for bad in (dict(t_end=-1.0), dict(dt0=0.0), dict(dt_max=-5.0), dict(dT_target=0.0), dict(max_cuts=-1),
                dict(max_steps=0)):
        kw = dict(t_end=10.0, dt0=5.0, dt_max=10.0)
        kw.update(bad)
        with pytest.raises(isc.IscError) as err:
            g.run(**kw)
        assert err.value.status == -1
    # max_steps stops the loop early
    info, dts = g.run(600.0, 5.0, 150.0, max_steps=3)
    assert info.steps == 3 and len(dts) == 3 and info.t == pytest.approx(dts.sum(), rel=1e-15)
    g.close()
