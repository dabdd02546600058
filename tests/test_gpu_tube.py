"""End-to-end parity on the 50-cell combustion tube over 2 simulated hours.

The oracle chooses the step sizes with its controller; the GPU replays the
same step sizes and the same number of Newton solves per step (so both run
the same sequence of linearise-decouple-solve-update operations), then the
final pressure, temperature and saturations must agree to 1e-7.
"""
import numpy as np
import pytest

import isc_inputs as inp
from oracle import sim

pytestmark = pytest.mark.gpu


def test_tube_trajectory_matches_oracle():
    from paper_1811_11992_gb300 import build
    build.build()
    from paper_1811_11992_gb300 import Simulator

    case = inp.tube_case()
    opts = sim.NewtonOptions(tol=1e-6)
    opts.solve.solver = "dense"
    u_o, c_o, dts, stats = sim.run(case, case.t_end, 5.0, 150.0, opts)
    assert 40 <= len(dts) <= 80
    g = Simulator(case, tol_newton=0.0, tol_lin=1e-12, maxit_lin=400)
    g.init_equilibrium()
    for dt, its in zip(dts, stats["its_per_step"]):
        for _ in range(its):
            g.newton_step(dt)
        g.assemble(dt)        # the convergence-check assembly solves C_c at the accepted state
        g.begin_step()
    u_g, c_g = g.get_state()
    rel_p = np.max(np.abs(u_g[0] - u_o[0]) / u_o[0])
    rel_T = np.max(np.abs(u_g[5] - u_o[5]) / u_o[5])
    So_g, So_o = 1 - u_g[6] - u_g[7], 1 - u_o[6] - u_o[7]
    d_S = max(np.max(np.abs(u_g[6] - u_o[6])), np.max(np.abs(u_g[7] - u_o[7])), np.max(np.abs(So_g - So_o)))
    assert rel_p < 1e-7 and rel_T < 1e-7 and d_S < 1e-7, (rel_p, rel_T, d_S)
    assert np.allclose(c_g, c_o, rtol=1e-6, atol=1e-12 * max(c_o.max(), 1.0))
    g.close()


def test_gpu_timestep_loop_runs_the_tube():
    from paper_1811_11992_gb300 import Simulator
    case = inp.tube_case()
    g = Simulator(case)
    g.init_equilibrium()
    t, dt = 0.0, 5.0
    steps = 0
    while t < 600.0:
        info = g.timestep(dt)
        assert info.status == 0
        t += dt
        steps += 1
        dt = min(2 * dt, 150.0)
    u, c = g.get_state()
    assert np.all(np.isfinite(u)) and np.all(u[6] > 0) and np.all(u[7] > 0)
    g.close()
