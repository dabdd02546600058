"""Multi-step parity in 3D: ten accepted implicit-Euler steps (Sec. 3.1) of an
8x6x4 field box with gravity, an ignited air injector in one corner column, a
producer in the opposite one, the four reactions and heat loss to the
overburden and underburden (Sec. 2.1), followed by the oracle and by the GPU.

The oracle chooses the step sizes with its controller and solves its Newton
systems densely; the GPU replays the same step sizes and the same number of
Newton solves per step (GMRES + block ILU(0) to 1e-12), then pressure and
temperature must agree to 1e-7 relative and the saturations to 1e-7 absolute
after the last step."""
import numpy as np
import pytest

import isc_inputs as inp
from oracle import sim

pytestmark = pytest.mark.gpu


def _case(heat_loss):
    case = inp.field_case(8, 6, 4, 0, 11, "field 8x6x4", 30 * inp.DAY, 40, air_rate_std=5e-4)
    return inp.with_heat_loss(case) if heat_loss else case


@pytest.mark.parametrize("heat_loss", [True, False], ids=["heat_loss", "no_heat_loss"])
@pytest.mark.parametrize("prec", ["bilu0", "cpr"])
def test_3d_trajectory_matches_oracle(heat_loss, prec):
    from paper_1811_11992_gb300 import build
    build.build()
    from paper_1811_11992_gb300 import Simulator

    case = _case(heat_loss)
    opts = sim.NewtonOptions(tol=1e-6)
    opts.solve.solver = "dense"
    u_o, c_o, dts, stats = sim.run(case, 1e9, 60.0, 4 * 3600.0, opts, max_steps=10)
    assert len(dts) == 10 and u_o[5].max() > 600.0          # still burning after the last step
    g = Simulator(case, tol_newton=0.0, tol_lin=1e-12, maxit_lin=2000, prec=prec)
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


def test_heat_loss_residual_and_jacobian_match_oracle():
    """Residual and Jacobian with the loss switched on, at a random state of a
    3-layer box (top and bottom layers lose heat, the middle one does not)."""
    from paper_1811_11992_gb300 import build
    build.build()
    from paper_1811_11992_gb300 import Simulator
    from oracle import model

    case = inp.with_heat_loss(inp.small_box(5, 4, 3))
    a = inp.random_state(case, 1301)
    b = inp.random_state(case, 1302)
    g = Simulator(case)
    g.set_state(a["u"], a["coke"])
    g.begin_step()
    g.set_state(b["u"])
    g.assemble(100.0)
    acc_old = model.old_accumulation(case, a["u"], a["coke"])
    Fo = model.residual(case, b["u"], a["coke"], acc_old, 100.0)
    F = g.residual()
    scale = np.abs(Fo).max(axis=1, keepdims=True)
    assert np.max(np.abs(F - Fo) / scale) < 1e-10
    rp, col, J = g.jacobian()
    _, _, Jo = model.jacobian(case, b["u"], a["coke"], acc_old, 100.0)
    rows = np.repeat(np.arange(case.n), np.diff(rp))
    diag = col == rows
    # the energy row's temperature entry carries the 17 W/K per face conductance
    assert np.allclose(J[diag][:, 6, 5], Jo[diag][:, 6, 5], rtol=1e-10)
    # every entry, relative to its block row's largest entry over the whole row (unknowns in their units)
    sc = np.array([1e6, 1, 1, 1, 1, 100.0, 1, 1])
    Js, Jos = J * sc[None, None, :], Jo * sc[None, None, :]
    rowmax = np.zeros((case.n, 8))
    np.maximum.at(rowmax, rows, np.abs(Jos).max(axis=2))
    assert np.max(np.abs(Js - Jos) / (rowmax[rows][:, :, None] + 1e-300)) < 1e-10
    # switching it off restores the plain residual
    g.set_heat_loss(1.7, 10.0, 300.0, 0.0, faces=0)
    g.assemble(100.0)
    F0 = model.residual(inp.small_box(5, 4, 3), b["u"], a["coke"], acc_old, 100.0)
    assert np.max(np.abs(g.residual() - F0) / np.abs(F0).max(axis=1, keepdims=True)) < 1e-10
    g.close()
