"""GPU coupled injectors (bottom-hole pressure unknown, Sec. 2.2 Well
Modeling, for injection) against the oracle: residual, perforation blocks and
the border (B, C, D, F_w) of the Newton system with one or both perforations
flowing, and Newton-converged time steps under a fixed bottom-hole pressure
and a fixed total rate; on a single perforation the rate-controlled coupled
injector reaches the state of the oracle's fixed-rate injector."""
import numpy as np
import pytest

import isc_inputs as inp
from oracle import model, sim

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def Simulator():
    from paper_1811_11992_gb300 import build
    build.build()
    from paper_1811_11992_gb300 import Simulator as S
    return S


def _box(control, target, bhp_init=5.0e6 + 1.0e3, ignited=True):
    base = inp.small_box(4, 3, 2)
    if not ignited:
        base.ignited = np.array([], np.int32)
    return inp.with_coupled_injector(base, control, target, bhp_init)


def _thresholds(case, u):
    """Bottom-hole pressure at which each perforation starts to inject."""
    bp = model.base_properties(case, u)
    cw = model.coupled_wells(case)[0]
    c = cw.cells
    return bp["p"][c] + bp["gam"][0 if cw.inj_phase == 0 else 2][c] * (cw.ref_depth - case.depth[c])


@pytest.mark.parametrize("control", ["bhp", "total"])
@pytest.mark.parametrize("flowing", ["both", "one"])
def test_residual_and_border_match_oracle(Simulator, control, flowing):
    ctl, target = (inp.CTRL_BHP, 5.2e6) if control == "bhp" else (inp.CTRL_TOTAL_RATE, 0.005)
    case = _box(ctl, target)
    a = inp.random_state(case, 301)
    b = inp.random_state(case, 302)
    t = _thresholds(case, b["u"])
    if flowing == "both":
        bhp = np.array([t.max() + 1.0e5])
    else:
        assert abs(t[1] - t[0]) > 1.0e4
        bhp = np.array([0.5 * (t[0] + t[1])])
    g = Simulator(case)
    g.set_state(a["u"], a["coke"])
    g.begin_step()
    g.set_state(b["u"])
    g.set_well_bhp(bhp)
    g.assemble(100.0)
    F = g.residual()
    rp, col, J = g.jacobian()
    B, C, D, Fw = g.well_system()
    acc = model.old_accumulation(case, a["u"], a["coke"])
    F_ref = model.residual(case, b["u"], a["coke"], acc, 100.0, bhp=bhp)
    rowscale = np.abs(F_ref).max(axis=1, keepdims=True) + 1e-300
    assert np.max(np.abs(F - F_ref) / rowscale) <= 1e-10
    _, _, J_ref = model.jacobian(case, b["u"], a["coke"], acc, 100.0, bhp=bhp)
    cells = model.coupled_wells(case)[0].cells
    rows = np.repeat(np.arange(case.n), np.diff(rp))
    for c in cells:
        blk = np.flatnonzero((rows == c) & (col == c))[0]
        assert np.max(np.abs(J[blk] - J_ref[blk])) <= 1e-10 * np.abs(J_ref[blk]).max()
    B_ref, C_ref, D_ref, Fw_ref = model.coupled_blocks(case, b["u"], bhp, a["coke"], acc, 100.0)
    flows = t < bhp[0]
    assert np.all(B_ref[~flows] == 0.0) and np.all(B[~flows] == 0.0)
    assert np.max(np.abs(B - B_ref)) <= 1e-10 * np.abs(B_ref).max()
    if control == "total":
        assert np.max(np.abs(C - C_ref)) <= 1e-10 * np.abs(C_ref).max()
        np.testing.assert_allclose(D, D_ref, rtol=1e-10)
    else:
        assert np.all(C == 0.0) and np.all(C_ref == 0.0) and D[0] == 1.0 == D_ref[0]
    np.testing.assert_allclose(Fw, Fw_ref, rtol=1e-10, atol=1e-12 * abs(target))
    g.close()


@pytest.mark.parametrize("control", ["total", "bhp"])
def test_time_step_matches_oracle(Simulator, control):
    ctl, target = (inp.CTRL_BHP, 5.05e6) if control == "bhp" else (inp.CTRL_TOTAL_RATE, 0.005)
    case = _box(ctl, target, ignited=False)
    u0, c0 = sim.initial_state(case)
    b0 = np.array([5.0e6 + 1.0e3])
    opts = sim.NewtonOptions(tol=1e-11, maxit=40)
    u_ref, b_ref, c_ref, its, ok = sim.timestep_coupled(case, u0, b0, c0, 60.0, opts)
    assert ok and its >= 2
    g = Simulator(case, tol_newton=1e-11, tol_lin=1e-12, maxit_newton=40)
    g.init_equilibrium()
    g.set_well_bhp(b0)
    g.timestep(60.0)
    u, coke = g.get_state()
    bhp = g.well_bhp()
    assert abs(bhp[0] - b_ref[0]) <= 1e-7 * b_ref[0]
    assert np.max(np.abs(u[0] - u_ref[0]) / u_ref[0]) <= 1e-7
    assert np.max(np.abs(u[5] - u_ref[5]) / u_ref[5]) <= 1e-7
    assert np.max(np.abs(u[6:] - u_ref[6:])) <= 1e-7
    if control == "total":
        bp = model.base_properties(case, u)
        Q = model.coupled_injection_rate(case, bp, model.coupled_wells(case)[0], bhp[0])
        assert np.sum(Q) == pytest.approx(target, rel=1e-8)
    g.close()


def test_single_perforation_rate_control_is_the_rate_injector(Simulator):
    base = inp.tube_case(n_cells=12)
    base.ignited = np.array([], np.int32)
    q = [w for w in base.wells if w.kind == inp.WELL_RATE_INJECTOR][0].target
    u0, c0 = sim.initial_state(base)
    b0 = np.array([u0[0, 0] + 10.0])
    opts = sim.NewtonOptions(tol=1e-10, maxit=40)
    opts.solve.solver = "dense"
    u_ref, _, _, ok = sim.timestep(base, u0, c0, 5.0, opts)
    assert ok
    case = inp.with_coupled_injector(base, inp.CTRL_TOTAL_RATE, q, b0[0])
    g = Simulator(case, tol_newton=1e-10, tol_lin=1e-12, maxit_newton=40)
    g.init_equilibrium()
    g.set_well_bhp(b0)
    g.timestep(5.0)
    u, _ = g.get_state()
    scale = np.array([1e6, 1, 1, 1, 1, 100.0, 1, 1])[:, None]
    assert np.max(np.abs(u - u_ref) / scale) < 1e-7
    assert g.well_bhp()[0] > u[0, 0]
    g.close()
