"""Pins of the oracle's coupled producers (bottom-hole pressure unknown, well
equations of Sec. 2.2 Well Modeling) to facts that do not come from the new
code: the existing fixed-BHP producer, the molar balance of the residual rows,
hydrostatics of a vertical well, finite differences, and the control being
met at Newton convergence."""
import copy

import numpy as np
import pytest

import isc_inputs as inp
from oracle import model, sim


def _no_gravity(case):
    c = copy.copy(case)
    c.fluid = dict(case.fluid)
    c.fluid["gravity"] = 0.0
    return c


@pytest.fixture(scope="module")
def box():
    case = inp.small_box(4, 3, 2)
    u, c = sim.initial_state(case)
    return case, u, c


def test_fixed_bhp_control_without_gravity_is_the_bhp_producer(box):
    case, u, c = box
    base = _no_gravity(case)
    target = [w for w in base.wells if w.kind == inp.WELL_BHP_PRODUCER][0].target
    coupled = inp.with_coupled_producer(base, inp.CTRL_BHP, target, target)
    acc = model.old_accumulation(base, u, c)
    F0 = model.residual(base, u, c, acc, 100.0)
    F1 = model.residual(coupled, u, c, acc, 100.0, bhp=np.array([target]))
    np.testing.assert_array_equal(F1, F0)
    np.testing.assert_array_equal(model.well_equations(coupled, u, np.array([target])), [0.0])


def test_total_rate_equation_is_the_molar_production_of_the_residual(box):
    """At a state whose gas fractions sum to one, the well terms of rows W..CO2
    add up to the well's total molar inflow; with the well removed they vanish."""
    case, u, c = box
    base = _no_gravity(case)
    bhp = 4.6e6
    coupled = inp.with_coupled_producer(base, inp.CTRL_TOTAL_RATE, 0.0, bhp)
    cw = model.coupled_wells(coupled)[0]
    y = model.base_properties(coupled, u)["y"]
    assert np.allclose(sum(y)[cw.cells], 1.0, atol=1e-14)
    acc = model.old_accumulation(base, u, c)
    no_well = copy.copy(base)
    no_well.wells = [w for w in base.wells if w.kind != inp.WELL_BHP_PRODUCER]
    F_with = model.residual(coupled, u, c, acc, 100.0, bhp=np.array([bhp]))
    F_without = model.residual(no_well, u, c, acc, 100.0)
    produced = np.sum(F_with[:6, cw.cells] - F_without[:6, cw.cells])   # -(inflow) = production
    Fw = model.well_equations(coupled, u, np.array([bhp]))[0]
    assert produced > 0
    assert Fw == pytest.approx(produced, rel=1e-12)


def test_equal_drawdown_along_a_hydrostatic_column():
    """Cell pressures in hydrostatic equilibrium with the water column: every
    perforation of a vertical well sees the same water-phase drawdown."""
    case = inp.field_case(1, 2, 8, 0, 1, "column", 30 * inp.DAY, 40)
    u, c = sim.initial_state(case)
    u[6] = 0.9       # water-filled column
    u[7] = 0.0
    coupled = inp.with_coupled_producer(case, inp.CTRL_BHP, 4.0e6, 4.0e6)
    cw = model.coupled_wells(coupled)[0]
    z_ref, p_ref = cw.ref_depth, 5.0e6
    for _ in range(50):   # gamma_w depends weakly on p: iterate to the hydrostatic state
        gam = model.base_properties(coupled, u)["gam"][0]
        u[0] = p_ref + gam * (case.depth - z_ref)
    bp = model.base_properties(coupled, u)
    eps = 2.0e5
    Q = model.coupled_phase_rates(coupled, bp, cw, p_ref - eps)
    drawdown = Q[0] / (cw.WI * bp["lam"][0][cw.cells])
    np.testing.assert_allclose(drawdown, -eps, rtol=1e-9)


def test_border_blocks_match_finite_differences(box):
    case, u, c = box
    coupled = inp.with_coupled_producer(case, inp.CTRL_OIL_RATE, 0.05, 4.6e6)
    bhp = np.array([4.6e6])
    acc = model.old_accumulation(case, u, c)
    B, C, D, Fw = model.coupled_blocks(coupled, u, bhp, c, acc, 100.0)
    cw = model.coupled_wells(coupled)[0]
    h = 1.0
    Fp = model.residual(coupled, u, c, acc, 100.0, bhp=bhp + h)
    Fm = model.residual(coupled, u, c, acc, 100.0, bhp=bhp - h)
    np.testing.assert_allclose(B, ((Fp - Fm) / (2 * h))[:, cw.cells].T, rtol=1e-6, atol=1e-12 * np.abs(B).max())
    D_fd = (model.well_equations(coupled, u, bhp + h) - model.well_equations(coupled, u, bhp - h)) / (2 * h)
    assert D[0] == pytest.approx(D_fd[0], rel=1e-6)
    scale = np.array([1e6, 1, 1, 1, 1, 100, 1, 1])
    for q, cell in enumerate(cw.cells):
        for j in range(8):
            hj = 1e-7 * max(abs(u[j, cell]), scale[j])
            up, um = u.copy(), u.copy()
            up[j, cell] += hj
            um[j, cell] -= hj
            fd = (model.well_equations(coupled, up, bhp)[0] - model.well_equations(coupled, um, bhp)[0]) / (2 * hj)
            assert C[q, j] == pytest.approx(fd, rel=1e-5, abs=1e-9 * np.abs(C).max())


def test_rate_control_is_met_at_newton_convergence(box):
    case, u, c = box
    target = 5.0   # mol/s total production (the 4.5 MPa producer makes ~8.8)
    coupled = inp.with_coupled_producer(case, inp.CTRL_TOTAL_RATE, target, 4.6e6)
    opts = sim.NewtonOptions(tol=1e-11, maxit=40)
    un, bn, cn, its, ok = sim.timestep_coupled(coupled, u, np.array([4.6e6]), c, 10.0, opts)
    assert ok
    bp = model.base_properties(coupled, un)
    Q = model.coupled_phase_rates(coupled, bp, model.coupled_wells(coupled)[0], bn[0])
    assert -sum(np.sum(q) for q in Q) == pytest.approx(target, rel=1e-10)
    assert 4.5e6 < bn[0] < 5.0e6    # a smaller rate than at 4.5 MPa needs a higher bottom-hole pressure


def test_producers_above_reservoir_pressure_are_shut(box):
    """Producers only take fluid out: with the bottom-hole pressure (fixed or
    coupled) above every perforated cell's pressure the well terms vanish, and
    the residual is the one without the well."""
    case, u, c = box
    base = _no_gravity(case)
    acc = model.old_accumulation(base, u, c)
    bhp = 1.5 * float(np.max(u[0]))
    shut = copy.copy(base)
    shut.wells = [copy.copy(w) for w in base.wells]
    for w in shut.wells:
        if w.kind == inp.WELL_BHP_PRODUCER:
            w.target = bhp
    none = copy.copy(base)
    none.wells = [w for w in base.wells if w.kind != inp.WELL_BHP_PRODUCER]
    F_none = model.residual(none, u, c, acc, 100.0)
    np.testing.assert_array_equal(model.residual(shut, u, c, acc, 100.0), F_none)
    coupled = inp.with_coupled_producer(base, inp.CTRL_BHP, bhp, bhp)
    w = model.coupled_wells(coupled)[0]
    Q = model.coupled_phase_rates(coupled, model.base_properties(coupled, u), w, bhp)
    assert all(np.all(q == 0.0) for q in Q)
    np.testing.assert_array_equal(model.residual(coupled, u, c, acc, 100.0, bhp=np.array([bhp])), F_none)
