"""Pins of the oracle's coupled injectors (Sec. 2.2, Well Modeling: the
bottom-hole pressure of an injection well becomes an unknown with a fixed
pressure or a fixed total rate). Reading: the injected stream enters each
perforation at Q = WI lambda_T (bhp - p - gamma (z_bh - z)), lambda_T the
cell's total molar mobility, inflow only. Pinned to facts that do not come
from the new code: the fixed-rate injector it must reproduce on a
single-perforation well, the molar and energy content of the injected stream,
finite differences, and the control met at Newton convergence."""
import copy

import numpy as np
import pytest

import isc_inputs as inp
from oracle import model, sim


def _tube_injector(control, target, bhp_init):
    return inp.with_coupled_injector(inp.tube_case(n_cells=12), control, target, bhp_init)


def test_rate_controlled_injector_on_one_perforation_is_the_rate_injector():
    """A single-perforation coupled injector held at the fixed-rate injector's
    rate injects the same stream into the same cell: after a Newton-converged
    time step the states agree to the Newton tolerance, and the bottom-hole
    pressure exceeds the perforated cell's pressure. The tube is not ignited:
    in the ignition step the cell pressure of the Newton iterates swings by
    tenths of a megapascal, and an iterate in which a rate-controlled injector
    stops flowing has a zero well row."""
    base = inp.tube_case(n_cells=12)
    base.ignited = np.array([], np.int32)
    q = [w for w in base.wells if w.kind == inp.WELL_RATE_INJECTOR][0].target
    u0, c0 = sim.initial_state(base)
    b0 = u0[0, 0] + 10.0
    coupled = inp.with_coupled_injector(base, inp.CTRL_TOTAL_RATE, q, b0)
    opts = sim.NewtonOptions(tol=1e-10, maxit=40)
    opts.solve.solver = "dense"
    dt = 5.0
    u1, c1, its, ok = sim.timestep(base, u0, c0, dt, opts)
    assert ok and u1[0, 0] - u0[0, 0] > 100.0         # the injection raised the pressure
    u2, b2, c2, its2, ok2 = sim.timestep_coupled(coupled, u0, np.array([b0]), c0, dt, opts)
    assert ok2
    scale = np.array([1e6, 1, 1, 1, 1, 100.0, 1, 1])[:, None]
    assert np.max(np.abs(u2 - u1) / scale) < 1e-7
    cw = model.coupled_wells(coupled)[0]
    assert b2[0] > u2[0, cw.cells[0]]
    Fw = model.well_equations(coupled, u2, b2)
    assert abs(Fw[0]) <= 1e-8 * q


def test_injected_moles_and_enthalpy_per_mole_of_the_stream():
    """The well terms of rows W..CO2 add up to the total injected molar rate
    (the stream's fractions sum to one) and the energy row carries that rate
    times the stream's molar enthalpy; below the cell pressure nothing flows."""
    case = _tube_injector(inp.CTRL_BHP, 6.0e6, 6.0e6)
    u, c = sim.initial_state(case)
    acc = model.old_accumulation(case, u, c)
    no_well = copy.copy(case)
    no_well.wells = [w for w in case.wells if w.kind != inp.WELL_COUPLED_INJECTOR]
    cw = model.coupled_wells(case)[0]
    assert np.sum(cw.inj_y) == pytest.approx(1.0, abs=1e-15)
    F0 = model.residual(no_well, u, c, acc, 10.0)
    bp = model.base_properties(case, u)
    for bhp, flows in ((6.0e6, True), (4.0e6, False)):
        F1 = model.residual(case, u, c, acc, 10.0, bhp=np.array([bhp]))
        Q = model.coupled_injection_rate(case, bp, cw, bhp)
        cell = cw.cells[0]
        injected = -np.sum(F1[:6, cell] - F0[:6, cell])
        if flows:
            assert Q[0] > 0 and injected == pytest.approx(Q[0], rel=1e-12)
            energy = -(F1[6, cell] - F0[6, cell])
            assert energy == pytest.approx(Q[0] * model.injected_enthalpy(case.fluid, cw), rel=1e-12)
        else:
            assert Q[0] == 0.0 and np.array_equal(F1, F0)


def test_injection_rate_is_linear_in_the_bottom_hole_pressure_above_the_cell():
    """Doubling the overpressure doubles the rate (the mobility is the cell's)."""
    case = _tube_injector(inp.CTRL_BHP, 6.0e6, 6.0e6)
    u, c = sim.initial_state(case)
    bp = model.base_properties(case, u)
    cw = model.coupled_wells(case)[0]
    p = bp["p"][cw.cells[0]]            # horizontal tube: no head between the reference and the cell
    q1 = model.coupled_injection_rate(case, bp, cw, p + 1.0e5)[0]
    q2 = model.coupled_injection_rate(case, bp, cw, p + 2.0e5)[0]
    assert q1 > 0 and q2 == pytest.approx(2 * q1, rel=1e-12)


def test_injector_border_blocks_match_finite_differences():
    case = inp.with_coupled_injector(inp.small_box(4, 3, 2), inp.CTRL_TOTAL_RATE, 0.01, 5.4e6)
    u, c = sim.initial_state(case)
    bhp = np.array([5.4e6])
    acc = model.old_accumulation(case, u, c)
    B, C, D, Fw = model.coupled_blocks(case, u, bhp, c, acc, 100.0)
    cw = model.coupled_wells(case)[0]
    h = 1.0e3        # the rate is linear in bhp while the well flows: the difference is exact but for rounding
    Fp = model.residual(case, u, c, acc, 100.0, bhp=bhp + h)
    Fm = model.residual(case, u, c, acc, 100.0, bhp=bhp - h)
    np.testing.assert_allclose(B, ((Fp - Fm) / (2 * h))[:, cw.cells].T, rtol=1e-6, atol=1e-12 * np.abs(B).max())
    assert np.all(B[:, :6] <= 0.0)       # more pressure, more injection: the sources grow
    D_fd = (model.well_equations(case, u, bhp + h) - model.well_equations(case, u, bhp - h)) / (2 * h)
    assert D[0] > 0 and D[0] == pytest.approx(D_fd[0], rel=1e-6)


def test_rate_control_is_met_on_a_3d_box():
    """Two perforations 1 m apart: the bottom-hole pressure found by Newton
    meets the total rate, and the deeper perforation, whose cell pressure
    includes the gas head, takes the smaller share (not ignited, as above)."""
    base = inp.small_box(4, 3, 2)
    base.ignited = np.array([], np.int32)
    u0, c0 = sim.initial_state(base)
    b0 = 5.0e6 + 1.0e3
    case = inp.with_coupled_injector(base, inp.CTRL_TOTAL_RATE, 0.005, b0)
    opts = sim.NewtonOptions(tol=1e-10, maxit=40)
    u, b, c, its, ok = sim.timestep_coupled(case, u0, np.array([b0]), c0, 60.0, opts)
    assert ok and its >= 2
    bp = model.base_properties(case, u)
    cw = model.coupled_wells(case)[0]
    Q = model.coupled_injection_rate(case, bp, cw, b[0])
    assert np.sum(Q) == pytest.approx(0.005, rel=1e-8)
    assert case.depth[cw.cells[1]] > case.depth[cw.cells[0]] and 0.0 < Q[1] < Q[0]
