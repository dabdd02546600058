"""Pins of the oracle's heat loss to the overburden and underburden (Sec. 2.1,
the last term of the energy equation; + V Q_loss in the discrete energy
residual of Sec. 3.1). Reading: conduction A K_ob ((T - T_ini)/d - rho)
through the horizontal face of each top- and / or bottom-layer cell.

The expected numbers are worked by hand for the HEAT_LOSS data of the inputs
(K_ob = 1.7 W/m/K, d = 10 m, T_ini = 300 K, rho = 0) on 10 m x 10 m cells:
the face area is 100 m^2, so a face conducts 100 * 1.7 / 10 = 17 W per kelvin
of excess temperature."""
import numpy as np

import isc_inputs as inp
from oracle import model, sim


def _residual_pair(case, u, coke, acc_old, dt=100.0):
    off = model.residual(case, u, coke, acc_old, dt)
    on = model.residual(inp.with_heat_loss(case), u, coke, acc_old, dt)
    return off, on


def _state_at(case, T):
    u, c = sim.initial_state(case)
    u = u.copy()
    u[5] = T
    return u, c


def test_one_layer_cell_loses_through_both_faces_by_hand():
    # nz = 1: every cell is both top and bottom layer; at 400 K each face conducts
    # 17 W/K * 100 K = 1700 W, so the energy residual grows by 3400 W
    case = inp.small_box(3, 2, 1)
    u, c = _state_at(case, 400.0)
    acc_old = model.old_accumulation(case, u, c)
    off, on = _residual_pair(case, u, c, acc_old)
    assert np.allclose(on[6] - off[6], 3400.0, rtol=1e-13)
    assert np.array_equal(on[:6], off[:6]) and np.array_equal(on[7], off[7])


def test_only_the_boundary_layers_lose_heat():
    case = inp.small_box(3, 2, 3)
    u, c = _state_at(case, 350.0)                  # 50 K above T_ini: 850 W per face
    acc_old = model.old_accumulation(case, u, c)
    off, on = _residual_pair(case, u, c, acc_old)
    layer = np.arange(case.n) // (case.nx * case.ny)
    d = on[6] - off[6]
    assert np.allclose(d[layer == 0], 850.0, rtol=1e-13)
    assert np.allclose(d[layer == 2], 850.0, rtol=1e-13)
    assert np.all(d[layer == 1] == 0.0)
    # the top face only
    top = model.residual(inp.with_heat_loss(case, faces=1), u, c, acc_old, 100.0)
    d1 = top[6] - off[6]
    assert np.allclose(d1[layer == 0], 850.0, rtol=1e-13) and np.all(d1[layer > 0] == 0.0)


def test_no_loss_at_the_initial_temperature_and_the_offset_shifts_it():
    case = inp.small_box(2, 2, 1)
    u, c = _state_at(case, 300.0)
    acc_old = model.old_accumulation(case, u, c)
    off, on = _residual_pair(case, u, c, acc_old)
    assert np.array_equal(on, off)
    # rho = 2 K/m: the loss is A K_ob (0 - 2) = -340 W per face (a gain), 2 faces
    shifted = model.residual(inp.with_heat_loss(case, rho=2.0), u, c, acc_old, 100.0)
    assert np.allclose(shifted[6] - off[6], -680.0, rtol=1e-13)


def test_jacobian_gains_exactly_the_conductance_in_the_temperature_column():
    # d(loss)/dT = 17 W/K per face; nothing else in the Jacobian moves
    case = inp.small_box(3, 2, 2)
    st = inp.random_state(case, 77)
    u0, c0 = sim.initial_state(case)
    acc_old = model.old_accumulation(case, u0, c0)
    rp, col, J0 = model.jacobian(case, st["u"], st["coke"], acc_old, 100.0)
    _, _, J1 = model.jacobian(inp.with_heat_loss(case), st["u"], st["coke"], acc_old, 100.0)
    diff = J1 - J0
    rows = np.repeat(np.arange(case.n), np.diff(rp))
    diag = col == rows
    # every cell here is in a boundary layer; the difference of two Jacobians carries
    # the rounding of the entry itself (the stored-energy term, ~1e5 W/K)
    big = np.abs(J0[diag][:, 6, 5])
    assert np.all(np.abs(diff[diag][:, 6, 5] - 17.0) <= 1e-12 * big + 1e-12 * 17.0)
    diff[np.nonzero(diag)[0], 6, 5] = 0.0
    assert np.max(np.abs(diff)) <= 1e-12 * np.max(np.abs(J0))


def test_energy_balance_of_a_closed_box_includes_the_loss():
    # fluxes telescope: summed over the cells, the energy residual is the stored
    # energy change minus the sources plus the total loss (no wells, no reactions)
    case = inp.with_heat_loss(inp.small_box(3, 3, 2))
    case.wells = []
    rx = dict(case.reactions)
    rx["A"] = np.zeros_like(rx["A"])
    case.reactions = rx
    st = inp.random_state(case, 78)
    u0, c0 = sim.initial_state(case)
    acc_old = model.old_accumulation(case, u0, c0)
    dt = 100.0
    F, coke = model.residual(case, st["u"], c0, acc_old, dt, return_coke=True)
    bp = model.base_properties(case, st["u"])
    acc = np.array(model.accumulation(case, bp, coke))
    V = model.cell_volume(case)
    loss = model.heat_loss(case, st["u"][5])
    expect = (V / dt * (acc[6] - acc_old[6])).sum() + loss.sum()
    assert abs(F[6].sum() - expect) <= 1e-12 * np.abs(F[6]).sum()
