"""Pins of the oracle's residual and Jacobian (Sec. 3.1): conservation by
telescoping fluxes, reaction mass balance, and the analytical Jacobian
against the paper's numerical (finite-difference) Jacobian."""
import numpy as np
import pytest

import isc_inputs as inp
from oracle import model, sim

SCALE = np.array([1e6, 1, 1, 1, 1, 100.0, 1, 1])


def _state(case, seed):
    st = inp.random_state(case, seed)
    u0, c0 = sim.initial_state(case)
    acc_old = model.old_accumulation(case, u0, c0)
    return st["u"], st["coke"], acc_old


@pytest.mark.parametrize("mk", [lambda: inp.tube_case(n_cells=12), lambda: inp.small_box(4, 3, 2)])
def test_fluxes_telescope_global_balance(mk):
    # summed over all cells, the flux terms cancel: sum F = accumulation - sources
    case = mk()
    u, coke_old, acc_old = _state(case, 11)
    dt = 50.0
    F, coke = model.residual(case, u, coke_old, acc_old, dt, return_coke=True)
    bp = model.base_properties(case, u)
    acc = np.array(model.accumulation(case, bp, coke))
    V = model.cell_volume(case)
    rates = model.reaction_rates(case, bp, coke)
    st = case.reactions["stoich"]
    src = np.zeros((7, case.n))
    for r, rate in enumerate(rates):
        src[:6] += V * st[r, :6, None] * rate
        src[6] += V * case.reactions["dH"][r] * rate
    for w in case.wells:
        if w.kind == 0:
            share = w.WI / w.WI.sum()
            Hinj = model.injected_enthalpy(case.fluid, w)
            src[:6, w.cells] += share * w.target * w.inj_y[:, None]
            src[6, w.cells] += share * w.target * Hinj
        else:
            dp = w.target - bp["p"][w.cells]
            open_ = dp < 0
            for a, (rows, xs) in enumerate((([0], [np.ones(len(w.cells))]),
                                            ([1, 2], [bp["x_lo"][w.cells], bp["x_ho"][w.cells]]),
                                            (list(range(6)), [bp["y"][c][w.cells] for c in range(6)]))):
                Q = np.where(open_, w.WI * bp["lam"][a][w.cells] * dp, 0.0)
                for row, x in zip(rows, xs):
                    src[row, w.cells] += Q * x
                src[6, w.cells] += Q * (bp["H_w"], bp["H_o"], bp["H_g"])[a][w.cells]
    expect = (V / dt * (acc - acc_old) - src).sum(axis=1)
    got = F[:7].sum(axis=1)
    scale = np.abs(F[:7]).sum(axis=1)
    assert np.all(np.abs(got - expect) <= 1e-12 * scale)


def test_single_face_flux_is_antisymmetric():
    case = inp.tube_case(n_cells=2)
    u, coke_old, acc_old = _state(case, 12)
    case.wells = []
    case.reactions["A"] = np.zeros(4)
    dt = 10.0
    F = model.residual(case, u, coke_old, acc_old, dt)
    V = model.cell_volume(case)
    bp = model.base_properties(case, u)
    acc = np.array(model.accumulation(case, bp, coke_old))
    flux = F[:7] - V / dt * (acc - acc_old)
    assert np.all(np.abs(flux[:, 0] + flux[:, 1]) <= 1e-13 * np.abs(flux[:, 0]))


def test_reactions_conserve_mass_per_cell():
    case = inp.tube_case()
    u, coke_old, _ = _state(case, 13)
    u[5] = np.linspace(400, 900, case.n)
    bp = model.base_properties(case, u)
    rates = model.reaction_rates(case, bp, coke_old + 100.0)
    M = np.concatenate([case.fluid["M"], [case.fluid["coke_M"]]])
    st = case.reactions["stoich"]
    mass = sum(st[r] @ M * rates[r] for r in range(4))
    scale = sum(np.abs(st[r]) @ M * np.abs(rates[r]) for r in range(4))
    assert np.all(np.abs(mass) <= 1e-13 * scale)


def test_initial_state_satisfies_gas_constraint_away_from_ignition():
    case = inp.small_box(4, 3, 2)
    u, coke = sim.initial_state(case)
    F = model.residual(case, u, coke, model.old_accumulation(case, u, coke), 10.0)
    cold = np.setdiff1d(np.arange(case.n), case.ignited)
    assert np.max(np.abs(F[7, cold])) < 1e-15


def _scaled_rel_err(J, Jref, rowptr):
    n = len(rowptr) - 1
    Js = J * SCALE[None, None, :]
    Jr = Jref * SCALE[None, None, :]
    rows = np.repeat(np.arange(n), np.diff(rowptr))
    rowmax = np.zeros((n, 8))
    np.maximum.at(rowmax, rows, np.abs(Jr).max(axis=2))
    return np.abs(Js - Jr) / rowmax[rows][:, :, None]


@pytest.mark.parametrize("mk,seed", [(lambda: inp.tube_case(n_cells=12), 21), (lambda: inp.small_box(4, 3, 2), 22)])
def test_analytical_jacobian_matches_numerical_jacobian(mk, seed):
    case = mk()
    u, coke_old, acc_old = _state(case, seed)
    u[5] = np.clip(u[5], 300, 560)     # away from the water/light-oil critical points
    dt = 100.0
    rp, col, J = model.jacobian(case, u, coke_old, acc_old, dt)
    rp2, col2, Jfd = model.residual_fd_jacobian(case, u, coke_old, acc_old, dt, rel=1e-6)
    assert np.array_equal(rp, rp2) and np.array_equal(col, col2)
    err = _scaled_rel_err(J, Jfd, rp)
    assert err.max() < 1e-6


def test_jacobian_directional_derivative():
    case = inp.small_box(3, 3, 2)
    u, coke_old, acc_old = _state(case, 23)
    dt = 30.0
    rp, col, J = model.jacobian(case, u, coke_old, acc_old, dt)
    rng = np.random.default_rng(0)
    v = rng.standard_normal(u.shape) * SCALE[:, None]
    Jv = np.zeros_like(u)
    for r in range(case.n):
        for b in range(rp[r], rp[r + 1]):
            Jv[:, r] += J[b] @ v[:, col[b]]
    h = 1e-6
    fd = (model.residual(case, u + h * v, coke_old, acc_old, dt) - model.residual(case, u - h * v, coke_old, acc_old, dt)) / (2 * h)
    scale = np.abs(Jv).max(axis=1, keepdims=True)
    assert np.max(np.abs(Jv - fd) / scale) < 1e-6
