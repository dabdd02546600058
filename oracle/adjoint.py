"""Oracle: sensitivities of the cumulative oil production of a time loop.

Test infrastructure only (see ``oracle/__init__``).

Parameters theta = (ln k multiplier of every cell (applied to k_x, k_y, k_z),
Ea_R, ln A_R of every reaction). Loss L = sum_n dt_n P(u^n) with P the oil mass
produced per second (LO + HO in any phase) at the BHP producers.

``tangent`` is the forward (tangent-linear) model of the implicit-Euler loop,
an algorithm independent of a reverse adjoint: per step n

    du^n = -J_n^-1 (dR^n/d(u^{n-1}, C^{n-1}, theta) . (du^{n-1}, dC^{n-1}, v))
    dC^n = dPhi/d(u^n, C^{n-1}, theta) . (du^n, dC^{n-1}, v)
    dL  += dt_n dP/d(u^n, theta) . (du^n, v)

where the directional derivatives of the residual R^n, of the per-cell coke
solve Phi and of P are taken by complex-step differentiation and J_n is the
exact Jacobian of the converged step.
"""
from __future__ import annotations

import copy

import numpy as np

from . import model, sim

H = 1e-30


def param_case(case, lnk=None, Ea=None, lnA=None):
    """A copy of case with cell permeabilities and well indices scaled by
    exp(lnk) and the reactions' Ea, A replaced (values may be complex)."""
    c = copy.copy(case)
    c.reactions = dict(case.reactions)
    if lnk is not None:
        f = np.exp(lnk)
        c.perm = case.perm * f[None, :]
        wells = []
        for w in case.wells:
            nw = copy.copy(w)
            nw.WI = w.WI * f[w.cells]
            wells.append(nw)
        c.wells = wells
    if Ea is not None:
        c.reactions["Ea"] = Ea
    if lnA is not None:
        c.reactions["A"] = np.exp(lnA)
    return c


def oil_production_rate(case, u):
    """Oil mass produced per second (LO + HO in the oil and gas phases) at the
    BHP producers (Peaceman rates of Sec. 2.2, outflow only)."""
    bp = model.base_properties(case, u)
    M = case.fluid["M"]
    total = 0.0
    for w in case.wells:
        if w.kind != 1:
            continue
        c = w.cells
        dp = w.target - bp["p"][c]
        open_ = np.real(dp) < 0.0
        Qo = np.where(open_, w.WI * bp["lam"][1][c] * dp, 0.0 * dp)
        Qg = np.where(open_, w.WI * bp["lam"][2][c] * dp, 0.0 * dp)
        mo = M[1] * bp["x_lo"][c] + M[2] * bp["x_ho"][c]
        mg = M[1] * bp["y"][1][c] + M[2] * bp["y"][2][c]
        total = total + np.sum(-(Qo * mo + Qg * mg))
    return total


def trajectory(case, dts, tol=1e-11, maxit=40):
    """Converged states (u^n, C^n), n = 0..N, of the implicit-Euler loop with
    the given step sizes (dense linear solves)."""
    opts = sim.NewtonOptions(tol=tol, maxit=maxit)
    opts.solve.solver = "dense"
    geom = model.faces(case)
    u, c = sim.initial_state(case)
    us, cs = [u], [c]
    for dt in dts:
        un, cn, its, ok = sim.timestep(case, u, c, dt, opts, geom)
        if not ok:
            raise RuntimeError("oracle time step did not converge")
        u, c = un, cn
        us.append(u)
        cs.append(c)
    return us, cs


def loss(case, dts, us):
    return float(sum(dt * np.real(oil_production_rate(case, u)) for dt, u in zip(dts, us[1:])))


def tangent(case, dts, us, cs, v_lnk, v_Ea, v_lnA):
    """dL/dtheta . v by the forward tangent model (see the module docstring)."""
    rx = case.reactions
    lnk_c = 1j * H * np.asarray(v_lnk, dtype=float)
    Ea_c = rx["Ea"] + 1j * H * np.asarray(v_Ea, dtype=float)
    lnA_c = np.log(rx["A"]) + 1j * H * np.asarray(v_lnA, dtype=float)
    case_c = param_case(case, lnk_c, Ea_c, lnA_c)
    geom_c = model.faces(case_c)
    geom = model.faces(case)
    du = np.zeros_like(us[0])
    dc = np.zeros_like(cs[0])
    dL = 0.0
    for n, dt in enumerate(dts, start=1):
        u_old_c = us[n - 1] + 1j * H * du
        c_old_c = cs[n - 1] + 1j * H * dc
        acc_old_c = model.old_accumulation(case_c, u_old_c, c_old_c)
        R = model.residual(case_c, us[n].astype(complex), c_old_c, acc_old_c, dt, geom_c)
        rhs = np.imag(R) / H
        acc_old = model.old_accumulation(case, us[n - 1], cs[n - 1])
        rp, col, val = model.jacobian(case, us[n], cs[n - 1], acc_old, dt, geom=geom)
        from . import linalg
        A = linalg.bsr_to_dense(rp, col, val)
        du = -np.linalg.solve(A, rhs.T.reshape(-1)).reshape(case.n, 8).T
        u_c = us[n] + 1j * H * du
        bp = model.base_properties(case_c, u_c)
        dc = np.imag(model.solve_coke(case_c, bp, c_old_c, dt)) / H
        dL += dt * np.imag(oil_production_rate(case_c, u_c)) / H
    return float(dL)
