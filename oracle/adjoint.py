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

With coupled producers (Sec. 2.2, Well Modeling: the bottom-hole pressures
are unknowns with their own well equations F_w) the state is (u, bhp), J_n is
the bordered matrix [[J, B], [C, D]] of the converged step, the well equations
join the residual, and P adds the coupled producers' oil (``*_coupled``).
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


# ------------------------------------------------------------ coupled producers
def coupled_oil_rate(case, u, bhp):
    """Oil mass produced per second (LO + HO in the oil and gas phases) at the
    coupled producers, from their Peaceman phase rates at bottom-hole pressure
    bhp (Sec. 2.2, Well Modeling; outflow only)."""
    bp = model.base_properties(case, u)
    M = case.fluid["M"]
    total = 0.0
    for k, w in enumerate(model.coupled_wells(case)):
        if w.kind != 2:      # injectors produce no oil
            continue
        c = w.cells
        Q = model.coupled_phase_rates(case, bp, w, bhp[k])
        mo = M[1] * bp["x_lo"][c] + M[2] * bp["x_ho"][c]
        mg = M[1] * bp["y"][1][c] + M[2] * bp["y"][2][c]
        total = total + np.sum(-(Q[1] * mo + Q[2] * mg))
    return total


def trajectory_coupled(case, dts, tol=1e-11, maxit=40):
    """Converged states (u^n, bhp^n, C^n), n = 0..N, of the implicit-Euler loop
    with coupled producers (bordered Newton, dense solves)."""
    opts = sim.NewtonOptions(tol=tol, maxit=maxit)
    geom = model.faces(case)
    u, c = sim.initial_state(case)
    b = np.array([w.bhp_init for w in model.coupled_wells(case)], dtype=float)
    us, bs, cs = [u], [b], [c]
    for dt in dts:
        un, bn, cn, its, ok = sim.timestep_coupled(case, u, b, c, dt, opts, geom)
        if not ok:
            raise RuntimeError("oracle time step did not converge")
        u, b, c = un, bn, cn
        us.append(u)
        bs.append(b)
        cs.append(c)
    return us, bs, cs


def loss_coupled(case, dts, us, bs):
    return float(sum(dt * (np.real(oil_production_rate(case, u)) + np.real(coupled_oil_rate(case, u, b)))
                     for dt, u, b in zip(dts, us[1:], bs[1:])))


def _bordered(case, J, B, C, D):
    n, nw = case.n, len(D)
    A = np.zeros((8 * n + nw, 8 * n + nw))
    A[:8 * n, :8 * n] = J
    q = 0
    for k, w in enumerate(model.coupled_wells(case)):
        for cell in w.cells:
            A[8 * cell:8 * cell + 8, 8 * n + k] = B[q]
            A[8 * n + k, 8 * cell:8 * cell + 8] = C[q]
            q += 1
        A[8 * n + k, 8 * n + k] = D[k]
    return A


def tangent_coupled(case, dts, us, bs, cs, v_lnk, v_Ea, v_lnA):
    """dL/dtheta . v of the loop with coupled producers by the forward tangent
    model: per step the bordered system
        [[J, B], [C, D]] (du^n, dbhp^n) = -(dR^n, dF_w^n)/d(u^{n-1}, C^{n-1}, theta) . (du^{n-1}, dC^{n-1}, v)
    then dC^n from the coke solve and dL += dt_n dP/d(u^n, bhp^n, theta)."""
    from . import linalg
    rx = case.reactions
    lnk_c = 1j * H * np.asarray(v_lnk, dtype=float)
    Ea_c = rx["Ea"] + 1j * H * np.asarray(v_Ea, dtype=float)
    lnA_c = np.log(rx["A"]) + 1j * H * np.asarray(v_lnA, dtype=float)
    case_c = param_case(case, lnk_c, Ea_c, lnA_c)
    geom_c = model.faces(case_c)
    geom = model.faces(case)
    n = case.n
    du = np.zeros_like(us[0])
    db = np.zeros_like(bs[0])
    dc = np.zeros_like(cs[0])
    dL = 0.0
    for s, dt in enumerate(dts, start=1):
        u_old_c = us[s - 1] + 1j * H * du
        c_old_c = cs[s - 1] + 1j * H * dc
        acc_old_c = model.old_accumulation(case_c, u_old_c, c_old_c)
        R = model.residual(case_c, us[s].astype(complex), c_old_c, acc_old_c, dt, geom_c, bhp=bs[s].astype(complex))
        Fw = model.well_equations(case_c, us[s].astype(complex), bs[s].astype(complex))
        rhs = np.concatenate([(np.imag(R) / H).T.reshape(-1), np.imag(Fw) / H])
        acc_old = model.old_accumulation(case, us[s - 1], cs[s - 1])
        rp, col, val = model.jacobian(case, us[s], cs[s - 1], acc_old, dt, geom=geom, bhp=bs[s])
        B, C, D, _ = model.coupled_blocks(case, us[s], bs[s], cs[s - 1], acc_old, dt, geom=geom)
        A = _bordered(case, linalg.bsr_to_dense(rp, col, val), B, C, D)
        x = -np.linalg.solve(A, rhs)
        du = x[:8 * n].reshape(n, 8).T
        db = x[8 * n:]
        u_c = us[s] + 1j * H * du
        b_c = bs[s] + 1j * H * db
        bp = model.base_properties(case_c, u_c)
        dc = np.imag(model.solve_coke(case_c, bp, c_old_c, dt)) / H
        dL += dt * (np.imag(oil_production_rate(case_c, u_c)) + np.imag(coupled_oil_rate(case_c, u_c, b_c))) / H
    return float(dL)
