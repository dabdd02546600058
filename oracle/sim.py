"""Oracle: Newton linearise-decouple-solve-update step and time stepping.

Test infrastructure only (see ``oracle/__init__``).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import linalg, model

NU = 8


def initial_state(case):
    """Initial state recipe: uniform p, T, S_w, S_o, S_g and x_LO; the gas holds
    y_W = f(S_w) K_W, y_LO = K_LO x_LO, y_HO = f(S_o) K_HO x_HO (Tab4.4 with
    the PER of eq. PER1/PER2) and the remainder split over O2:N2:CO2 by the
    given ratios; cells listed as ignited start at T_ignite; C_c = 0.
    Returns (u (8, N), coke (N,))."""
    ini = case.init
    n = case.n
    p = np.full(n, ini["p"])
    T = np.full(n, ini["T"])
    Sw = np.full(n, ini["Sw"])
    Sg = np.full(n, ini["Sg"])
    So = 1.0 - Sw - Sg
    x_lo = np.full(n, ini["x_LO"])
    fl = case.fluid
    zero = np.zeros(n)
    y = model.gas_fractions(fl, p, T, x_lo, zero, zero, zero, Sw, So)
    rest = 1.0 - (y[0] + y[1] + y[2])
    u = np.empty((NU, n))
    u[0] = p
    u[1] = x_lo
    for g in range(3):
        u[2 + g] = ini["y_rest"][g] * rest
    u[5] = T
    u[5, case.ignited] = ini["T_ignite"]
    u[6] = Sw
    u[7] = Sg
    return u, np.zeros(n)


def convergence_norms(case, F, u, coke):
    """Scaled max-norms of the residual rows:
    mass rows |F_c| dt/(V N_tot) are returned WITHOUT the dt factor here and
    scaled by the caller: e_mass = max |F_c| / (V N_tot / dt);
    energy |F_E| / (V cv_rock * 1 K / dt); constraint |F_GS| raw."""
    V = model.cell_volume(case)
    bp = model.base_properties(case, u)
    acc = model.accumulation(case, bp, coke)
    ntot = np.abs(acc[0]) + np.abs(acc[1]) + np.abs(acc[2]) + np.abs(acc[3]) + np.abs(acc[4]) + np.abs(acc[5])
    e_mass = float(np.max(np.abs(F[:6]) / (V * ntot)))
    e_energy = float(np.max(np.abs(F[6]) / (V * case.rock["cv1"])))
    e_gs = float(np.max(np.abs(F[7])))
    return e_mass, e_energy, e_gs


def apply_update(u, du, max_dp_frac=0.2, max_dT=50.0):
    """u + du with the safeguards: |dp| <= 0.2 p, |dT| <= 50 K; a saturation or
    mole fraction that would turn negative is halved instead (the 0.5 S rule
    of Sec. 2.2, Phase Equilibrium); the same rule on S_o = 1 - S_w - S_g
    scales S_w and S_g so that S_o halves."""
    un = np.empty_like(u)
    p = u[0]
    un[0] = p + np.clip(du[0], -max_dp_frac * p, max_dp_frac * p)
    un[5] = u[5] + np.clip(du[5], -max_dT, max_dT)
    x = u[1] + du[1]
    x = np.where(x < 0.0, 0.5 * u[1], x)
    x = np.where(x > 1.0, 1.0 - 0.5 * (1.0 - u[1]), x)
    un[1] = x
    for k in (2, 3, 4, 6, 7):
        v = u[k] + du[k]
        un[k] = np.where(v < 0.0, 0.5 * u[k], v)
    so_old = 1.0 - u[6] - u[7]
    so_new = 1.0 - un[6] - un[7]
    bad = so_new < 0.0
    if np.any(bad):
        target = 1.0 - 0.5 * so_old[bad]
        s = un[6, bad] + un[7, bad]
        un[6, bad] *= target / s
        un[7, bad] *= target / s
    return un


@dataclass
class SolveOptions:
    solver: str = "gmres"        # "gmres", "bicgstab", "dense"
    prec: str = "ilu0"           # "ilu0", "bjacobi", "none"
    decouple: bool = True
    restart: int = 30
    rtol: float = 1e-8
    maxit: int = 1000


@dataclass
class NewtonOptions:
    tol: float = 1e-6
    maxit: int = 25
    solve: SolveOptions = field(default_factory=SolveOptions)


def linear_solve(rowptr, col, val, rhs, opts: SolveOptions):
    """Solve J du = rhs (rhs (N, 8) block-major). With decoupling the system is
    first left-scaled by C_L via Gauss-Jordan (Sec. 3.2)."""
    if opts.decouple:
        val, rhs = linalg.gauss_jordan_decouple(rowptr, col, val, rhs)
    if opts.solver == "dense":
        A = linalg.bsr_to_dense(rowptr, col, val)
        x = np.linalg.solve(A, rhs.reshape(-1)).reshape(rhs.shape)
        return x, 0, 0.0
    A = linalg.bsr_to_scipy(rowptr, col, val)
    mv = lambda v: (A @ v.reshape(-1)).reshape(v.shape)
    if opts.prec == "ilu0":
        M = linalg.ILU0Preconditioner(rowptr, col, val)
    elif opts.prec == "bjacobi":
        M = linalg.BlockJacobiPreconditioner(rowptr, col, val)
    else:
        M = linalg.IdentityPreconditioner()
    if opts.solver == "gmres":
        return linalg.gmres(mv, rhs, M, opts.restart, opts.rtol, opts.maxit)
    return linalg.bicgstab(mv, rhs, M, opts.rtol, opts.maxit)


def newton_step(case, u, coke_old, acc_old, dt, opts: NewtonOptions, geom=None):
    """One Newton linearise-and-solve step: residual and Jacobian (Sec. 3.1),
    convergence test, Gauss-Jordan decoupling (Sec. 3.2), preconditioned Krylov
    solve of J du = -F, safeguarded update. Returns a dict."""
    if geom is None:
        geom = model.faces(case)
    F, coke = model.residual(case, u, coke_old, acc_old, dt, geom, return_coke=True)
    e = convergence_norms(case, F, u, coke)
    norm = max(e[0] * dt, e[1] * dt, e[2])
    if norm <= opts.tol:
        return dict(u=u, coke=coke, converged=True, norm=norm, norms=e, F=F, its=0)
    rowptr, col, val = model.jacobian(case, u, coke_old, acc_old, dt, geom=geom)
    rhs = -F.T.copy()
    du, its, rel = linear_solve(rowptr, col, val, rhs, opts.solve)
    un = apply_update(u, du.T)
    return dict(u=un, du=du.T, coke=coke, converged=False, norm=norm, norms=e, F=F, its=its, rel=rel)


def timestep(case, u, coke, dt, opts: NewtonOptions, geom=None):
    """Implicit-Euler step t -> t + dt (Sec. 3.1): Newton until the scaled
    residual is below tol. Returns (u, coke, newton_iterations, ok)."""
    if geom is None:
        geom = model.faces(case)
    acc_old = model.old_accumulation(case, u, coke)
    un = u.copy()
    for it in range(opts.maxit + 1):
        r = newton_step(case, un, coke, acc_old, dt, opts, geom)
        if r["converged"]:
            return r["u"], r["coke"], it, True
        un = r["u"]
        if not np.all(np.isfinite(un)):
            break
    return u, coke, opts.maxit, False


def well_norms(case, Fw):
    """Scaled well-equation residuals: |F_w| / |c| with c the well's target
    (Pa for a fixed bottom-hole pressure, mol/s for a fixed rate)."""
    return [abs(float(f)) / abs(w.target) for f, w in zip(Fw, model.coupled_wells(case))]


def newton_step_coupled(case, u, bhp, coke_old, acc_old, dt, opts: NewtonOptions, geom=None):
    """Newton step with coupled producers (Sec. 2.2, Well Modeling): unknowns
    (u, bhp), equations (F, F_w); the bordered system
        [ J  B ] [du  ]     [F  ]
        [ C  D ] [dbhp] = - [F_w]
    is solved densely (small cases). bhp takes the pressure safeguard
    |dbhp| <= max_dp_frac bhp. Returns a dict like newton_step plus bhp."""
    if geom is None:
        geom = model.faces(case)
    bhp = np.asarray(bhp, dtype=float)
    F, coke = model.residual(case, u, coke_old, acc_old, dt, geom, return_coke=True, bhp=bhp)
    e = convergence_norms(case, F, u, coke)
    Fw = np.real(model.well_equations(case, u, bhp))
    ew = well_norms(case, Fw)
    norm = max([e[0] * dt, e[1] * dt, e[2]] + ew)
    if norm <= opts.tol:
        return dict(u=u, bhp=bhp, coke=coke, converged=True, norm=norm, norms=e, F=F, Fw=Fw, its=0)
    rowptr, col, val = model.jacobian(case, u, coke_old, acc_old, dt, geom=geom, bhp=bhp)
    B, C, D, _ = model.coupled_blocks(case, u, bhp, coke_old, acc_old, dt, geom=geom)
    n, nw = case.n, len(bhp)
    A = np.zeros((8 * n + nw, 8 * n + nw))
    A[:8 * n, :8 * n] = linalg.bsr_to_dense(rowptr, col, val)
    q = 0
    for k, w in enumerate(model.coupled_wells(case)):
        for c in w.cells:
            A[8 * c:8 * c + 8, 8 * n + k] = B[q]
            A[8 * n + k, 8 * c:8 * c + 8] = C[q]
            q += 1
        A[8 * n + k, 8 * n + k] = D[k]
    rhs = -np.concatenate([F.T.reshape(-1), Fw])
    x = np.linalg.solve(A, rhs)
    du = x[:8 * n].reshape(n, 8).T
    dbhp = np.clip(x[8 * n:], -0.2 * bhp, 0.2 * bhp)
    un = apply_update(u, du)
    return dict(u=un, bhp=bhp + dbhp, du=du, dbhp=x[8 * n:], coke=coke, converged=False, norm=norm, norms=e,
                F=F, Fw=Fw, its=0)


def timestep_coupled(case, u, bhp, coke, dt, opts: NewtonOptions, geom=None):
    """Implicit-Euler step with coupled producers. Returns (u, bhp, coke, its, ok)."""
    if geom is None:
        geom = model.faces(case)
    acc_old = model.old_accumulation(case, u, coke)
    un, bn = u.copy(), np.asarray(bhp, dtype=float).copy()
    for it in range(opts.maxit + 1):
        r = newton_step_coupled(case, un, bn, coke, acc_old, dt, opts, geom)
        if r["converged"]:
            return r["u"], r["bhp"], r["coke"], it, True
        un, bn = r["u"], r["bhp"]
        if not (np.all(np.isfinite(un)) and np.all(np.isfinite(bn))):
            break
    return u, bhp, coke, opts.maxit, False


def next_dt(dt, u_old, u_new, dt_max, dT_target=20.0, dS_target=0.2):
    dT = float(np.max(np.abs(u_new[5] - u_old[5])))
    dS = float(max(np.max(np.abs(u_new[6] - u_old[6])), np.max(np.abs(u_new[7] - u_old[7]))))
    f = min(dT_target / max(dT, 1e-12), dS_target / max(dS, 1e-12))
    return min(dt * min(max(f, 0.5), 2.0), dt_max)


def run(case, t_end, dt0, dt_max, opts: NewtonOptions, max_cuts=8, max_steps=100000, dts=None):
    """Time loop with the deterministic controller; with ``dts`` given the
    accepted step sizes are replayed instead. Returns (u, coke, accepted dts,
    stats); stats["its_per_step"] holds the Newton solves of each accepted step."""
    geom = model.faces(case)
    u, coke = initial_state(case)
    t = 0.0
    dt = dt0
    accepted = []
    its_per_step = []
    newton_total = 0
    cuts = 0
    steps = 0
    while t < t_end * (1 - 1e-12) and steps < max_steps:
        if dts is not None:
            if steps >= len(dts):
                break
            dt = dts[steps]
        dt = min(dt, t_end - t) if dts is None else dt
        for c in range(max_cuts + 1):
            un, cn, its, ok = timestep(case, u, coke, dt, opts, geom)
            newton_total += its
            if ok:
                break
            if dts is not None:
                raise RuntimeError(f"replayed step {steps} (dt={dt}) did not converge")
            cuts += 1
            dt *= 0.5
        if not ok:
            raise RuntimeError(f"time step failed after {max_cuts} cuts at t={t}")
        accepted.append(dt)
        its_per_step.append(its)
        t += dt
        steps += 1
        nd = next_dt(dt, u, un, dt_max)
        u, coke = un, cn
        dt = nd
    return u, coke, accepted, dict(newton=newton_total, cuts=cuts, steps=steps, t=t, its_per_step=its_per_step)
