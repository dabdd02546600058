"""Oracle: properties, residual and Jacobian of the discrete ISC model.

Test infrastructure only (see ``oracle/__init__``).

Primary unknowns per cell (Tab:nco&ncg with x_HO eliminated by the oil
constraint and C_c eliminated by the coke equation):

    u = (p, x_LO, y_O2, y_N2, y_CO2, T, S_w, S_g)

Equation rows per cell: mass of W, LO, HO, O2, N2, CO2, energy, and the gas
composition constraint F_GS = sum_c y_c - 1 (Sec. 3.1).

Every function accepts complex arrays so that the Jacobian can be taken by
complex-step differentiation: all branch decisions look at real parts.
"""
from __future__ import annotations

import numpy as np

R_GAS = 8.314462618
OMEGA_A = 0.427480      # Redlich-Kwong A coefficient (Sec. 2.2, Z factor)
OMEGA_B = 0.086640      # Redlich-Kwong B coefficient
W, LO, HO, O2, N2, CO2 = range(6)
NU = 8


def _re(z):
    return np.real(z)


def _where(cond, a, b):
    return np.where(cond, a, b)


# ---------------------------------------------------------------- properties
def k_value(fl, c, p, T):
    """K = (kv1/p + kv2 p + kv3) exp(kv4/(T - kv5)) (Sec. 2.2, Phase Equilibrium)."""
    kv = fl["kv"][c]
    return (kv[0] / p + kv[1] * p + kv[2]) * np.exp(kv[3] / (T - kv[4]))


def per_factor(s, eps):
    """PER correction s/(s+eps) (Sec. 2.2, eq. PER1/PER2; eps replaces the
    printed n_cg in the water formula, see the text that follows it)."""
    return s / (s + eps)


def gas_fractions(fl, p, T, x_lo, y_o2, y_n2, y_co2, Sw, So):
    """Gas mole fractions y_c (Tab4.4 with the modified PER of eq. PER1/PER2):
    y_W = f(S_w) K_W (pure water phase), y_LO = K_LO x_LO (no correction),
    y_HO = f(S_o) K_HO x_HO (correction on the heaviest oil component only)."""
    eps = fl["per_eps"]
    x_ho = 1.0 - x_lo
    yW = per_factor(Sw, eps) * k_value(fl, W, p, T)
    yLO = k_value(fl, LO, p, T) * x_lo
    yHO = per_factor(So, eps) * k_value(fl, HO, p, T) * x_ho
    return [yW, yLO, yHO, y_o2, y_n2, y_co2]


def cubic_largest_real_root(a1, a0):
    """Largest real root of Z^3 - Z^2 + a1 Z + a0 = 0 for real coefficients
    (trigonometric form for three real roots, Cardano otherwise), then two
    Newton polishes."""
    a2 = -1.0
    pp = a1 - a2 * a2 / 3.0
    qq = 2.0 * a2 ** 3 / 27.0 - a2 * a1 / 3.0 + a0
    disc = (qq / 2.0) ** 2 + (pp / 3.0) ** 3
    z = np.empty_like(a1)
    three = disc < 0
    if np.any(three):
        m = 2.0 * np.sqrt(-pp[three] / 3.0)
        arg = np.clip(3.0 * qq[three] / (pp[three] * m), -1.0, 1.0)
        z[three] = m * np.cos(np.arccos(arg) / 3.0)
    one = ~three
    if np.any(one):
        sd = np.sqrt(disc[one])
        z[one] = np.cbrt(-qq[one] / 2.0 + sd) + np.cbrt(-qq[one] / 2.0 - sd)
    z = z - a2 / 3.0
    for _ in range(2):
        f = ((z - 1.0) * z + a1) * z + a0
        df = (3.0 * z - 2.0) * z + a1
        z = z - f / df
    return z


def z_factor(fl, p, T, y):
    """Redlich-Kwong compressibility factor with the mixing rule of Sec. 2.2.

    The printed mixing parameter a is dimensionally garbled; it is read as the
    standard RK rule a = sum y_i Tc_i^(5/4)/sqrt(pc_i), which makes
    Tc = (a^2/b)^(2/3) and pc = Tc/b reproduce a single component's critical
    point. The largest real root of the cubic is taken.
    """
    Tc, pc = fl["Tc"], fl["pc"]
    a = sum(y[c] * Tc[c] ** 1.25 / np.sqrt(pc[c]) for c in range(6))
    b = sum(y[c] * Tc[c] / pc[c] for c in range(6))
    Tcm = (a * a / b) ** (2.0 / 3.0)
    pcm = Tcm / b
    A = OMEGA_A * (p / pcm) * (Tcm / T) ** 2.5
    B = OMEGA_B * (p / pcm) * (Tcm / T)
    a1 = A - B - B * B
    a0 = -A * B
    z = cubic_largest_real_root(_re(a1).astype(np.float64), _re(a0).astype(np.float64)).astype(a1.dtype)
    if np.iscomplexobj(a1):
        for _ in range(3):   # Newton on the complex-perturbed cubic carries the derivative
            f = ((z - 1.0) * z + a1) * z + a0
            df = (3.0 * z - 2.0) * z + a1
            z = z - f / df
    return z


def liquid_density(fl, c, p, T):
    """rho = rho_ref exp(cp dp - ct1 dT - ct2/2 dT^2 + cpt dp dT) (Sec. 2.2, Density)."""
    dp = p - fl["p_ref"]
    dT = T - fl["T_ref"]
    return fl["rho_ref"][c] * np.exp(fl["cp"][c] * dp - fl["ct1"][c] * dT
                                     - 0.5 * fl["ct2"][c] * dT * dT + fl["cpt"][c] * dp * dT)


def gas_enthalpy_component(fl, c, T):
    """H_g,c = integral from T_ref to T of the cpg polynomial (Sec. 2.2)."""
    Tr = fl["T_ref"]
    cpg = fl["cpg"][c]
    return sum(cpg[k] / (k + 1) * (T ** (k + 1) - Tr ** (k + 1)) for k in range(4))


def vaporisation_enthalpy(fl, c, T):
    """H_v,c = u(Tc - T) hvr (Tc - T)^ev (Sec. 2.2), Heaviside on the real part."""
    d = fl["Tc"][c] - T
    pos = _re(d) > 0
    dsafe = _where(pos, d, 1.0)
    return _where(pos, fl["hvr"][c] * dsafe ** fl["ev"][c], 0.0 * d)


def corey_unit(s):
    """clamp(s, 0, 1) with zero derivative outside (0, 1)."""
    rs = _re(s)
    return _where(rs <= 0.0, 0.0 * s, _where(rs >= 1.0, 1.0 + 0.0 * s, s))


def rel_perms(fl, Sw, Sg):
    """Corey curves (exponent 2) for the two-phase tables and Stone's model II
    for k_ro (Sec. 2.2, Relative Permeabilities), with k_rocw = k_row(Swc) = 1."""
    Swc, Sorw, Sgc, Sorg = fl["Swc"], fl["Sorw"], fl["Sgc"], fl["Sorg"]
    krw = corey_unit((Sw - Swc) / (1.0 - Swc - Sorw)) ** 2
    krow = corey_unit((1.0 - Sw - Sorw) / (1.0 - Swc - Sorw)) ** 2
    krg = corey_unit((Sg - Sgc) / (1.0 - Swc - Sgc)) ** 2
    krog = corey_unit((1.0 - Sg - Swc - Sorg) / (1.0 - Swc - Sorg)) ** 2
    krocw = 1.0
    kro = krocw * ((krow / krocw + krw) * (krog / krocw + krg) - krw - krg)
    kro = _where(_re(kro) < 0.0, 0.0 * kro, kro)
    return krw, kro, krg


def base_properties(case, u):
    """Everything that depends on u alone (not on coke): Sec. 2.2."""
    fl = case.fluid
    rock = case.rock
    p, x_lo, y_o2, y_n2, y_co2, T, Sw, Sg = (u[k] for k in range(NU))
    So = 1.0 - Sw - Sg
    x_ho = 1.0 - x_lo
    y = gas_fractions(fl, p, T, x_lo, y_o2, y_n2, y_co2, Sw, So)
    Z = z_factor(fl, p, T, y)
    rho_g = p / (Z * R_GAS * T)
    rho_w = liquid_density(fl, W, p, T)
    rho_lo = liquid_density(fl, LO, p, T)
    rho_ho = liquid_density(fl, HO, p, T)
    rho_o = 1.0 / (x_lo / rho_lo + x_ho / rho_ho)
    M = fl["M"]
    mu_w = fl["avisc"][W] * np.exp(fl["bvisc"][W] / T)
    mu_lo = fl["avisc"][LO] * np.exp(fl["bvisc"][LO] / T)
    mu_ho = fl["avisc"][HO] * np.exp(fl["bvisc"][HO] / T)
    mu_o = np.exp(x_lo * np.log(mu_lo) + x_ho * np.log(mu_ho))   # log mixing (product form)
    sqM = np.sqrt(M)
    num = sum(fl["avg"][c] * T ** fl["bvg"][c] * y[c] * sqM[c] for c in range(6))
    den = sum(y[c] * sqM[c] for c in range(6))
    mu_g = num / den
    krw, kro, krg = rel_perms(fl, Sw, Sg)
    Hg_c = [gas_enthalpy_component(fl, c, T) for c in range(6)]
    Hl_c = [Hg_c[c] - vaporisation_enthalpy(fl, c, T) for c in range(3)]
    H_w = Hl_c[W]
    H_o = x_lo * Hl_c[LO] + x_ho * Hl_c[HO]
    H_g = sum(y[c] * Hg_c[c] for c in range(6))
    U_w = H_w - p / rho_w
    U_o = H_o - p / rho_o
    U_g = H_g - p / rho_g
    dpr = p - rock["p_ref"]
    dTr = T - rock["T_ref"]
    phi = case.phi_ref * (1.0 + rock["cpor"] * dpr - rock["ctpor"] * dTr + rock["cptpor"] * dpr * dTr)
    U_r = rock["cv1"] * dTr + 0.5 * rock["cv2"] * (T * T - rock["T_ref"] ** 2)
    U_c = fl["coke_cp"] * (T - fl["T_ref"])
    g = fl["gravity"]
    gam_w = rho_w * M[W] * g
    gam_o = rho_o * (x_lo * M[LO] + x_ho * M[HO]) * g
    gam_g = rho_g * sum(y[c] * M[c] for c in range(6)) * g
    return dict(p=p, T=T, Sw=Sw, So=So, Sg=Sg, x_lo=x_lo, x_ho=x_ho, y=y, Z=Z,
                rho_w=rho_w, rho_o=rho_o, rho_g=rho_g, mu_w=mu_w, mu_o=mu_o, mu_g=mu_g,
                krw=krw, kro=kro, krg=krg, H_w=H_w, H_o=H_o, H_g=H_g, Hg_c=Hg_c,
                U_w=U_w, U_o=U_o, U_g=U_g, U_r=U_r, U_c=U_c, phi=phi,
                gam=(gam_w, gam_o, gam_g),
                lam=(rho_w * krw / mu_w, rho_o * kro / mu_o, rho_g * krg / mu_g))


def reaction_rates(case, bp, coke):
    """Arrhenius rates r_R (Sec. 2.2, Reaction Model), mol/(m3 bulk s).

    Oil concentrations use the fluid porosity phi_f = phi - C_c/rho_coke
    (Sec. 2.2, Porosity); the gas pressure is p (capillary pressure zero).
    """
    rx = case.reactions
    fl = case.fluid
    T, p = bp["T"], bp["p"]
    phi_f = bp["phi"] - coke / fl["coke_rho"]
    oil_conc = [phi_f * bp["So"] * bp["rho_o"] * bp["x_lo"], phi_f * bp["So"] * bp["rho_o"] * bp["x_ho"]]
    pO2 = bp["y"][O2] * p
    rates = []
    for r in range(rx["nr"]):
        k = rx["A"][r] * np.exp(-rx["Ea"][r] / (R_GAS * T))
        kind = rx["kind"][r]
        if kind == 0:
            rates.append(k * pO2 * oil_conc[rx["comp"][r] - 1])
        elif kind == 1:
            rates.append(k * oil_conc[rx["comp"][r] - 1] * (1.0 - (coke / rx["coke_max"]) ** 5))
        else:
            rates.append(k * pO2 * coke)
    return rates


def solve_coke(case, bp, coke_old, dt, tol=1e-14, maxit=60):
    """Coke conservation dC_c/dt = q_coke,reac by backward Euler (Sec. 3.1,
    F_Coke), solved per cell: g(C) = C - C^n - dt sum_R s_coke,R r_R(C) = 0.

    g is increasing in C wherever the rates are physical, so Newton from
    C^n converges; the derivative dg/dC is written out here. With complex u
    the iteration continues until the imaginary part has converged too.
    """
    rx = case.reactions
    fl = case.fluid
    s_c = rx["stoich"][:, 6]
    C = np.asarray(coke_old, dtype=bp["p"].dtype).copy()
    T, p = bp["T"], bp["p"]
    base_oil = bp["So"] * bp["rho_o"]
    xs = [bp["x_lo"], bp["x_ho"]]
    pO2 = bp["y"][O2] * p
    for it in range(maxit):
        phi_f = bp["phi"] - C / fl["coke_rho"]
        g = C - coke_old
        dg = np.ones_like(C)
        for r in range(rx["nr"]):
            if s_c[r] == 0.0:
                continue
            k = rx["A"][r] * np.exp(-rx["Ea"][r] / (R_GAS * T))
            kind = rx["kind"][r]
            if kind == 0:
                conc = phi_f * base_oil * xs[rx["comp"][r] - 1]
                rate = k * pO2 * conc
                drate = k * pO2 * (-1.0 / fl["coke_rho"]) * base_oil * xs[rx["comp"][r] - 1]
            elif kind == 1:
                cm = rx["coke_max"]
                conc = phi_f * base_oil * xs[rx["comp"][r] - 1]
                lim = 1.0 - (C / cm) ** 5
                rate = k * conc * lim
                drate = k * ((-1.0 / fl["coke_rho"]) * base_oil * xs[rx["comp"][r] - 1] * lim
                             + conc * (-5.0 * C ** 4 / cm ** 5))
            else:
                rate = k * pO2 * C
                drate = k * pO2
            g = g - dt * s_c[r] * rate
            dg = dg - dt * s_c[r] * drate
        step = g / dg
        C = C - step
        scale = np.abs(_re(C)) + np.abs(_re(coke_old)) + 1e-300
        if np.all(np.abs(_re(step)) <= tol * scale) and (
                not np.iscomplexobj(C) or it > 3 and np.all(np.abs(np.imag(step)) <= tol * (np.abs(np.imag(C)) + 1e-300))):
            return C
    return C


def accumulation(case, bp, coke):
    """Moles per bulk volume N_c (c = W..CO2) and energy per bulk volume E
    (the accumulation terms of F_W, F_O[i], F_G[i] and F_E in Sec. 3.1)."""
    fl = case.fluid
    phi_f = bp["phi"] - coke / fl["coke_rho"]
    y = bp["y"]
    gas = bp["rho_g"] * bp["Sg"]
    oil = bp["rho_o"] * bp["So"]
    N = [phi_f * (bp["rho_w"] * bp["Sw"] + gas * y[W]),
         phi_f * (oil * bp["x_lo"] + gas * y[LO]),
         phi_f * (oil * bp["x_ho"] + gas * y[HO]),
         phi_f * gas * y[O2], phi_f * gas * y[N2], phi_f * gas * y[CO2]]
    E = (phi_f * (bp["rho_w"] * bp["Sw"] * bp["U_w"] + oil * bp["U_o"] + gas * bp["U_g"])
         + (1.0 - bp["phi"]) * bp["U_r"] + coke * bp["U_c"])
    return N + [E]


def thermal_conductivity(case, bp, coke):
    """K_T = phi_f (S_w K_w + S_o K_o + S_g K_g) + (1 - phi) K_r + C_c K_c (Sec. 2.1)."""
    fl = case.fluid
    Kp = fl["K_phase"]
    phi_f = bp["phi"] - coke / fl["coke_rho"]
    return phi_f * (bp["Sw"] * Kp[0] + bp["So"] * Kp[1] + bp["Sg"] * Kp[2]) + (1.0 - bp["phi"]) * case.rock["K_rock"] + coke * fl["coke_K"]


def injected_enthalpy(fl, w):
    """Molar enthalpy of an injected stream at T_inj: a gas stream carries
    sum_c y_c H_g,c; a liquid-water stream carries H_w = H_g,W - H_v,W."""
    T = np.float64(w.inj_T)
    if w.inj_phase == 0:
        return w.inj_y[W] * (gas_enthalpy_component(fl, W, T) - vaporisation_enthalpy(fl, W, np.array([T]))[0])
    return sum(w.inj_y[c] * gas_enthalpy_component(fl, c, T) for c in range(6))


# ------------------------------------------------------------------ geometry
def faces(case):
    """Interior faces (lo, hi, T_face, Gamma_face, z_lo - z_hi).

    T_face is the harmonic average of (A k/h) of the two cells (Sec. 3.1);
    Gamma_face = (A/h)_avg for conduction.
    """
    nx, ny, nz = case.nx, case.ny, case.nz
    idx = np.arange(case.n).reshape(nz, ny, nx)
    out = []
    specs = ((0, case.dy * case.dz, case.dx, idx[:, :, :-1], idx[:, :, 1:]),
             (1, case.dx * case.dz, case.dy, idx[:, :-1, :], idx[:, 1:, :]),
             (2, case.dx * case.dy, case.dz, idx[:-1, :, :], idx[1:, :, :]))
    for d, area, h, a, b in specs:
        lo = a.reshape(-1)
        hi = b.reshape(-1)
        if lo.size == 0:
            continue
        t_lo = area * case.perm[d, lo] / h
        t_hi = area * case.perm[d, hi] / h
        T = 2.0 * t_lo * t_hi / (t_lo + t_hi)
        gam = np.full(lo.size, area / h)
        out.append((lo, hi, T, gam))
    if not out:   # a single cell has no interior faces
        e = np.zeros(0, dtype=np.int64)
        return e, e, np.zeros(0), np.zeros(0), np.zeros(0)
    lo = np.concatenate([o[0] for o in out])
    hi = np.concatenate([o[1] for o in out])
    T = np.concatenate([o[2] for o in out])
    G = np.concatenate([o[3] for o in out])
    dz = case.depth[lo] - case.depth[hi]
    return lo, hi, T, G, dz


def cell_volume(case):
    return case.dx * case.dy * case.dz


# ------------------------------------------------------------------ residual
def old_accumulation(case, u_old, coke_old):
    """Accumulation of the accepted state (N^n, E^n): shape (7, N)."""
    bp = base_properties(case, u_old)
    return np.array(accumulation(case, bp, coke_old))


def coupled_wells(case):
    """The coupled wells (bottom-hole pressure unknown: producers, kind 2, and
    injectors, kind 3), in case order."""
    return [w for w in case.wells if w.kind in (2, 3)]


def coupled_phase_rates(case, bp, w, bhp):
    """Peaceman phase rates (Sec. 2.2, Well Modeling) of a coupled producer's
    perforations, positive into the reservoir:
        Q_alpha = WI lambda_alpha (bhp - p - gamma_alpha (z_bh - z))
    with gamma_alpha the phase's specific weight in the perforated cell
    (gravity included) and z depth; outflow only (a perforation whose driving
    difference is positive does not inject). Returns the three (nperf,) arrays."""
    c = w.cells
    p = bp["p"][c]
    out = []
    for a in range(3):
        dphi = bhp - p - bp["gam"][a][c] * (w.ref_depth - case.depth[c])
        out.append(_where(_re(dphi) < 0.0, w.WI * bp["lam"][a][c] * dphi, 0.0 * dphi))
    return out


def coupled_injection_rate(case, bp, w, bhp):
    """Molar rate (mol/s, into the reservoir) of the injected stream at each
    perforation of a coupled injector (Sec. 2.2, Well Modeling, for injection).
    Reading: Peaceman's formula with the perforated cell's total molar
    mobility, Q = WI sum_alpha(rho_alpha k_r,alpha / mu_alpha)
    (bhp - p - gamma (z_bh - z)), gamma the specific weight of the injected
    phase (gas, or water for inj_phase 0) in the cell; inflow only (no
    back-flow into the well). Returns an (nperf,) array."""
    c = w.cells
    lam_t = bp["lam"][0][c] + bp["lam"][1][c] + bp["lam"][2][c]
    gam = bp["gam"][0 if w.inj_phase == 0 else 2][c]
    dphi = bhp - bp["p"][c] - gam * (w.ref_depth - case.depth[c])
    return _where(_re(dphi) > 0.0, w.WI * lam_t * dphi, 0.0 * dphi)


def well_equations(case, u, bhp):
    """Well equations of the coupled wells (Sec. 2.2): bhp - c for a fixed
    bottom-hole pressure; for a producer the summed production rate (mol/s,
    positive out of the reservoir) of the controlled phases minus c; for an
    injector the total injected molar rate minus c."""
    bp = base_properties(case, u)
    F = []
    for k, w in enumerate(coupled_wells(case)):
        if w.control == 0:
            F.append(bhp[k] - w.target)
            continue
        if w.kind == 3:
            F.append(np.sum(coupled_injection_rate(case, bp, w, bhp[k])) - w.target)
            continue
        Q = coupled_phase_rates(case, bp, w, bhp[k])
        rate = sum(-np.sum(Q[a]) for a in range(3) if w.control & (1 << a))
        F.append(rate - w.target)
    return np.array(F, dtype=np.result_type(u, np.asarray(bhp)))


def residual(case, u, coke_old, acc_old, dt, geom=None, return_coke=False, bhp=None):
    """Discrete residual F (8, N) of Sec. 3.1 at unknowns u (8, N).

    Sign convention (the printed flux sign is inverted relative to its own
    Delta-Phi definition; this is the outflow-positive reading):
        F_c = V/dt (N_c - N_c^n) + sum_faces T lam_up xi_up dPhi - Q_c,well - V q_c,reac
        F_E = V/dt (E - E^n) + sum_faces (T lam_up H_up dPhi + G K_T,harm dT)
              - Q_E,well - V Q_reac
        F_GS = sum_c y_c - 1
    dPhi over face (lo, hi) = p_lo - p_hi - gamma_avg (z_lo - z_hi), gamma_avg
    the arithmetic mean of the two cells; upstream = lo if dPhi >= 0 else hi.
    Each face is evaluated once and added to lo, subtracted from hi.
    """
    if geom is None:
        geom = faces(case)
    lo, hi, Tf, Gf, dzf = geom
    V = cell_volume(case)
    bp = base_properties(case, u)
    coke = solve_coke(case, bp, coke_old, dt)
    acc = accumulation(case, bp, coke)
    n = case.n
    F = np.zeros((NU, n), dtype=u.dtype)
    for r in range(7):
        F[r] = V / dt * (acc[r] - acc_old[r])
    y = bp["y"]
    carried = (  # per phase: [(row, quantity)], energy carried by enthalpy
        [(W, 1.0)],
        [(LO, bp["x_lo"]), (HO, bp["x_ho"])],
        [(c, y[c]) for c in range(6)],
    )
    H = (bp["H_w"], bp["H_o"], bp["H_g"])
    p = bp["p"]
    for a in range(3):
        gam = bp["gam"][a]
        dphi = (p[lo] - p[hi]) - 0.5 * (gam[lo] + gam[hi]) * dzf
        up = _where(_re(dphi) >= 0.0, lo, hi)
        lam = bp["lam"][a]
        for (row, xi) in carried[a]:
            q = lam * xi if not np.isscalar(xi) else lam * xi
            flux = Tf * q[up] * dphi
            np.add.at(F[row], lo, flux)
            np.add.at(F[row], hi, -flux)
        fluxE = Tf * (lam * H[a])[up] * dphi
        np.add.at(F[6], lo, fluxE)
        np.add.at(F[6], hi, -fluxE)
    KT = thermal_conductivity(case, bp, coke)
    Kh = 2.0 * KT[lo] * KT[hi] / (KT[lo] + KT[hi])
    cond = Gf * Kh * (bp["T"][lo] - bp["T"][hi])
    np.add.at(F[6], lo, cond)
    np.add.at(F[6], hi, -cond)
    # wells (Peaceman, Sec. 2.2 Well Modeling)
    for w in case.wells:
        cells = w.cells
        if w.kind == 0:   # fixed-rate injector: constant source
            share = w.WI / np.sum(w.WI)
            Hinj = injected_enthalpy(case.fluid, w)
            for c in range(6):
                F[c, cells] -= share * w.target * w.inj_y[c]
            F[6, cells] -= share * w.target * Hinj
        elif w.kind == 3:  # coupled injector: the injected stream at a rate set by the bottom-hole pressure
            k = next(i for i, cw in enumerate(coupled_wells(case)) if cw is w)
            Q = coupled_injection_rate(case, bp, w, bhp[k])
            Hinj = injected_enthalpy(case.fluid, w)
            for c in range(6):
                F[c, cells] -= Q * w.inj_y[c]
            F[6, cells] -= Q * Hinj
        elif w.kind == 2:  # coupled producer: the bottom-hole pressure is an unknown
            k = next(i for i, cw in enumerate(coupled_wells(case)) if cw is w)
            Q = coupled_phase_rates(case, bp, w, bhp[k])
            xi = ([1.0], [bp["x_lo"][cells], bp["x_ho"][cells]], [y[c][cells] for c in range(6)])
            rows = ([W], [LO, HO], list(range(6)))
            for a in range(3):
                for row, x in zip(rows[a], xi[a]):
                    F[row, cells] -= Q[a] * x
                F[6, cells] -= Q[a] * H[a][cells]
        else:             # fixed-BHP producer, outflow only
            dp = w.target - p[cells]
            open_ = _re(dp) < 0.0
            xi = ([1.0], [bp["x_lo"][cells], bp["x_ho"][cells]], [y[c][cells] for c in range(6)])
            rows = ([W], [LO, HO], list(range(6)))
            for a in range(3):
                Q = _where(open_, w.WI * bp["lam"][a][cells] * dp, 0.0 * dp)
                for row, x in zip(rows[a], xi[a]):
                    F[row, cells] -= Q * x
                F[6, cells] -= Q * H[a][cells]
    # reactions (q_c,reac = sum_R s_cR r_R, Q_reac = sum_R H_R r_R)
    rates = reaction_rates(case, bp, coke)
    st = case.reactions["stoich"]
    for r, rate in enumerate(rates):
        for c in range(6):
            if st[r, c] != 0.0:
                F[c] -= V * st[r, c] * rate
        F[6] -= V * case.reactions["dH"][r] * rate
    F[6] += heat_loss(case, bp["T"])
    F[7] = sum(y) - 1.0
    if return_coke:
        return F, coke
    return F


def heat_loss(case, T):
    """Heat lost to the overburden and underburden (Sec. 2.1, last term of the
    energy equation; + V Q_loss in the discrete energy residual of Sec. 3.1).
    Reading: the loss leaves through the horizontal face (area A = dx dy) of
    every cell of the top layer (k = 0) and / or the bottom layer (k = nz - 1)
    by conduction, K_ob ((T(ob) - T_ini)/d - rho) per unit area, into a
    confining layer of thickness d whose far side stays at the initial
    temperature T_ini; T(ob), the temperature at the interface, is the cell's
    temperature and rho the fitted offset (K/m). Returns W per cell (N,)."""
    hl = getattr(case, "heat_loss", None)
    if not hl:
        return np.zeros(case.n, dtype=T.dtype)
    k = np.arange(case.n) // (case.nx * case.ny)
    nfaces = ((k == 0) & bool(hl["faces"] & 1)).astype(float) + ((k == case.nz - 1) & bool(hl["faces"] & 2))
    return nfaces * (case.dx * case.dy * hl["K_ob"]) * ((T - hl["T_ini"]) / hl["d"] - hl["rho"])


# ------------------------------------------------------------------ Jacobian
def bsr_pattern(case):
    """Block-sparse pattern of the 7-point stencil, columns sorted per row."""
    nx, ny, nz = case.nx, case.ny, case.nz
    n = case.n
    rowptr = [0]
    col = []
    for c in range(n):
        i = c % nx
        j = (c // nx) % ny
        k = c // (nx * ny)
        nb = []
        if k > 0:
            nb.append(c - nx * ny)
        if j > 0:
            nb.append(c - nx)
        if i > 0:
            nb.append(c - 1)
        nb.append(c)
        if i < nx - 1:
            nb.append(c + 1)
        if j < ny - 1:
            nb.append(c + nx)
        if k < nz - 1:
            nb.append(c + nx * ny)
        col.extend(nb)
        rowptr.append(len(col))
    return np.array(rowptr, dtype=np.int64), np.array(col, dtype=np.int64)


def stencil_colouring(case):
    """Colour classes such that every 7-point stencil holds at most one cell of
    each colour: colour = (sum_d m_d i_d) mod (2D + 1) over the D grid axes of
    length > 1, with multipliers m = 1, 2, 3."""
    n = case.n
    ijk = (np.arange(n) % case.nx, (np.arange(n) // case.nx) % case.ny, np.arange(n) // (case.nx * case.ny))
    dims = [d for d, m in enumerate((case.nx, case.ny, case.nz)) if m > 1]
    color = np.zeros(n, dtype=np.int64)
    for m, d in enumerate(dims):
        color += (m + 1) * ijk[d]
    ncolor = 2 * len(dims) + 1
    return color % ncolor, ncolor


def jacobian(case, u, coke_old, acc_old, dt, h=1e-30, geom=None, bhp=None):
    """Exact Jacobian dF/du in BSR form (rowptr, col, val[nnzb, 8, 8]) with
    val[b][r][k] = dF_r(row cell)/du_k(col cell) (the coupled producers'
    bottom-hole pressures held at bhp).

    Computed by complex-step differentiation of ``residual`` (derivative
    accurate to rounding, no subtraction error), with the cells split into
    colour classes (``stencil_colouring``) so that each 7-point stencil holds
    at most one perturbed cell.
    """
    if geom is None:
        geom = faces(case)
    rowptr, col = bsr_pattern(case)
    n = case.n
    color, ncolor = stencil_colouring(case)
    rows = np.repeat(np.arange(n), np.diff(rowptr))
    val = np.zeros((col.size, NU, NU))
    for c in range(ncolor):
        sel = color == c
        if not np.any(sel):
            continue
        blocks = color[col] == c
        for k in range(NU):
            uc = u.astype(np.complex128)
            uc[k, sel] += 1j * h
            F = residual(case, uc, coke_old, acc_old, dt, geom, bhp=bhp)
            dF = np.imag(F) / h
            val[blocks, :, k] = dF[:, rows[blocks]].T
    return rowptr, col, val


def coupled_blocks(case, u, bhp, coke_old, acc_old, dt, h=1e-30, geom=None):
    """The border of the Newton system of the coupled producers (Sec. 2.2,
    Well Modeling: the bottom-hole pressure becomes an unknown), by complex
    step. For the perforations of the coupled wells in case order:
        B[q] = dF(cell of q)/d bhp(well of q)       (8,)
        C[q] = dF_w(well of q)/d u(cell of q)       (8,)
    and per coupled well D[w] = dF_w/d bhp_w, Fw = the well equations."""
    if geom is None:
        geom = faces(case)
    wells = coupled_wells(case)
    bhp = np.asarray(bhp, dtype=float)
    B, C = [], []
    D = np.zeros(len(wells))
    for k, w in enumerate(wells):
        bc = bhp.astype(np.complex128)
        bc[k] += 1j * h
        dF = np.imag(residual(case, u.astype(np.complex128), coke_old, acc_old, dt, geom, bhp=bc)) / h
        D[k] = np.imag(well_equations(case, u.astype(np.complex128), bc)[k]) / h
        for c in w.cells:
            B.append(dF[:, c].copy())
            row = np.zeros(NU)
            for j in range(NU):
                uc = u.astype(np.complex128)
                uc[j, c] += 1j * h
                row[j] = np.imag(well_equations(case, uc, bhp.astype(np.complex128))[k]) / h
            C.append(row)
    Fw = np.real(well_equations(case, u, bhp))
    return np.array(B).reshape(-1, NU), np.array(C).reshape(-1, NU), D, Fw


def residual_fd_jacobian(case, u, coke_old, acc_old, dt, rel=1e-7, geom=None):
    """Central finite-difference Jacobian (the paper's numerical Jacobian),
    same BSR layout, perturbation h = rel * max(|u|, u_scale)."""
    if geom is None:
        geom = faces(case)
    rowptr, col = bsr_pattern(case)
    n = case.n
    color, ncolor = stencil_colouring(case)
    rows = np.repeat(np.arange(n), np.diff(rowptr))
    scale = np.array([1e6, 1.0, 1.0, 1.0, 1.0, 100.0, 1.0, 1.0])
    val = np.zeros((col.size, NU, NU))
    for c in range(ncolor):
        sel = color == c
        if not np.any(sel):
            continue
        blocks = color[col] == c
        for k in range(NU):
            hk = rel * np.maximum(np.abs(u[k, sel]), scale[k])
            up = u.copy()
            um = u.copy()
            up[k, sel] += hk
            um[k, sel] -= hk
            hfull = np.zeros(n)
            hfull[sel] = hk
            dF = (residual(case, up, coke_old, acc_old, dt, geom) - residual(case, um, coke_old, acc_old, dt, geom))
            hb = hfull[col[blocks]]
            val[blocks, :, k] = dF[:, rows[blocks]].T / (2.0 * hb[:, None])
    return rowptr, col, val
