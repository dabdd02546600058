"""Pins of the oracle's property correlations (Sec. 2.2) against values the
paper prints, textbook physics, closed forms and library routines."""
import json
import os

import numpy as np
import pytest

import isc_inputs as inp
from oracle import model

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "printed_values.json")))
FL = inp.tube_fluid()


def test_water_k_value_is_one_at_boiling_point():
    g = GOLD["water_K_at_boiling"]
    K = model.k_value(FL, inp.W, g["p_psi"] * inp.PSI, inp.degF_to_K(g["T_F"]))
    assert abs(K - g["K"]) <= g["rtol"]


def test_k_value_field_units_match_si_conversion():
    # the correlation in the paper's own units (psi, F) against the SI form
    for c in range(3):
        kv1 = [1.7202e6, 1.4546e5, 2.7454e5][c]
        kv4 = [-6869.59, -4458.73, -8424.83][c]
        kv5 = [-376.64, -387.78, -205.69][c]
        for p_psi, T_F in ((100.0, 150.0), (725.2, 300.0), (2014.7, 700.0)):
            K_field = kv1 / p_psi * np.exp(kv4 / (T_F - kv5))
            K_si = model.k_value(FL, c, p_psi * inp.PSI, inp.degF_to_K(T_F))
            assert K_si == pytest.approx(K_field, rel=1e-12)


def test_oil_viscosity_at_initial_temperature():
    g = GOLD["oil_viscosity_initial"]
    T = inp.degF_to_K(g["T_F"])
    for c in (inp.LO, inp.HO):
        mu = FL["avisc"][c] * np.exp(FL["bvisc"][c] / T) / inp.CP
        assert mu == pytest.approx(g["mu_cp"], rel=g["rtol"])
    # the oil-phase mixture of two equal-viscosity components keeps that value
    case = inp.tube_case()
    u = np.array([[5e6], [0.744], [0.2], [0.7], [0.0], [T], [0.3], [0.1]])
    bp = model.base_properties(case, u)
    assert bp["mu_o"][0] / inp.CP == pytest.approx(g["mu_cp"], rel=g["rtol"])


def test_water_latent_heat_matches_steam_tables():
    g = GOLD["water_latent_heat_212F"]
    Hv = model.vaporisation_enthalpy(FL, inp.W, np.array([inp.degF_to_K(g["T_F"])]))[0]
    assert Hv / inp.BTU_PER_LBMOL == pytest.approx(g["Hv_btu_per_lbmol"], rel=g["rtol"])
    # Heaviside: no latent heat above the critical temperature
    assert model.vaporisation_enthalpy(FL, inp.W, np.array([FL["Tc"][0] + 1.0]))[0] == 0.0


def test_gas_enthalpy_derivative_is_heat_capacity():
    g = GOLD["steam_cp_100F"]
    T = inp.degF_to_K(g["T_F"])
    h = 1e-3
    cp = (model.gas_enthalpy_component(FL, inp.W, T + h) - model.gas_enthalpy_component(FL, inp.W, T - h)) / (2 * h)
    assert cp / (inp.BTU_PER_LBMOL * 1.8) == pytest.approx(g["cp_btu_per_lbmol_F"], rel=g["rtol"])
    assert model.gas_enthalpy_component(FL, inp.W, FL["T_ref"]) == 0.0


def test_gas_viscosity_nitrogen():
    g = GOLD["nitrogen_viscosity_100F"]
    T = inp.degF_to_K(g["T_F"])
    mu = FL["avg"][inp.N2] * T ** FL["bvg"][inp.N2] / inp.CP
    assert mu == pytest.approx(g["mu_cp"], rel=g["rtol"])


def test_per_factor_values():
    eps = FL["per_eps"]
    assert model.per_factor(GOLD["per_half_at_eps"]["s_over_eps"] * eps, eps) == pytest.approx(GOLD["per_half_at_eps"]["f"], rel=1e-15)
    d = np.imag(model.per_factor(1e-30j, eps)) / 1e-30
    assert d * eps == pytest.approx(GOLD["per_slope_at_zero"]["fprime_times_eps"], rel=1e-14)


def test_printed_stoichiometry_nearly_conserves_mass():
    g = GOLD["tube_stoichiometry_printed"]
    for row in g["reactions"]:
        imb = sum(v * g["M"][k] for k, v in row.items())
        scale = sum(abs(v) * g["M"][k] for k, v in row.items()) / 2
        assert abs(imb) / scale <= g["max_rel_imbalance"]


def test_build_stoichiometry_conserves_mass_exactly():
    rx = inp.tube_reactions()
    M = np.concatenate([FL["M"], [FL["coke_M"]]])
    NM = rx["stoich"] @ M
    assert np.all(np.abs(NM) <= 1e-14 * np.abs(rx["stoich"]) @ M)


@pytest.mark.parametrize("c", range(6))
def test_rk_mixing_single_component_reproduces_critical_point(c):
    # with a pure component the mixing rule must give back its own Tc and pc
    Tc, pc = FL["Tc"], FL["pc"]
    a = Tc[c] ** 1.25 / np.sqrt(pc[c])
    b = Tc[c] / pc[c]
    Tcm = (a * a / b) ** (2.0 / 3.0)
    assert Tcm == pytest.approx(Tc[c], rel=1e-13)
    assert Tcm / b == pytest.approx(pc[c], rel=1e-13)
    # and the Z factor equals the pure-component RK root from np.roots
    y = [np.zeros(1) for _ in range(6)]
    y[c] = np.ones(1)
    p, T = np.array([3e6]), np.array([500.0])
    Z = model.z_factor(FL, p, T, y)[0]
    A = 0.42748 * (p[0] / pc[c]) * (Tc[c] / T[0]) ** 2.5
    B = 0.08664 * (p[0] / pc[c]) * (Tc[c] / T[0])
    roots = np.roots([1.0, -1.0, A - B - B * B, -A * B])
    zr = max(r.real for r in roots if abs(r.imag) < 1e-9 * abs(r))
    assert Z == pytest.approx(zr, rel=1e-12)


def test_z_factor_ideal_gas_limit_and_cubic_residual():
    rng = np.random.default_rng(3)
    n = 400
    y = [rng.uniform(0.0, 1.0, n) for _ in range(6)]
    s = sum(y)
    y = [v / s for v in y]
    T = rng.uniform(280.0, 900.0, n)
    p = np.full(n, 1.0)
    assert np.all(np.abs(model.z_factor(FL, p, T, y) - 1.0) < 1e-5)
    p = rng.uniform(1e5, 2e7, n)
    Z = model.z_factor(FL, p, T, y)
    # recompute A, B from the mixing rule and check the cubic and the root choice
    Tc, pc = FL["Tc"], FL["pc"]
    a = sum(y[c] * Tc[c] ** 1.25 / np.sqrt(pc[c]) for c in range(6))
    b = sum(y[c] * Tc[c] / pc[c] for c in range(6))
    Tcm = (a * a / b) ** (2 / 3)
    A = 0.42748 * p / (Tcm / b) * (Tcm / T) ** 2.5
    B = 0.08664 * p / (Tcm / b) * (Tcm / T)
    res = Z ** 3 - Z ** 2 + (A - B - B * B) * Z - A * B
    assert np.max(np.abs(res)) < 1e-13
    for i in range(0, n, 7):
        roots = np.roots([1.0, -1.0, A[i] - B[i] - B[i] ** 2, -A[i] * B[i]])
        zr = max(r.real for r in roots if abs(r.imag) <= 1e-7 * max(1.0, abs(r)))
        assert Z[i] == pytest.approx(zr, rel=1e-9)


def test_liquid_density_reference_and_oil_harmonic_mixing():
    p, T = np.array([FL["p_ref"]]), np.array([FL["T_ref"]])
    for c in range(3):
        assert model.liquid_density(FL, c, p, T)[0] == FL["rho_ref"][c]
    case = inp.tube_case()
    u = np.array([[FL["p_ref"]], [0.3], [0.2], [0.7], [0.0], [FL["T_ref"]], [0.3], [0.1]])
    bp = model.base_properties(case, u)
    v = 0.3 / FL["rho_ref"][1] + 0.7 / FL["rho_ref"][2]
    assert bp["rho_o"][0] == pytest.approx(1.0 / v, rel=1e-14)


def test_stone2_reduces_to_two_phase_curves():
    # no gas: k_ro equals k_row; water at connate: k_ro equals k_rog
    Sw = np.linspace(0.15, 0.8, 27)
    krw, kro, krg = model.rel_perms(FL, Sw, np.zeros_like(Sw))
    krow = np.clip((1 - Sw - FL["Sorw"]) / (1 - FL["Swc"] - FL["Sorw"]), 0, 1) ** 2
    assert np.allclose(kro, krow, rtol=0, atol=1e-15)
    Sg = np.linspace(0.0, 0.6, 25)
    krw, kro, krg = model.rel_perms(FL, np.full_like(Sg, FL["Swc"]), Sg)
    krog = np.clip((1 - Sg - FL["Swc"] - FL["Sorg"]) / (1 - FL["Swc"] - FL["Sorg"]), 0, 1) ** 2
    assert np.allclose(kro, krog, rtol=0, atol=1e-15)
    assert np.all(krw == 0.0)


def test_coke_backward_euler_closed_form_for_coke_oxidation_only():
    # with cracking switched off, C = C^n / (1 + dt k4 y_O2 p)
    case = inp.tube_case()
    case.reactions["A"] = case.reactions["A"].copy()
    case.reactions["A"][2] = 0.0
    st = inp.random_state(case, 5)
    u = st["u"]
    bp = model.base_properties(case, u)
    dt = 37.0
    C = model.solve_coke(case, bp, st["coke"], dt)
    k4 = case.reactions["A"][3] * np.exp(-case.reactions["Ea"][3] / (model.R_GAS * u[5]))
    expect = st["coke"] / (1.0 + dt * k4 * u[2] * u[0])
    assert np.allclose(C, expect, rtol=1e-13, atol=0)


def test_coke_solve_satisfies_its_equation():
    case = inp.tube_case()
    st = inp.random_state(case, 6)
    u = st["u"].copy()
    u[5] = np.linspace(500, 900, case.n)
    bp = model.base_properties(case, u)
    dt = 300.0
    C = model.solve_coke(case, bp, st["coke"], dt)
    rates = model.reaction_rates(case, bp, C)
    s = case.reactions["stoich"][:, 6]
    g = C - st["coke"] - dt * sum(s[r] * rates[r] for r in range(4))
    assert np.max(np.abs(g) / (np.abs(C) + np.abs(st["coke"]))) < 1e-13


def _cells(case, p, T, x_lo=0.6, Sw=0.3, Sg=0.2, n=None):
    """A column of states u (8, n) with the given pressure, temperature, oil
    composition and saturations (gas composition away from the constraint is
    irrelevant to the properties tested here)."""
    n = n or np.broadcast(np.asarray(p), np.asarray(T), np.asarray(x_lo)).size
    u = np.zeros((8, n))
    u[0], u[1], u[2], u[3], u[4], u[5], u[6], u[7] = p, x_lo, 0.05, 0.7, 0.1, T, Sw, Sg
    return u


def test_gas_fractions_of_pure_oils_and_linear_in_the_oil_composition():
    """y_LO = K_LO x_LO and y_HO = f(S_o) K_HO x_HO with x_HO = 1 - x_LO: a pure
    LO oil sends no HO to the gas and a pure HO oil no LO; y_HO is proportional
    to x_HO."""
    p, T = 3e6, 500.0
    y1 = model.gas_fractions(FL, p, T, 1.0, 0.1, 0.7, 0.1, 0.3, 0.5)
    y0 = model.gas_fractions(FL, p, T, 0.0, 0.1, 0.7, 0.1, 0.3, 0.5)
    assert y1[inp.HO] == 0.0 and y1[inp.LO] > 0.0
    assert y0[inp.LO] == 0.0 and y0[inp.HO] > 0.0
    for x in (0.25, 0.6):
        y = model.gas_fractions(FL, p, T, x, 0.1, 0.7, 0.1, 0.3, 0.5)
        assert y[inp.HO] == pytest.approx((1.0 - x) * y0[inp.HO], rel=1e-14)
        assert y[inp.LO] == pytest.approx(x * y1[inp.LO], rel=1e-14)


def test_latent_heat_vanishes_at_the_critical_temperature():
    Tc = FL["Tc"][inp.W]
    Hv = model.vaporisation_enthalpy(FL, inp.W, np.array([Tc - 0.5, Tc, Tc + 0.5]))
    assert Hv[0] > 0.0
    assert Hv[1] == 0.0 and Hv[2] == 0.0


def test_liquid_enthalpy_does_not_depend_on_pressure():
    """The liquid enthalpies are H_gas - H_vap, functions of T (and the oil
    composition) only; the internal energies are those minus the flow work p/rho."""
    case = inp.tube_case(n_cells=3)
    T = 450.0
    bp = model.base_properties(case, _cells(case, np.array([1e5, 3e6, 2e7]), T))
    for ph in ("w", "o"):
        H = bp["U_" + ph] + bp["p"] / bp["rho_" + ph]
        np.testing.assert_allclose(H, H[0], rtol=1e-12)
        assert np.all(bp["U_" + ph] < H)


def test_porosity_and_rock_energy_at_their_reference():
    """phi(p_ref, T_ref) = phi_ref with (1/phi) dphi/dp = c_por there (the pore
    compressibility), and the rock's internal energy is zero at T_ref with
    dU_r/dT = cv1 + cv2 T (its volumetric heat capacity)."""
    case = inp.field_case(4, 3, 2, 0, 1, "f", 30 * inp.DAY, 40)
    rock = case.rock
    u = _cells(case, rock["p_ref"], rock["T_ref"], n=case.n)
    bp = model.base_properties(case, u)
    np.testing.assert_allclose(bp["phi"], case.phi_ref, rtol=1e-15)
    assert np.all(bp["U_r"] == 0.0)
    h = 1e-20
    for k, expect in ((0, rock["cpor"]), (5, None)):
        uc = u.astype(complex)
        uc[k] += 1j * h
        bc = model.base_properties(case, uc)
        if k == 0:
            np.testing.assert_allclose(bc["phi"].imag / h / case.phi_ref, expect, rtol=1e-12)
        else:
            np.testing.assert_allclose(bc["U_r"].imag / h, rock["cv1"] + rock["cv2"] * rock["T_ref"], rtol=1e-12)


def test_coke_takes_pore_volume_and_carries_its_own_energy():
    """Coke C_c (mol per bulk volume) fills C_c / rho_c of the pore space, so every
    fluid amount scales by phi_f / phi; at T_ref (rock and coke energies zero) the
    energy does too. Away from T_ref the energy changes by C_c (cp_c (T - T_ref)
    - e_f / rho_c), e_f the fluids' energy per pore volume."""
    case = inp.tube_case(n_cells=4)
    fl = case.fluid
    for T in (case.rock["T_ref"], 650.0):
        u = _cells(case, 2e6, T, n=case.n)
        bp = model.base_properties(case, u)
        c = np.array([0.0, 0.1, 0.5, 1.0]) * 0.3 * bp["phi"] * fl["coke_rho"]
        a0 = model.accumulation(case, bp, 0.0 * c)
        a1 = model.accumulation(case, bp, c)
        scale = (bp["phi"] - c / fl["coke_rho"]) / bp["phi"]
        for k in range(6):
            np.testing.assert_allclose(a1[k], a0[k] * scale, rtol=1e-13)
        e_f = (a0[6] - (1.0 - bp["phi"]) * bp["U_r"]) / bp["phi"]
        dE = c * (fl["coke_cp"] * (T - fl["T_ref"]) - e_f / fl["coke_rho"])
        np.testing.assert_allclose(a1[6], a0[6] + dE, rtol=1e-12, atol=1e-9 * np.abs(a0[6]).max())


def test_reaction_rates_special_cases_orders_and_arrhenius():
    """Crookston rate laws (Sec. 2.2, Reaction Model): the LO and HO oxidations are
    first order in the oxygen partial pressure and in their oil component's
    concentration phi_f S_o rho_o x_c, vanish without oxygen, without that
    component or without oil; cracking stops at the coke cap; coke burning is
    first order in p_O2 and in C_c with k = A exp(-E_a / RT)."""
    case = inp.tube_case(n_cells=1)
    rx = case.reactions
    kinds = list(rx["kind"])
    ox = [r for r in range(rx["nr"]) if kinds[r] == inp.RXN_OIL_OXIDATION]
    crk = [r for r in range(rx["nr"]) if kinds[r] == inp.RXN_CRACKING]
    cb = [r for r in range(rx["nr"]) if kinds[r] == inp.RXN_COKE_OXIDATION]
    assert ox and crk and cb
    coke = np.array([0.3 * rx["coke_max"]])

    def rates(p=3e6, T=600.0, x_lo=0.6, Sw=0.2, Sg=0.3, y_o2=0.1, c=coke):
        u = _cells(case, p, T, x_lo=x_lo, Sw=Sw, Sg=Sg, n=1)
        u[2] = y_o2
        return np.array([r[0] for r in model.reaction_rates(case, model.base_properties(case, u), c)])

    base = rates()
    assert np.all(base > 0.0)
    np.testing.assert_allclose(rates(y_o2=0.2)[ox + cb], 2.0 * base[ox + cb], rtol=1e-13)
    np.testing.assert_allclose(rates(y_o2=0.2)[crk], base[crk], rtol=1e-13)
    assert np.all(rates(y_o2=0.0)[ox + cb] == 0.0)
    # oil amount: S_o halves (gas takes its place), the oil reactions halve
    np.testing.assert_allclose(rates(Sg=0.55)[ox + crk], 0.5 * base[ox + crk], rtol=1e-13)
    assert np.all(rates(Sg=0.8)[ox + crk] == 0.0)
    for r in ox + crk:
        pure_other = 0.0 if rx["comp"][r] == inp.LO else 1.0
        assert rates(x_lo=pure_other)[r] == 0.0
    assert np.all(rates(c=np.array([rx["coke_max"]]))[crk] == 0.0)
    np.testing.assert_allclose(rates(c=2 * coke)[cb], 2.0 * base[cb], rtol=1e-13)
    T1, T2 = 600.0, 750.0
    for r in cb:
        ratio = rates(T=T2)[r] / rates(T=T1)[r]
        assert ratio == pytest.approx(np.exp(-rx["Ea"][r] / model.R_GAS * (1 / T2 - 1 / T1)), rel=1e-12)


@pytest.mark.parametrize("phase", [0, 1, 2])
def test_specific_weight_is_g_times_the_stored_mass_density(phase):
    """gamma_alpha / g equals the mass per volume of phase alpha that the
    accumulation stores when alpha fills the pores alone: sum_c M_c N_c / phi."""
    case = inp.tube_case(n_cells=1)
    sat = [(1.0, 0.0), (0.0, 0.0), (0.0, 1.0)][phase]
    u = _cells(case, 3e6, 500.0, x_lo=0.4, Sw=sat[0], Sg=sat[1], n=1)
    bp = model.base_properties(case, u)
    N = model.accumulation(case, bp, np.zeros(1))[:6]
    mass = sum(case.fluid["M"][c] * N[c] for c in range(6)) / bp["phi"]
    assert bp["gam"][phase][0] == pytest.approx(case.fluid["gravity"] * mass[0], rel=1e-13)


def test_corey_end_points_and_exponent():
    """Corey curves of exponent two: each relative permeability is zero at its
    critical or residual saturation, one at the other end of its mobile range,
    a quarter half way; Stone II gives k_ro = k_rocw = 1 at connate water
    without gas and zero at the residual oil of the water-oil table."""
    Swc, Sorw, Sgc = FL["Swc"], FL["Sorw"], FL["Sgc"]
    a = np.array
    krw, kro, krg = model.rel_perms(FL, a([Swc, 1 - Sorw, 0.5 * (Swc + 1 - Sorw), Swc, Swc, Swc]),
                                    a([0.0, 0.0, 0.0, Sgc, 1 - Swc, 0.5 * (Sgc + 1 - Swc)]))
    np.testing.assert_allclose(krw[:3], [0.0, 1.0, 0.25], atol=1e-15)
    np.testing.assert_allclose(krg[3:], [0.0, 1.0, 0.25], atol=1e-15)
    assert kro[0] == pytest.approx(1.0, abs=1e-15)
    assert kro[1] == pytest.approx(0.0, abs=1e-15)
    assert kro[4] == pytest.approx(0.0, abs=1e-15)
    # without gas Stone II is k_row, down to the small values next to residual oil
    for d in (0.01, 0.002):
        _, k, _ = model.rel_perms(FL, a([1 - Sorw - d]), a([0.0]))
        assert k[0] == pytest.approx((d / (1 - Swc - Sorw)) ** 2, rel=1e-12)
