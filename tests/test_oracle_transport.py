"""Pins of the oracle's inter-cell transport (Sec. 3.1) to the physics it
discretises: Darcy's law across one face in each direction with anisotropic
permeability and non-cubic cells (harmonic transmissibility), zero flux in a
hydrostatic column, Fourier conduction through two cells in series, the bulk
conductivity of a cell filled with one material, the gas-viscosity mixing rule
and reaction rates per stored mole. Each case isolates the term under test:
no wells, no reactions (A = 0) unless stated, and the old accumulation equal
to the current one, so the residual rows hold the face terms alone."""
import copy
import dataclasses

import numpy as np
import pytest

import isc_inputs as inp
from oracle import model


def _line(d, n=2, dxyz=(3.0, 5.0, 2.0), perm=None, gravity=0.0, phi=0.3, no_reactions=True):
    """n cells in a row along direction d (0 = x, 1 = y, 2 = z)."""
    base = inp.small_box(2, 1, 1)
    dims = [1, 1, 1]
    dims[d] = n
    fl = copy.deepcopy(base.fluid)
    fl["gravity"] = gravity
    rx = copy.deepcopy(base.reactions)
    if no_reactions:
        rx["A"] = np.zeros_like(rx["A"])
    depth = np.full(n, 100.0)
    if d == 2:
        depth = 100.0 + dxyz[2] * np.arange(n)
    perm = np.full((3, n), 1e-12) if perm is None else np.asarray(perm, dtype=float)
    return dataclasses.replace(base, nx=dims[0], ny=dims[1], nz=dims[2], dx=dxyz[0], dy=dxyz[1], dz=dxyz[2],
                               depth=depth, phi_ref=np.full(n, phi), perm=perm, fluid=fl, reactions=rx, wells=[],
                               ignited=np.zeros(0, dtype=np.int32))


def _state(n, p, T, Sw, Sg, x_lo=0.5, y=(0.0, 0.7, 0.2)):
    u = np.zeros((8, n))
    u[0], u[1], u[5], u[6], u[7] = p, x_lo, T, Sw, Sg
    u[2], u[3], u[4] = y
    return u


def _face_rows(case, u, coke=None):
    coke = np.zeros(case.n) if coke is None else coke
    bp = model.base_properties(case, u)
    acc = model.accumulation(case, bp, coke)
    return model.residual(case, u, coke, acc, 1.0e3), bp


@pytest.mark.parametrize("d", [0, 1, 2])
def test_darcy_flux_across_one_face_in_each_direction(d):
    """Molar water flux from cell 0 to cell 1 = T_face lambda_w (p_0 - p_1), with
    T_face the harmonic mean of k_d A_d / h_d of the two cells (A_d the face area,
    h_d the cell length along d); no gravity, water only."""
    dxyz = (3.0, 5.0, 2.0)
    perm = np.array([[1e-12, 3e-12], [2e-13, 5e-13], [7e-14, 1e-14]])
    case = _line(d, dxyz=dxyz, perm=perm)
    u = _state(2, np.array([5.2e6, 5.0e6]), 420.0, 1.0, 0.0)
    F, bp = _face_rows(case, u)
    area = dxyz[0] * dxyz[1] * dxyz[2] / dxyz[d]
    t = perm[d] * area / dxyz[d]
    Tf = 2 * t[0] * t[1] / (t[0] + t[1])
    q = Tf * bp["lam"][0][0] * (u[0, 0] - u[0, 1])
    assert F[inp.W, 0] == pytest.approx(q, rel=1e-13)
    assert F[inp.W, 1] == pytest.approx(-q, rel=1e-13)
    assert F[6, 0] == pytest.approx(q * bp["H_w"][0], rel=1e-12)


def test_hydrostatic_column_has_no_flux():
    """Three water-filled cells stacked in z at one temperature, pressures in
    discrete hydrostatic equilibrium (p_{k+1} - p_k = mean specific weight x dz):
    no phase moves, so every balance row vanishes."""
    case = _line(2, n=3, dxyz=(10.0, 10.0, 4.0), gravity=9.80665)
    u = _state(3, 5.0e6, 400.0, 1.0, 0.0)
    for _ in range(60):
        gam = model.base_properties(case, u)["gam"][0]
        for k in range(1, 3):
            u[0, k] = u[0, k - 1] + 0.5 * (gam[k - 1] + gam[k]) * case.dz
    F, bp = _face_rows(case, u)
    flow_scale = case.perm[2, 0] * case.dx * case.dy / case.dz * bp["lam"][0][0] * bp["gam"][0][0] * case.dz
    assert np.max(np.abs(F[:6])) <= 1e-9 * flow_scale
    assert np.max(np.abs(F[6])) <= 1e-9 * flow_scale * abs(bp["H_w"][0])
    # the same pressures without gravity drive water up the column
    case0 = _line(2, n=3, dxyz=(10.0, 10.0, 4.0), gravity=0.0)
    F0, _ = _face_rows(case0, u)
    assert F0[inp.W, 2] > 0.0 and F0[inp.W, 0] < 0.0


def test_conduction_through_two_cells_in_series():
    """No pressure difference, two temperatures: the heat flow leaving cell 0 is
    (T_0 - T_1) / R with R the two half-cell resistances in series,
    R = (h/2)/(K_0 A) + (h/2)/(K_1 A)."""
    dxyz = (3.0, 5.0, 2.0)
    case = _line(0, dxyz=dxyz)
    u = _state(2, 5.0e6, np.array([520.0, 450.0]), np.array([0.9, 0.2]), np.array([0.0, 0.5]))
    F, bp = _face_rows(case, u)
    K = model.thermal_conductivity(case, bp, np.zeros(2))
    A, h = dxyz[1] * dxyz[2], dxyz[0]
    R = (h / 2) / (K[0] * A) + (h / 2) / (K[1] * A)
    heat = (u[5, 0] - u[5, 1]) / R
    assert F[6, 0] == pytest.approx(heat, rel=1e-13)
    assert F[6, 1] == pytest.approx(-heat, rel=1e-13)
    assert np.all(F[:6] == 0.0)


@pytest.mark.parametrize("fill", ["water", "oil", "gas", "rock"])
def test_bulk_conductivity_of_a_cell_filled_with_one_material(fill):
    """K_T of a cell whose pores are filled by one phase with porosity one is that
    phase's conductivity; with porosity zero it is the rock's."""
    phi = 0.0 if fill == "rock" else 1.0
    case = _line(0, n=1, phi=phi)
    sat = dict(water=(1.0, 0.0), oil=(0.0, 0.0), gas=(0.0, 1.0), rock=(0.3, 0.3))[fill]
    u = _state(1, case.rock["p_ref"], case.rock["T_ref"], sat[0], sat[1])
    bp = model.base_properties(case, u)
    assert bp["phi"][0] == phi
    K = model.thermal_conductivity(case, bp, np.zeros(1))[0]
    expect = case.rock["K_rock"] if fill == "rock" else case.fluid["K_phase"][["water", "oil", "gas"].index(fill)]
    assert K == pytest.approx(expect, rel=1e-15)


def test_gas_viscosity_mixes_by_the_square_root_of_molar_mass():
    """A binary O2/N2 gas (no water, no oil in the pores): a pure gas keeps its own
    viscosity, and the mixture sits between the pure ones at the lever position
    given by the weights y_c sqrt(M_c)."""
    case = _line(0, n=1)
    M = case.fluid["M"]

    def mu(yo2, yn2):
        u = _state(1, 3e6, 500.0, 0.0, 1.0, x_lo=0.0, y=(yo2, yn2, 0.0))
        return model.base_properties(case, u)["mu_g"][0]

    m_o2, m_n2 = mu(1.0, 0.0), mu(0.0, 1.0)
    # a pure gas has its own correlation's viscosity avg T^bvg
    fl = case.fluid
    assert m_o2 == pytest.approx(fl["avg"][inp.O2] * 500.0 ** fl["bvg"][inp.O2], rel=1e-13)
    assert m_n2 == pytest.approx(fl["avg"][inp.N2] * 500.0 ** fl["bvg"][inp.N2], rel=1e-13)
    for yo2 in (0.21, 0.5, 0.8):
        m = mu(yo2, 1.0 - yo2)
        w_o2, w_n2 = yo2 * np.sqrt(M[inp.O2]), (1.0 - yo2) * np.sqrt(M[inp.N2])
        assert (m - m_n2) / (m_o2 - m) == pytest.approx(w_o2 / w_n2, rel=1e-10)


def test_stored_mass_is_the_saturation_weighted_phase_mass_density():
    """With all three phases present, sum_c M_c N_c / phi_f = sum_alpha S_alpha
    gamma_alpha / g: every component's gas and liquid parts are stored."""
    case = _line(0, n=1, gravity=9.80665)
    u = _state(1, 3e6, 480.0, 0.3, 0.25, x_lo=0.4, y=(0.1, 0.6, 0.1))
    bp = model.base_properties(case, u)
    coke = np.array([0.2 * case.reactions["coke_max"]])
    N = model.accumulation(case, bp, coke)[:6]
    phi_f = bp["phi"] - coke / case.fluid["coke_rho"]
    mass = sum(case.fluid["M"][c] * N[c] for c in range(6)) / phi_f
    S = (bp["Sw"], bp["So"], bp["Sg"])
    expect = sum(S[a] * bp["gam"][a] for a in range(3)) / 9.80665
    assert mass[0] == pytest.approx(expect[0], rel=1e-13)


def test_oil_reaction_rates_per_stored_mole_of_their_component():
    """Without gas in the pores the oil component's moles per bulk volume are
    phi_f S_o rho_o x_c, the concentration of the rate laws: at fixed T, p and
    y_O2 the rate per stored mole is the same whatever S_o, x_LO and coke."""
    case = _line(0, n=1, no_reactions=False)
    rx = case.reactions
    ratios = []
    for Sw, x_lo, c in ((0.2, 0.3, 0.0), (0.5, 0.6, 0.1), (0.7, 0.9, 0.05)):
        u = _state(1, 3e6, 600.0, Sw, 0.0, x_lo=x_lo, y=(0.1, 0.7, 0.1))
        bp = model.base_properties(case, u)
        coke = np.array([c * rx["coke_max"]])
        N = model.accumulation(case, bp, coke)
        r = model.reaction_rates(case, bp, coke)
        row = []
        for k in range(rx["nr"]):
            if rx["kind"][k] == inp.RXN_OIL_OXIDATION:
                row.append(r[k][0] / N[rx["comp"][k]][0])
            elif rx["kind"][k] == inp.RXN_CRACKING:
                row.append(r[k][0] / N[rx["comp"][k]][0] / (1.0 - (coke[0] / rx["coke_max"]) ** 5))
        ratios.append(row)
    ratios = np.array(ratios)
    np.testing.assert_allclose(ratios, ratios[0][None, :].repeat(3, 0), rtol=1e-12)


def test_a_single_cell_has_no_face_terms():
    """One cell, no wells, no reactions: the balance rows are the accumulation
    change alone, V/dt (N - N_old)."""
    case = _line(0, n=1)
    u = _state(1, 4e6, 500.0, 0.3, 0.2)
    bp = model.base_properties(case, u)
    acc = model.accumulation(case, bp, np.zeros(1))
    F0 = model.residual(case, u, np.zeros(1), acc, 50.0)
    assert np.all(F0[:7] == 0.0)
    old = [a * 0.9 for a in acc]
    F1 = model.residual(case, u, np.zeros(1), old, 50.0)
    V = case.dx * case.dy * case.dz
    for r in range(7):
        assert F1[r, 0] == pytest.approx(V / 50.0 * 0.1 * acc[r][0], rel=1e-12)


@pytest.mark.parametrize("c", [inp.W, inp.LO, inp.HO])
def test_liquid_compressibility_and_thermal_expansion(c):
    """At the reference state (1/rho) d rho/dp is the liquid's compressibility
    c_p and -(1/rho) d rho/dT its thermal expansion c_T1: liquids expand on
    heating."""
    fl = inp.small_box(2, 1, 1).fluid
    p0, T0 = fl["p_ref"], fl["T_ref"]
    h = 1e-20
    rho = model.liquid_density(fl, c, np.array([p0]), np.array([T0]))[0]
    assert rho == pytest.approx(fl["rho_ref"][c], rel=1e-15)
    dp = model.liquid_density(fl, c, np.array([p0 + 1j * h]), np.array([T0]))[0].imag / h
    dT = model.liquid_density(fl, c, np.array([p0]), np.array([T0 + 1j * h]))[0].imag / h
    assert dp / rho == pytest.approx(fl["cp"][c], rel=1e-12)
    assert -dT / rho == pytest.approx(fl["ct1"][c], rel=1e-12)
    assert fl["ct1"][c] > 0.0


@pytest.mark.parametrize("phase", [0, 1, 2])
def test_stored_energy_of_a_single_phase_is_enthalpy_density_minus_pressure(phase):
    """A cell of porosity one filled with one phase stores E = rho h - p per
    volume (u = h - p v), at any temperature (no rock to heat)."""
    case = _line(0, n=1, phi=1.0)
    sat = [(1.0, 0.0), (0.0, 0.0), (0.0, 1.0)][phase]
    u = _state(1, case.rock["p_ref"], 560.0, sat[0], sat[1], x_lo=0.35, y=(0.1, 0.6, 0.1))
    bp = model.base_properties(case, u)
    E = model.accumulation(case, bp, np.zeros(1))[6][0]
    rho = (bp["rho_w"], bp["rho_o"], bp["rho_g"])[phase][0]
    H = (bp["H_w"], bp["H_o"], bp["H_g"])[phase][0]
    assert E == pytest.approx(rho * H - bp["p"][0], rel=1e-12)
