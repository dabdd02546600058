"""Seeded synthetic inputs for the in-situ-combustion Newton step.

This module is shared by the oracle, the tests, the CUDA binding and the
benchmark. It holds DATA only: the paper's fluid and reaction tables
(Tab:input3 and Tab:input6 of the combustion-tube model, the CO2 column from
Tab:in2) converted to SI units, the constants chosen here where the
paper gives none, and seeded generators for grids, permeability fields and
wells. It evaluates none of the method's correlations or equations.

Unit conventions (SI everywhere): Pa, K, m, s, mol, J, kg/mol, Pa*s.
Component order: W, LO, HO, O2, N2, CO2 (Tab4.4 with the inert pseudo
component split into N2 and CO2); coke is the seventh species in the
stoichiometry rows.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# --- unit conversions (exact definitions) ---------------------------------
PSI = 6894.757293168361          # Pa per psi
FT = 0.3048                      # m per ft
LBMOL = 453.59237                # mol per lbmol
BTU = 1055.05585262              # J per Btu (IT)
BTU_PER_LBMOL = BTU / LBMOL      # J/mol per Btu/lbmol (= 2.326)
LBMOL_PER_FT3 = LBMOL / FT ** 3  # mol/m3 per lbmol/ft3
DARCY = 9.869233e-13             # m2
CP = 1.0e-3                      # Pa*s per cP
DAY = 86400.0


def degF_to_K(t_f):
    return (t_f + 459.67) / 1.8


NC = 6
COMP_NAMES = ("W", "LO", "HO", "O2", "N2", "CO2")
W, LO, HO, O2, N2, CO2 = range(6)
COKE = 6

# reaction rate-law kinds (the four forms of the Arrhenius rates in Sec. 2.2)
RXN_OIL_OXIDATION = 0   # k(T) * (y_O2 p) * (phi_f S_o rho_o x_i)
RXN_CRACKING = 1        # k(T) * (phi_f S_o rho_o x_i) * (1 - (C_c/C_max)^5)
RXN_COKE_OXIDATION = 2  # k(T) * (y_O2 p) * C_c

WELL_RATE_INJECTOR = 0
WELL_BHP_PRODUCER = 1
WELL_COUPLED_PRODUCER = 2      # producer with a bottom-hole-pressure unknown and a well equation
WELL_COUPLED_INJECTOR = 3      # injector with a bottom-hole-pressure unknown and a well equation

# controls of a coupled producer: 0 fixes the bottom-hole pressure; otherwise the
# bits select the phases (1 water, 2 oil, 4 gas) whose summed molar production
# rate (mol/s, positive out of the reservoir) is fixed
CTRL_BHP, CTRL_WATER_RATE, CTRL_OIL_RATE, CTRL_LIQUID_RATE, CTRL_GAS_RATE, CTRL_TOTAL_RATE = 0, 1, 2, 3, 4, 7


def tube_fluid() -> dict:
    """Fluid data of the combustion-tube model (Tab:input3) in SI units.

    N2 takes the tube's inert-gas column except its pseudo molar mass (28 is
    used for nitrogen); CO2 takes the inert-gas column of Tab:in2 (M = 44,
    p_c = 1073 psi, T_c = 88.03 F, cpg1 = 11). Correlations that the paper
    evaluates in field units with absolute temperature (cpg, avisc/bvisc,
    avg/bvg) are converted so that they take T in kelvin.
    """
    M = np.array([18.0, 156.7, 675.0, 32.0, 28.0, 44.0]) * 1e-3
    pc = np.array([3155.0, 305.7, 120.0, 730.0, 500.0, 1073.0]) * PSI
    Tc = degF_to_K(np.array([705.7, 651.7, 1138.0, -181.0, -232.0, 88.03]))
    # liquid-capable components W, LO, HO
    rho_ref = np.array([3.466, 0.3195, 0.0914]) * LBMOL_PER_FT3
    cp = np.array([3e-6, 5e-6, 5e-6]) / PSI
    ct1 = np.array([1.2e-4, 2.839e-4, 1.496e-4]) * 1.8
    ct2 = np.zeros(3)
    cpt = np.zeros(3)
    cpg_field = np.array([
        [7.613, 8.616e-4, 0.0, 0.0],
        [-1.89, 0.1275, -3.9e-5, 4.6e-9],
        [-8.14, 0.549, -1.68e-4, 1.98e-8],
        [6.713, -4.883e-7, 1.287e-6, -4.36e-10],
        [7.44, -0.0018, 1.975e-6, -4.78e-10],
        [11.0, 0.0, 0.0, 0.0],
    ])
    # cp(T_R)[Btu/lbmol/F] = sum_k cpg_k T_R^k, T_R = 1.8 T_K
    cpg = cpg_field * (BTU_PER_LBMOL * 1.8) * (1.8 ** np.arange(4))[None, :]
    ev = np.array([0.38, 0.38, 0.38])
    hvr = np.array([1657.0, 1917.0, 12198.0]) * BTU_PER_LBMOL * 1.8 ** ev
    bvg = np.array([1.116, 0.943, 1.102, 0.721, 0.702, 0.702])
    avg = np.array([8.822e-6, 2.166e-6, 3.926e-6, 2.196e-4, 2.127e-4, 2.127e-4]) * CP * 1.8 ** bvg
    avisc = np.array([4.7352e-3, 4.02e-4, 4.02e-4]) * CP
    bvisc = np.array([2728.2, 6121.6, 6121.6]) / 1.8
    # K = (kv1/p + kv2 p + kv3) exp(kv4 / (T - kv5))
    kv = np.zeros((3, 5))
    kv[:, 0] = np.array([1.7202e6, 1.4546e5, 2.7454e5]) * PSI
    kv[:, 3] = np.array([-6869.59, -4458.73, -8424.83]) / 1.8
    kv[:, 4] = degF_to_K(np.array([-376.64, -387.78, -205.69]))
    return dict(
        M=M, pc=pc, Tc=Tc, rho_ref=rho_ref, cp=cp, ct1=ct1, ct2=ct2, cpt=cpt,
        p_ref=101325.0, T_ref=298.15,
        cpg=cpg, hvr=hvr, ev=ev, avg=avg, bvg=bvg, avisc=avisc, bvisc=bvisc, kv=kv,
        K_phase=np.array([0.6, 0.13, 0.03]),        # W/m/K, water/oil/gas (chosen)
        coke_rho=57.2 * LBMOL_PER_FT3,               # Tab:input3 as printed
        coke_cp=4.06 * BTU_PER_LBMOL * 1.8,          # J/mol/K
        coke_K=0.0,
        coke_M=13.0e-3,
        Swc=0.15, Sorw=0.2, Sgc=0.05, Sorg=0.2,      # Corey endpoints
        per_eps=1.0e-4,
        gravity=9.80665,
    )


def _balanced_stoich() -> np.ndarray:
    """Tab:input6 stoichiometry with IR -> CO2; CO2 (or coke) is set so that
    the molar masses balance exactly (the paper's N M = 0 check)."""
    M = np.array([18.0, 156.7, 675.0, 32.0, 28.0, 44.0, 13.0])
    s = np.zeros((4, 7))
    # r1: LO + 14.06 O2 -> a CO2 + 6.58 H2O
    s[0, [LO, O2, W]] = [-1.0, -14.06, 6.58]
    # r2: HO + 60.55 O2 -> a CO2 + 28.34 H2O
    s[1, [HO, O2, W]] = [-1.0, -60.55, 28.34]
    # r3: HO -> 2.154 LO + a coke
    s[2, [HO, LO]] = [-1.0, 2.154]
    # r4: coke + 1.18 O2 -> a CO2 + 0.55 H2O
    s[3, [COKE, O2, W]] = [-1.0, -1.18, 0.55]
    for r, target in ((0, CO2), (1, CO2), (2, COKE), (3, CO2)):
        s[r, target] = -(s[r] @ M) / M[target]
    return s


def tube_reactions(seed: int = 0, phi_ref: float = 0.35) -> dict:
    """Crookston four-reaction model (Tab4.5, Tab:input6) in SI units.

    Pre-exponential factors are drawn log-uniformly within one decade of the
    tube's values (seeded); activation energies and reaction enthalpies are
    the tube's.
    """
    rng = np.random.default_rng(np.random.SeedSequence([seed, 0x5eed]))
    A_field = np.array([7.248e11, 7.248e11, 1.00008e7, 1.00008e4])  # 1/(psi*day)
    A_si = A_field / (PSI * DAY)
    lnA = np.log(A_si) + rng.uniform(-math.log(10.0), math.log(10.0), size=4)
    fl = tube_fluid()
    return dict(
        nr=4,
        stoich=_balanced_stoich(),
        kind=np.array([RXN_OIL_OXIDATION, RXN_OIL_OXIDATION, RXN_CRACKING, RXN_COKE_OXIDATION], dtype=np.int32),
        comp=np.array([LO, HO, HO, -1], dtype=np.int32),
        A=np.exp(lnA),
        Ea=np.array([59450.0, 59450.0, 27000.0, 25200.0]) * BTU_PER_LBMOL,
        dH=np.array([2.9075e6, 1.2525e7, 4.0e4, 2.25e5]) * BTU_PER_LBMOL,
        coke_max=0.1 * phi_ref * fl["coke_rho"],
    )


@dataclass
class Well:
    kind: int
    cells: np.ndarray          # int32 perforated cell ids
    WI: np.ndarray             # m3, per perforation
    target: float              # mol/s (injector, total) or Pa (producer BHP)
    inj_y: np.ndarray = field(default_factory=lambda: np.zeros(NC))
    inj_T: float = 300.0
    inj_phase: int = 2         # phase of the injected stream: 0 water (liquid), 2 gas
    control: int = CTRL_BHP    # coupled producer: CTRL_* (target in Pa for CTRL_BHP, else mol/s)
    ref_depth: float = 0.0     # coupled producer: depth (m) at which the bottom-hole pressure is defined
    bhp_init: float = 0.0      # coupled producer: initial bottom-hole pressure (Pa)


@dataclass
class Case:
    """One synthetic workload: grid, rock, fluid, reactions, wells, initial state."""
    name: str
    nx: int
    ny: int
    nz: int
    dx: float
    dy: float
    dz: float
    depth: np.ndarray          # (N,) m, cell-centre depth
    phi_ref: np.ndarray        # (N,)
    perm: np.ndarray           # (3, N) m2
    rock: dict
    fluid: dict
    reactions: dict
    wells: list
    init: dict                 # scalars of the initial-state recipe
    ignited: np.ndarray        # int32 cells started at T_ignite
    t_end: float
    n_steps: int
    dt0: float
    # heat loss to the overburden / underburden: None, or dict(K_ob W/m/K, d m,
    # T_ini K, rho K/m, faces: 1 top layer (k = 0), 2 bottom layer (k = nz - 1), 3 both)
    heat_loss: dict = None

    @property
    def n(self) -> int:
        return self.nx * self.ny * self.nz


def cell_id(i, j, k, nx, ny):
    return i + nx * (j + ny * k)


def _rock(cpor=1e-9, p_ref=5.0e6):
    return dict(cpor=cpor, ctpor=0.0, cptpor=0.0, p_ref=p_ref, T_ref=298.15,
                cv1=2.35e6, cv2=0.0, K_rock=2.0)


def _init(T0=300.0, p0=5.0e6):
    return dict(p=p0, T=T0, Sw=0.3, So=0.6, Sg=0.1, x_LO=0.744,
                y_rest=np.array([0.21, 0.79, 0.0]), T_ignite=650.0)


AIR = np.array([0.0, 0.0, 0.0, 0.21, 0.79, 0.0])
P_STD, T_STD = 101325.0, degF_to_K(60.0)


def std_rate_to_mol(q_m3s: float) -> float:
    """Gas rate at standard conditions (m3/s) to mol/s (ideal gas at 14.696 psi, 60 F)."""
    return q_m3s * P_STD / (8.314462618 * T_STD)


def tube_case(seed: int = 0, n_cells: int = 50) -> Case:
    """50-cell horizontal combustion tube (dx 0.02 m, area 5e-3 m2)."""
    nx = n_cells
    dx, area = 0.02, 5.0e-3
    dy = dz = math.sqrt(area)
    k = 10.0 * DARCY
    phi = 0.35
    fluid = tube_fluid()
    inj = Well(WELL_RATE_INJECTOR, np.array([0], np.int32), np.array([2 * k * area / dx]),
               std_rate_to_mol(1.0e-6), AIR.copy(), 300.0)
    prod = Well(WELL_BHP_PRODUCER, np.array([nx - 1], np.int32), np.array([2 * k * area / dx]), 5.0e6)
    return Case(
        name=f"tube {nx}x1x1", nx=nx, ny=1, nz=1, dx=dx, dy=dy, dz=dz,
        depth=np.full(nx, 0.5 * dz), phi_ref=np.full(nx, phi), perm=np.full((3, nx), k),
        rock=_rock(), fluid=fluid, reactions=tube_reactions(seed, phi), wells=[inj, prod],
        init=_init(), ignited=np.array([0], np.int32), t_end=7200.0, n_steps=60, dt0=20.0,
    )


def _smooth_gaussian_field(rng, shape, corr_cells):
    """White noise convolved with a separable Gaussian kernel, normalised to
    zero mean and unit standard deviation (shape is (nz, ny, nx))."""
    z = rng.standard_normal(shape)
    sig = float(corr_cells)
    half = int(math.ceil(3 * sig))
    t = np.arange(-half, half + 1)
    ker = np.exp(-0.5 * (t / sig) ** 2)
    ker /= ker.sum()
    for ax in range(3):
        if shape[ax] > 1:
            z = np.apply_along_axis(lambda v: np.convolve(np.pad(v, half, mode="wrap"), ker, mode="valid"), ax, z)
    z -= z.mean()
    sd = z.std()
    return z / sd if sd > 0 else z


def _well_index(k_h, dx, dy, dz, rw=0.1, skin=0.0):
    re = 0.14 * math.sqrt(dx * dx + dy * dy)
    return 2 * math.pi * k_h * dz / (math.log(re / rw) + skin)


def _vertical_well(kind, i, j, nx, ny, nz, perm, dx, dy, dz, target, inj_y=None):
    cells = np.array([cell_id(i, j, k, nx, ny) for k in range(nz)], np.int32)
    WI = np.array([_well_index(math.sqrt(perm[0, c] * perm[1, c]), dx, dy, dz) for c in cells])
    return Well(kind, cells, WI, target, AIR.copy() if inj_y is None else inj_y, 300.0)


def field_case(nx=60, ny=60, nz=20, seed=0, stream=1, name="field 60x60x20",
               t_end=30 * DAY, n_steps=40, air_rate_std=1.0e-2, bhp=4.5e6) -> Case:
    """3D block with a seeded log-normal permeability field (mean 1 D,
    sigma_ln 1, 5-cell correlation length, kv/kh 0.1), one air injector and
    one producer in opposite corners with full-depth completions."""
    rng = np.random.default_rng(np.random.SeedSequence([seed, stream]))
    dx = dy = 10.0
    dz = 1.0
    g = _smooth_gaussian_field(rng, (nz, ny, nx), 5.0).reshape(-1)
    kh = DARCY * np.exp(1.0 * g)
    perm = np.stack([kh, kh, 0.1 * kh])
    n = nx * ny * nz
    depth = (1000.0 + (np.arange(n) // (nx * ny) + 0.5) * dz).astype(np.float64)
    inj = _vertical_well(WELL_RATE_INJECTOR, 0, 0, nx, ny, nz, perm, dx, dy, dz, std_rate_to_mol(air_rate_std))
    prod = _vertical_well(WELL_BHP_PRODUCER, nx - 1, ny - 1, nx, ny, nz, perm, dx, dy, dz, bhp)
    return Case(
        name=name, nx=nx, ny=ny, nz=nz, dx=dx, dy=dy, dz=dz, depth=depth,
        phi_ref=np.full(n, 0.35), perm=perm, rock=_rock(), fluid=tube_fluid(),
        reactions=tube_reactions(seed, 0.35), wells=[inj, prod], init=_init(),
        ignited=inj.cells.copy(), t_end=t_end, n_steps=n_steps, dt0=t_end / n_steps,
    )


def large_case(nx=200, ny=200, nz=50, seed=0, air_rate_std=2.5e-2, bhp=4.5e6) -> Case:
    """3-facies log-normal field (0.1 / 1 / 5 D means) with a 5-spot pattern."""
    rng = np.random.default_rng(np.random.SeedSequence([seed, 5]))
    dx = dy = 10.0
    dz = 1.0
    shape = (nz, ny, nx)
    fac = np.argmax(np.stack([_smooth_gaussian_field(rng, shape, 5.0) for _ in range(3)]), axis=0).reshape(-1)
    means = np.array([0.1, 1.0, 5.0]) * DARCY
    noise = _smooth_gaussian_field(rng, shape, 2.0).reshape(-1)
    kh = means[fac] * np.exp(0.5 * noise)
    perm = np.stack([kh, kh, 0.1 * kh])
    n = nx * ny * nz
    depth = (1000.0 + (np.arange(n) // (nx * ny) + 0.5) * dz).astype(np.float64)
    wells = []
    for (i, j) in ((0, 0), (nx - 1, 0), (0, ny - 1), (nx - 1, ny - 1)):
        wells.append(_vertical_well(WELL_RATE_INJECTOR, i, j, nx, ny, nz, perm, dx, dy, dz, std_rate_to_mol(air_rate_std)))
    wells.append(_vertical_well(WELL_BHP_PRODUCER, nx // 2, ny // 2, nx, ny, nz, perm, dx, dy, dz, bhp))
    ign = np.concatenate([w.cells for w in wells[:4]])
    return Case(
        name=f"large {nx}x{ny}x{nz}", nx=nx, ny=ny, nz=nz, dx=dx, dy=dy, dz=dz, depth=depth,
        phi_ref=np.full(n, 0.35), perm=perm, rock=_rock(), fluid=tube_fluid(),
        reactions=tube_reactions(seed, 0.35), wells=wells, init=_init(),
        ignited=ign, t_end=10 * DAY, n_steps=15, dt0=10 * DAY / 15,
    )


def config(n: int, seed: int = 0) -> Case:
    """The five synthetic workloads (1 tube, 2 field, 3 mixed, 4 adjoint, 5 large)."""
    if n == 1:
        return tube_case(seed)
    if n == 2:
        return field_case(60, 60, 20, seed, 1, "field 60x60x20", 30 * DAY, 40)
    if n == 3:
        return field_case(100, 100, 30, seed, 3, "mixed 100x100x30", 30 * DAY, 40)
    if n == 4:
        return field_case(40, 40, 10, seed, 4, "adjoint 40x40x10", 20 * DAY, 20)
    if n == 5:
        return large_case(seed=seed)
    raise ValueError(n)


def adjoint_steps(case: Case, first: float = 60.0, ratio: float = 1.8) -> list:
    """Frozen step sizes of a sensitivity run: a geometric ramp from ``first``
    seconds by ``ratio`` per step, capped at the case's nominal step, for the
    case's number of steps. Newton from the ignited initial state needs the
    short first steps; for the 40x40x10 adjoint workload (20 steps, cap 1 day)
    the loop covers 8.8 days."""
    return [min(first * ratio ** k, case.dt0) for k in range(case.n_steps)]


def with_coupled_producer(case: Case, control: int, target: float, bhp_init: float) -> Case:
    """A copy of the case whose BHP producers become coupled producers with the
    given control and target, their bottom-hole pressure defined at the depth
    of the shallowest perforation and starting at bhp_init."""
    import copy
    c = copy.copy(case)
    wells = []
    for w in case.wells:
        if w.kind == WELL_BHP_PRODUCER:
            w = copy.copy(w)
            w.kind = WELL_COUPLED_PRODUCER
            w.control = control
            w.target = target
            w.ref_depth = float(np.min(case.depth[w.cells]))
            w.bhp_init = bhp_init
        wells.append(w)
    c.wells = wells
    return c


# heat loss of the workloads that enable it: shale cap and base rock conducting
# 1.7 W/m/K over a 10 m layer back to the initial 300 K, no fitted offset
HEAT_LOSS = dict(K_ob=1.7, d=10.0, T_ini=300.0, rho=0.0, faces=3)


def with_heat_loss(case: Case, **kw) -> Case:
    """A copy of the case with heat loss to the overburden and underburden
    (HEAT_LOSS, with any entry overridden by keyword)."""
    import copy
    c = copy.copy(case)
    c.heat_loss = dict(HEAT_LOSS, **kw)
    return c


def with_coupled_injector(case: Case, control: int, target: float, bhp_init: float) -> Case:
    """A copy of the case whose rate injectors become coupled injectors (the
    injected stream's rate set by a bottom-hole pressure unknown) with the given
    control (CTRL_BHP or CTRL_TOTAL_RATE) and target, the bottom-hole pressure
    defined at the depth of the shallowest perforation and starting at bhp_init."""
    import copy
    c = copy.copy(case)
    wells = []
    for w in case.wells:
        if w.kind == WELL_RATE_INJECTOR:
            w = copy.copy(w)
            w.kind = WELL_COUPLED_INJECTOR
            w.control = control
            w.target = target
            w.ref_depth = float(np.min(case.depth[w.cells]))
            w.bhp_init = bhp_init
        wells.append(w)
    c.wells = wells
    return c


def small_box(nx=4, ny=3, nz=2, seed=0) -> Case:
    """A tiny 3D case for dense-LU comparisons and element-by-element parity."""
    return field_case(nx, ny, nz, seed, 7, f"box {nx}x{ny}x{nz}", 1 * DAY, 4, air_rate_std=2e-4)


def random_state(case: Case, seed: int, spread: float = 1.0) -> dict:
    """A seeded random (not converged) state in the physical ranges of the
    workload: primary unknowns (p, x_LO, y_O2, y_N2, y_CO2, T, S_w, S_g) and
    coke, used for element-by-element residual/Jacobian parity."""
    rng = np.random.default_rng(np.random.SeedSequence([seed, 0xabc]))
    n = case.n
    u = np.empty((8, n))
    u[0] = 5.0e6 * (1 + 0.05 * spread * rng.uniform(-1, 1, n))
    u[1] = rng.uniform(0.3, 0.9, n)
    y = rng.uniform(0.05, 0.4, (3, n))
    u[2:5] = y
    u[5] = rng.uniform(300.0, 300.0 + 350.0 * spread, n)
    sw = rng.uniform(0.16, 0.5, n)
    sg = rng.uniform(0.06, 0.3, n)
    u[6] = sw
    u[7] = sg
    coke = rng.uniform(0.0, 0.05, n) * case.reactions["coke_max"]
    return dict(u=u, coke=coke)
