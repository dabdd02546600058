"""Pins of the oracle's Newton step and time loop: quadratic convergence of
Newton with the exact Jacobian, invariance of the Newton update under
Gauss-Jordan decoupling (Sec. 3.2), and a non-reacting water flood against
the Buckley-Leverett solution."""
import copy

import numpy as np
import pytest

import isc_inputs as inp
from oracle import linalg, model, sim


def test_newton_converges_quadratically_on_the_tube():
    case = inp.tube_case()
    u, coke = sim.initial_state(case)
    acc_old = model.old_accumulation(case, u, coke)
    opts = sim.NewtonOptions(tol=1e-13)
    opts.solve.solver = "dense"
    norms = []
    for _ in range(30):
        r = sim.newton_step(case, u, coke, acc_old, 20.0, opts)
        norms.append(r["norm"])
        if r["converged"]:
            break
        u = r["u"]
    # the tail of the sequence shows e_{k+1} ~ C e_k^2 (exact Jacobian)
    tail = [n for n in norms if 1e-12 < n < 1e-1]
    assert len(tail) >= 2
    ratios = [np.log(tail[i + 1]) / np.log(tail[i]) for i in range(len(tail) - 1)]
    assert max(ratios) > 1.7


def test_decoupling_leaves_the_newton_update_unchanged():
    case = inp.small_box(3, 2, 2)
    st = inp.random_state(case, 41)
    u0, c0 = sim.initial_state(case)
    acc_old = model.old_accumulation(case, u0, c0)
    o1 = sim.NewtonOptions(tol=0.0)
    o1.solve.solver = "dense"
    o1.solve.decouple = True
    o2 = copy.deepcopy(o1)
    o2.solve.decouple = False
    r1 = sim.newton_step(case, st["u"], st["coke"], acc_old, 100.0, o1)
    r2 = sim.newton_step(case, st["u"], st["coke"], acc_old, 100.0, o2)
    scale = np.array([1e6, 1, 1, 1, 1, 100.0, 1, 1])[:, None]
    d = np.max(np.abs(r1["du"] - r2["du"]) / scale) / np.max(np.abs(r2["du"]) / scale)
    assert d < 1e-9


def test_saturation_safeguard_halves_instead_of_going_negative():
    u = np.array([[5e6], [0.4], [0.2], [0.3], [0.1], [400.0], [0.2], [0.3]])
    du = np.array([[4e6], [-0.9], [-0.5], [0.1], [0.0], [120.0], [-0.5], [0.1]])
    un = sim.apply_update(u, du)
    assert un[0, 0] == pytest.approx(6e6)        # |dp| <= 0.2 p
    assert un[5, 0] == pytest.approx(450.0)      # |dT| <= 50 K
    assert un[1, 0] == pytest.approx(0.2)        # x_LO halves
    assert un[2, 0] == pytest.approx(0.1)        # y_O2 halves
    assert un[6, 0] == pytest.approx(0.1)        # S_w halves
    du2 = np.array([[0.0], [0.0], [0.0], [0.0], [0.0], [0.0], [0.2], [0.5]])
    un2 = sim.apply_update(u, du2)
    assert 1 - un2[6, 0] - un2[7, 0] == pytest.approx(0.5 * (1 - 0.2 - 0.3))


def test_tube_runs_to_two_hours():
    case = inp.tube_case()
    opts = sim.NewtonOptions(tol=1e-6)
    opts.solve.solver = "dense"
    u, coke, dts, stats = sim.run(case, case.t_end, 5.0, 150.0, opts)
    assert stats["t"] == pytest.approx(case.t_end)
    assert sum(dts) == pytest.approx(case.t_end, rel=1e-12)
    assert stats["steps"] == len(dts) == len(stats["its_per_step"])
    assert stats["newton"] >= sum(stats["its_per_step"])
    assert (stats["cuts"] == 0) == (stats["newton"] == sum(stats["its_per_step"]))
    assert 40 <= stats["steps"] <= 80
    So = 1 - u[6] - u[7]
    assert np.all(u[6] > 0) and np.all(u[7] > 0) and np.all(So > 0)
    assert np.all(np.abs(u[2] + u[3] + u[4] - 1) < 1.0)


# ------------------------------------------------------------ Buckley-Leverett
def _waterflood_case(n):
    case = inp.tube_case(n_cells=n)
    length = 1.0
    case.dx = length / n
    fl = case.fluid
    fl["cp"] = np.zeros(3)
    fl["ct1"] = np.zeros(3)
    fl["kv"] = fl["kv"].copy()
    fl["kv"][:, 0] = 0.0                 # non-volatile water and oil
    case.rock["cpor"] = 0.0
    case.reactions["A"] = np.zeros(4)
    case.init.update(Sw=0.15, Sg=0.02, So=0.83)
    case.ignited = np.array([], np.int32)
    rho_w = fl["rho_ref"][0]
    q_vol = 1.7e-8                           # m3/s of water
    k = case.perm[0, 0]
    area = case.dy * case.dz
    inj = inp.Well(inp.WELL_RATE_INJECTOR, np.array([0], np.int32), np.array([1.0]), q_vol * rho_w,
                   np.array([1.0, 0, 0, 0, 0, 0]), 300.0, inj_phase=0)
    prod = inp.Well(inp.WELL_BHP_PRODUCER, np.array([n - 1], np.int32), np.array([2 * k * area / case.dx]), 5.0e6)
    case.wells = [inj, prod]
    return case, q_vol, area


def _bl_profile(case, q_vol, area, t, x):
    fl = case.fluid
    T = 300.0
    mu_w = fl["avisc"][0] * np.exp(fl["bvisc"][0] / T)
    ln_mu_o = 0.744 * np.log(fl["avisc"][1] * np.exp(fl["bvisc"][1] / T)) + 0.256 * np.log(fl["avisc"][2] * np.exp(fl["bvisc"][2] / T))
    mu_o = np.exp(ln_mu_o)
    S = np.linspace(0.15, 0.8, 20001)
    krw, kro, _ = model.rel_perms(fl, S, np.full_like(S, 0.02))
    fw = (krw / mu_w) / (krw / mu_w + kro / mu_o)
    dfw = np.gradient(fw, S)
    swi = 0.15
    slope = fw / np.maximum(S - swi, 1e-12)
    i_f = int(np.argmax(np.where(S > swi + 1e-3, slope, 0)))   # Welge tangent point
    Sf = S[i_f]
    phi = case.phi_ref[0]
    xd = q_vol * t / (area * phi)
    xf = xd * fw[i_f] / (Sf - swi)
    prof = np.full_like(x, swi)
    behind = x < xf
    # rarefaction: dfw/dS (S) = x / xd for S >= Sf
    Sr = S[i_f:]
    dr = dfw[i_f:]
    order = np.argsort(dr)
    prof[behind] = np.interp(x[behind] / xd, dr[order], Sr[order])
    return prof, xf, Sf


def _flood(n, t_end, steps):
    case, q_vol, area = _waterflood_case(n)
    opts = sim.NewtonOptions(tol=1e-8)
    opts.solve.solver = "gmres"
    opts.solve.prec = "ilu0"
    opts.solve.rtol = 1e-12
    dt = t_end / steps
    u, coke, dts, stats = sim.run(case, t_end, dt, dt, opts, dts=[dt] * steps)
    x = (np.arange(n) + 0.5) * case.dx
    prof, xf, Sf = _bl_profile(case, q_vol, area, t_end, x)
    return u[6], prof, xf, Sf, case.dx, x


def test_waterflood_matches_buckley_leverett():
    """Front and profile converge to the Buckley-Leverett solution under grid
    refinement (first-order upwinding smears the shock over a few cells at
    this oil/water mobility ratio of about 45), and the injected water is
    all accounted for."""
    t_end = 1.0e4
    errs, front = [], []
    for n in (16, 32, 64):
        sw, prof, xf, Sf, dx, x = _flood(n, t_end, 2 * n)
        errs.append(np.mean(np.abs(sw - prof)))
        mid = 0.5 * (0.15 + Sf)
        i = int(np.argmax(sw < mid))
        x_num = x[i - 1] + (mid - sw[i - 1]) / (sw[i] - sw[i - 1]) * dx
        front.append(abs(x_num - xf))
        assert 0.4 < xf < 0.8
        # water balance: injected volume = water gained (incompressible, closed tube)
        case, q_vol, area = _waterflood_case(n)
        gained = np.sum(sw - 0.15) * dx * area * case.phi_ref[0]
        assert gained == pytest.approx(q_vol * t_end, rel=1e-9)
        if n == 32:
            assert front[-1] <= 4 * dx
    assert errs[1] < errs[0] and errs[2] < errs[1]
    assert front[1] < front[0] and front[2] < front[1]


def test_safeguard_other_branches():
    """The remaining branches of the update rule: x_LO pushed above one moves half
    way to one, y_N2, y_CO2 and S_g halve when they would turn negative, and the
    pressure and temperature limits hold in the negative direction too."""
    u = np.array([[5e6], [0.4], [0.2], [0.3], [0.1], [400.0], [0.2], [0.3]])
    du = np.array([[-3e6], [0.9], [0.0], [-0.5], [-0.2], [-80.0], [0.0], [-0.4]])
    un = sim.apply_update(u, du)
    assert un[0, 0] == pytest.approx(4e6)        # dp >= -0.2 p
    assert un[5, 0] == pytest.approx(350.0)      # dT >= -50 K
    assert un[1, 0] == pytest.approx(0.7)        # 1 - (1 - 0.4) / 2
    assert un[2, 0] == 0.2                       # unchanged
    assert un[3, 0] == pytest.approx(0.15)       # y_N2 halves
    assert un[4, 0] == pytest.approx(0.05)       # y_CO2 halves
    assert un[6, 0] == 0.2
    assert un[7, 0] == pytest.approx(0.15)       # S_g halves
    # a small update passes through untouched
    small = 1e-3 * du
    np.testing.assert_allclose(sim.apply_update(u, small), u + small, rtol=1e-15)


def test_step_size_controller():
    """dt grows or shrinks so that the largest temperature change would be 20 K
    and the largest saturation change 0.2, by a factor in [0.5, 2], capped at
    dt_max."""
    u0 = np.zeros((8, 3))
    u0[5] = 400.0

    def moved(dT, dS):
        u1 = u0.copy()
        u1[5, 1] += dT
        u1[6, 2] += dS
        return u1

    assert sim.next_dt(10.0, u0, moved(10.0, 0.05), 1e9) == pytest.approx(20.0)   # both small: x2
    assert sim.next_dt(10.0, u0, moved(2.0, 0.01), 1e9) == pytest.approx(20.0)    # growth capped at x2
    assert sim.next_dt(10.0, u0, moved(16.0, 0.05), 1e9) == pytest.approx(12.5)   # 20 / 16
    assert sim.next_dt(10.0, u0, moved(5.0, 0.16), 1e9) == pytest.approx(12.5)    # 0.2 / 0.16
    assert sim.next_dt(10.0, u0, moved(100.0, 0.0), 1e9) == pytest.approx(5.0)    # floor 0.5
    assert sim.next_dt(10.0, u0, moved(1.0, 0.0), 15.0) == pytest.approx(15.0)    # dt_max
    u1 = u0.copy()
    u1[7, 0] -= 0.4                                                              # S_g counts too
    assert sim.next_dt(10.0, u0, u1, 1e9) == pytest.approx(5.0)


def test_initial_state_recipe():
    """Uniform p, T, S_w, S_g and x_LO from the recipe, ignited cells at T_ignite,
    no coke; O2, N2 and CO2 share what the water and oil vapours leave of the gas
    in the recipe's ratios, so the gas constraint holds in every cell at the
    initial temperature."""
    case = inp.tube_case()
    ini = case.init
    u, coke = sim.initial_state(case)
    assert np.all(coke == 0.0)
    for k, key in ((0, "p"), (1, "x_LO"), (6, "Sw"), (7, "Sg")):
        assert np.all(u[k] == ini[key])
    hot = np.zeros(case.n, dtype=bool)
    hot[case.ignited] = True
    assert hot.any() and not hot.all()
    assert np.all(u[5, hot] == ini["T_ignite"]) and np.all(u[5, ~hot] == ini["T"])
    y = model.gas_fractions(case.fluid, u[0], u[5], u[1], u[2], u[3], u[4], u[6], 1 - u[6] - u[7])
    np.testing.assert_allclose(sum(y)[~hot], 1.0, rtol=1e-14)
    r = np.asarray(ini["y_rest"], dtype=float)
    for g in range(3):
        np.testing.assert_allclose(u[2 + g] * r.sum(), r[g] * (u[2] + u[3] + u[4]), rtol=1e-14)


def test_convergence_norms_are_relative_mass_and_rock_kelvin():
    """e_mass dt is the residual's mole imbalance as a fraction of the cell's
    stored moles; e_energy dt is its energy imbalance in kelvin of rock heating."""
    case = inp.small_box(3, 2, 2)
    st = inp.random_state(case, 5)
    u, coke = st["u"], st["coke"]
    acc = model.accumulation(case, model.base_properties(case, u), coke)
    ntot = sum(np.abs(acc[c]) for c in range(6))
    V, dt = model.cell_volume(case), 250.0
    F = np.zeros((8, case.n))
    F[3, 4] = V / dt * 1e-6 * ntot[4]
    F[6, 7] = V / dt * case.rock["cv1"] * 1e-3
    F[7, 2] = 3e-9
    e = sim.convergence_norms(case, F, u, coke)
    assert e[0] * dt == pytest.approx(1e-6, rel=1e-12)
    assert e[1] * dt == pytest.approx(1e-3, rel=1e-12)
    assert e[2] == pytest.approx(3e-9, rel=1e-15)


def _one_cell_no_sources():
    import dataclasses
    base = inp.small_box(2, 1, 1)
    rx = copy.deepcopy(base.reactions)
    rx["A"] = np.zeros_like(rx["A"])
    return dataclasses.replace(base, nx=1, depth=base.depth[:1], phi_ref=base.phi_ref[:1], perm=base.perm[:, :1],
                               reactions=rx, wells=[], ignited=np.zeros(0, dtype=np.int32))


def test_newton_norm_is_relative_mass_kelvin_and_gas_constraint():
    """The Newton step's convergence measure is the largest of the relative mole
    imbalance, the energy imbalance in kelvin of rock heating and |sum y - 1|,
    whatever the step size. One cell whose gas fractions sum to one, storing 10 %
    more moles (energy unchanged), then 10 % more energy (moles unchanged), then
    with the N2 fraction off by 0.2."""
    case = _one_cell_no_sources()
    u = np.array([[4e6], [0.5], [0.05], [0.0], [0.1], [420.0], [0.3], [0.2]])
    y = model.gas_fractions(case.fluid, u[0], u[5], u[1], u[2], u[3], u[4], u[6], 1 - u[6] - u[7])
    u[3] = 1.0 - sum(y)
    assert 0.0 < u[3, 0] < 1.0
    acc = model.accumulation(case, model.base_properties(case, u), np.zeros(1))
    mass = 0.1 * max(abs(acc[c][0]) for c in range(6)) / sum(abs(acc[c][0]) for c in range(6))
    kelvin = 0.1 * abs(acc[6][0]) / case.rock["cv1"]
    more_moles = [0.9 * a for a in acc[:6]] + [acc[6]]
    more_energy = list(acc[:6]) + [0.9 * acc[6]]
    off = u.copy()
    off[3] += 0.2
    acc_off = model.accumulation(case, model.base_properties(case, off), np.zeros(1))
    for dt in (50.0, 5000.0):
        opts = sim.NewtonOptions(tol=1e-300)
        assert sim.newton_step(case, u, np.zeros(1), more_moles, dt, opts)["norm"] == pytest.approx(mass, rel=1e-10)
        assert sim.newton_step(case, u, np.zeros(1), more_energy, dt, opts)["norm"] == pytest.approx(kelvin, rel=1e-10)
        assert sim.newton_step(case, off, np.zeros(1), acc_off, dt, opts)["norm"] == pytest.approx(0.2, rel=1e-10)
    done = sim.newton_step(case, u, np.zeros(1), acc, 50.0, sim.NewtonOptions(tol=1e300))
    assert done["converged"] and done["its"] == 0


def test_newton_iteration_cap_counts_updates():
    """timestep succeeds with maxit equal to the number of Newton updates it needs
    and fails with one fewer."""
    case = inp.small_box(3, 2, 1)
    u, c = sim.initial_state(case)
    opts = sim.NewtonOptions(tol=1e-8)
    opts.solve.solver = "dense"
    _, _, its, ok = sim.timestep(case, u, c, 500.0, opts)
    assert ok and its >= 2
    opts.maxit = its
    assert sim.timestep(case, u, c, 500.0, opts)[3]
    opts.maxit = its - 1
    assert not sim.timestep(case, u, c, 500.0, opts)[3]


def test_well_norm_is_relative_to_the_target():
    case = inp.with_coupled_producer(inp.small_box(3, 2, 2), inp.CTRL_BHP, 4.0e6, 4.0e6)
    w = model.coupled_wells(case)[0]
    assert sim.well_norms(case, [0.01 * w.target]) == [pytest.approx(0.01, rel=1e-15)]


def test_oil_saturation_rule_leaves_small_positive_oil_alone():
    u = np.array([[5e6], [0.4], [0.2], [0.3], [0.1], [400.0], [0.2], [0.3]])
    du = np.zeros((8, 1))
    du[7, 0] = 0.4995                            # S_o = 1 - 0.2 - 0.7995 = 5e-4 > 0
    un = sim.apply_update(u, du)
    assert un[6, 0] == 0.2 and un[7, 0] == pytest.approx(0.7995, rel=1e-15)
    # x_LO: small positive values pass, values just above one move half way to one
    for dx, expect in ((-0.3995, 5e-4), (0.65, 0.7)):
        du = np.zeros((8, 1))
        du[1, 0] = dx
        assert sim.apply_update(u, du)[1, 0] == pytest.approx(expect, rel=1e-12)


def test_coupled_newton_iteration_cap_counts_updates():
    """The bordered Newton loop of a case with a coupled producer: maxit is the
    number of updates allowed, as for the plain loop."""
    case = inp.with_coupled_producer(inp.small_box(3, 2, 1), inp.CTRL_BHP, 4.5e6, 4.5e6)
    u, c = sim.initial_state(case)
    opts = sim.NewtonOptions(tol=1e-8)
    _, _, _, its, ok = sim.timestep_coupled(case, u, np.array([4.5e6]), c, 500.0, opts)
    assert ok and its >= 2
    opts.maxit = its
    assert sim.timestep_coupled(case, u, np.array([4.5e6]), c, 500.0, opts)[4]
    opts.maxit = its - 1
    assert not sim.timestep_coupled(case, u, np.array([4.5e6]), c, 500.0, opts)[4]


def test_dense_solve_reports_no_krylov_iterations():
    case = inp.small_box(2, 2, 1)
    st = inp.random_state(case, 3)
    u0, c0 = sim.initial_state(case)
    acc_old = model.old_accumulation(case, u0, c0)
    rp, col, val = model.jacobian(case, st["u"], st["coke"], acc_old, 100.0)
    rhs = np.random.default_rng(2).standard_normal((case.n, 8))
    x, its, rel = sim.linear_solve(rp, col, val, rhs, sim.SolveOptions(solver="dense"))
    assert its == 0 and rel == 0.0
    A = linalg.bsr_to_dense(rp, col, val)
    ref = np.linalg.solve(A, rhs.reshape(-1))
    assert np.linalg.norm(x.reshape(-1) - ref) <= 1e-8 * np.linalg.norm(ref)


def test_failed_steps_are_halved_and_counted():
    """A first tube step of 2000 s does not converge within 25 Newton updates; it is
    halved until it does (twice, to 500 s), each halving is counted, and max_cuts
    bounds the number of halvings."""
    case = inp.tube_case(n_cells=10)
    opts = sim.NewtonOptions(tol=1e-6)
    opts.solve.solver = "dense"
    _, _, dts, st = sim.run(case, 2000.0, 2000.0, 1e9, opts, max_steps=1)
    assert dts == [500.0] and st["cuts"] == 2 and st["steps"] == 1
    assert sim.run(case, 2000.0, 2000.0, 1e9, opts, max_cuts=2, max_steps=1)[2] == [500.0]
    with pytest.raises(RuntimeError):
        sim.run(case, 2000.0, 2000.0, 1e9, opts, max_cuts=1, max_steps=1)


def test_coupled_newton_step_limits_the_bottom_hole_pressure_change():
    """Under a bottom-hole-pressure control the well equation is linear, so the
    Newton correction is target - bhp; it is limited to 20 % of bhp either way."""
    for target, expect in ((8.0e6, 4.8e6), (2.0e6, 3.2e6), (4.2e6, 4.2e6)):
        case = inp.with_coupled_producer(inp.small_box(3, 2, 1), inp.CTRL_BHP, target, 4.0e6)
        u, c = sim.initial_state(case)
        acc = model.old_accumulation(case, u, c)
        r = sim.newton_step_coupled(case, u, np.array([4.0e6]), c, acc, 100.0, sim.NewtonOptions(tol=1e-300))
        assert r["dbhp"][0] == pytest.approx(target - 4.0e6, rel=1e-9)
        assert r["bhp"][0] == pytest.approx(expect, rel=1e-12)
        assert r["its"] == 0


def test_coupled_newton_norm_scales_like_the_plain_one():
    """With its producer shut (bottom-hole pressure above the reservoir, at its
    target) a coupled case has the residual of the case without the well, and the
    bordered Newton step reports the plain step's convergence measure at any dt,
    whether stored moles or stored energy dominate it."""
    import dataclasses
    box = inp.small_box(3, 2, 1)
    rx = copy.deepcopy(box.reactions)
    rx["A"] = np.zeros_like(rx["A"])
    # one layer, no injector, no reactions, no ignition: only the stored amounts change
    base = dataclasses.replace(box, reactions=rx, ignited=np.zeros(0, dtype=np.int32),
                               wells=[w for w in box.wells if w.kind == inp.WELL_BHP_PRODUCER])
    u, c = sim.initial_state(base)
    bhp = 1.5 * float(np.max(u[0]))
    coupled = inp.with_coupled_producer(base, inp.CTRL_BHP, bhp, bhp)
    plain = copy.copy(base)
    plain.wells = [w for w in base.wells if w.kind != inp.WELL_BHP_PRODUCER]
    acc = model.accumulation(base, model.base_properties(base, u), c)
    variants = ([0.5 * a for a in acc[:6]] + [acc[6]], list(acc[:6]) + [0.9 * acc[6]])
    opts = sim.NewtonOptions(tol=1e-300)
    for old in variants:
        for dt in (50.0, 5000.0):
            r0 = sim.newton_step(plain, u, c, old, dt, opts)
            n1 = sim.newton_step_coupled(coupled, u, np.array([bhp]), c, old, dt, opts)["norm"]
            assert n1 == pytest.approx(r0["norm"], rel=1e-12)
            e = r0["norms"]
            assert r0["norm"] == pytest.approx(max(e[0], e[1]) * dt, rel=1e-12)   # not the gas constraint
    big = sim.newton_step_coupled(coupled, u, np.array([bhp]), c, acc, 50.0, sim.NewtonOptions(tol=1e300))
    assert big["converged"] and big["its"] == 0
