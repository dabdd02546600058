"""GPU parity: libisc (through the C ABI) against the CPU oracle, element by
element on seeded inputs.

Tolerances: residual and Jacobian 1e-10 relative (to the row's scale, since
single entries can cancel to ~0); decoupled system and preconditioner 1e-11
on identical inputs; Newton updates to the solver tolerance measured with the
oracle's own matrix.
"""
import numpy as np
import pytest

import isc_inputs as inp
from oracle import linalg, model, sim
from oracle_system import assembled, decoupled

pytestmark = pytest.mark.gpu

SCALE = np.array([1e6, 1, 1, 1, 1, 100.0, 1, 1])


@pytest.fixture(scope="module")
def Simulator():
    from paper_1811_11992_gb300 import build
    build.build()
    from paper_1811_11992_gb300 import Simulator as S
    return S


def row_scaled_err(F, Fo):
    scale = np.abs(Fo).max(axis=1, keepdims=True) + 1e-300
    return np.max(np.abs(F - Fo) / scale)


def jac_err(J, Jo, rowptr, n):
    rows = np.repeat(np.arange(n), np.diff(rowptr))
    Js = J * SCALE[None, None, :]
    Jos = Jo * SCALE[None, None, :]
    rowmax = np.zeros((n, 8))
    np.maximum.at(rowmax, rows, np.abs(Jos).max(axis=2))
    return np.max(np.abs(Js - Jos) / (rowmax[rows][:, :, None] + 1e-300))


CASES = {
    "tube12": lambda: inp.tube_case(n_cells=12),
    "tube50": lambda: inp.tube_case(),
    "box432": lambda: inp.small_box(4, 3, 2),
    "box755": lambda: inp.small_box(7, 5, 5),
}


def _gpu_assembled(S, case, st_a, st_b, dt, **opt):
    g = S(case, **opt)
    g.set_state(st_a["u"], st_a["coke"])
    g.begin_step()
    g.set_state(st_b["u"])
    g.assemble(dt)
    return g


@pytest.mark.parametrize("name", list(CASES))
def test_residual_and_jacobian_match_oracle(Simulator, name):
    case = CASES[name]()
    a = inp.random_state(case, 101)
    b = inp.random_state(case, 202)
    dt = 150.0
    g = _gpu_assembled(Simulator, case, a, b, dt)
    F = g.residual()
    rp, col, J = g.jacobian()
    acc_old = model.old_accumulation(case, a["u"], a["coke"])
    Fo, co = model.residual(case, b["u"], a["coke"], acc_old, dt, return_coke=True)
    rpo, colo, Jo = model.jacobian(case, b["u"], a["coke"], acc_old, dt)
    assert np.array_equal(rp, rpo) and np.array_equal(col, colo)
    assert np.allclose(g.coke(), co, rtol=1e-12, atol=1e-300)
    assert row_scaled_err(F, Fo) < 1e-10
    assert jac_err(J, Jo, rp, case.n) < 1e-10
    g.close()


def test_initial_state_and_ignited_assembly(Simulator):
    case = inp.small_box(5, 4, 3)
    g = Simulator(case)
    g.init_equilibrium()
    u0, c0 = sim.initial_state(case)
    ug, cg = g.get_state()
    assert np.allclose(ug, u0, rtol=1e-13, atol=1e-300)
    assert np.all(cg == 0)
    dt = 3600.0
    g.assemble(dt)
    acc_old = model.old_accumulation(case, u0, c0)
    Fo = model.residual(case, u0, c0, acc_old, dt)
    assert row_scaled_err(g.residual(), Fo) < 1e-10
    rp, col, J = g.jacobian()
    _, _, Jo = model.jacobian(case, u0, c0, acc_old, dt)
    assert jac_err(J, Jo, rp, case.n) < 1e-10


@pytest.mark.parametrize("name", ["tube12", "box432", "box755"])
def test_gauss_jordan_kernel_matches_oracle_on_identical_input(Simulator, name):
    """The oracle's assembled system loaded through isc_set_system, decoupled by
    the GPU, against the oracle's Gauss-Jordan decoupling of the same system."""
    case = CASES[name]()
    rp, col, J, F = assembled(case, 303, 404)
    g = Simulator(case)
    g.set_system(J, F)
    g.decouple()
    Fd = g.residual()
    _, _, Jd = g.jacobian()
    vo, ro = linalg.gauss_jordan_decouple(rp, col, J, F.T.copy())
    rows = np.repeat(np.arange(case.n), np.diff(rp))
    assert np.all(Jd[col == rows] == np.eye(8))
    err = np.abs(Jd - vo).reshape(len(col), -1).max(axis=1) / np.maximum(np.abs(vo).reshape(len(col), -1).max(axis=1), 1e-300)
    assert err.max() < 1e-11
    assert row_scaled_err(Fd, ro.T) < 1e-11
    g.close()


@pytest.mark.parametrize("name", ["tube12", "box432", "box755"])
def test_spmv_and_ilu0_apply_match_oracle(Simulator, name):
    case = CASES[name]()
    rp, col, _, _, Jd, Fd = decoupled(case, 505, 606)
    g = Simulator(case)
    g.set_system(Jd, Fd, decoupled=True)
    rng = np.random.default_rng(7)
    x = rng.standard_normal((8, case.n))
    y = g.spmv(x)
    yo = linalg.bsr_matvec(rp, col, Jd, x.T.copy()).T
    assert np.max(np.abs(y - yo)) <= 1e-13 * np.abs(yo).max()
    g.build_preconditioner()
    z = g.precond_apply(x)
    M = linalg.ILU0Preconditioner(rp, col, Jd)
    zo = M.apply(x.T.copy()).T
    assert np.max(np.abs(z - zo)) <= 1e-11 * np.abs(zo).max()
    g.close()


@pytest.mark.parametrize("dims", [(2, 1, 1), (3, 1, 1), (33, 1, 1), (5, 4, 3), (17, 3, 2), (13, 7, 5)],
                         ids=lambda d: "x".join(map(str, d)))
def test_row_panel_spmv_on_ragged_grids(Simulator, dims):
    """The decoupled SpMV on degenerate and ragged grids (single cells in a line,
    odd sizes, rows with 1 to 6 neighbours): exact up to summation order against
    the oracle's BSR product."""
    case = inp.small_box(*dims)
    rp, col, _, _, Jd, Fd = decoupled(case, 515, 616)
    g = Simulator(case)
    g.set_system(Jd, Fd, decoupled=True)
    x = np.random.default_rng(8).standard_normal((8, case.n))
    y = g.spmv(x)
    yo = linalg.bsr_matvec(rp, col, Jd, x.T.copy()).T
    assert np.max(np.abs(y - yo)) <= 1e-13 * np.abs(yo).max()
    g.close()


@pytest.mark.parametrize("krylov,prec", [("gmres", "bilu0"), ("gmres", "bjacobi"), ("bicgstab", "bilu0"), ("gmres", "none")])
def test_krylov_solution_has_small_residual_in_oracle_matrix(Simulator, krylov, prec):
    case = inp.small_box(4, 3, 2)
    rp, col, J, F = assembled(case, 707, 808)
    g = Simulator(case, krylov=krylov, prec=prec, tol_lin=1e-11, maxit_lin=2000)
    g.set_system(J, F)
    g.decouple()
    info = g.solve()
    du = g.newton_update()
    assert info.krylov_rel_residual <= 1e-11
    # residual of the GPU update in the oracle's decoupled system
    vo, ro = linalg.gauss_jordan_decouple(rp, col, J, -F.T.copy())
    r = ro - linalg.bsr_matvec(rp, col, vo, du.T.copy())
    assert np.linalg.norm(r) <= 2e-11 * np.linalg.norm(ro)
    ref = np.linalg.solve(linalg.bsr_to_dense(rp, col, J), -F.T.reshape(-1)).reshape(case.n, 8).T
    assert np.max(np.abs(du - ref) / SCALE[:, None]) <= 1e-6 * np.max(np.abs(ref) / SCALE[:, None])
    g.close()


def test_reassembly_after_decoupling_overwrites_every_block(Simulator):
    # the Jacobian buffer is reused: a second assembly must not see the
    # previous (decoupled) system
    case = inp.small_box(4, 3, 2)
    a = inp.random_state(case, 11)
    b = inp.random_state(case, 12)
    g = _gpu_assembled(Simulator, case, a, b, 100.0)
    g.decouple()
    g.assemble(100.0)
    rp, col, J = g.jacobian()
    acc_old = model.old_accumulation(case, a["u"], a["coke"])
    _, _, Jo = model.jacobian(case, b["u"], a["coke"], acc_old, 100.0)
    assert jac_err(J, Jo, rp, case.n) < 1e-10
    g.close()


def test_newton_step_matches_oracle_on_tube(Simulator):
    case = inp.tube_case()
    dt = 20.0
    g = Simulator(case, tol_lin=1e-12, maxit_lin=400, tol_newton=0.0)
    g.init_equilibrium()
    u0, c0 = sim.initial_state(case)
    acc_old = model.old_accumulation(case, u0, c0)
    opts = sim.NewtonOptions(tol=0.0)
    opts.solve.solver = "dense"
    u = u0
    for k in range(3):
        info = g.newton_step(dt)
        r = sim.newton_step(case, u, c0, acc_old, dt, opts)
        u = r["u"]
        ug, _ = g.get_state()
        d = np.max(np.abs(ug - u) / SCALE[:, None])
        assert d < 1e-7, (k, d)
        g.set_state(u)   # continue both from the oracle's iterate
    g.close()


def _degenerate(name):
    if name == "single":
        case = inp.tube_case(n_cells=1)
        case.wells = case.wells[:1]           # one cell holds one well
        return case
    if name == "pair":
        return inp.tube_case(n_cells=2)
    if name == "nx1":
        return inp.small_box(1, 4, 3)
    if name == "flat":
        return inp.small_box(5, 3, 1)
    if name == "ny1":
        return inp.small_box(5, 1, 4)
    if name == "column":
        case = inp.small_box(1, 1, 6)
        case.wells = case.wells[:1]           # both wells of the box would share the column
        return case
    if name == "nowells":
        case = inp.small_box(3, 3, 2)
        case.wells = []                       # a closed box: no source term anywhere
        return case
    raise ValueError(name)


@pytest.mark.parametrize("name", ["single", "pair", "nx1", "flat", "ny1", "column", "nowells"])
def test_degenerate_grids(Simulator, name):
    case = _degenerate(name)
    a = inp.random_state(case, 31)
    b = inp.random_state(case, 32)
    dt = 60.0
    g = _gpu_assembled(Simulator, case, a, b, dt)
    acc_old = model.old_accumulation(case, a["u"], a["coke"])
    Fo = model.residual(case, b["u"], a["coke"], acc_old, dt)
    rp, col, J = g.jacobian()
    _, _, Jo = model.jacobian(case, b["u"], a["coke"], acc_old, dt)
    assert row_scaled_err(g.residual(), Fo) < 1e-10
    assert jac_err(J, Jo, rp, case.n) < 1e-10
    # the preconditioner on the oracle's decoupled system of the same grid
    _, _, Jo_, Fo_ = assembled(case, 31, 32, dt)
    vd, rd = linalg.gauss_jordan_decouple(rp.astype(np.int64), col.astype(np.int64), Jo_, Fo_.T.copy())
    g.set_system(vd, rd.T, decoupled=True)
    x = np.random.default_rng(2).standard_normal((8, case.n))
    g.build_preconditioner()
    z = g.precond_apply(x)
    zo = linalg.ILU0Preconditioner(rp.astype(np.int64), col.astype(np.int64), vd).apply(x.T.copy()).T
    assert np.max(np.abs(z - zo)) <= 1e-11 * np.abs(zo).max()
    info = g.solve()
    assert info.krylov_rel_residual <= 1e-6
    g.close()
