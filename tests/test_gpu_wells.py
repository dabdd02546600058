"""GPU coupled producers (bottom-hole pressure unknown, Sec. 2.2 Well
Modeling) against the oracle: residual, perforation blocks and the border
(B, C, D, F_w) of the Newton system; the bordered SpMV after decoupling; the
preconditioner's well rows; and a rate-controlled time step."""
import numpy as np
import pytest

import isc_inputs as inp
from oracle import linalg, model, sim

pytestmark = pytest.mark.gpu

CONTROLS = {"bhp": (inp.CTRL_BHP, 4.55e6), "oil": (inp.CTRL_OIL_RATE, 0.05), "total": (inp.CTRL_TOTAL_RATE, 5.0),
            "liquid": (inp.CTRL_LIQUID_RATE, 4.0)}


@pytest.fixture(scope="module")
def Simulator():
    from paper_1811_11992_gb300 import build
    build.build()
    from paper_1811_11992_gb300 import Simulator as S
    return S


def _case(control):
    ctl, target = CONTROLS[control]
    return inp.with_coupled_producer(inp.small_box(4, 3, 2), ctl, target, 4.6e6)


@pytest.mark.parametrize("control", list(CONTROLS))
def test_residual_and_border_match_oracle(Simulator, control):
    case = _case(control)
    a = inp.random_state(case, 301)
    b = inp.random_state(case, 302)
    bhp = np.array([4.4e6])
    g = Simulator(case)
    g.set_state(a["u"], a["coke"])
    g.begin_step()
    g.set_state(b["u"])
    g.set_well_bhp(bhp)
    g.assemble(100.0)
    F = g.residual()
    rp, col, J = g.jacobian()
    B, C, D, Fw = g.well_system()
    acc = model.old_accumulation(case, a["u"], a["coke"])
    F_ref = model.residual(case, b["u"], a["coke"], acc, 100.0, bhp=bhp)
    rowscale = np.abs(F_ref).max(axis=1, keepdims=True) + 1e-300
    assert np.max(np.abs(F - F_ref) / rowscale) <= 1e-10
    rp_o, col_o, J_ref = model.jacobian(case, b["u"], a["coke"], acc, 100.0, bhp=bhp)
    cells = model.coupled_wells(case)[0].cells
    rows = np.repeat(np.arange(case.n), np.diff(rp))
    for c in cells:
        blk = np.flatnonzero((rows == c) & (col == c))[0]
        sc = np.abs(J_ref[blk]).max()
        assert np.max(np.abs(J[blk] - J_ref[blk])) <= 1e-10 * sc
    B_ref, C_ref, D_ref, Fw_ref = model.coupled_blocks(case, b["u"], bhp, a["coke"], acc, 100.0)
    assert np.max(np.abs(B - B_ref)) <= 1e-10 * np.abs(B_ref).max()
    if control != "bhp":
        assert np.max(np.abs(C - C_ref)) <= 1e-10 * np.abs(C_ref).max()
    else:
        assert np.all(C == 0.0) and np.all(C_ref == 0.0)
    np.testing.assert_allclose(D, D_ref, rtol=1e-10)
    np.testing.assert_allclose(Fw, Fw_ref, rtol=1e-10, atol=1e-12 * abs(case.wells[-1].target))
    g.close()


def _dense_bordered(case, rp, col, J, B, C, D):
    n, nw = case.n, len(D)
    A = np.zeros((8 * n + nw, 8 * n + nw))
    A[:8 * n, :8 * n] = linalg.bsr_to_dense(rp.astype(np.int64), col.astype(np.int64), J)
    q = 0
    for k, w in enumerate(model.coupled_wells(case)):
        for c in w.cells:
            A[8 * c:8 * c + 8, 8 * n + k] = B[q]
            A[8 * n + k, 8 * c:8 * c + 8] = C[q]
            q += 1
        A[8 * n + k, 8 * n + k] = D[k]
    return A


def test_bordered_spmv_after_decoupling_and_preconditioner_well_rows(Simulator):
    case = _case("oil")
    u, c = sim.initial_state(case)
    g = Simulator(case)
    g.init_equilibrium()
    g.assemble(100.0)
    rp, col, J = g.jacobian()
    B, C, D, _ = g.well_system()
    g.decouple()
    g.build_preconditioner()
    # decoupling scales each cell row, the border column included, by J_ii^-1
    rows = np.repeat(np.arange(case.n), np.diff(rp))
    Jd, Bd = J.copy(), B.copy()
    diag = {int(r): np.flatnonzero((rows == r) & (col == r))[0] for r in range(case.n)}
    for r in range(case.n):
        Jd[rows == r] = np.linalg.solve(J[diag[r]], J[rows == r].transpose(1, 0, 2).reshape(8, -1)).reshape(
            8, -1, 8).transpose(1, 0, 2)
    for q, cell in enumerate(model.coupled_wells(case)[0].cells):
        Bd[q] = np.linalg.solve(J[diag[int(cell)]], B[q])
    A = _dense_bordered(case, rp, col, Jd, Bd, C, D)
    x = np.random.default_rng(4).standard_normal(8 * case.n + 1)
    y = g.spmv_full(x)
    np.testing.assert_allclose(y, A @ x, rtol=1e-10, atol=1e-10 * np.abs(A @ x).max())
    # the preconditioner's well row: z_w = (r_w - C . z_cells) / D
    r = np.random.default_rng(5).standard_normal(8 * case.n + 1)
    z = g.precond_apply_full(r)
    cells = model.coupled_wells(case)[0].cells
    zc = z[:8 * case.n].reshape(case.n, 8)
    expect = (r[-1] - sum(C[q] @ zc[cell] for q, cell in enumerate(cells))) / D[0]
    assert z[-1] == pytest.approx(expect, rel=1e-12)
    g.close()


@pytest.mark.parametrize("control", ["total", "bhp"])
def test_time_step_matches_oracle(Simulator, control):
    case = _case(control)
    u0, c0 = sim.initial_state(case)
    opts = sim.NewtonOptions(tol=1e-11, maxit=40)
    u_ref, b_ref, c_ref, its, ok = sim.timestep_coupled(case, u0, np.array([4.6e6]), c0, 10.0, opts)
    assert ok
    g = Simulator(case, tol_newton=1e-11, tol_lin=1e-12, maxit_newton=40)
    g.init_equilibrium()
    g.timestep(10.0)
    u, coke = g.get_state()
    bhp = g.well_bhp()
    assert abs(bhp[0] - b_ref[0]) <= 1e-7 * b_ref[0]
    assert np.max(np.abs(u[0] - u_ref[0]) / u_ref[0]) <= 1e-7
    assert np.max(np.abs(u[5] - u_ref[5]) / u_ref[5]) <= 1e-7
    assert np.max(np.abs(u[6:] - u_ref[6:])) <= 1e-7
    if control == "total":
        bp = model.base_properties(case, u)
        Q = model.coupled_phase_rates(case, bp, model.coupled_wells(case)[0], bhp[0])
        assert -sum(np.sum(q) for q in Q) == pytest.approx(CONTROLS["total"][1], rel=1e-8)
    g.close()


@pytest.mark.parametrize("prec,precision", [("cpr", "fp64"), ("cpr", "mixed"), ("bilu0", "mixed_fgmres"),
                                            ("cpr", "mixed_fgmres")])
def test_coupled_well_time_step_under_other_solvers(Simulator, prec, precision):
    """The bordered system with CPR-PF and the mixed-precision solves: the well rows
    follow the cells' preconditioner (block lower-triangular), and the time step
    reaches the FP64 ILU(0) state and bottom-hole pressure within the Newton
    tolerance."""
    case = _case("total")
    res = {}
    for key, p, q in (("ref", "bilu0", "fp64"), ("alt", prec, precision)):
        g = Simulator(case, prec=p, precision=q, tol_newton=1e-10, tol_lin=1e-10, maxit_newton=40)
        g.init_equilibrium()
        g.timestep(10.0)
        res[key] = (g.get_state()[0], g.well_bhp())
        g.close()
    (u_r, b_r), (u_a, b_a) = res["ref"], res["alt"]
    assert abs(b_a[0] - b_r[0]) <= 1e-7 * b_r[0]
    scale = np.array([5e6, 1, 1, 1, 1, 300, 1, 1])[:, None]
    assert np.max(np.abs(u_a - u_r) / scale) <= 1e-7
