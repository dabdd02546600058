"""Parity where the pencil kernels change schedule: grids with more x-pencils
(ny*nz) than the factorisation and sweep kernels keep resident warps, so that
warps take several pencils from the counter and the hand-off ordering runs
past its first round. The inputs come from the oracle alone (its assembly and
Gauss-Jordan decoupling of Sec. 3.2), loaded through isc_set_system; the GPU's
D^-1 blocks and ILU(0) apply are compared element by element with the
oracle's textbook block ILU(0) (IKJ form). FP64 at 1e-11 (apply) and 1e-10
(inverse blocks, relative to the block); FP32 factors and sweeps at the FP32
unit roundoff times the blocks' condition numbers, against the oracle on the
FP32-rounded matrix."""
import numpy as np
import pytest

import isc_inputs as inp
from oracle import linalg, model

pytestmark = pytest.mark.gpu

# 4 x 80 x 64: 20,480 cells and 5,120 pencils, more than the 152 SMs x 32 resident warps
# of the factorisation (4,864, one pencil per warp). The sweeps hold two pencils per warp on
# grids this large: 2 x 160 x 100 (32,000 cells, 16,000 pencils, 8,000 pencil pairs) is
# beyond both the FP64 sweeps' 152 x 24 resident warps (3,648) and the FP32 sweeps'
# 152 x 32 (4,864), so that there warps take a second pair from the counter as well.
GRIDS = [(4, 80, 64), (3, 90, 70), (2, 160, 100)]


@pytest.fixture(scope="module")
def Simulator():
    from paper_1811_11992_gb300 import build
    build.build()
    from paper_1811_11992_gb300 import Simulator as S
    return S


def _oracle_system(case, seed):
    """The oracle's residual and Jacobian at a random state, decoupled by the
    oracle's Gauss-Jordan elimination."""
    a = inp.random_state(case, seed)
    b = inp.random_state(case, seed + 1)
    acc = model.old_accumulation(case, a["u"], a["coke"])
    F = model.residual(case, b["u"], a["coke"], acc, 100.0)
    rp, col, J = model.jacobian(case, b["u"], a["coke"], acc, 100.0)
    vd, rd = linalg.gauss_jordan_decouple(rp, col, J, F.T.copy())
    return rp, col, J, F, vd, rd


@pytest.fixture(scope="module", params=GRIDS, ids=lambda d: "x".join(map(str, d)))
def system(request):
    nx, ny, nz = request.param
    case = inp.field_case(nx, ny, nz, 0, 9, f"field {nx}x{ny}x{nz}", inp.DAY, 4)
    assert ny * nz > 152 * 32
    rp, col, J, F, vd, rd = _oracle_system(case, 2101)
    Fi = linalg.block_ilu0(rp, col, vd)
    rows = np.repeat(np.arange(case.n), np.diff(rp))
    Dinv_o = np.linalg.inv(Fi[col == rows])
    M = linalg.ILU0Preconditioner(rp, col, vd)
    x = np.random.default_rng(17).standard_normal((case.n, 8))
    zo = M.apply(x)
    return dict(case=case, rp=rp, col=col, vd=vd, rd=rd, Dinv=Dinv_o, x=x, zo=zo)


def test_fp64_ilu0_factor_and_sweeps_beyond_one_round_of_warps(Simulator, system):
    case = system["case"]
    g = Simulator(case, precision="fp64")
    g.set_system(system["vd"], system["rd"].T, decoupled=True)
    g.build_preconditioner()
    D = g.ilu_diag()
    Do = system["Dinv"]
    scale = np.abs(Do).reshape(case.n, -1).max(axis=1)
    err_d = (np.abs(D - Do).reshape(case.n, -1).max(axis=1) / scale).max()
    assert err_d < 1e-10, err_d
    z = g.precond_apply(system["x"].T)
    zo = system["zo"].T
    err = np.max(np.abs(z - zo)) / np.abs(zo).max()
    assert err < 1e-11, err
    # the same apply twice (fresh sentinels and counters each call)
    assert np.array_equal(z, g.precond_apply(system["x"].T))
    g.close()


U32 = 2.0 ** -24   # FP32 unit roundoff


def test_fp32_ilu0_factor_and_sweeps_beyond_one_round_of_warps(Simulator, system):
    """FP32 factors and sweeps against the oracle's FP64 block ILU(0) of the
    FP32-rounded matrix (the rounding of the inputs is the mixed scheme's
    choice; what is compared is the kernels' FP32 arithmetic). Each inverse
    block within 64 kappa(D_i) u32 of the oracle's (kappa the block's
    infinity-norm condition number), the apply within 64 kappa_max u32 of
    max |z|, and further than FP64 rounding from the unrounded oracle."""
    case = system["case"]
    rp, col = system["rp"], system["col"]
    v32 = system["vd"].astype(np.float32).astype(np.float64)
    Fi = linalg.block_ilu0(rp, col, v32)
    rows = np.repeat(np.arange(case.n), np.diff(rp))
    Dd = Fi[col == rows]
    Do = np.linalg.inv(Dd)
    kappa = np.abs(Dd).sum(axis=2).max(axis=1) * np.abs(Do).sum(axis=2).max(axis=1)
    g = Simulator(case, precision="mixed")
    g.set_system(system["vd"], system["rd"].T, decoupled=True)
    g.build_preconditioner()
    D = g.ilu_diag()
    scale = np.abs(Do).reshape(case.n, -1).max(axis=1)
    err_d = np.abs(D - Do).reshape(case.n, -1).max(axis=1) / scale
    assert np.all(err_d <= 64 * kappa * U32), (err_d / (kappa * U32)).max()
    x32 = system["x"].astype(np.float32).astype(np.float64)
    zo = linalg.ILU0Preconditioner(rp, col, v32).apply(x32).T
    z = g.precond_apply(system["x"].T)
    err = np.max(np.abs(z - zo)) / np.abs(zo).max()
    assert err <= 64 * kappa.max() * U32, (err, kappa.max())
    assert np.max(np.abs(z - system["zo"].T)) / np.abs(zo).max() > 1e-12     # really FP32
    assert np.array_equal(z, g.precond_apply(system["x"].T))
    g.close()


@pytest.mark.parametrize("orth", ["cgs2", "cgs1"])
def test_spmv_and_gmres_on_the_oracle_system(Simulator, system, orth):
    """GMRES with classical Gram-Schmidt twice or once: either way the update's
    residual in the oracle's own decoupled system meets the tolerance."""
    case = system["case"]
    g = Simulator(case, tol_lin=1e-10, maxit_lin=3000, orth=orth)
    g.set_system(system["vd"], system["rd"].T, decoupled=True)
    x = system["x"]
    y = g.spmv(x.T)
    yo = linalg.bsr_to_scipy(system["rp"], system["col"], system["vd"]) @ x.reshape(-1)
    yo = yo.reshape(case.n, 8).T
    assert np.max(np.abs(y - yo)) <= 1e-13 * np.abs(yo).max()
    if case.n > 25_000:
        # the 2 x 160 x 100 grid is here for the sweeps' second round of pencil pairs; the
        # system of a random state on it is beyond GMRES(30) with ILU(0) at this tolerance
        # (the oracle's own GMRES stands at a relative residual of 8e-3 after 300
        # iterations), so there only the SpMV is compared
        g.close()
        return
    info = g.solve()
    du = g.newton_update()
    # the update's residual in the oracle's own decoupled system (J du = -F)
    A = linalg.bsr_to_scipy(system["rp"], system["col"], system["vd"])
    b = -system["rd"].reshape(-1)
    res = np.linalg.norm(b - A @ du.T.reshape(-1)) / np.linalg.norm(b)
    assert info.krylov_rel_residual <= 1e-10
    assert res <= 2e-10, res
    g.close()


def test_solve_external_matches_dense_lu_on_a_tiny_system(Simulator):
    """isc_solve_external on the oracle's (not decoupled) system of a 4x3x2
    box: decoupling, ILU(0) and GMRES inside, x against the oracle's dense LU."""
    case = inp.small_box(4, 3, 2)
    rp, col, J, F, _, _ = _oracle_system(case, 2201)
    g = Simulator(case, tol_lin=1e-12, maxit_lin=500)
    b = np.random.default_rng(4).standard_normal((8, case.n))
    x, info = g.solve_external(rp, col, J, b)
    ref = np.linalg.solve(linalg.bsr_to_dense(rp, col, J), b.T.reshape(-1)).reshape(case.n, 8).T
    scale = np.array([1e6, 1, 1, 1, 1, 100.0, 1, 1])[:, None]
    # the dense solution in the unknowns' own units, against the solver tolerance times the condition
    assert np.max(np.abs(x - ref) / scale) <= 1e-6 * np.max(np.abs(ref) / scale)
    assert info.krylov_rel_residual <= 1e-12
    # a matrix off the handle's pattern is refused
    bad = rp.copy()
    bad[1] += 1
    with pytest.raises(Exception):
        g.solve_external(bad, col, J, b)
    g.close()


def test_set_system_checks_the_declared_unit_diagonal(Simulator):
    case = inp.small_box(3, 3, 2)
    rp, col, J, F, vd, rd = _oracle_system(case, 2301)
    g = Simulator(case)
    with pytest.raises(Exception):
        g.set_system(J, F, decoupled=True)      # the assembled diagonal blocks are not I
    g.set_system(vd, rd.T, decoupled=True)
    g.close()
