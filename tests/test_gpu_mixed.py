"""Mixed precision. `mixed`: the block ILU(0) factors are computed, stored and
applied in FP32 inside the FP64 GMRES; the preconditioner agrees with the FP64
oracle to FP32 accuracy. `mixed_fgmres`: the FP64 GMRES is flexible and its
preconditioner is a fixed number of FP32 GMRES iterations (FP32 SpMV, FP32
Gram-Schmidt, FP32 ILU(0)); that inner solve agrees with the oracle's GMRES
iterate of the same length to FP32 accuracy. Both reach the FP64 relative
residual of the Newton update (error against the oracle stated in the
assertions)."""
import numpy as np
import pytest

import isc_inputs as inp
from oracle import linalg, model
from oracle_system import assembled, decoupled

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def Simulator():
    from paper_1811_11992_gb300 import build
    build.build()
    from paper_1811_11992_gb300 import Simulator as S
    return S


def _assembled(S, case, **opt):
    a = inp.random_state(case, 1201)
    b = inp.random_state(case, 1202)
    g = S(case, **opt)
    g.set_state(a["u"], a["coke"])
    g.begin_step()
    g.set_state(b["u"])
    g.assemble(100.0)
    return g, a, b


@pytest.mark.parametrize("dims", [(7, 5, 5), (13, 4, 3), (1, 6, 4)])
def test_fp32_ilu0_apply_matches_fp64_oracle(Simulator, dims):
    case = inp.small_box(*dims)
    rp, col, _, _, Jd, Fd = decoupled(case, 1201, 1202)
    g = Simulator(case, precision="mixed")
    g.set_system(Jd, Fd, decoupled=True)
    g.build_preconditioner()
    x = np.random.default_rng(9).standard_normal((8, case.n))
    z = g.precond_apply(x)
    zo = linalg.ILU0Preconditioner(rp, col, Jd).apply(x.T.copy()).T
    err = np.max(np.abs(z - zo)) / np.abs(zo).max()
    assert err < 2e-5, err          # FP32 factors and sweeps
    assert err > 1e-12              # really FP32
    g.close()


def test_mixed_solve_reaches_fp64_tolerance(Simulator):
    case = inp.small_box(7, 5, 5)
    tol = 1e-10
    rp, col, J, F = assembled(case, 1201, 1202)
    g = Simulator(case, precision="mixed", tol_lin=tol, maxit_lin=2000)
    g.set_system(J, F)
    g.decouple()
    info = g.solve()
    du = g.newton_update()
    vo, ro = linalg.gauss_jordan_decouple(rp, col, J, -F.T.copy())
    res = np.linalg.norm(ro - linalg.bsr_matvec(rp, col, vo, du.T.copy())) / np.linalg.norm(ro)
    assert res <= 2 * tol, res      # FP64 residual in the oracle's own decoupled system
    ref = np.linalg.solve(linalg.bsr_to_dense(rp, col, J), -F.T.reshape(-1)).reshape(case.n, 8).T
    scale = np.array([1e6, 1, 1, 1, 1, 100.0, 1, 1])[:, None]
    rel = np.max(np.abs(du - ref) / scale) / np.max(np.abs(ref) / scale)
    assert rel < 1e-5, rel
    g.close()


def test_mixed_newton_step_on_field_block(Simulator):
    case = inp.field_case(12, 12, 6, 0, 1, "field 12x12x6", 30 * inp.DAY, 40)
    res = {}
    for prec in ("fp64", "mixed"):
        g = Simulator(case, precision=prec, tol_lin=1e-6)
        g.init_equilibrium()
        info = g.newton_step(case.dt0)
        u, _ = g.get_state()
        res[prec] = (u, info.krylov_iterations, info.krylov_rel_residual)
        g.close()
    assert res["mixed"][2] <= 1e-6
    assert res["mixed"][1] <= res["fp64"][1] + 3
    scale = np.array([1e6, 1, 1, 1, 1, 100.0, 1, 1])[:, None]
    # both Newton updates solve the same system to 1e-6: they agree to about that level
    assert np.max(np.abs(res["mixed"][0] - res["fp64"][0]) / scale) < 1e-3


U32 = 2.0 ** -24   # FP32 unit roundoff


def _oracle_decoupled(case, dt):
    """The oracle's decoupled system (assembly of Sec. 3.1, Gauss-Jordan of Sec. 3.2)
    at the case's initial state for step size dt."""
    from oracle import sim
    u0, c0 = sim.initial_state(case)
    acc = model.old_accumulation(case, u0, c0)
    F = model.residual(case, u0, c0, acc, dt)
    rp, col, J = model.jacobian(case, u0, c0, acc, dt)
    vd, rd = linalg.gauss_jordan_decouple(rp, col, J, F.T.copy())
    return rp, col, vd, rd


def _gmres_iterate(rp, col, A, b, m, M, rng=None):
    """The oracle's GMRES iterate after m iterations from x0 = 0 (b, x as (8, N)).
    With rng, every matrix-vector product and preconditioner application is
    perturbed by a relative +-u32 per entry: a model of FP32 kernels rounding
    their outputs at each iteration."""
    def noisy(v):
        return v if rng is None else v * (1 + U32 * rng.choice([-1.0, 1.0], v.shape))

    class P:
        def apply(self, v):
            return noisy(M.apply(v))

    x, its, _ = linalg.gmres(lambda v: noisy(linalg.bsr_matvec(rp, col, A, v)), b.T.copy(), P(), restart=m,
                             rtol=1e-300, maxit=m)
    assert its == m
    return x.T


@pytest.mark.parametrize("dt,m", [(1000.0, 1), (1000.0, 8), (1000.0, 20), (None, 8), (None, 20)])
def test_fgmres_inner_solve_is_the_oracle_gmres_iterate(Simulator, dt, m):
    """The preconditioner of mixed_fgmres is m iterations of ILU(0)-preconditioned
    GMRES from x0 = 0 on the FP32 copy of the decoupled matrix: the oracle's FP64
    GMRES stopped after m iterations on that same rounded matrix (and the ILU(0)
    of it) gives the same iterate, to the FP32 arithmetic of the GPU's Krylov
    vectors, sweeps and SpMV. The bound is S u32 times 64: S is the iterate's
    measured sensitivity to FP32 rounding (two more oracle runs whose every
    product and preconditioner output carries a relative +-u32 perturbation,
    largest deviation over u32), 64 covers the rounding accumulated inside each
    kernel's output (up to 48 products per SpMV row, the sweeps' chains). At
    the workload's first step GMRES stagnates and S is in the thousands; at a
    1000 s step it is about 60. (The residual in that matrix is not compared: a
    1e-6 relative change of the iterate moves it by the condition number times
    as much.) The system is the oracle's, loaded through isc_set_system."""
    case = inp.field_case(13, 7, 3, 0, 1, "field 13x7x3", 30 * inp.DAY, 40)
    rp, col, vd, rd = _oracle_decoupled(case, dt or case.dt0)
    g = Simulator(case, precision="mixed_fgmres", inner_its=m)
    g.set_system(vd, rd.T, decoupled=True)
    g.build_preconditioner()
    A32 = vd.astype(np.float32).astype(np.float64)
    r = np.random.default_rng(31).standard_normal((8, case.n))
    r32 = r.astype(np.float32).astype(np.float64)
    z = g.precond_apply(r)
    M = linalg.ILU0Preconditioner(rp, col, A32)
    x = _gmres_iterate(rp, col, A32, r32, m, M)
    rng = np.random.default_rng(32)
    sens = max(np.max(np.abs(_gmres_iterate(rp, col, A32, r32, m, M, rng) - x)) for _ in range(2))
    sens = sens / np.abs(x).max() / U32
    err = np.max(np.abs(z - x)) / np.abs(x).max()
    assert err <= 64 * max(sens, 1.0) * U32, (err, sens, err / (max(sens, 1.0) * U32))
    assert err > 1e-9, err         # really FP32
    g.close()


def test_mixed_fgmres_solve_reaches_fp64_tolerance(Simulator):
    case = inp.small_box(7, 5, 5)
    tol = 1e-10
    rp, col, J, F = assembled(case, 1201, 1202)
    g = Simulator(case, precision="mixed_fgmres", inner_its=10, tol_lin=tol, maxit_lin=400)
    g.set_system(J, F)
    g.decouple()
    info = g.solve()
    du = g.newton_update()
    vo, ro = linalg.gauss_jordan_decouple(rp, col, J, -F.T.copy())
    res = np.linalg.norm(ro - linalg.bsr_matvec(rp, col, vo, du.T.copy())) / np.linalg.norm(ro)
    assert res <= 2 * tol, res      # FP64 residual in the oracle's own decoupled system
    ref = np.linalg.solve(linalg.bsr_to_dense(rp, col, J), -F.T.reshape(-1)).reshape(case.n, 8).T
    scale = np.array([1e6, 1, 1, 1, 1, 100.0, 1, 1])[:, None]
    rel = np.max(np.abs(du - ref) / scale) / np.max(np.abs(ref) / scale)
    assert rel < 1e-5, rel
    g.close()


def test_mixed_fgmres_newton_step_on_field_block(Simulator):
    case = inp.field_case(12, 12, 6, 0, 1, "field 12x12x6", 30 * inp.DAY, 40)
    res = {}
    for prec in ("fp64", "mixed_fgmres"):
        g = Simulator(case, precision=prec, tol_lin=1e-6)
        g.init_equilibrium()
        info = g.newton_step(case.dt0)
        u, _ = g.get_state()
        res[prec] = (u, info.krylov_iterations, info.krylov_rel_residual)
        g.close()
    assert res["mixed_fgmres"][2] <= 1e-6
    scale = np.array([1e6, 1, 1, 1, 1, 100.0, 1, 1])[:, None]
    assert np.max(np.abs(res["mixed_fgmres"][0] - res["fp64"][0]) / scale) < 1e-3


@pytest.mark.parametrize("opt", [dict(prec="bjacobi"), dict(krylov="bicgstab"), dict(inner_its=0), dict(inner_its=33)])
def test_mixed_fgmres_option_checks(Simulator, opt):
    from paper_1811_11992_gb300.isc import IscError
    case = inp.small_box(3, 3, 2)
    with pytest.raises(IscError):
        Simulator(case, precision="mixed_fgmres", **opt)
