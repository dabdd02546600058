"""Pins of the oracle's decoupling and linear solvers (Sec. 3.2 and the
solver settings of Sec. 4.3) against dense LAPACK solves and the defining
properties of ILU(0)."""
import numpy as np
import pytest

import isc_inputs as inp
from oracle import linalg, model, sim


def _system(case, seed, dt=200.0):
    st = inp.random_state(case, seed)
    u0, c0 = sim.initial_state(case)
    acc_old = model.old_accumulation(case, u0, c0)
    rp, col, val = model.jacobian(case, st["u"], st["coke"], acc_old, dt)
    F = model.residual(case, st["u"], st["coke"], acc_old, dt)
    return rp, col, val, -F.T.copy()


def test_gauss_jordan_gives_identity_diagonal_and_equals_inverse_scaling():
    case = inp.small_box(4, 3, 2)
    rp, col, val, b = _system(case, 31)
    vd, bd = linalg.gauss_jordan_decouple(rp, col, val, b)
    rows = np.repeat(np.arange(case.n), np.diff(rp))
    diag = col == rows
    assert np.all(vd[diag] == np.eye(8))
    Dinv = np.linalg.inv(val[diag])          # LAPACK inverse of every J_ii
    ref = np.einsum("bij,bjk->bik", Dinv[rows], val)
    scale = np.abs(ref).reshape(len(ref), -1).max(axis=1)
    err = np.abs(vd - ref).reshape(len(ref), -1).max(axis=1)
    assert np.all(err[~diag] <= 1e-11 * np.maximum(scale[~diag], 1.0))
    assert np.allclose(bd, np.einsum("nij,nj->ni", Dinv, b), rtol=1e-11, atol=1e-11 * np.abs(bd).max())


def test_gauss_jordan_pivoting_handles_zero_leading_entry_and_detects_singular():
    rp = np.array([0, 1])
    col = np.array([0])
    A = np.random.default_rng(1).standard_normal((8, 8))
    A[:, 0] = 0.0
    A[3, 0] = 2.0                            # only row 3 can pivot column 0
    b = np.arange(8.0)[None, :]
    vd, bd = linalg.gauss_jordan_decouple(rp, col, A[None], b)
    assert np.allclose(bd[0], np.linalg.solve(A, b[0]), rtol=1e-12)
    A[3, 0] = 0.0
    with pytest.raises(linalg.SingularBlockError):
        linalg.gauss_jordan_decouple(rp, col, A[None], b)


def test_gauss_jordan_singularity_is_judged_against_the_pivot_row():
    """A pivot counts as zero when it is below 1e-300 times the largest entry of its
    own row in the diagonal block: an all-zero row is singular (also as the last pivot), and a 1e-290 pivot
    beside a 1e12 entry is singular while a 1e-280 one is still eliminated exactly."""
    rp, col = np.array([0, 1]), np.array([0])
    b = np.linspace(1.0, 2.0, 8)[None, :]
    for zero_row in (5, 7):
        A = np.eye(8)
        A[zero_row] = 0.0
        with pytest.raises(linalg.SingularBlockError):
            linalg.gauss_jordan_decouple(rp, col, A[None], b)
    A = np.eye(8)
    A[6, 7] = 1e12
    A[6, 6] = 1e-290
    with pytest.raises(linalg.SingularBlockError):
        linalg.gauss_jordan_decouple(rp, col, A[None], b)
    A[6, 6] = 1e-280
    vd, bd = linalg.gauss_jordan_decouple(rp, col, A[None], b)
    ref = np.linalg.solve(A, b[0])
    assert np.allclose(bd[0], ref, rtol=1e-12, atol=0)


def test_decoupled_and_original_systems_have_the_same_solution():
    case = inp.small_box(3, 2, 2)
    rp, col, val, b = _system(case, 32)
    x0 = np.linalg.solve(linalg.bsr_to_dense(rp, col, val), b.reshape(-1))
    vd, bd = linalg.gauss_jordan_decouple(rp, col, val, b)
    A1 = linalg.bsr_to_dense(rp, col, vd)
    x1 = np.linalg.solve(A1, bd.reshape(-1))
    # both are backward-stable solves of the same system: they differ by at
    # most cond * eps in the variable-scaled norm
    scale = np.tile(np.array([1e6, 1, 1, 1, 1, 100.0, 1, 1]), case.n)
    cond = np.linalg.cond(A1 * scale[None, :])
    d = np.max(np.abs(x1 - x0) / scale) / np.max(np.abs(x0) / scale)
    assert d <= 100 * cond * 2.2e-16


def test_ilu0_is_exact_lu_on_a_tube():
    # a block-tridiagonal matrix has no fill, so ILU(0) is the exact LU
    case = inp.tube_case(n_cells=20)
    rp, col, val, b = _system(case, 33)
    vd, bd = linalg.gauss_jordan_decouple(rp, col, val, b)
    M = linalg.ILU0Preconditioner(rp, col, vd)
    x = M.apply(bd)
    ref = np.linalg.solve(linalg.bsr_to_dense(rp, col, vd), bd.reshape(-1))
    assert np.allclose(x.reshape(-1), ref, rtol=1e-10, atol=1e-12 * np.abs(ref).max())


def test_ilu0_product_reproduces_matrix_on_its_pattern():
    # defining property: (L U)_ij = A_ij for every (i, j) in the pattern
    case = inp.small_box(4, 3, 3)
    rp, col, val, b = _system(case, 34)
    vd, _ = linalg.gauss_jordan_decouple(rp, col, val, b)
    F = linalg.block_ilu0(rp, col, vd)
    n = case.n
    rows = np.repeat(np.arange(n), np.diff(rp))
    L = np.zeros((n * 8, n * 8))
    U = np.zeros((n * 8, n * 8))
    for bb in range(len(col)):
        r, c = rows[bb], col[bb]
        (L if c < r else U)[r * 8:r * 8 + 8, c * 8:c * 8 + 8] = F[bb]
    L += np.eye(n * 8)
    P = L @ U
    A = linalg.bsr_to_dense(rp, col, vd)
    for bb in range(len(col)):
        r, c = rows[bb], col[bb]
        assert np.allclose(P[r * 8:r * 8 + 8, c * 8:c * 8 + 8], A[r * 8:r * 8 + 8, c * 8:c * 8 + 8], atol=1e-11 * np.abs(A).max())


@pytest.mark.parametrize("solver", ["gmres", "bicgstab"])
@pytest.mark.parametrize("prec", ["ilu0", "bjacobi", "none"])
def test_krylov_matches_dense_lu(solver, prec):
    case = inp.small_box(4, 3, 2)      # 192 unknowns
    rp, col, val, b = _system(case, 35)
    opts = sim.SolveOptions(solver=solver, prec=prec, rtol=1e-11, maxit=2000, restart=30)
    x, its, rel = sim.linear_solve(rp, col, val, b, opts)
    A = linalg.bsr_to_dense(rp, col, val)
    ref = np.linalg.solve(A, b.reshape(-1))
    vd, bd = linalg.gauss_jordan_decouple(rp, col, val, b)
    res = np.linalg.norm(bd.reshape(-1) - linalg.bsr_to_dense(rp, col, vd) @ x.reshape(-1)) / np.linalg.norm(bd)
    assert res <= 2e-11
    cond = np.linalg.cond(linalg.bsr_to_dense(rp, col, vd))
    assert np.linalg.norm(x.reshape(-1) - ref) <= 10 * cond * 1e-11 * np.linalg.norm(ref)


def test_bsr_matvec_is_the_library_bsr_product():
    """The oracle's block loop y_i = sum_b A_ib x_col(b) against scipy's BSR product."""
    import scipy.sparse as sp
    case = inp.small_box(5, 3, 2)
    rp, col, val, b = _system(case, 36)
    x = np.random.default_rng(3).standard_normal(b.shape)
    A = sp.bsr_matrix((val, col, rp), shape=(case.n * 8, case.n * 8))
    ref = A @ x.reshape(-1)
    y = linalg.bsr_matvec(rp, col, val, x).reshape(-1)
    bound = 1e-13 * (abs(A) @ np.abs(x.reshape(-1)))
    assert np.all(np.abs(y - ref) <= bound)


def _k_eigenvalue_matrix(n, lams, seed):
    """A = Q diag(lam) Q^T with len(set(lam)) distinct eigenvalues: for a generic b the
    Krylov space K_j(A, b) has dimension min(j, k), so GMRES from x0 = 0 reaches the
    exact solution at iteration k and not before."""
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    d = np.resize(np.asarray(lams, dtype=float), n)
    return (Q * d) @ Q.T, rng.standard_normal(n)


@pytest.mark.parametrize("lams", [[2.0], [1.0, 3.0], [1.0, 2.0, 5.0, 9.0], [0.5, 1.0, 2.0, 4.0, 7.0, 11.0]])
def test_gmres_terminates_at_the_degree_of_the_minimal_polynomial(lams):
    A, b = _k_eigenvalue_matrix(48, lams, 70 + len(lams))
    x, its, rel = linalg.gmres(lambda v: A @ v, b, restart=30, rtol=1e-10, maxit=100)
    assert its == len(lams)
    assert np.linalg.norm(b - A @ x) <= 1e-10 * np.linalg.norm(b)
    assert rel == pytest.approx(np.linalg.norm(b - A @ x) / np.linalg.norm(b), rel=1e-6, abs=1e-15)


def test_gmres_restart_and_iteration_cap():
    """GMRES(2) needs more than one cycle on six distinct eigenvalues; maxit caps the
    total count of Arnoldi steps over all cycles, and each cycle's correction
    minimises the residual over its Krylov space, so the residual never grows."""
    A, b = _k_eigenvalue_matrix(48, [0.5, 1.0, 2.0, 4.0, 7.0, 11.0], 81)
    prev = np.linalg.norm(b)
    for m in range(1, 8):
        x, its, rel = linalg.gmres(lambda v: A @ v, b, restart=2, rtol=1e-300, maxit=m)
        assert its == m
        r = np.linalg.norm(b - A @ x)
        assert r <= prev * (1 + 1e-12)
        prev = r
    x1, _, _ = linalg.gmres(lambda v: A @ v, b, restart=2, rtol=1e-300, maxit=1)
    # one Arnoldi step: x = (b.Ab / |Ab|^2) b, the 1-D residual minimiser
    Ab = A @ b
    assert np.allclose(x1, (b @ Ab) / (Ab @ Ab) * b, rtol=1e-12, atol=0)


@pytest.mark.parametrize("lams", [[3.0], [1.0, 3.0], [1.0, 2.0, 5.0, 9.0]])
def test_bicgstab_terminates_at_the_degree_of_the_minimal_polynomial(lams):
    """For symmetric positive definite A and shadow residual r^ = r0, BiCG is CG, whose
    polynomial annihilates r0 at step k; BiCGSTAB's intermediate residual s is that
    BiCG residual times the earlier stabilising factors, so it vanishes at step k."""
    A, b = _k_eigenvalue_matrix(40, lams, 90 + len(lams))
    for maxit in (100, len(lams)):
        x, its, rel = linalg.bicgstab(lambda v: A @ v, b, rtol=1e-10, maxit=maxit)
        assert its == len(lams)
        assert rel <= 1e-10
        assert np.linalg.norm(b - A @ x) <= 1e-9 * np.linalg.norm(b)


@pytest.mark.parametrize("solver", ["gmres", "bicgstab"])
def test_krylov_solvers_are_scale_invariant(solver):
    """Scaling b or A by a power of two scales every rounded operation exactly, so
    x(s b) = s x(b) and x(s A) = x(A) / s bit for bit, with the same iteration count
    and relative residual, down to right-hand sides near 1e-120 (where the squares
    in the residual norm are still normal numbers); only b = 0 returns
    x = 0 at once."""
    A, b = _k_eigenvalue_matrix(40, [1.0, 2.0, 5.0, 9.0], 95)
    f = getattr(linalg, solver)
    x1, i1, r1 = f(lambda v: A @ v, b, rtol=1e-10, maxit=100)
    for s in (2.0 ** -20, 2.0 ** -400):
        xs, i_s, rs = f(lambda v: A @ v, s * b, rtol=1e-10, maxit=100)
        assert i_s == i1 and rs == r1
        assert np.array_equal(xs, s * x1)
    for sa in (2.0 ** -14, 2.0 ** 14):
        xa, i_a, ra = f(lambda v: sa * (A @ v), b, rtol=1e-10, maxit=100)
        assert i_a == i1 and ra == r1
        assert np.array_equal(xa, x1 / sa)
    x0, i0, r0 = f(lambda v: A @ v, 0 * b, rtol=1e-10, maxit=100)
    assert i0 == 0 and r0 == 0.0 and not np.any(x0)


def test_bicgstab_step_minimises_the_residual_along_its_stabilising_direction():
    """One BiCGSTAB step from x0 = 0 (no preconditioner, shadow residual r0 = b): the
    BiCG half-step x = alpha b with alpha = b.b / b.Ab leaves s = b - alpha Ab, then the
    stabilising step x += omega s picks omega so that the new residual is orthogonal
    to A s (the one-dimensional minimal residual)."""
    A, b = _k_eigenvalue_matrix(40, [1.0, 2.0, 5.0, 9.0], 97)
    A = A + 0.3 * np.triu(np.random.default_rng(5).standard_normal((40, 40)), 1) / 40
    x1, its, rel = linalg.bicgstab(lambda v: A @ v, b, rtol=1e-300, maxit=1)
    assert its == 1
    alpha = (b @ b) / (b @ (A @ b))
    s = b - alpha * (A @ b)
    d = x1 - alpha * b                      # the stabilising correction: a multiple of s
    assert np.linalg.norm(d - (d @ s) / (s @ s) * s) <= 1e-12 * np.linalg.norm(d)
    r1 = b - A @ x1
    As = A @ s
    assert abs(r1 @ As) <= 1e-12 * np.linalg.norm(r1) * np.linalg.norm(As)
    assert rel == pytest.approx(np.linalg.norm(r1) / np.linalg.norm(b), rel=1e-10)
