"""Pins of the oracle's CPR-PF preconditioner (oracle/cpr.py) to facts that do
not come from the oracle itself: exact solves where the method reduces to one,
properties of the Galerkin product, convergence of the smoother and the
V-cycle on textbook problems, and the two-stage formula (an exact second stage
must give the exact inverse)."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import isc_inputs as inp
from oracle import cpr, linalg, model, sim


def _lap1(m, w):
    return sp.diags([-w * np.ones(m - 1), 2 * w * np.ones(m), -w * np.ones(m - 1)], [-1, 0, 1])


def _poisson(nx, ny, nz, wz=10.0, shift=1e-3):
    I = sp.identity
    A = (sp.kron(I(nz), sp.kron(I(ny), _lap1(nx, 1.0))) + sp.kron(I(nz), sp.kron(_lap1(ny, 1.0), I(nx)))
         + sp.kron(_lap1(nz, wz), sp.kron(I(ny), I(nx))))
    return (A + shift * sp.identity(nx * ny * nz)).tocsr()


def _random_stencil(nx, ny, nz, seed, symmetric, margin=(0.01, 0.1)):
    """A 7-point M-matrix with random couplings, strictly diagonally dominant
    by a random margin per row."""
    rng = np.random.default_rng(seed)
    n = nx * ny * nz
    idx = np.arange(n).reshape(nz, ny, nx)
    rows, cols, vals = [], [], []
    for a, b in ((idx[:, :, :-1], idx[:, :, 1:]), (idx[:, :-1, :], idx[:, 1:, :]), (idx[:-1], idx[1:])):
        a, b = a.reshape(-1), b.reshape(-1)
        w = rng.uniform(0.1, 2.0, a.size)
        w2 = w if symmetric else w * rng.uniform(0.5, 1.5, a.size)
        rows += [a, b]
        cols += [b, a]
        vals += [-w, -w2]
    off = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n, n))
    d = -np.asarray(off.sum(axis=1)).ravel() + rng.uniform(*margin, n)
    return (off + sp.diags(d)).tocsr()


def test_single_column_level_is_an_exact_tridiagonal_solve():
    A = _random_stencil(1, 1, 17, 3, symmetric=False)
    mg = cpr.AggregationMG(A, 1, 1, 17)
    assert len(mg.A) == 1
    b = np.random.default_rng(4).standard_normal(17)
    np.testing.assert_allclose(mg.vcycle(b), spla.spsolve(A.tocsc(), b), rtol=1e-12)


def test_galerkin_coarse_operator_row_sums_symmetry_and_pattern():
    nx, ny, nz = 7, 6, 3
    A = _random_stencil(nx, ny, nz, 5, symmetric=True)
    mg = cpr.AggregationMG(A, nx, ny, nz)
    assert mg.dims == [(7, 6, 3), (4, 3, 3), (2, 2, 3), (1, 1, 3)]
    for l, P in enumerate(mg.P):
        Ac = mg.A[l + 1]
        # P^T A 1 = A_c 1 (P 1_c = 1_f for a piecewise-constant P)
        np.testing.assert_allclose(Ac @ np.ones(Ac.shape[0]), P.T @ (mg.A[l] @ np.ones(P.shape[0])), rtol=1e-13)
        np.testing.assert_allclose(Ac.toarray(), Ac.toarray().T, rtol=1e-13, atol=1e-15)
        # aggregates that only touch at a corner are not coupled (5-point x-y structure)
        cx, cy, _ = mg.dims[l + 1]
        if cx > 1 and cy > 1:
            assert Ac[0, 1 + cx] == 0.0
    # every fine cell lies in exactly one aggregate
    for P in mg.P:
        np.testing.assert_array_equal(np.asarray(P.sum(axis=1)).ravel(), 1.0)


def test_red_black_line_gauss_seidel_converges_to_the_solution():
    nx, ny, nz = 6, 5, 4
    # Gauss-Seidel converges for strictly diagonally dominant matrices
    A = _random_stencil(nx, ny, nz, 7, symmetric=False, margin=(0.5, 1.0))
    mg = cpr.AggregationMG(A, nx, ny, nz)
    b = np.random.default_rng(8).standard_normal(A.shape[0])
    x = mg.smooth(0, np.zeros_like(b), b, 100)
    np.testing.assert_allclose(x, spla.spsolve(A.tocsc(), b), rtol=1e-9)


def test_vcycle_reduces_an_anisotropic_poisson_residual():
    A = _poisson(16, 16, 8)
    mg = cpr.AggregationMG(A, 16, 16, 8)
    b = np.random.default_rng(1).standard_normal(A.shape[0])
    x = np.zeros_like(b)
    prev = np.linalg.norm(b)
    for _ in range(4):
        x = x + mg.vcycle(b - A @ x)
        cur = np.linalg.norm(b - A @ x)
        assert cur < 0.1 * prev
        prev = cur


@pytest.fixture(scope="module")
def field_block():
    case = inp.field_case(16, 12, 6, 0, 1, "f", 30 * inp.DAY, 40)
    u, c = sim.initial_state(case)
    acc = model.old_accumulation(case, u, c)
    F = model.residual(case, u, c, acc, case.dt0)
    rp, col, val = model.jacobian(case, u, c, acc, case.dt0)
    vd, rhs = linalg.gauss_jordan_decouple(rp, col, val, -F.T.copy())
    return case, rp, col, vd, rhs


def test_pressure_matrix_holds_the_pressure_entries(field_block):
    case, rp, col, vd, _ = field_block
    Ap = cpr.pressure_matrix(rp, col, vd).toarray()
    D = linalg.bsr_to_dense(rp, col, vd)
    np.testing.assert_array_equal(Ap, D[0::8, 0::8])
    np.testing.assert_allclose(np.diag(Ap), 1.0, rtol=0, atol=1e-14)   # decoupled: unit diagonal blocks


class _Exact:
    def __init__(self, A, n):
        self.lu = spla.splu(A.tocsc())
        self.n = n

    def apply(self, r):
        return self.lu.solve(np.asarray(r).reshape(-1)).reshape(self.n, 8)


class _Zero:
    def apply(self, r):
        return np.zeros_like(r)


def test_two_stage_formula(field_block):
    case, rp, col, vd, _ = field_block
    n = case.n
    A = linalg.bsr_to_scipy(rp, col, vd)
    r = np.random.default_rng(11).standard_normal((n, 8))
    # an exact second stage makes the preconditioner the exact inverse
    M = cpr.CPRPreconditioner(rp, col, vd, case.nx, case.ny, case.nz, second=_Exact(A, n))
    np.testing.assert_allclose(M.apply(r), spla.spsolve(A.tocsc(), r.reshape(-1)).reshape(n, 8), rtol=1e-8,
                               atol=1e-10 * np.abs(r).max())
    # without a second stage only the pressure correction remains
    M0 = cpr.CPRPreconditioner(rp, col, vd, case.nx, case.ny, case.nz, second=_Zero())
    z = M0.apply(r)
    assert np.all(z[:, 1:] == 0.0)
    np.testing.assert_array_equal(z[:, 0], M0.mg.vcycle(r[:, 0].copy()))


def test_cpr_cuts_gmres_iterations_on_a_field_block(field_block):
    case, rp, col, vd, rhs = field_block
    A = linalg.bsr_to_scipy(rp, col, vd)
    mv = lambda v: (A @ v.reshape(-1)).reshape(v.shape)
    _, its_ilu, _ = linalg.gmres(mv, rhs, linalg.ILU0Preconditioner(rp, col, vd), 30, 1e-6, 3000)
    x, its_cpr, rel = linalg.gmres(mv, rhs, cpr.CPRPreconditioner(rp, col, vd, case.nx, case.ny, case.nz),
                                   30, 1e-6, 3000)
    assert rel <= 1e-6
    assert its_cpr <= 12 and 3 * its_cpr <= its_ilu, (its_cpr, its_ilu)


@pytest.mark.parametrize("dims", [(2, 1, 1), (1, 2, 1)])
def test_vcycle_on_two_cells_by_hand(dims):
    """Two cells side by side in x or in y (one column of height 1 each): colour 0 is
    cell 0, colour 1 is cell 1, and one aggregation step leaves one coarse cell
    with A_c = a + b + c + d. One pre-smoothing sweep (cell 0 then cell 1), the
    coarse correction added to both cells, one post-smoothing sweep, written out
    by hand for A = [[a, b], [c, d]]."""
    a, b, c, d = 4.0, -1.5, -0.5, 3.0
    A = sp.csr_matrix(np.array([[a, b], [c, d]]))
    mg = cpr.AggregationMG(A, *dims)
    assert mg.dims == [dims, (1, 1, 1)]
    f0, f1 = 1.0, 2.0
    x0 = f0 / a                            # pre-smoothing, colour 0 (x1 = 0)
    x1 = (f1 - c * x0) / d                 # pre-smoothing, colour 1
    r0 = f0 - a * x0 - b * x1              # r1 = 0 after its own solve
    r1 = f1 - c * x0 - d * x1
    e = (r0 + r1) / (a + b + c + d)        # coarse solve, prolonged to both cells
    x0, x1 = x0 + e, x1 + e
    x0 = (f0 - b * x1) / a                 # post-smoothing, colour 0
    x1 = (f1 - c * x0) / d                 # post-smoothing, colour 1
    np.testing.assert_allclose(mg.vcycle(np.array([f0, f1])), [x0, x1], rtol=1e-14)


def test_red_black_half_sweeps_solve_their_own_columns():
    """In one line-smoothing sweep from x = 0, every colour-0 column is solved
    with its neighbours still zero (x-y neighbours always have the other colour),
    and after the colour-1 half-sweep every colour-1 column's equations hold."""
    nx, ny, nz = 5, 4, 6
    A = _random_stencil(nx, ny, nz, 11, symmetric=False)
    mg = cpr.AggregationMG(A, nx, ny, nz)
    f = np.random.default_rng(12).standard_normal(A.shape[0])
    x = mg.smooth(0, np.zeros_like(f), f, 1)
    r = f - A @ x
    for cy in range(ny):
        for cx in range(nx):
            idx = cx + nx * cy + nx * ny * np.arange(nz)
            if (cx + cy) % 2 == 0:
                T = A[idx][:, idx].toarray()
                np.testing.assert_allclose(x[idx], np.linalg.solve(T, f[idx]), rtol=1e-12)
            else:
                assert np.max(np.abs(r[idx])) <= 1e-12 * np.max(np.abs(f))


def test_cpr_defaults_one_pre_and_one_post_sweep_and_pairwise_aggregation(field_block):
    """The CPR-PF reading: one V-cycle with one pre- and one post-smoothing sweep,
    aggregates of 2 x 2 cells in x-y, z kept."""
    case, rp, col, vd = field_block[:4]
    P = cpr.CPRPreconditioner(rp, col, vd, case.nx, case.ny, case.nz)
    assert (P.mg.nu1, P.mg.nu2) == (1, 1)
    assert P.mg.dims[1] == ((case.nx + 1) // 2, (case.ny + 1) // 2, case.nz)
