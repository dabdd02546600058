"""Parity at full size, in the configuration bench.py times (field 60x60x20,
first Newton step from the ignited state), plus sampled rows of the largest
workload (200x200x50, 2 million cells, 7 GB Jacobian).

At full size the oracle checks everything that holds at any size: the whole
residual; J v against one complex-step evaluation of the oracle residual
(exact directional derivative); the decoupled operator against
blockdiag(J_ii)^-1 J v; the Krylov residual in the exported matrix; the
safeguarded update. Rows of the 2M-cell grid are checked against the oracle
run on a window of that grid (interior cells of a window have the same
residual and Jacobian rows as in the whole grid), and the GPU's linear step at
that size is checked by the residual of its update recomputed on the host.
"""
import copy

import numpy as np
import pytest
import scipy.sparse as sp

import isc_inputs as inp
from oracle import linalg, model, sim

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def Simulator():
    from paper_1811_11992_gb300 import build
    build.build()
    from paper_1811_11992_gb300 import Simulator as S
    return S


def test_bench_workload_full_size(Simulator):
    case = inp.config(2)
    dt = case.dt0
    g = Simulator(case, tol_lin=1e-6)
    g.init_equilibrium()
    u0, c0 = sim.initial_state(case)
    ug, _ = g.get_state()
    assert np.allclose(ug, u0, rtol=1e-13, atol=1e-300)
    g.assemble(dt)
    acc_old = model.old_accumulation(case, u0, c0)
    geom = model.faces(case)
    Fo = model.residual(case, u0, c0, acc_old, dt, geom)
    F = g.residual()
    scale = np.abs(Fo).max(axis=1, keepdims=True)
    assert np.max(np.abs(F - Fo) / scale) < 1e-10
    # J v against the complex-step directional derivative of the oracle residual
    rng = np.random.default_rng(5)
    v = rng.standard_normal((8, case.n)) * np.array([1e5, 0.1, 0.1, 0.1, 0.1, 10.0, 0.1, 0.1])[:, None]
    h = 1e-30
    Jv_o = np.imag(model.residual(case, u0.astype(complex) + 1j * h * v, c0, acc_old, dt, geom)) / h
    Jv = g.spmv(v)
    sc = np.abs(Jv_o).max(axis=1, keepdims=True)
    assert np.max(np.abs(Jv - Jv_o) / sc) < 1e-10
    # decoupling: diagonal blocks exactly I and C_L J v = blockdiag(J_ii)^-1 (J v)
    rp, col, J = g.jacobian()
    rows = np.repeat(np.arange(case.n), np.diff(rp))
    Dinv = np.linalg.inv(J[col == rows])
    g.decouple()
    _, _, Jd = g.jacobian()
    assert np.all(Jd[col == rows] == np.eye(8))
    CJv = np.einsum("nij,nj->ni", Dinv, Jv.T).T
    assert np.max(np.abs(g.spmv(v) - CJv) / np.abs(CJv).max(axis=1, keepdims=True)) < 1e-9
    # Krylov: relative residual of the GPU update in the exported decoupled system
    Fd = g.residual()
    info = g.solve()
    du = g.newton_update()
    A = linalg.bsr_to_scipy(rp.astype(np.int64), col.astype(np.int64), Jd)
    b = -Fd.T.reshape(-1)
    res = np.linalg.norm(b - A @ du.T.reshape(-1)) / np.linalg.norm(b)
    assert res <= 1.05e-6 and abs(res - info.krylov_rel_residual) < 1e-7
    # the update kernel applies the paper's safeguards exactly
    g.update()
    un, _ = g.get_state()
    assert np.array_equal(un, sim.apply_update(ug, du))   # from the GPU's own iterate
    g.close()


def _window(case, i0, j0, k0, w):
    """Sub-case made of the cells [i0, i0+w) x [j0, j0+w) x [k0, k0+w) of case."""
    nx, ny = case.nx, case.ny
    ii, jj, kk = np.meshgrid(np.arange(i0, i0 + w), np.arange(j0, j0 + w), np.arange(k0, k0 + w), indexing="ij")
    cells = (ii + nx * (jj + ny * kk)).transpose(2, 1, 0).reshape(-1)   # sub-grid natural order
    sub = copy.copy(case)
    sub.nx = sub.ny = sub.nz = w
    sub.depth = case.depth[cells]
    sub.phi_ref = case.phi_ref[cells]
    sub.perm = case.perm[:, cells]
    pos = {int(c): q for q, c in enumerate(cells)}
    wells = []
    for wl in case.wells:
        keep = [q for q, c in enumerate(wl.cells) if int(c) in pos]
        if not keep:
            continue
        nw = copy.copy(wl)
        nw.cells = np.array([pos[int(wl.cells[q])] for q in keep], np.int32)
        nw.WI = wl.WI[keep]
        if wl.kind == 0:   # keep each perforation's share of the injection rate
            nw.target = wl.target * nw.WI.sum() / wl.WI.sum()
        wells.append(nw)
    sub.wells = wells
    return sub, cells


def test_largest_workload_sampled_rows(Simulator):
    case = inp.config(5)
    dt = case.dt0
    g = Simulator(case, tol_lin=1e-6)
    g.init_equilibrium()
    g.assemble(dt)
    F = g.residual()
    rp, col, J = g.jacobian()
    u, _ = g.get_state()
    row_scale = np.abs(F).max(axis=1)       # residual rows scaled over the whole grid
    w = 6
    windows = [(0, 0, 0), (97, 97, 22), (194, 0, 44), (97, 194, 0), (30, 150, 20)]
    for (i0, j0, k0) in windows:
        sub, cells = _window(case, i0, j0, k0, w)
        us = u[:, cells]
        cs = np.zeros(len(cells))
        acc = model.old_accumulation(sub, us, cs)
        Fo = model.residual(sub, us, cs, acc, dt)
        rps, cols, Jo = model.jacobian(sub, us, cs, acc, dt)
        for q in range(len(cells)):
            x, y, z = q % w, (q // w) % w, q // (w * w)
            gx, gy, gz = i0 + x, j0 + y, k0 + z
            # a window cell's row is complete when none of its grid neighbours lies outside the window
            ok = all((0 < c < w - 1) or (gc == 0 and c == 0) or (gc == n - 1 and c == w - 1)
                     for c, gc, n in ((x, gx, case.nx), (y, gy, case.ny), (z, gz, case.nz)))
            if not ok:
                continue
            c = cells[q]
            assert np.all(np.abs(F[:, c] - Fo[:, q]) <= 1e-10 * row_scale), (i0, j0, k0, q)
            # the row's blocks: same neighbours in the same sorted order
            gb = list(range(rp[c], rp[c + 1]))
            ob = list(range(rps[q], rps[q + 1]))
            assert [cells[cols[b]] for b in ob] == [col[b] for b in gb]
            Gs = np.concatenate([J[b] for b in gb], axis=1) * np.tile([1e6, 1, 1, 1, 1, 100, 1, 1], len(gb))
            Os = np.concatenate([Jo[b] for b in ob], axis=1) * np.tile([1e6, 1, 1, 1, 1, 100, 1, 1], len(ob))
            rs = np.abs(Os).max(axis=1, keepdims=True) + 1e-300
            assert np.max(np.abs(Gs - Os) / rs) < 1e-10
    del J
    # the whole linear step at this size: decoupling, ILU(0) over 10,000 pencils (more
    # than the sweeps keep resident, so warps take several), GMRES(30) to 1e-6. The
    # update's residual is recomputed on the host from the exported decoupled system,
    # independently of the solver's own estimate.
    g.decouple()
    info = g.solve()
    assert info.krylov_rel_residual <= 1e-6
    du = g.newton_update().T.copy()          # (N, 8)
    Fd = g.residual().T.copy()               # decoupled residual, (N, 8)
    _, _, Jd = g.jacobian()
    r = _bsr_residual(rp, col, Jd, du, -Fd)
    rel = np.linalg.norm(r) / np.linalg.norm(Fd)
    assert rel <= 1.05e-6, rel
    g.close()


def _bsr_residual(rp, col, val, x, b, chunk=200_000):
    """b - A x for a BSR matrix, rows in chunks (numpy, float64)."""
    n = len(rp) - 1
    r = b.copy()
    for r0 in range(0, n, chunk):
        r1 = min(n, r0 + chunk)
        b0, b1 = rp[r0], rp[r1]
        prod = np.einsum("bij,bj->bi", val[b0:b1], x[col[b0:b1]])
        r[r0:r1] -= np.add.reduceat(prod, rp[r0:r1] - b0, axis=0)
    return r
