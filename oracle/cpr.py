"""Oracle: the CPR-PF two-stage preconditioner.

Test infrastructure only (see ``oracle/__init__``).

Sec. 4 (Example 2) switches the linear solver's preconditioner from RAS to
CPR-PF, a member of the platform's family of constrained-pressure-residual
preconditioners; the paper gives no further detail of it. Readings taken here:

* System: the Gauss-Jordan-decoupled Jacobian (Sec. 3.2), whose diagonal
  blocks are I, so row 0 of block row i is the equation paired with the
  pressure unknown of cell i. The pressure matrix A_p holds the (0, 0) entry of
  every block (same 7-point pattern).
* CPR-PF ("pressure first"): with r_p the pressure rows of r and E the
  injection of a pressure vector into unknown 0 of every cell,
      x1 = E M_p^-1 r_p,   z = x1 + M^-1 (r - A x1),
  M_p^-1 one multigrid V-cycle on A_p from a zero guess, M^-1 the block ILU(0)
  preconditioner of the whole system.
* Pressure multigrid (the platform's pressure solver is not described): x-y
  aggregation of agg x agg cells, agg = 2 (piecewise-constant prolongation P, restriction
  P^T, Galerkin coarse operator P^T A P), z not coarsened, repeated until one
  column remains; smoothing by red-black z-line Gauss-Seidel (columns coloured
  by (x + y) mod 2, colour 0 first; each column's z-tridiagonal system is
  solved exactly with the other columns' current values); nu1 pre- and nu2
  post-smoothing sweeps; on the single-column level the tridiagonal system is
  solved exactly.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from . import linalg


def pressure_matrix(rowptr, col, val):
    """A_p: the (0, 0) entry of every block, as a scalar CSR matrix."""
    n = len(rowptr) - 1
    rows = np.repeat(np.arange(n), np.diff(rowptr))
    return sp.csr_matrix((val[:, 0, 0], (rows, col)), shape=(n, n))


def aggregation_1d(m, agg=2):
    """Piecewise-constant prolongation of one direction: fine cell x belongs to
    aggregate x // agg (the trailing aggregate may hold fewer cells)."""
    mc = (m + agg - 1) // agg
    return sp.csr_matrix((np.ones(m), (np.arange(m), np.arange(m) // agg)), shape=(m, mc)), mc


class AggregationMG:
    """Levels (A_l, dims_l) with P_l from level l to l + 1; cell index
    x + nx (y + ny z) on every level."""

    def __init__(self, A, nx, ny, nz, nu1=1, nu2=1, agg=2):
        self.nu1, self.nu2 = nu1, nu2
        self.A, self.P, self.dims = [A.tocsr()], [], [(nx, ny, nz)]
        while nx > 1 or ny > 1:
            Px, cx = aggregation_1d(nx, agg)
            Py, cy = aggregation_1d(ny, agg)
            P = sp.kron(sp.identity(nz), sp.kron(Py, Px)).tocsr()
            self.P.append(P)
            self.A.append((P.T @ self.A[-1] @ P).tocsr())
            nx, ny = cx, cy
            self.dims.append((nx, ny, nz))

    def _column_solve(self, l, b, x, colour):
        """Solve the z-tridiagonal system of every column of the colour (all
        columns if colour is None) with the other columns' current x."""
        A = self.A[l]
        nx, ny, nz = self.dims[l]
        nxy = nx * ny
        r = b - A @ x
        xn = x.copy()
        for cy in range(ny):
            for cx in range(nx):
                if colour is not None and (cx + cy) % 2 != colour:
                    continue
                idx = cx + nx * cy + nxy * np.arange(nz)
                T = A[idx][:, idx].toarray()
                # r holds b - A x; adding back the column's own part gives b - (off-column part) x
                rhs = r[idx] + T @ x[idx]
                ab = np.zeros((3, nz))
                ab[0, 1:] = np.diag(T, 1)
                ab[1] = np.diag(T)
                ab[2, :-1] = np.diag(T, -1)
                xn[idx] = sla.solve_banded((1, 1), ab, rhs)
        return xn

    def smooth(self, l, x, b, sweeps):
        for _ in range(sweeps):
            x = self._column_solve(l, b, x, 0)
            x = self._column_solve(l, b, x, 1)
        return x

    def vcycle(self, b, l=0):
        if l == len(self.A) - 1:
            return self._column_solve(l, b, np.zeros_like(b), None)
        x = self.smooth(l, np.zeros_like(b), b, self.nu1)
        r = b - self.A[l] @ x
        xc = self.vcycle(self.P[l].T @ r, l + 1)
        x = x + self.P[l] @ xc
        return self.smooth(l, x, b, self.nu2)


class CPRPreconditioner:
    """z = E M_p^-1 r_p + M^-1 (r - A E M_p^-1 r_p) on the decoupled system."""

    def __init__(self, rowptr, col, val, nx, ny, nz, nu1=1, nu2=1, second=None, agg=2):
        self.n = len(rowptr) - 1
        self.A = linalg.bsr_to_scipy(rowptr, col, val)
        self.mg = AggregationMG(pressure_matrix(rowptr, col, val), nx, ny, nz, nu1, nu2, agg)
        self.second = second if second is not None else linalg.ILU0Preconditioner(rowptr, col, val)

    def apply(self, r):
        r = np.asarray(r, dtype=float).reshape(self.n, linalg.BS)
        p = self.mg.vcycle(r[:, 0].copy())
        x1 = np.zeros_like(r)
        x1[:, 0] = p
        r1 = r - (self.A @ x1.reshape(-1)).reshape(self.n, linalg.BS)
        return x1 + self.second.apply(r1)
