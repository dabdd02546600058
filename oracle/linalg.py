"""Oracle: decoupling and linear solvers on block-sparse (BSR) systems.

Test infrastructure only (see ``oracle/__init__``).

A BSR matrix here is (rowptr, col, val) with val[b] the dense 8x8 block at
(row of b, col[b]), columns sorted within a row.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

BS = 8


class SingularBlockError(RuntimeError):
    pass


def bsr_to_dense(rowptr, col, val):
    n = len(rowptr) - 1
    A = np.zeros((n * BS, n * BS))
    for r in range(n):
        for b in range(rowptr[r], rowptr[r + 1]):
            c = col[b]
            A[r * BS:(r + 1) * BS, c * BS:(c + 1) * BS] = val[b]
    return A


def bsr_to_scipy(rowptr, col, val):
    n = len(rowptr) - 1
    return sp.bsr_matrix((val, col, rowptr), shape=(n * BS, n * BS)).tocsr()


def bsr_matvec(rowptr, col, val, x):
    """y = A x, x and y of shape (n, 8) (row-block major)."""
    n = len(rowptr) - 1
    y = np.zeros((n, BS))
    for r in range(n):
        for b in range(rowptr[r], rowptr[r + 1]):
            y[r] += val[b] @ x[col[b]]
    return y


def gauss_jordan_decouple(rowptr, col, val, rhs, pivot_floor=1e-300):
    """ABF decoupling by Gauss-Jordan elimination with partial pivoting (Sec. 3.2).

    For every block row i the augmented matrix [J_i,* | f_i] is transformed by
    elementary row operations (row exchange, row scaling, row addition) until
    its diagonal block is the identity. The result equals C_L J and C_L f with
    C_L = blockdiag(J_ii^-1), without forming J_ii^-1. Pivot: largest |a| in
    the pivot column among the remaining rows, ties to the lowest row index.
    A pivot below pivot_floor * (row max) raises SingularBlockError.

    rhs: (n, 8). Returns (val_out, rhs_out); the diagonal blocks of val_out
    are exactly the identity.
    """
    n = len(rowptr) - 1
    val_out = val.copy()
    rhs_out = rhs.copy()
    for i in range(n):
        b0, b1 = rowptr[i], rowptr[i + 1]
        nb = b1 - b0
        d = int(np.nonzero(col[b0:b1] == i)[0][0])
        M = np.concatenate([val_out[b0 + k] for k in range(nb)] + [rhs_out[i][:, None]], axis=1)
        c0 = d * BS
        for k in range(BS):
            piv = k + int(np.argmax(np.abs(M[k:, c0 + k])))
            rowmax = np.max(np.abs(M[piv, c0:c0 + BS]))
            if not (abs(M[piv, c0 + k]) > pivot_floor * max(rowmax, 1e-300)):
                raise SingularBlockError(f"zero pivot in block row {i}, column {k}")
            if piv != k:
                M[[k, piv]] = M[[piv, k]]
            M[k] = M[k] / M[k, c0 + k]
            for r in range(BS):
                if r != k:
                    M[r] = M[r] - M[r, c0 + k] * M[k]
        for k in range(nb):
            val_out[b0 + k] = M[:, k * BS:(k + 1) * BS]
        val_out[b0 + d] = np.eye(BS)
        rhs_out[i] = M[:, nb * BS]
    return val_out, rhs_out


def block_ilu0(rowptr, col, val):
    """Block ILU(0), IKJ form (textbook), on the matrix's own sparsity pattern.

    for i = 1..n: for k < i in row i: A_ik <- A_ik A_kk^-1;
                  for j > k in row i that are also in row k: A_ij <- A_ij - A_ik A_kj
    Returns the factor blocks in the same layout: strictly lower blocks hold L
    (unit block diagonal implied), diagonal and upper blocks hold U.
    """
    n = len(rowptr) - 1
    F = val.copy()
    pos = [dict() for _ in range(n)]
    for r in range(n):
        for b in range(rowptr[r], rowptr[r + 1]):
            pos[r][int(col[b])] = b
    diag_inv = {}
    for i in range(n):
        for b in range(rowptr[i], rowptr[i + 1]):
            k = int(col[b])
            if k >= i:
                break
            if k not in diag_inv:
                diag_inv[k] = np.linalg.inv(F[pos[k][k]])
            F[b] = F[b] @ diag_inv[k]
            for bj in range(rowptr[i], rowptr[i + 1]):
                j = int(col[bj])
                if j <= k:
                    continue
                bk = pos[k].get(j)
                if bk is not None:
                    F[bj] = F[bj] - F[b] @ F[bk]
    return F


class ILU0Preconditioner:
    """z = (LU)^-1 r with the block ILU(0) factors; the two triangular solves
    use scipy's sparse triangular solver on the scalar form of L and of
    blockdiag(U)^-1 U (both triangular with a stored unit diagonal)."""

    def __init__(self, rowptr, col, val, factors=None):
        """factors: the block ILU(0) factor blocks F (as block_ilu0 returns
        them) when already known; by default they are computed from val."""
        self.n = len(rowptr) - 1
        F = block_ilu0(rowptr, col, val) if factors is None else factors
        rows = np.repeat(np.arange(self.n), np.diff(rowptr))
        low = col < rows
        dia = col == rows
        upp = col > rows
        eye = np.broadcast_to(np.eye(BS), (self.n, BS, BS))
        # L: unit lower
        lval = np.concatenate([F[low], eye])
        lrow = np.concatenate([rows[low], np.arange(self.n)])
        lcol = np.concatenate([col[low], np.arange(self.n)])
        self.L = _blocks_to_csr(lrow, lcol, lval, self.n)
        self.Dinv = np.linalg.inv(F[dia])            # row order
        uval = np.einsum("bij,bjk->bik", self.Dinv[rows[upp]], F[upp])
        urow = np.concatenate([rows[upp], np.arange(self.n)])
        ucol = np.concatenate([col[upp], np.arange(self.n)])
        self.U = _blocks_to_csr(urow, ucol, np.concatenate([uval, eye]), self.n)

    def apply(self, r):
        y = spla.spsolve_triangular(self.L, r.reshape(-1), lower=True, unit_diagonal=False)
        yd = np.einsum("nij,nj->ni", self.Dinv, y.reshape(self.n, BS)).reshape(-1)
        z = spla.spsolve_triangular(self.U, yd, lower=False, unit_diagonal=False)
        return z.reshape(self.n, BS)


class BlockJacobiPreconditioner:
    """z_i = A_ii^-1 r_i."""

    def __init__(self, rowptr, col, val):
        n = len(rowptr) - 1
        rows = np.repeat(np.arange(n), np.diff(rowptr))
        self.Dinv = np.linalg.inv(val[col == rows])

    def apply(self, r):
        return np.einsum("nij,nj->ni", self.Dinv, r)


class IdentityPreconditioner:
    def apply(self, r):
        return r.copy()


def _blocks_to_csr(brow, bcol, bval, n):
    r = (brow[:, None, None] * BS + np.arange(BS)[None, :, None]) * np.ones((1, 1, BS), dtype=np.int64)
    c = (bcol[:, None, None] * BS + np.arange(BS)[None, None, :]) * np.ones((1, BS, 1), dtype=np.int64)
    M = sp.coo_matrix((bval.reshape(-1), (r.reshape(-1), c.reshape(-1))), shape=(n * BS, n * BS)).tocsr()
    M.sum_duplicates()
    M.sort_indices()
    return M


def gmres(A_mv, b, M=None, restart=30, rtol=1e-8, maxit=1000):
    """Right-preconditioned restarted GMRES(m) with modified Gram-Schmidt and
    Givens rotations. Stops when ||b - A x|| <= rtol ||b|| (x0 = 0).
    Returns (x, iterations, relative residual estimate)."""
    M = M or IdentityPreconditioner()
    shape = b.shape
    bn = np.linalg.norm(b)
    x = np.zeros_like(b)
    if bn == 0.0:
        return x, 0, 0.0
    its = 0
    rel = 1.0
    while its < maxit:
        r = b - A_mv(x)
        beta = np.linalg.norm(r)
        rel = beta / bn
        if rel <= rtol:
            break
        V = [r / beta]
        Z = []
        Hm = np.zeros((restart + 1, restart))
        cs = np.zeros(restart)
        sn = np.zeros(restart)
        g = np.zeros(restart + 1)
        g[0] = beta
        j_done = 0
        for j in range(restart):
            z = M.apply(V[j])
            Z.append(z)
            w = A_mv(z)
            for i in range(j + 1):
                Hm[i, j] = np.sum(w * V[i])
                w = w - Hm[i, j] * V[i]
            hn = np.linalg.norm(w)
            Hm[j + 1, j] = hn
            for i in range(j):
                t = cs[i] * Hm[i, j] + sn[i] * Hm[i + 1, j]
                Hm[i + 1, j] = -sn[i] * Hm[i, j] + cs[i] * Hm[i + 1, j]
                Hm[i, j] = t
            den = np.hypot(Hm[j, j], Hm[j + 1, j])
            cs[j] = Hm[j, j] / den
            sn[j] = Hm[j + 1, j] / den
            Hm[j, j] = den
            Hm[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            its += 1
            j_done = j + 1
            rel = abs(g[j + 1]) / bn
            if rel <= rtol or its >= maxit or hn == 0.0:
                break
            V.append(w / hn)
        y = np.zeros(j_done)
        for i in range(j_done - 1, -1, -1):
            y[i] = (g[i] - Hm[i, i + 1:j_done] @ y[i + 1:j_done]) / Hm[i, i]
        for i in range(j_done):
            x = x + y[i] * Z[i]
        if rel <= rtol:
            rel = np.linalg.norm(b - A_mv(x)) / bn
            if rel <= rtol:
                break
    return x.reshape(shape), its, rel


def bicgstab(A_mv, b, M=None, rtol=1e-8, maxit=1000):
    """Right-preconditioned BiCGSTAB (van der Vorst), x0 = 0.
    Returns (x, iterations, relative residual)."""
    M = M or IdentityPreconditioner()
    bn = np.linalg.norm(b)
    x = np.zeros_like(b)
    if bn == 0.0:
        return x, 0, 0.0
    r = b.copy()
    rhat = r.copy()
    rho_old = alpha = omega = 1.0
    v = np.zeros_like(b)
    p = np.zeros_like(b)
    rel = 1.0
    for it in range(1, maxit + 1):
        rho = np.sum(rhat * r)
        if rho == 0.0:
            return x, it, rel
        beta = (rho / rho_old) * (alpha / omega) if it > 1 else 0.0
        p = r + beta * (p - omega * v) if it > 1 else r.copy()
        phat = M.apply(p)
        v = A_mv(phat)
        alpha = rho / np.sum(rhat * v)
        s = r - alpha * v
        if np.linalg.norm(s) / bn <= rtol:
            x = x + alpha * phat
            return x, it, np.linalg.norm(s) / bn
        shat = M.apply(s)
        t = A_mv(shat)
        tt = np.sum(t * t)
        omega = np.sum(t * s) / tt if tt > 0 else 0.0
        x = x + alpha * phat + omega * shat
        r = s - omega * t
        rho_old = rho
        rel = np.linalg.norm(r) / bn
        if rel <= rtol:
            return x, it, rel
        if omega == 0.0:
            return x, it, rel
    return x, maxit, rel
