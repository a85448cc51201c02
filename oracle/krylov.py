"""Textbook Krylov solvers and a direct solve for the oracle (FP64, CPU).

TEST INFRASTRUCTURE ONLY: nothing in the product path may import this module.

The paper solves the pressure system with conjugate gradients and the
advection-diffusion system with BiCGStab (App. A.5).  These are the standard
algorithms: Jacobi-preconditioned CG (Hestenes-Stiefel with a diagonal
preconditioner) and BiCGStab (van der Vorst 1992), each stopping when
||r||_2 <= max(rtol*||b||_2, atol).  App. A.5 also offers an incomplete-LU
preconditioner for the BiCGStab, on its own or only after the unpreconditioned
solve failed: ``ilu0`` is the textbook zero-fill incomplete factorisation
(Saad, Iterative Methods for Sparse Linear Systems, Sec. 10.3.2, IKJ order)
and ``bicgstab`` takes it as a right preconditioner.  ``direct_solve`` is the
plain definition x = A^-1 b used to pin all of them.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


class SolveInfo:
    def __init__(self, iters: int, converged: bool, resid: float, breakdown: bool = False):
        self.iters, self.converged, self.resid, self.breakdown = iters, converged, resid, breakdown

    def __repr__(self):
        return f"SolveInfo(iters={self.iters}, converged={self.converged}, resid={self.resid:.3e})"


def pcg(matvec, diag, b, x0, rtol=1e-13, atol=0.0, maxit=100000):
    """Jacobi-preconditioned CG for a symmetric positive (semi-)definite operator."""
    x = np.array(x0, dtype=np.float64, copy=True)
    r = b - matvec(x)
    bnorm = float(np.linalg.norm(b))
    tol = max(rtol * bnorm, atol)
    rn = float(np.linalg.norm(r))
    if rn <= tol:
        return x, SolveInfo(0, True, rn)
    z = r / diag
    d = z.copy()
    rz = float(r @ z)
    for it in range(1, maxit + 1):
        q = matvec(d)
        alpha = rz / float(d @ q)
        x += alpha * d
        r -= alpha * q
        rn = float(np.linalg.norm(r))
        if rn <= tol:
            return x, SolveInfo(it, True, rn)
        z = r / diag
        rz_new = float(r @ z)
        d = z + (rz_new / rz) * d
        rz = rz_new
    return x, SolveInfo(maxit, False, rn)


def bicgstab(matvec, b, x0, rtol=1e-13, atol=0.0, maxit=100000, precond=None):
    """BiCGStab with shadow residual r0; ``precond`` (a callable applying K^-1)
    makes it right-preconditioned: the search directions are y = K^-1 p and
    z = K^-1 s, and x is updated with them (van der Vorst 1992, Alg. 3.1 with
    K1 = I).  Without it K = I."""
    K = precond if precond is not None else (lambda w: w)
    x = np.array(x0, dtype=np.float64, copy=True)
    r = b - matvec(x)
    bnorm = float(np.linalg.norm(b))
    tol = max(rtol * bnorm, atol)
    rn = float(np.linalg.norm(r))
    if rn <= tol:
        return x, SolveInfo(0, True, rn)
    rhat = r.copy()
    rho_old = alpha = omega = 1.0
    v = np.zeros_like(b)
    p = np.zeros_like(b)
    for it in range(1, maxit + 1):
        rho = float(rhat @ r)
        if rho == 0.0:
            return x, SolveInfo(it, False, rn, breakdown=True)
        beta = (rho / rho_old) * (alpha / omega)
        p = r + beta * (p - omega * v)
        y = K(p)
        v = matvec(y)
        alpha = rho / float(rhat @ v)
        s = r - alpha * v
        sn = float(np.linalg.norm(s))
        if sn <= tol:
            x += alpha * y
            return x, SolveInfo(it, True, sn)
        z = K(s)
        t = matvec(z)
        omega = float(t @ s) / float(t @ t)
        x += alpha * y + omega * z
        r = s - omega * t
        rn = float(np.linalg.norm(r))
        if not np.isfinite(rn):
            return x, SolveInfo(it, False, rn, breakdown=True)
        if rn <= tol:
            return x, SolveInfo(it, True, rn)
        rho_old = rho
    return x, SolveInfo(maxit, False, rn)


def ilu0(A):
    """Zero-fill incomplete LU of a square sparse matrix in its given row
    order: L unit lower and U upper triangular, both on the sparsity pattern of
    A, with (L U)_ij = a_ij at every (i, j) of that pattern.  IKJ elimination
    in which every update that would land outside the pattern is dropped.
    Plain Python loops over the rows (small and moderate sizes only)."""
    A = sp.csr_matrix(A, dtype=np.float64)
    A.sum_duplicates()
    A.sort_indices()
    n = A.shape[0]
    ptr, idx = A.indptr, A.indices
    W = A.data.copy()                       # becomes L (strictly lower) and U (upper) in place
    pos = [dict(zip(idx[ptr[i]:ptr[i + 1]].tolist(), range(ptr[i], ptr[i + 1]))) for i in range(n)]
    diag = np.empty(n, dtype=np.int64)
    for i in range(n):
        if i not in pos[i]:
            raise ValueError(f"ILU(0) needs a stored diagonal (row {i})")
        diag[i] = pos[i][i]
    for i in range(1, n):
        row = pos[i]
        for kk in range(ptr[i], ptr[i + 1]):
            k = int(idx[kk])
            if k >= i:
                break
            W[kk] /= W[diag[k]]
            lik = W[kk]
            for jj in range(diag[k] + 1, ptr[k + 1]):        # row k of U, right of its diagonal
                q = row.get(int(idx[jj]))
                if q is not None:
                    W[q] -= lik * W[jj]
    F = sp.csr_matrix((W, idx.copy(), ptr.copy()), shape=A.shape)
    L = sp.tril(F, k=-1, format="csr") + sp.identity(n, format="csr")
    U = sp.triu(F, k=0, format="csr")
    return L, U


def ilu0_preconditioner(A):
    """The callable w -> (L U)^-1 w of ``ilu0(A)``: two triangular solves."""
    L, U = ilu0(A)
    L, U = L.tocsr(), U.tocsr()

    def apply(w):
        y = spla.spsolve_triangular(L, w, lower=True, unit_diagonal=True)
        return spla.spsolve_triangular(U, y, lower=False)
    return apply


def direct_solve(A, b):
    """x = A^-1 b by sparse LU (scipy SuperLU)."""
    return spla.spsolve(A.tocsc(), b)


def direct_solve_singular(A, b):
    """Solve a symmetric system whose null space is the constant vector, with
    b orthogonal to it: fix x_0 = 0, solve the remaining rows, return the
    mean-free solution."""
    A = A.tocsr()
    n = A.shape[0]
    sub = A[1:, 1:].tocsc()
    x = np.zeros(n)
    x[1:] = spla.spsolve(sub, b[1:])
    return x - x.mean()
