"""Textbook Krylov solvers and a direct solve for the oracle (FP64, CPU).

TEST INFRASTRUCTURE ONLY: nothing in the product path may import this module.

The paper solves the pressure system with conjugate gradients and the
advection-diffusion system with BiCGStab (App. A.5).  These are the standard
algorithms: Jacobi-preconditioned CG (Hestenes-Stiefel with a diagonal
preconditioner) and unpreconditioned BiCGStab (van der Vorst 1992), each
stopping when ||r||_2 <= max(rtol*||b||_2, atol).  ``direct_solve`` is the plain
definition x = A^-1 b used to pin both.
"""
from __future__ import annotations

import numpy as np
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


def bicgstab(matvec, b, x0, rtol=1e-13, atol=0.0, maxit=100000):
    """Unpreconditioned BiCGStab with shadow residual r0."""
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
        v = matvec(p)
        alpha = rho / float(rhat @ v)
        s = r - alpha * v
        sn = float(np.linalg.norm(s))
        if sn <= tol:
            x += alpha * p
            return x, SolveInfo(it, True, sn)
        t = matvec(s)
        omega = float(t @ s) / float(t @ t)
        x += alpha * p + omega * s
        r = s - omega * t
        rn = float(np.linalg.norm(r))
        if rn <= tol:
            return x, SolveInfo(it, True, rn)
        rho_old = rho
    return x, SolveInfo(maxit, False, rn)


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
