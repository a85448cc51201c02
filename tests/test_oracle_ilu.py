"""Pins of the oracle's ILU(0) factorisation and of its preconditioned
BiCGStab (App. A.5: incomplete-LU preconditioning of the advection-diffusion
solve, optionally only after the unpreconditioned solve failed), against
facts that do not depend on the oracle: an exact LU where no fill can occur,
the defining pattern identity, the closed-form pivots of the five-point
stencil, exact preconditioning, and the direct solution."""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle as O
from oracle import krylov as K
from oracle import piso as OP
from paper_2505_16992_b300 import workloads as W


def _five_point(nx, ny, seed, periodic_x=False):
    """Nonsymmetric diagonally dominant 5-point matrix on an nx x ny grid
    (x fastest): random advection-diffusion-like off-diagonals."""
    rng = np.random.default_rng(seed)
    n = nx * ny
    rows, cols, vals = [], [], []
    for y in range(ny):
        for x in range(nx):
            i = x + nx * y
            off = 0.0
            for dx, dy in ((-1, 0), (1, 0), (0, -1), (0, 1)):
                xx, yy = x + dx, y + dy
                if periodic_x:
                    xx %= nx
                if not (0 <= xx < nx and 0 <= yy < ny):
                    continue
                v = -1.0 + 0.6 * rng.uniform(-1, 1)
                rows.append(i), cols.append(xx + nx * yy), vals.append(v)
                off += abs(v)
            rows.append(i), cols.append(i), vals.append(off + 0.5 + rng.uniform())
    return sp.csr_matrix((vals, (rows, cols)), shape=(n, n))


def test_ilu0_is_exact_lu_of_a_tridiagonal_matrix():
    """No fill position exists for a tridiagonal matrix, so ILU(0) is its LU."""
    rng = np.random.default_rng(0)
    n = 40
    A = sp.diags([rng.uniform(-1, 0, n - 1), 3 + rng.uniform(0, 1, n), rng.uniform(-1, 0.5, n - 1)],
                 [-1, 0, 1], format="csr")
    L, U = K.ilu0(A)
    assert np.abs((L @ U - A).toarray()).max() <= 1e-14 * np.abs(A.toarray()).max()
    x = rng.standard_normal(n)
    assert np.allclose(K.ilu0_preconditioner(A)(A @ x), x, rtol=0, atol=1e-12)


def test_ilu0_matches_a_on_its_pattern_and_fills_only_outside():
    A = _five_point(9, 7, 1)
    L, U = K.ilu0(A)
    Ad = A.toarray()
    R = (L @ U).toarray() - Ad
    pat = Ad != 0
    assert np.abs(R[pat]).max() <= 1e-13 * np.abs(Ad).max()
    # L and U keep A's pattern (L unit lower, U upper)
    Ld, Ud = L.toarray(), U.toarray()
    assert np.all(np.diag(Ld) == 1.0)
    assert not np.any((np.tril(Ld, -1) != 0) & ~pat) and not np.any((Ud != 0) & ~pat)
    # the dropped fill of a 5-point stencil sits at (i, i - nx + 1) and (i, i + nx - 1)
    nx = 9
    fill = np.zeros_like(pat)
    n = Ad.shape[0]
    for i in range(n):
        for j in (i - nx + 1, i + nx - 1):
            if 0 <= j < n:
                fill[i, j] = True
    assert np.abs(R[~pat & ~fill]).max() == 0.0
    assert np.abs(R[fill]).max() > 0.0


def test_ilu0_pivots_follow_the_five_point_closed_form():
    """For a five-point matrix in natural order the pivots of ILU(0) satisfy
    d_i = a_ii - a_{i,i-1} a_{i-1,i} / d_{i-1} - a_{i,i-nx} a_{i-nx,i} / d_{i-nx}
    (Meijerink and van der Vorst 1977); the IKJ elimination must agree."""
    nx, ny = 11, 6
    A = _five_point(nx, ny, 2)
    _, U = K.ilu0(A)
    Ad = A.toarray()
    n = Ad.shape[0]
    d = np.zeros(n)
    for i in range(n):
        d[i] = Ad[i, i]
        if i % nx:
            d[i] -= Ad[i, i - 1] * Ad[i - 1, i] / d[i - 1]
        if i >= nx:
            d[i] -= Ad[i, i - nx] * Ad[i - nx, i] / d[i - nx]
    assert np.abs(U.diagonal() - d).max() <= 1e-13 * np.abs(d).max()


def test_ilu0_with_a_periodic_wrap_keeps_the_pattern_identity():
    A = _five_point(6, 5, 3, periodic_x=True)
    L, U = K.ilu0(A)
    Ad = A.toarray()
    R = (L @ U).toarray() - Ad
    assert np.abs(R[Ad != 0]).max() <= 1e-13 * np.abs(Ad).max()


def test_right_preconditioned_bicgstab_with_the_exact_inverse_takes_one_step():
    A = _five_point(8, 8, 4)
    b = np.random.default_rng(5).standard_normal(A.shape[0])
    exact = lambda w: K.direct_solve(A, w)
    x, info = K.bicgstab(lambda v: A @ v, b, np.zeros_like(b), 1e-12, precond=exact)
    assert info.converged and info.iters == 1
    assert np.allclose(x, K.direct_solve(A, b), rtol=0, atol=1e-12 * np.abs(x).max())


def _predictor_system(c, m):
    """C and the predictor right-hand side of the first step, from the oracle's
    own step record."""
    opts = OP.Options(solver="direct")
    _, _, tape = O.piso_step(m, c.u0, c.p0, c.dt, c.nu, c.S, opts=opts)
    C = tape["C"]
    return C, tape["rhs"], OP.to_sparse(m, C)


@pytest.mark.parametrize("precond", ["none", "ilu"])
def test_preconditioned_predictor_solve_matches_the_direct_solution(precond):
    c = W.channel3d(10, 16, 4, gamma=3.0, dt=0.5)
    m = O.mesh_from_case(c)
    C, rhs, Cs = _predictor_system(c, m)
    opts = OP.Options(solver="krylov", adv_rtol=1e-13, adv_precond=precond)
    x, infos = OP.solve_C(m, C, rhs, c.u0, opts)
    for k in range(3):
        ref = K.direct_solve(Cs, rhs[k])
        assert np.abs(x[k] - ref).max() <= 1e-10 * np.abs(ref).max()
        assert infos[k].converged and infos[k].precond == precond
    if precond == "ilu":
        plain = OP.solve_C(m, C, rhs, c.u0, OP.Options(solver="krylov", adv_rtol=1e-13))[1]
        assert sum(i.iters for i in infos) < 0.7 * sum(i.iters for i in plain)


def test_transposed_solve_with_ilu_matches_the_direct_solution():
    c = W.channel3d(10, 16, 4, gamma=3.0, dt=0.5)
    m = O.mesh_from_case(c)
    C, rhs, Cs = _predictor_system(c, m)
    g = np.random.default_rng(6).standard_normal(rhs.shape)
    z = OP.solve_C_T(m, C, g, OP.Options(solver="krylov", adv_rtol=1e-13, adv_precond="ilu"))
    for k in range(3):
        ref = K.direct_solve(Cs.T.tocsr(), g[k])
        assert np.abs(z[k] - ref).max() <= 1e-10 * np.abs(ref).max()


def test_ilu_on_failure_restarts_preconditioned():
    """An iteration limit the plain solve cannot meet but the ILU(0) solve can:
    the fallback restarts from x0 and reaches the direct solution."""
    c = W.channel3d(10, 16, 4, gamma=3.0, dt=0.5)
    m = O.mesh_from_case(c)
    C, rhs, Cs = _predictor_system(c, m)
    tight = OP.Options(solver="krylov", adv_rtol=1e-12)
    _, plain = OP.solve_C(m, C, rhs, c.u0, tight)
    _, ilu = OP.solve_C(m, C, rhs, c.u0, OP.Options(solver="krylov", adv_rtol=1e-12, adv_precond="ilu"))
    lim = max(i.iters for i in ilu) + 1
    assert min(i.iters for i in plain) > lim
    opts = OP.Options(solver="krylov", adv_rtol=1e-12, maxit=lim, adv_precond="ilu_on_failure")
    x, infos = OP.solve_C(m, C, rhs, c.u0, opts)
    for k in range(3):
        assert infos[k].converged and infos[k].precond == "ilu_after_failure"
        assert infos[k].iters == lim + ilu[k].iters
        ref = K.direct_solve(Cs, rhs[k])
        assert np.abs(x[k] - ref).max() <= 1e-9 * np.abs(ref).max()
    # without the fallback the same limit fails
    _, none = OP.solve_C(m, C, rhs, c.u0, OP.Options(solver="krylov", adv_rtol=1e-12, maxit=lim))
    assert not any(i.converged for i in none)
