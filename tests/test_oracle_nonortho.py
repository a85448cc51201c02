"""Pins of the oracle's non-orthogonal terms (App. A.2 "Non-Orthogonal
Grids": the cross derivatives alpha_jk d_j d_k, j != k, of the viscous term
and of the pressure operator; the direct-neighbour part of the viscous ones in
the matrix (Eq. difNonOrthoMatDiscrete), the rest deferred to the right-hand
sides with the previous iterate over non-orthogonal corrector steps), against
facts that do
not depend on the oracle: exactness of the full discrete operators on
quadratic fields of affine (sheared) grids, vanishing cross terms on
orthogonal grids, the fixed point of the corrector loops, and the
Taylor-Green decay on a sheared periodic grid."""
import math

import numpy as np
import pytest

import oracle as O
from oracle import piso as OP
from paper_2505_16992_b300 import workloads as W


def _verts(res, h, shear):
    """Vertices of an affine sheared block: x = A (xi h), A = I + strict upper
    shear (x gets a*y + b*z, y gets c*z)."""
    nd = len(res)
    axes = [np.arange(r + 1) * hh for r, hh in zip(res, h)]
    if nd == 2:
        Y, X = np.meshgrid(axes[1], axes[0], indexing="ij")
        return np.stack([X + shear[0] * Y, Y], axis=-1)               # [y][x][2]
    Z, Y, X = np.meshgrid(axes[2], axes[1], axes[0], indexing="ij")
    return np.stack([X + shear[0] * Y + shear[1] * Z, Y + shear[2] * Z, Z], axis=-1)   # [z][y][x][3]


def _walled_mesh(res, h, shear, seed=0):
    """One sheared block with Dirichlet values (seeded) on every side."""
    nd = len(res)
    rng = np.random.default_rng(seed)
    r3 = tuple(res) + ((1,) if nd == 2 else ())
    dirichlet = []
    for s in range(2 * nd):
        ax = s // 2
        nf = int(np.prod([r3[a] for a in range(3) if a != ax]))
        dirichlet.append((0, s, rng.standard_normal((nf, nd))))
    return O.Mesh(nd, [(r3, _verts(res, h, shear))], (), dirichlet, allow_nonorthogonal=True)


def _centres(m, res, h, shear):
    """Cell centres of the affine block (the images of the computational centres)."""
    nd = len(res)
    if nd == 2:
        yy, xx = np.meshgrid((np.arange(res[1]) + 0.5) * h[1], (np.arange(res[0]) + 0.5) * h[0], indexing="ij")
        return np.stack([(xx + shear[0] * yy).ravel(), yy.ravel()])
    zz, yy, xx = np.meshgrid(*[(np.arange(res[a]) + 0.5) * h[a] for a in (2, 1, 0)], indexing="ij")
    return np.stack([(xx + shear[0] * yy + shear[1] * zz).ravel(), (yy + shear[2] * zz).ravel(), zz.ravel()])


def _interior(res, depth=2):
    nd = len(res)
    idx = np.indices(tuple(reversed(res))).reshape(nd, -1)[::-1]    # x first
    keep = np.ones(idx.shape[1], dtype=bool)
    for a in range(nd):
        keep &= (idx[a] >= depth) & (idx[a] < res[a] - depth)
    return keep


@pytest.mark.parametrize("res,h,shear", [((10, 9), (0.1, 0.12), (0.6,)),
                                         ((7, 8, 7), (0.1, 0.12, 0.09), (0.5, -0.3, 0.4))])
def test_full_viscous_operator_exact_on_quadratics(res, h, shear):
    """On an affine grid the orthogonal part (matrix C) plus the cross part
    equals nu times the Laplacian of any quadratic field, at every cell whose
    stencil stays inside (J, T, alpha constant; central differences exact)."""
    m = _walled_mesh(res, h, shear)
    assert m.has_cross
    nd = len(res)
    xc = _centres(m, res, h, shear)
    rng = np.random.default_rng(1)
    Q = rng.standard_normal((nd, nd))
    Q = Q + Q.T                                   # q = x.Q.x/2 + g.x + c
    g = rng.standard_normal(nd)
    q = 0.5 * np.einsum("in,ij,jn->n", xc, Q, xc) + g @ xc + 0.3
    nu, dt = 0.7, 1e30
    u = np.zeros((nd, m.N))
    C, _ = OP.assemble_C(m, u, nu, dt, None, m.bval)
    qq = np.zeros((nd, m.N))
    qq[0] = q
    orth = -((C.diag - 1.0 / dt) * q + OP.offdiag_matvec(m, C, qq)[0])
    total = orth + OP.cross_diffusion(m, qq, nu, m.bval)[0]
    keep = _interior(res)
    want = nu * np.trace(Q)
    assert np.abs(total[keep] - want).max() <= 1e-10 * abs(want)
    # the cross part is really needed: the orthogonal part alone is off
    assert np.abs(orth[keep] - want).max() > 1e-3 * abs(want)


@pytest.mark.parametrize("res,h,shear", [((10, 9), (0.1, 0.12), (0.6,)),
                                         ((7, 8, 7), (0.1, 0.12, 0.09), (0.5, -0.3, 0.4))])
def test_full_pressure_operator_exact_on_quadratics(res, h, shear):
    """P (Eq. pMatDiscrete with A = 1) plus the cross part equals the cell
    volume J times the Laplacian of a quadratic field in the interior."""
    m = _walled_mesh(res, h, shear)
    nd = len(res)
    xc = _centres(m, res, h, shear)
    rng = np.random.default_rng(2)
    Q = rng.standard_normal((nd, nd))
    Q = Q + Q.T
    q = 0.5 * np.einsum("in,ij,jn->n", xc, Q, xc) + rng.standard_normal(nd) @ xc
    A = np.ones(m.N)
    Pm = OP.assemble_P(m, A)
    full = OP.matvec(m, Pm, q) + OP.cross_pressure(m, q, A)
    keep = _interior(res)
    want = m.J * np.trace(Q)
    assert np.abs(full[keep] - want[keep]).max() <= 1e-10 * np.abs(want).max()


def test_cross_terms_vanish_on_orthogonal_grids():
    c = W.channel3d(8, 6, 4)
    m = OP.mesh_from_case(c, allow_nonorthogonal=True)
    assert not m.has_cross
    rng = np.random.default_rng(3)
    u = rng.standard_normal((3, m.N))
    assert np.all(OP.cross_diffusion(m, u, 0.1, m.bval) == 0.0)
    assert np.all(OP.cross_pressure(m, rng.standard_normal(m.N), 1.0 + rng.random(m.N)) == 0.0)


def test_nonorthogonal_meshes_still_rejected_by_default():
    with pytest.raises(ValueError):
        O.Mesh(2, [((6, 5, 1), _verts((6, 5), (0.1, 0.1), (0.5,)))], (),
               [(0, s, np.zeros((5 if s < 2 else 6, 2))) for s in range(4)])


@pytest.mark.parametrize("split", ["paper", "deferred"])
def test_corrector_loops_converge_to_the_full_discrete_system(split):
    """With enough non-orthogonal corrector steps the predictor solves the
    momentum system with the cross terms included (C u* = rhs + X(u*), C the
    orthogonal matrix of Eqs. advMatDiscrete / difMatDiscrete) and every
    pressure solve the full pressure system ((P + Y) p = b), to the solver
    tolerance, whichever part of the viscous cross terms the matrix holds."""
    res, h, shear = (9, 8), (0.1, 0.1), (0.7,)
    m = _walled_mesh(res, h, shear, seed=4)
    rng = np.random.default_rng(5)
    u0 = rng.standard_normal((2, m.N))
    p0 = rng.standard_normal(m.N)
    S = rng.standard_normal((2, m.N))
    nu, dt = 0.05, 0.02
    opts = OP.Options(n_nonortho=60, solver="direct", nonortho_split=split)
    u1, p1, tape = O.piso_step(m, u0, p0, dt, nu, S, None, opts)
    C, rhs = OP.assemble_C(m, u0, nu, dt, S, tape["bval"])
    us = tape["ustar"]
    res_u = rhs + OP.cross_diffusion(m, us, nu, tape["bval"]) - OP.matvec(m, C, us)
    assert np.abs(res_u).max() <= 1e-10 * np.abs(rhs).max()
    A = tape["C"].diag
    for cr in tape["corr"]:
        r = cr["b"] - OP.matvec(m, tape["Pm"], cr["x"]) - OP.cross_pressure(m, cr["x"], A)
        r -= r.mean()
        assert np.abs(r).max() <= 1e-10 * np.abs(cr["b"]).max()
    # one step is not the same as the orthogonal scheme on this mesh
    u1a, _, _ = O.piso_step(m, u0, p0, dt, nu, S, None, OP.Options(n_nonortho=1, solver="direct",
                                                                   nonortho_split=split))
    assert np.abs(u1a - u1).max() > 0


def test_paper_split_matrix_holds_the_direct_neighbour_terms():
    """The split of Eq. difNonOrthoMatDiscrete / Eq. velRHSnonOrtho: the cross
    terms with P's own central differences are an affine map of u whose matrix
    touches only P and its direct neighbours (the 2d+1 stencil of C), the rest
    uses P's diagonal neighbours; together they are the whole cross term."""
    m = _walled_mesh((7, 6, 5), (0.1, 0.12, 0.09), (0.5, -0.3, 0.4), seed=13)
    rng = np.random.default_rng(14)
    u = rng.standard_normal((3, m.N))
    nu = 0.2
    M = OP.cross_matrix(m, nu)
    own = OP.cross_diffusion(m, u, nu, m.bval, part="own")
    const = OP.cross_diffusion(m, np.zeros_like(u), nu, m.bval, part="own")
    np.testing.assert_allclose(own, OP.matvec(m, M, u) + const, rtol=1e-12, atol=1e-13 * np.abs(own).max())
    nbr = OP.cross_diffusion(m, u, nu, m.bval, part="nbr")
    np.testing.assert_allclose(own + nbr, OP.cross_diffusion(m, u, nu, m.bval), rtol=1e-12,
                               atol=1e-13 * np.abs(own).max())
    # the neighbour part does not see P's direct neighbours: perturbing one
    # cell moves it only at cells for which that cell is a diagonal neighbour
    # (or a direct neighbour of theirs across a boundary ghost, none here in
    # the interior)
    i = 3 + 7 * (3 + 6 * 2)
    du = np.zeros_like(u)
    du[1, i] = 1.0
    moved = np.nonzero(np.abs(OP.cross_diffusion(m, u + du, nu, m.bval, part="nbr") - nbr)[1] > 0)[0]
    direct = {int(m.nb[s, i]) for s in range(m.nsides)}
    assert not (set(moved.tolist()) & (direct | {i}))


def _wavy_periodic(n, L=2 * math.pi, a=0.35):
    """A curved periodic box: x = xi + a sin(eta), y = eta + a sin(xi) (period
    L = 2 pi in both, so the mesh wraps onto itself); alpha_jk varies from
    cell to cell.  Seeded smooth initial field."""
    t = np.arange(n + 1) * L / n
    E, X = np.meshgrid(t, t, indexing="ij")
    V = np.stack([X + a * np.sin(E), E + a * np.sin(X)], axis=-1)
    m = O.Mesh(2, [((n, n, 1), V)], [(0, 0, 0, 1), (0, 2, 0, 3)], allow_nonorthogonal=True)
    rng = np.random.default_rng(16)
    u0 = rng.standard_normal((2, m.N))
    return m, u0, rng.standard_normal(m.N)


def test_splits_differ_at_one_corrector_step_and_agree_when_converged():
    """Both splits converge to the same full momentum system, so the converged
    predictors agree.  A = diag C differs only where a Dirichlet ghost puts a
    cross entry on the diagonal, so on a mesh without walls (the sheared
    periodic box) whole converged steps agree too; at n_nonortho = 1 the two
    are different approximations of it."""
    m = _walled_mesh((9, 8), (0.1, 0.1), (0.7,), seed=4)
    rng = np.random.default_rng(15)
    u0 = rng.standard_normal((2, m.N))
    p0 = rng.standard_normal(m.N)
    nu, dt = 0.05, 0.02
    us = {sp: O.piso_step(m, u0, p0, dt, nu, None, None, OP.Options(n_nonortho=60, solver="direct",
                                                                    nonortho_split=sp))[2]["ustar"]
          for sp in ("paper", "deferred")}
    assert np.abs(us["paper"] - us["deferred"]).max() <= 1e-10 * np.abs(us["paper"]).max()
    assert np.abs(OP.cross_matrix(m, nu).diag).max() > 0          # walls: A differs at the wall cells
    mp, u0, p0 = _wavy_periodic(12)
    assert np.all(OP.cross_matrix(mp, 0.1).diag == 0)               # no walls: A is the same
    assert np.abs(OP.cross_matrix(mp, 0.1).off).max() > 0           # alpha_jk varies: direct entries
    out = {}
    for split in ("paper", "deferred"):
        for n in (1, 60):
            out[split, n] = O.piso_step(mp, u0, p0, 0.05, 0.1, None, None,
                                        OP.Options(n_nonortho=n, solver="direct", nonortho_split=split))[0]
    scale = np.abs(out["paper", 60]).max()
    assert np.abs(out["paper", 60] - out["deferred", 60]).max() <= 1e-10 * scale
    d1 = np.abs(out["paper", 1] - out["deferred", 1]).max() / scale
    assert d1 > 1e-6, d1


def _tg_sheared(n, nu, dt):
    """Taylor-Green vortex on [0, 2 pi)^2 with parallelogram cells x = xi h + eta
    h, y = eta h: shifting eta by the period moves x by 2 pi, so both
    directions wrap periodically."""
    h = 2 * math.pi / n
    V = _verts((n, n), (h, h), (1.0,))
    m = O.Mesh(2, [((n, n, 1), V)], [(0, 0, 0, 1), (0, 2, 0, 3)], allow_nonorthogonal=True)
    xc = _centres(m, (n, n), (h, h), (1.0,))
    x, y = xc
    u0 = np.stack([-np.cos(x) * np.sin(y), np.sin(x) * np.cos(y)])
    p0 = -0.25 * (np.cos(2 * x) + np.cos(2 * y))
    return m, u0, p0


def test_taylor_green_decay_on_a_sheared_periodic_grid():
    """u(t) = u(0) exp(-2 nu t) on cells sheared by 45 degrees: with the cross
    terms (two non-orthogonal corrector steps) the error falls at second order
    as h and dt are refined together (measured 2.10, 2.07); with the cross terms
    left out it stalls (0.79, 0.37), so this pins them."""
    T_end, nu = 0.2, 0.1
    errs = []
    for n in (16, 32, 64):
        dt = 0.025 * 16 / n
        steps = int(round(T_end / dt))
        m, u, p = _tg_sheared(n, nu, dt)
        exact = u * math.exp(-2 * nu * T_end)
        opts = OP.Options(n_nonortho=2)
        for _ in range(steps):
            u, p, _ = O.piso_step(m, u, p, dt, nu, None, None, opts)
        errs.append(np.abs(u - exact).max())
    order = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert min(order) > 1.5, (errs, order)
    assert errs[-1] < 5e-3, errs


def _fd4(f, eps):
    return (-f(2 * eps) + 8 * f(eps) - 8 * f(-eps) + f(-2 * eps)) / (12 * eps)


def test_cross_operator_transposes_are_exact():
    """<X(u), g> = <u, X_u^T g> + <bval, X_b^T g> and <Y(p), g> = <p, Y^T g>,
    with the A-derivative of Y checked by central differences."""
    res, h, shear = (7, 6), (0.1, 0.12), (0.6,)
    m = _walled_mesh(res, h, shear, seed=8)
    rng = np.random.default_rng(9)
    u = rng.standard_normal((2, m.N))
    g = rng.standard_normal((2, m.N))
    nu = 0.3
    for part in ("all", "own", "nbr"):
        gu, gb = OP.cross_diffusion_T(m, g, nu, part)
        lhs = float(np.sum(OP.cross_diffusion(m, u, nu, m.bval, part) * g))
        rhs = float(np.sum(gu * u)) + sum(float(np.sum(gb[s] * m.bval[s])) for s in range(m.nsides))
        assert abs(lhs - rhs) <= 1e-12 * abs(lhs), part
    p = rng.standard_normal(m.N)
    A = 1.0 + rng.random(m.N)
    gy = rng.standard_normal(m.N)
    gp, gA = OP.cross_pressure_T(m, gy, p, A)
    assert abs(float(np.sum(OP.cross_pressure(m, p, A) * gy)) - float(np.sum(gp * p))) <= 1e-12 * np.abs(gp).sum()
    dA = rng.standard_normal(m.N)
    fd = _fd4(lambda t: float(np.sum(OP.cross_pressure(m, p, A + t * dA) * gy)), 1e-4)
    assert abs(float(np.sum(gA * dA)) - fd) <= 1e-8 * abs(fd)


@pytest.mark.parametrize("split", ["paper", "deferred"])
@pytest.mark.parametrize("periodic", [False, True])
def test_nonorthogonal_adjoint_matches_central_differences(periodic, split):
    """The adjoint of the non-orthogonal step (two corrector steps): every
    input's directional derivative (u^n, p^n, which now enters through the
    pressure cross terms, S, nu and the boundary values) equals 4th-order
    central differences of the forward step."""
    res, h, shear = (7, 6), (0.1, 0.12), (0.6,)
    if periodic:
        m0 = _walled_mesh(res, h, shear, seed=10)
        dirichlet = [(0, s, m0.side_values(m0.bval, 0, s)) for s in (2, 3)]
        m = O.Mesh(2, [((7, 6, 1), _verts(res, h, shear))], [(0, 0, 0, 1)], dirichlet, allow_nonorthogonal=True)
    else:
        m = _walled_mesh(res, h, shear, seed=10)
    d, N = 2, m.N
    rng = np.random.default_rng(12)
    u0 = 0.5 * rng.standard_normal((d, N))
    p0 = rng.standard_normal(N)
    S0 = rng.standard_normal((d, N))
    nu, dt = 0.05, 0.03
    opts = OP.Options(n_nonortho=2, solver="direct", nonortho_split=split)
    ubar, pbar = rng.standard_normal((d, N)), rng.standard_normal(N)
    _, _, tape = O.piso_step(m, u0, p0, dt, nu, S0, None, opts)
    gu, gp, gS, gnu, gbv = O.piso_step_adjoint(m, tape, ubar, pbar, opts, want_bval=True)
    assert np.abs(gp).max() > 0
    dirs = [rng.standard_normal((d, N)), rng.standard_normal(N), rng.standard_normal((d, N)), 0.01]
    bdir = [rng.standard_normal((d, N)) * m.is_bface[s][None, :] for s in range(m.nsides)]
    for k in range(5):
        def L(t):
            args = [u0, p0, S0, nu]
            bv = m.bval
            if k < 4:
                args[k] = args[k] + t * dirs[k]
            else:
                bv = np.stack([m.bval[s] + t * bdir[s] for s in range(m.nsides)])
            u1, p1, _ = O.piso_step(m, args[0], args[1], dt, args[3], args[2], bv, opts)
            return float(np.sum(ubar * u1) + np.sum(pbar * p1))
        fd = _fd4(L, 1e-4)
        if k < 3:
            adj = float(np.sum([gu, gp, gS][k] * dirs[k]))
        elif k == 3:
            adj = gnu * dirs[3]
        else:
            adj = sum(float(np.sum(gbv[s] * bdir[s])) for s in range(m.nsides))
        assert abs(adj - fd) <= 1e-6 * max(abs(fd), 1e-12), (k, adj, fd)
