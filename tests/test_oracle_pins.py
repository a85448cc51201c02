"""Pins of the FP64 oracle against things other than itself: closed forms,
textbook special cases, brute-force transposes, dense direct solves and
invariants of the paper's scheme (arXiv:2505.16992, App. A and B)."""
import json
import math
import os

import numpy as np
import pytest

import oracle as O
from oracle import krylov
from paper_2505_16992_b300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def mesh_of(case):
    return O.mesh_from_case(case)


# ---------------------------------------------------------------------------
# metrics (App. A.2 "Grid Transformations")
# ---------------------------------------------------------------------------

def test_metrics_rectilinear_closed_form():
    xv = np.array([0.0, 0.5, 1.5, 1.75])
    yv = np.array([0.0, 0.2, 0.7])
    zv = np.array([1.0, 1.3, 2.3])
    b = W.rect_block(xv, yv, zv)
    m = O.Mesh(3, [(b.res, b.vertices)], [], [(0, s, W.wall(b, s, 3)) for s in range(6)])
    hx, hy, hz = np.diff(xv), np.diff(yv), np.diff(zv)
    HZ, HY, HX = np.meshgrid(hz, hy, hx, indexing="ij")
    HX, HY, HZ = HX.ravel(), HY.ravel(), HZ.ravel()
    np.testing.assert_allclose(m.J, HX * HY * HZ, rtol=1e-14)
    for j, h in enumerate((HX, HY, HZ)):
        np.testing.assert_allclose(m.T[:, j, j], 1.0 / h, rtol=1e-14)
        np.testing.assert_allclose(m.alpha[j], HX * HY * HZ / h ** 2, rtol=1e-14)
    off = m.T.copy()
    for j in range(3):
        off[:, j, j] = 0
    assert np.abs(off).max() < 1e-14


def test_metrics_rotated_grid():
    """A uniform grid rotated by theta: dx/dxi = h R, so T = R^T / h, J = h^2."""
    th, h, n = 0.3, 0.1, 4
    R = np.array([[math.cos(th), -math.sin(th)], [math.sin(th), math.cos(th)]])
    V = W.tensor_vertices(np.arange(n + 1) * h, np.arange(n + 1) * h)
    Vr = V @ R.T
    walls = [(0, s, np.zeros((n, 2))) for s in range(4)]
    m = O.Mesh(2, [((n, n, 1), Vr)], [], walls)
    np.testing.assert_allclose(m.J, h * h, rtol=1e-12)
    for i in range(m.N):
        np.testing.assert_allclose(m.T[i], R.T / h, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(m.alpha, 1.0, rtol=1e-12)


def test_nonorthogonal_mesh_rejected():
    n = 3
    V = W.tensor_vertices(np.arange(n + 1.0), np.arange(n + 1.0))
    V[..., 0] += 0.3 * V[..., 1]          # shear
    walls = [(0, s, np.zeros((n, 2))) for s in range(4)]
    with pytest.raises(ValueError):
        O.Mesh(2, [((n, n, 1), V)], [], walls)


def test_missing_or_double_boundary_rejected():
    b = W.rect_block(np.arange(4.0), np.arange(3.0))
    walls = [(0, s, W.wall(b, s, 2)) for s in range(3)]
    with pytest.raises(ValueError):
        O.Mesh(2, [(b.res, b.vertices)], [], walls)
    walls = [(0, s, W.wall(b, s, 2)) for s in range(4)]
    with pytest.raises(ValueError):
        O.Mesh(2, [(b.res, b.vertices)], [(0, 1, 0, 0)], walls)


# ---------------------------------------------------------------------------
# operators: closed forms and brute-force transposes (App. A.2)
# ---------------------------------------------------------------------------

def _periodic_mesh(nx=8, ny=6, L=(2.0, 1.5)):
    c = W.periodic2d(nx, L=L[0], ny=ny, Ly=L[1])
    return c, mesh_of(c)


def test_diffusion_exact_on_quadratic():
    """With no advecting velocity, (C phi)_P = phi_P/dt - nu lap(phi); the
    compact stencil is exact for phi = x^2 + 3 y^2 at interior cells."""
    c = W.cavity2d(8)
    m = mesh_of(c)
    nu, dt = 0.7, 0.1
    C, _ = O.assemble_C(m, np.zeros((2, m.N)), nu, dt, None, m.bval)
    xc, yc = W.cell_centres(c.blocks[0])
    phi = xc ** 2 + 3 * yc ** 2
    y = O.matvec(m, C, phi)
    inner = m.inner.all(axis=0)
    np.testing.assert_allclose(y[inner], phi[inner] / dt - nu * 8.0, rtol=1e-12)


def test_central_advection_closed_form():
    """Constant velocity on a periodic grid: the face-averaged central flux
    gives c (sin(x+h) - sin(x-h)) / (2h) for phi = sin x (2 pi periodic)."""
    n = 16
    c = W.periodic2d(n, L=2 * math.pi)
    m = mesh_of(c)
    u = np.zeros((2, m.N))
    u[0] = 0.8
    u[1] = -0.3
    dt = 0.5
    C, rhs0 = O.assemble_C(m, u, 0.0, dt, None, m.bval)
    xc, yc = W.cell_centres(c.blocks[0])
    h = 2 * math.pi / n
    phi = np.sin(xc) + np.cos(2 * yc)
    exact = phi / dt + 0.8 * np.cos(xc) * math.sin(h) / h - 0.3 * (-2 * np.sin(2 * yc)) * math.sin(2 * h) / (2 * h)
    np.testing.assert_allclose(O.matvec(m, C, phi), exact, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(rhs0, u / dt, rtol=1e-15)


def test_pressure_gradient_exact_on_linear():
    xv = np.cumsum(np.r_[0.0, np.full(6, 0.2)])
    b = W.rect_block(xv, xv * 1.5, xv * 0.5)
    m = O.Mesh(3, [(b.res, b.vertices)], [], [(0, s, W.wall(b, s, 3)) for s in range(6)])
    xc = W.cell_centres(b)
    p = 2.0 * xc[0] - 3.0 * xc[1] + 0.5 * xc[2]
    g = O.grad_p(m, p)
    inner = m.inner.all(axis=0)
    for i, v in enumerate((2.0, -3.0, 0.5)):
        np.testing.assert_allclose(g[i, inner], v, rtol=1e-12)


def test_divergence_exact_on_linear_field():
    """div(h) integrated over a cell equals J (dh_x/dx + dh_y/dy) for a linear
    field at interior cells of a uniform grid."""
    c = W.cavity2d(6)
    m = mesh_of(c)
    xc, yc = W.cell_centres(c.blocks[0])
    h = np.stack([3 * xc + yc, -xc + 0.5 * yc])
    b = O.divergence(m, h, np.zeros_like(m.bval))
    inner = m.inner.all(axis=0)
    np.testing.assert_allclose(b[inner], m.J[inner] * 3.5, rtol=1e-12)


def _dense(f, n_in, shape_in):
    cols = []
    for k in range(n_in):
        e = np.zeros(n_in)
        e[k] = 1.0
        cols.append(np.ravel(f(e.reshape(shape_in))))
    return np.stack(cols, axis=1)


@pytest.mark.parametrize("case", ["bfs_small", "channel3d_small", "periodic"])
def test_transposes_brute_force(case):
    if case == "bfs_small":
        c = W.bfs2d(n_in=(4, 3), n_ch=6, n_out=3, half=3)
    elif case == "channel3d_small":
        c = W.channel3d(5, 4, 3)
    else:
        c = W.periodic2d(5, ny=4)
    m = mesh_of(c)
    d, N = m.ndim, m.N
    rng = np.random.default_rng(0)
    u = rng.standard_normal((d, N))
    C, _ = O.assemble_C(m, u, 0.37, 0.1, None, m.bval)
    Cd = _dense(lambda v: O.matvec(m, C, v), N, (N,))
    CTd = _dense(lambda v: O.matvec_T(m, C, v), N, (N,))
    np.testing.assert_allclose(CTd, Cd.T, atol=1e-13)
    np.testing.assert_allclose(O.to_sparse(m, C).toarray(), Cd, atol=1e-13)
    G = _dense(lambda v: O.grad_p(m, v), N, (N,))
    GT = _dense(lambda v: O.grad_p_T(m, v), d * N, (d, N))
    np.testing.assert_allclose(GT, G.T, atol=1e-13)
    D = _dense(lambda v: O.divergence(m, v, np.zeros_like(m.bval)), d * N, (d, N))
    DT = _dense(lambda v: O.divergence_T(m, v), N, (N,))
    np.testing.assert_allclose(DT, D.T, atol=1e-13)


def test_pressure_matrix_symmetric_and_laplacian():
    c = W.bfs2d(n_in=(4, 3), n_ch=6, n_out=3, half=3)
    m = mesh_of(c)
    rng = np.random.default_rng(1)
    A = 1.0 + rng.random(m.N)
    Pm = O.assemble_P(m, A)
    Ps = O.to_sparse(m, Pm)
    assert (Ps - Ps.T).count_nonzero() == 0          # bit-exact symmetry
    np.testing.assert_allclose(np.asarray(Ps.sum(axis=1)).ravel(), 0.0, atol=1e-13)
    # uniform grid, constant A: P = (1/A) * textbook 5-point Laplacian (Neumann walls)
    c2 = W.cavity2d(5)
    m2 = mesh_of(c2)
    P2 = O.to_sparse(m2, O.assemble_P(m2, np.full(m2.N, 2.0))).toarray()
    n = 5
    L = np.zeros((n * n, n * n))
    for y in range(n):
        for x in range(n):
            i = x + n * y
            for dx, dy in ((1, 0), (-1, 0), (0, 1), (0, -1)):
                if 0 <= x + dx < n and 0 <= y + dy < n:
                    L[i, i + dx + n * dy] += 1.0
                    L[i, i] -= 1.0
    np.testing.assert_allclose(P2, L / 2.0, atol=1e-15)


# ---------------------------------------------------------------------------
# Krylov solvers vs dense direct solves
# ---------------------------------------------------------------------------

def test_krylov_matches_dense_solve():
    c = W.cavity2d(8)
    m = mesh_of(c)
    rng = np.random.default_rng(2)
    u = rng.standard_normal((2, m.N))
    C, _ = O.assemble_C(m, u, 0.01, 0.05, None, m.bval)
    Cd = O.to_sparse(m, C).toarray()
    b = rng.standard_normal(m.N)
    x, info = krylov.bicgstab(lambda v: O.matvec(m, C, v), b, np.zeros(m.N), 1e-14)
    assert info.converged
    np.testing.assert_allclose(x, np.linalg.solve(Cd, b), rtol=1e-11, atol=1e-12)
    xt, info = krylov.bicgstab(lambda v: O.matvec_T(m, C, v), b, np.zeros(m.N), 1e-14)
    np.testing.assert_allclose(xt, np.linalg.solve(Cd.T, b), rtol=1e-11, atol=1e-12)
    # pressure: singular, consistent rhs
    Pm = O.assemble_P(m, C.diag)
    bp = rng.standard_normal(m.N)
    bp -= bp.mean()
    xp, _ = O.piso.solve_P(m, Pm, bp, np.zeros(m.N), O.Options(solver="krylov", p_rtol=1e-14))
    Pd = O.to_sparse(m, Pm).toarray()
    ref = np.linalg.lstsq(Pd, bp, rcond=None)[0]
    ref -= ref.mean()
    np.testing.assert_allclose(xp, ref, rtol=1e-9, atol=1e-11 * np.abs(ref).max())
    np.testing.assert_allclose(Pd @ xp, bp, atol=1e-11)


def test_step_krylov_equals_direct():
    c = W.channel3d(6, 5, 4)
    m = mesh_of(c)
    u1, p1, _ = O.piso_step(m, c.u0, c.p0, c.dt, c.nu, c.S, None, O.Options(solver="krylov"))
    u2, p2, _ = O.piso_step(m, c.u0, c.p0, c.dt, c.nu, c.S, None, O.Options(solver="direct"))
    np.testing.assert_allclose(u1, u2, rtol=0, atol=1e-12 * np.abs(u2).max())
    np.testing.assert_allclose(p1, p2, rtol=0, atol=1e-11 * np.abs(p2).max())


# ---------------------------------------------------------------------------
# whole-step pins: closed forms and invariants (App. A.1, App. B)
# ---------------------------------------------------------------------------

def test_divergence_free_after_correction():
    """Compact (Rhie-Chow) face-flux divergence b - P x vanishes after each
    corrector up to the solver tolerance."""
    c = W.bfs2d(n_in=(8, 4), n_ch=16, n_out=8, half=4, dt=0.05)
    m = mesh_of(c)
    u, p = c.u0, c.p0
    bval = m.bval
    for _ in range(3):
        u, p, tape = O.piso_step(m, u, p, c.dt, c.nu, c.S, bval)
        bval = tape["bval"]
        for k in range(2):
            r = O.rhie_chow_residual(m, tape, k)
            assert np.abs(r).max() <= 1e-10 * max(np.abs(tape["corr"][k]["b"]).max(), 1e-300)


def test_uniform_flow_is_preserved():
    """Uniform inflow = outflow through a y-periodic channel: u = (1, 0) must be
    an exact fixed point (pins the boundary advective flux sign, R6 and the
    outflow rescaling)."""
    n = 6
    b = W.rect_block(np.linspace(0, 1, n + 1), np.linspace(0, 0.5, n + 1))
    inflow = W.wall(b, 0, 2)
    inflow[:, 0] = 1.0
    out = W.wall(b, 1, 2)
    out[:, 0] = 1.0
    m = O.Mesh(2, [(b.res, b.vertices)], [(0, 3, 0, 2)], [(0, 0, inflow)],
               [(0, 1, np.array([1.0, 0.0]), out)])
    u = np.zeros((2, m.N))
    u[0] = 1.0
    u1, p1, tape = O.piso_step(m, u, np.zeros(m.N), 0.1, 0.05, None)
    np.testing.assert_allclose(u1, u, atol=1e-12)
    np.testing.assert_allclose(p1, 0.0, atol=1e-12)
    np.testing.assert_allclose(tape["bval"], m.bval, atol=1e-14)


def test_couette_linear_profile_exact():
    """Steady Couette flow on a uniform grid: the discrete scheme with the
    half-cell wall flux reproduces u = y exactly."""
    n = 8
    b = W.rect_block(np.linspace(0, 1, 5), np.linspace(0, 1, n + 1))
    top = W.wall(b, 3, 2)
    top[:, 0] = 1.0
    m = O.Mesh(2, [(b.res, b.vertices)], [(0, 1, 0, 0)], [(0, 2, W.wall(b, 2, 2)), (0, 3, top)])
    u = np.zeros((2, m.N))
    p = np.zeros(m.N)
    for _ in range(60):
        u, p, _ = O.piso_step(m, u, p, 5.0, 1.0, None)
    yc = W.cell_centres(b)[1]
    np.testing.assert_allclose(u[0], yc, atol=1e-12)
    np.testing.assert_allclose(u[1], 0.0, atol=1e-12)


def _poiseuille_steady(ny, gamma, steps=80):
    c = W.channel2d(nx=4, ny=ny, gamma=gamma, G=1.0, nu=1.0, dt=5.0)
    m = mesh_of(c)
    u, p = c.u0, c.p0
    for _ in range(steps):
        u, p, _ = O.piso_step(m, u, p, c.dt, c.nu, c.S)
    return c, m, u


@pytest.mark.parametrize("gamma", [0.0, 1.5])
def test_poiseuille_steady_state_equals_1d_diffusion_solve(gamma):
    """At steady state advection and the pressure gradient vanish; the profile
    is the direct solve of the 1D finite-volume diffusion problem with source G
    (face coefficient = mean of 1/h of the two cells, half-cell wall distance)."""
    ny = 12
    c, m, u = _poiseuille_steady(ny, gamma)
    yv = W.tanh_vertices(ny, 0.0, 1.0, gamma) if gamma > 0 else np.linspace(0, 1, ny + 1)
    h = np.diff(yv)
    Amat = np.zeros((ny, ny))
    rhs = h * 1.0                              # G times cell height
    for k in range(ny):
        if k > 0:
            w = 0.5 * (1 / h[k] + 1 / h[k - 1])
            Amat[k, k] += w
            Amat[k, k - 1] -= w
        else:
            Amat[k, k] += 2 / h[k]
        if k < ny - 1:
            w = 0.5 * (1 / h[k] + 1 / h[k + 1])
            Amat[k, k] += w
            Amat[k, k + 1] -= w
        else:
            Amat[k, k] += 2 / h[k]
    prof = np.linalg.solve(Amat, rhs)
    U = u[0].reshape(ny, 4)
    for x in range(4):
        np.testing.assert_allclose(U[:, x], prof, rtol=1e-11)
    np.testing.assert_allclose(u[1], 0.0, atol=1e-12)


def test_poiseuille_golden_umax_and_order():
    """App. B.1: u_max = 0.125 for G = nu = 1 on [0,1]; the discrete maximum
    converges to it at second order on uniform grids."""
    g = json.load(open(os.path.join(GOLDEN, "poiseuille_umax.json")))
    errs = []
    for ny in (8, 16, 32):
        c, m, u = _poiseuille_steady(ny, 0.0)
        yc = W.cell_centres(c.blocks[0])[1]
        exact = g["G"] / (2 * g["nu"]) * yc * (g["height"] - yc)
        errs.append(np.abs(u[0] - exact).max())
        umax_disc = u[0].max()
    assert abs(umax_disc - g["u_max"]) < 2e-3
    order = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert min(order) > 1.8


def test_taylor_green_decay_convergence():
    """Taylor-Green vortex: u(t) = u(0) exp(-2 nu t).  Refining h and dt
    together (dt ~ h) reduces the error at first order or better."""
    T_end, nu = 0.2, 0.1
    errs = []
    for n in (16, 32, 64):
        dt = 0.025 * 16 / n
        steps = int(round(T_end / dt))
        c = W.taylor_green2d(n, nu=nu, dt=dt)
        m = mesh_of(c)
        u, p = c.u0, c.p0
        for _ in range(steps):
            u, p, _ = O.piso_step(m, u, p, dt, nu, None)
        exact = c.u0 * math.exp(-2 * nu * T_end)
        errs.append(np.abs(u - exact).max())
    order = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert min(order) > 0.9, (errs, order)
    assert errs[-1] < 2e-3


def test_cavity_lid_rotation_invariance():
    """App. B.2: permutations of the lid give identical results.  A lid on +y
    moving +x and a lid on -x moving +y are the same flow rotated by 90 deg."""
    n = 8
    a = W.cavity2d(n, steps=3)
    bcase = W.cavity2d(n, steps=3, lid_side=W.SIDE_XM, lid_speed=1.0)
    ma, mb = mesh_of(a), mesh_of(bcase)
    ua, pa = a.u0, a.p0
    ub, pb = bcase.u0, bcase.p0
    for _ in range(3):
        ua, pa, _ = O.piso_step(ma, ua, pa, a.dt, a.nu, None)
        ub, pb, _ = O.piso_step(mb, ub, pb, a.dt, a.nu, None)
    # rotation by +90 deg maps point (x, y) -> (1 - y, x) and (u, v) -> (-v, u);
    # here lid (+y side, +x motion) -> (-x side, +y motion)
    Ua = ua.reshape(2, n, n)          # [c, y, x]
    Ub = ub.reshape(2, n, n)
    # b at (x', y') = (1 - y, x): Ub[:, x, n-1-y] relates to Ua[:, y, x]
    rot_u = np.empty_like(Ua)
    for y in range(n):
        for x in range(n):
            rot_u[0, x, n - 1 - y] = -Ua[1, y, x]
            rot_u[1, x, n - 1 - y] = Ua[0, y, x]
    np.testing.assert_allclose(Ub, rot_u, atol=1e-12)


def test_stokes_cavity_mirror_symmetry():
    """Without advection (tiny velocities, linear regime) mirroring x -> 1-x maps
    the flow to that of the reversed lid, which by linearity is its negative:
    u(x,y) = u(1-x,y), v(x,y) = -v(1-x,y)."""
    n = 10
    c = W.cavity2d(n, lid_speed=1e-9, nu=1.0, dt=0.01)
    m = mesh_of(c)
    u, p = c.u0, c.p0
    for _ in range(4):
        u, p, _ = O.piso_step(m, u, p, c.dt, c.nu, None)
    U = u.reshape(2, n, n)
    scale = np.abs(U).max()
    assert np.abs(U[0] - U[0][:, ::-1]).max() < 1e-8 * scale
    assert np.abs(U[1] + U[1][:, ::-1]).max() < 1e-8 * scale


def test_z_invariant_3d_equals_2d_inviscid():
    """With nu = 0 and w = 0 a z-invariant 3D periodic flow reproduces the 2D
    run exactly (with viscosity the z-diffusion enters diag(C) = A and hence the
    pressure equation, so PISO's iterates differ by design)."""
    n, nz = 6, 3
    c2 = W.turbulence2d(n, steps=2)
    m2 = mesh_of(c2)
    v = np.linspace(0, 2 * math.pi, n + 1)
    b = W.rect_block(v, v, np.linspace(0, 1.0, nz + 1))
    m3 = O.Mesh(3, [(b.res, b.vertices)], [(0, 1, 0, 0), (0, 3, 0, 2), (0, 5, 0, 4)], [])
    u2, p2 = c2.u0, c2.p0
    u3 = np.zeros((3, m3.N))
    u3[:2] = np.tile(u2, (1, nz))
    p3 = np.zeros(m3.N)
    for _ in range(2):
        u2, p2, _ = O.piso_step(m2, u2, p2, c2.dt, 0.0, None)
        u3, p3, _ = O.piso_step(m3, u3, p3, c2.dt, 0.0, None)
    U3 = u3.reshape(3, nz, n * n)
    for z in range(nz):
        np.testing.assert_allclose(U3[:2, z], u2, atol=1e-12)
        np.testing.assert_allclose(p3.reshape(nz, -1)[z], p2, atol=1e-11)
    np.testing.assert_allclose(U3[2], 0.0, atol=1e-12)


def test_poiseuille_3d_steady_state_matches_2d():
    """The 3D channel (periodic x and z, tanh walls in y) relaxes to the same
    steady profile as the 2D channel on the same y vertices."""
    ny, gamma = 8, 1.2
    c2 = W.channel2d(nx=3, ny=ny, gamma=gamma, G=1.0, nu=1.0, dt=5.0)
    m2 = mesh_of(c2)
    c3 = W.channel3d(3, ny, 2, gamma=gamma, nu=1.0, dt=5.0, amp=0.0)
    m3 = mesh_of(c3)
    u2, p2, u3, p3 = c2.u0, c2.p0, np.zeros_like(c3.u0), c3.p0
    S3 = np.zeros_like(c3.u0)
    S3[0] = 1.0
    for _ in range(60):
        u2, p2, _ = O.piso_step(m2, u2, p2, 5.0, 1.0, c2.S)
        u3, p3, _ = O.piso_step(m3, u3, p3, 5.0, 1.0, S3)
    # 2D channel spans y in [0,1], the 3D one y in [-1,1]: height 2 -> profile x4
    U3 = u3[0].reshape(2, ny, 3)
    U2 = u2[0].reshape(ny, 3)
    for z in range(2):
        np.testing.assert_allclose(U3[z], 4.0 * U2, rtol=1e-10)


def test_periodic_shift_equivariance():
    c = W.turbulence2d(16, steps=2)
    m = mesh_of(c)
    u1, p1, _ = O.piso_step(m, c.u0, c.p0, c.dt, c.nu, c.S)
    sh = lambda a: np.roll(a.reshape(a.shape[:-1] + (16, 16)), 3, axis=-1).reshape(a.shape)
    u2, p2, _ = O.piso_step(m, sh(c.u0), sh(c.p0), c.dt, c.nu, sh(c.S))
    np.testing.assert_allclose(u2, sh(u1), atol=1e-12)


def test_block_split_equivalence():
    """The same cavity as one block and as four connected blocks gives the same
    step (block connections only change the neighbour lookup, App. A.3)."""
    n = 8
    c = W.cavity2d(n, steps=2)
    m1 = mesh_of(c)
    v = np.linspace(0, 1, n + 1)
    halves = [v[: n // 2 + 1], v[n // 2:]]
    blocks, order = [], []
    for yi in range(2):
        for xi in range(2):
            blocks.append(W.rect_block(halves[xi], halves[yi]))
    # block id = xi + 2*yi
    conns = [(0, 1, 1, 0), (2, 1, 3, 0), (0, 3, 2, 2), (1, 3, 3, 2)]
    dirichlet = []
    for bid in range(4):
        xi, yi = bid % 2, bid // 2
        for s, on in ((0, xi == 0), (1, xi == 1), (2, yi == 0), (3, yi == 1)):
            if on:
                val = W.wall(blocks[bid], s, 2)
                if s == 3:
                    val[:, 0] = 1.0
                dirichlet.append((bid, s, val))
    m4 = O.Mesh(2, [(b.res, b.vertices) for b in blocks], conns, dirichlet)
    # map single-block cell (x, y) -> four-block global index
    h = n // 2
    perm = np.empty(m1.N, dtype=int)
    for y in range(n):
        for x in range(n):
            bid = (x // h) + 2 * (y // h)
            perm[x + n * y] = bid * h * h + (x % h) + h * (y % h)
    u1, p1 = c.u0, c.p0
    u4, p4 = np.zeros((2, m4.N)), np.zeros(m4.N)
    for _ in range(2):
        u1, p1, _ = O.piso_step(m1, u1, p1, c.dt, c.nu, None)
        u4, p4, _ = O.piso_step(m4, u4, p4, c.dt, c.nu, None)
    np.testing.assert_allclose(u4[:, perm], u1, atol=1e-13)
    np.testing.assert_allclose(p4[perm], p1, atol=1e-12)


def test_predictor_pressure_gradient_reading_r4():
    """Reading R4: with -grad p^n in the predictor the pressure iteration of the
    compact-Laplacian / central-gradient pair amplifies on anisotropic cells
    (aspect 8 here), while the predictor of Eq. velRHSdiscrete stays at the
    Poiseuille steady state to roundoff."""
    c = W.channel2d(nx=4, ny=32, gamma=0.0, G=1.0, nu=1.0, dt=0.05)
    m = mesh_of(c)
    out = {}
    for pg in (False, True):
        u, p = c.u0, c.p0
        for _ in range(40):
            u, p, _ = O.piso_step(m, u, p, c.dt, c.nu, c.S, None, O.Options(pred_grad_p=pg))
        out[pg] = np.abs(p).max()
    assert out[False] < 1e-12
    assert out[True] > 1.0


def test_outflow_update_balances_flux():
    c = W.bfs2d(n_in=(8, 4), n_ch=16, n_out=8, half=4)
    m = mesh_of(c)
    rng = np.random.default_rng(3)
    u = rng.standard_normal((2, m.N))
    bval = O.outflow_update(m, u, m.bval, 0.05)
    net = 0.0
    for s in range(m.nsides):
        B = np.nonzero(m.is_bface[s])[0]
        net += np.sum(O.piso.sign(s) * m.face_flux_b(s, bval[s])[B])
    assert abs(net) < 1e-13
