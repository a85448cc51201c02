"""Pins of block connections with permuted or flipped axes (Sec. 2.2: blocks
joined side to side with matching resolution; App. A.3: a connection only
changes the neighbour lookup; App. B: O- and C-grids need such cuts).

The same cells described by two block layouts must give the same step: a
block whose index frame is turned (180 degrees, +-90 degrees, a 3D turn that
exchanges two tangential axes) joins its neighbour through a flipped or
permuted connection, and the result must equal that of the plain layout,
forward and adjoint, on orthogonal and on slanted (non-orthogonal) cells.  A
C-grid whose cut is a side joined to itself with its tangential axis
reversed must equal the same mesh cut into two blocks; its adjoint must
equal central differences."""
import math

import numpy as np
import pytest

import oracle as O
from oracle import piso as OP
from paper_2505_16992_b300 import workloads as W


def _centres(case):
    return np.concatenate([W.cell_centres(b) for b in case.blocks], axis=1)


def _step(case, opts):
    m = O.mesh_from_case(case, allow_nonorthogonal=True)
    u1, p1, tape = O.piso_step(m, case.u0, case.p0, case.dt, case.nu, case.S, None, opts)
    return m, u1, p1, tape


def _compare(c, idx, c0, opts, seed):
    """Forward and adjoint of layout c against the plain layout c0 (cell k of c
    is cell idx[k] of c0)."""
    m, u1, p1, t = _step(c, opts)
    m0, u0, p0, t0 = _step(c0, opts)
    assert m.twisted and not m0.twisted
    np.testing.assert_allclose(_centres(c), _centres(c0)[:, idx], atol=1e-14)
    su = np.abs(u0).max()
    assert np.abs(u1 - u0[:, idx]).max() <= 1e-12 * su
    assert np.abs(p1 - p0[idx]).max() <= 1e-11 * np.abs(p0).max()
    rng = np.random.default_rng(seed)
    gu, gp = rng.standard_normal(u0.shape), rng.standard_normal(p0.shape)
    a0 = O.piso_step_adjoint(m0, t0, gu, gp, opts)
    a1 = O.piso_step_adjoint(m, t, gu[:, idx], gp[idx], opts)
    for k, (x1, x0) in enumerate(zip(a1[:3], a0[:3])):
        x0 = x0[..., idx]
        assert np.abs(x1 - x0).max() <= 1e-11 * max(np.abs(x0).max(), 1e-300), k
    assert abs(a1[3] - a0[3]) <= 1e-11 * abs(a0[3])


@pytest.mark.parametrize("shear", [0.0, 0.4])
@pytest.mark.parametrize("rot", [1, 2, 3])
def test_turned_block_equals_plain_layout_2d(rot, shear):
    c, idx = W.two_block_cavity2d(8, 6, rot=rot, shear=shear)
    c0, _ = W.two_block_cavity2d(8, 6, rot=0, shear=shear)
    _compare(c, idx, c0, OP.Options(n_nonortho=2), seed=rot)


@pytest.mark.parametrize("shear", [0.0, 0.4])
def test_turned_block_equals_plain_layout_3d(shear):
    """The turn about x exchanges the joint's tangential axes (axis_perm = 1)
    and reverses one of them (flip_mask bit 0)."""
    c, idx = W.two_block_channel3d(turned=True, shear=shear)
    c0, _ = W.two_block_channel3d(turned=False, shear=shear)
    _compare(c, idx, c0, OP.Options(n_nonortho=2), seed=7)


def test_neighbours_across_turned_joints_are_adjacent():
    """Every neighbour across a permuted or flipped joint is the physically
    adjacent cell (one cell width away, through the shared face)."""
    for c in (W.two_block_cavity2d(8, 6, rot=3)[0], W.two_block_channel3d(turned=True)[0],
              W.slit_cgrid2d(12, 6)):
        m = O.mesh_from_case(c, allow_nonorthogonal=True)
        xc = _centres(c)
        for s in range(m.nsides):
            P = np.nonzero(m.inner[s] & np.any(m.nbax[s] != np.arange(3), axis=1)
                           | m.inner[s] & np.any(m.nbsg[s] != 1.0, axis=1))[0]
            if not len(P):
                continue
            F = m.nb[s, P]
            # the neighbour's face towards P is P's face: the midpoint of the
            # two centres lies on it, so both cells are half a width from it
            h = np.sqrt(np.abs(m.J[P])) if m.ndim == 2 else np.cbrt(np.abs(m.J[P]))
            dist = np.linalg.norm(xc[:, F] - xc[:, P], axis=0)
            assert np.all(dist < 3.0 * h), (c.name, s, dist.max())


def _slit_two_blocks(n_xi, n_eta):
    """The slit C-grid cut at xi = 0 into two blocks, the left one turned by 180
    degrees: the cut becomes a plain side-to-side connection and the joint at
    xi = 0 (the negative x-axis) one between two -x sides with the tangential
    axis reversed.  Returns (case, cell_index into the one-block layout)."""
    one = W.slit_cgrid2d(n_xi, n_eta)
    V = one.blocks[0].vertices
    h = n_xi // 2
    left = W.Block((h, n_eta, 1), V[:, : h + 1].copy())
    right = W.Block((h, n_eta, 1), V[:, h:].copy())
    lt, old, side_map = W.rotate_block_2d(left, 2)
    ui = np.array([1.0, 0.0])
    dirichlet = [(0, side_map[s], np.tile(ui, (W.side_nfaces(lt.res, side_map[s], 2), 1))) for s in (0, 3)]
    dirichlet += [(1, s, np.tile(ui, (W.side_nfaces(right.res, s, 2), 1))) for s in (1, 3)]
    conns = [(0, side_map[2], 1, 2), (0, side_map[1], 1, 0, 0, 1)]
    # cell index of the one-block layout: left cells (x < h) and right cells
    gx = np.arange(n_xi * n_eta).reshape(n_eta, n_xi)
    idx = np.concatenate([gx[:, :h].ravel()[old], gx[:, h:].ravel()])
    c = W.Case("slit2", 2, [lt, right], conns, dirichlet, [], one.u0[:, idx], one.p0[idx], None, one.nu, one.dt, 1)
    return c, idx, one


def test_cgrid_fold_equals_two_block_layout():
    """A side joined to itself with its axis reversed (the C-grid cut) against
    the same cells as two blocks (a plain cut and a flipped joint elsewhere):
    equal steps, forward and adjoint, over two steps."""
    c2, idx, one = _slit_two_blocks(12, 6)
    opts = OP.Options(n_nonortho=2)
    m1 = O.mesh_from_case(one, allow_nonorthogonal=True)
    m2 = O.mesh_from_case(c2, allow_nonorthogonal=True)
    assert m1.twisted and m2.twisted and m1.has_cross
    u1, p1, u2, p2 = one.u0, one.p0, c2.u0, c2.p0
    for _ in range(2):
        u1, p1, t1 = O.piso_step(m1, u1, p1, one.dt, one.nu, None, None, opts)
        u2, p2, t2 = O.piso_step(m2, u2, p2, one.dt, one.nu, None, None, opts)
        assert np.abs(u2 - u1[:, idx]).max() <= 1e-12 * np.abs(u1).max()
        assert np.abs(p2 - p1[idx]).max() <= 1e-11 * np.abs(p1).max()
    rng = np.random.default_rng(3)
    gu, gp = rng.standard_normal(u1.shape), rng.standard_normal(p1.shape)
    a1 = O.piso_step_adjoint(m1, t1, gu, gp, opts)
    a2 = O.piso_step_adjoint(m2, t2, gu[:, idx], gp[idx], opts)
    for k in range(2):
        assert np.abs(a2[k] - a1[k][..., idx]).max() <= 1e-11 * np.abs(a1[k]).max(), k
    assert abs(a2[3] - a1[3]) <= 1e-11 * abs(a1[3])


def _fd4(f, eps):
    return (-f(2 * eps) + 8 * f(eps) - 8 * f(-eps) + f(-2 * eps)) / (12 * eps)


def test_cgrid_adjoint_matches_central_differences():
    """dL/du^n, dL/dp^n and dL/dnu of the step on the C-grid with its folded cut
    equal 4th-order central differences."""
    c = W.slit_cgrid2d(12, 6)
    m = O.mesh_from_case(c, allow_nonorthogonal=True)
    opts = OP.Options(n_nonortho=2, solver="direct")
    rng = np.random.default_rng(4)
    ubar, pbar = rng.standard_normal(c.u0.shape), rng.standard_normal(c.p0.shape)
    _, _, tape = O.piso_step(m, c.u0, c.p0, c.dt, c.nu, None, None, opts)
    gu, gp, _, gnu = O.piso_step_adjoint(m, tape, ubar, pbar, opts)
    du, dp = rng.standard_normal(c.u0.shape), rng.standard_normal(c.p0.shape)
    for k, (adj, f) in enumerate([
            (float(np.sum(gu * du)), lambda t: O.piso_step(m, c.u0 + t * du, c.p0, c.dt, c.nu, None, None, opts)),
            (float(np.sum(gp * dp)), lambda t: O.piso_step(m, c.u0, c.p0 + t * dp, c.dt, c.nu, None, None, opts)),
            (gnu * 0.01, lambda t: O.piso_step(m, c.u0, c.p0, c.dt, c.nu + 0.01 * t, None, None, opts))]):
        def L(t, f=f):
            u1, p1, _ = f(t)
            return float(np.sum(ubar * u1) + np.sum(pbar * p1))
        fd = _fd4(L, 1e-4)
        assert abs(adj - fd) <= 1e-6 * abs(fd), (k, adj, fd)


def test_connection_descriptions_rejected():
    c = W.slit_cgrid2d(12, 6)
    b = (c.blocks[0].res, c.blocks[0].vertices)
    walls = [(0, s, np.zeros((W.side_nfaces(b[0], s, 2), 2))) for s in (0, 1, 3)]
    with pytest.raises(ValueError):                  # a 2D joint has one tangential axis: no exchange
        O.Mesh(2, [b], [(0, 2, 0, 2, 1, 1)], walls, allow_nonorthogonal=True)
    with pytest.raises(ValueError):                  # a fold without the reversal pairs each cell with itself
        O.Mesh(2, [b], [(0, 2, 0, 2, 0, 0)], walls, allow_nonorthogonal=True)
    odd = W.slit_cgrid2d(11, 6)
    bo = (odd.blocks[0].res, odd.blocks[0].vertices)
    wo = [(0, s, np.zeros((W.side_nfaces(bo[0], s, 2), 2))) for s in (0, 1, 3)]
    with pytest.raises(ValueError):                  # odd count: the middle cell would meet itself
        O.Mesh(2, [bo], [(0, 2, 0, 2, 0, 1)], wo, allow_nonorthogonal=True)
    c2, _ = W.two_block_cavity2d(8, 6, rot=0)
    bl = [(x.res, x.vertices) for x in c2.blocks]
    with pytest.raises(ValueError):                  # resolutions of the joined sides differ (8 vs 6 cells)
        O.Mesh(2, bl, [(0, 1, 1, 2)], c2.dirichlet)


def test_ignoring_the_frames_breaks_the_equivalence():
    """Planted slip: read the neighbour across a turned joint as if its axes
    were P's (identity frame, opposite return side); the turned layout then
    no longer reproduces the plain one (so the equivalence pins the frames).
    The 3D joint keeps its normal axis, so there the frames matter through the
    tangential cross terms of the slanted cells."""
    for c, idx, c0 in [(*W.two_block_cavity2d(8, 6, rot=2, shear=0.4), W.two_block_cavity2d(8, 6, rot=0, shear=0.4)[0]),
                       (*W.two_block_channel3d(turned=True, shear=0.4),
                        W.two_block_channel3d(turned=False, shear=0.4)[0])]:
        m = O.mesh_from_case(c, allow_nonorthogonal=True)
        m.nbax[:] = np.arange(3)
        m.nbsg[:] = 1.0
        m.nbret[:] = np.array([s ^ 1 for s in range(m.nsides)])[:, None]
        opts = OP.Options(n_nonortho=2)
        u1, _, _ = O.piso_step(m, c.u0, c.p0, c.dt, c.nu, c.S, None, opts)
        m0 = O.mesh_from_case(c0, allow_nonorthogonal=True)
        u0, _, _ = O.piso_step(m0, c0.u0, c0.p0, c0.dt, c0.nu, c0.S, None, opts)
        assert np.abs(u1 - u0[:, idx]).max() > 1e-4 * np.abs(u0).max()
