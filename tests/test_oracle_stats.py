"""Pins of the turbulence-statistics oracle (arXiv:2505.16992, Sec. 2.5 and
Sec. 3.3) against brute force, closed forms and finite differences."""
import math

import numpy as np
import pytest

import oracle as O
from oracle import stats as OS
from paper_2505_16992_b300 import workloads as W


def _brute_record(q, res):
    """Pure-Python loops over the cells of each plane (tiny inputs)."""
    nx, ny, nz = res
    nq = q.shape[0]
    out_mean = np.zeros((ny, nq))
    out_m2 = np.zeros((ny, nq, nq))
    out_m3 = np.zeros((ny, nq, nq, nq))
    for y in range(ny):
        cells = [x + nx * (y + ny * z) for z in range(nz) for x in range(nx)]
        n = len(cells)
        for i in range(nq):
            out_mean[y, i] = sum(q[i, c] for c in cells) / n
        for i in range(nq):
            for j in range(nq):
                out_m2[y, i, j] = sum((q[i, c] - out_mean[y, i]) * (q[j, c] - out_mean[y, j]) for c in cells) / n
                for k in range(nq):
                    out_m3[y, i, j, k] = sum((q[i, c] - out_mean[y, i]) * (q[j, c] - out_mean[y, j]) *
                                             (q[k, c] - out_mean[y, k]) for c in cells) / n
    return out_mean, out_m2, out_m3


def test_frame_record_equals_brute_force():
    rng = np.random.default_rng(0)
    res = (3, 4, 2)
    q = rng.standard_normal((2, 24)) + np.arange(2)[:, None]
    rec = OS.frame_record(q, res)
    m, m2, m3 = _brute_record(q, res)
    assert np.allclose(rec["mean"], m, rtol=0, atol=1e-14)
    assert np.allclose(rec["m2"], m2, rtol=0, atol=1e-14)
    assert np.allclose(rec["m3"], m3, rtol=0, atol=1e-14)
    assert np.all(rec["n"] == 6)


def test_frame_record_closed_form_cosine_fluctuation():
    """u = U(y) + A cos(2 pi k x / nx): per plane mean U, variance A^2 / 2,
    third moment 0 (discrete orthogonality of the sampled cosines)."""
    nx, ny, nz, k, A = 16, 5, 3, 3, 0.7
    x = np.arange(nx)
    res = (nx, ny, nz)
    N = nx * ny * nz
    idx = np.arange(N)
    xi, yi = idx % nx, (idx // nx) % ny
    U = 1.0 + 0.25 * yi
    q = np.stack([U + A * np.cos(2 * math.pi * k * xi / nx)])
    rec = OS.frame_record(q, res)
    assert np.allclose(rec["mean"][:, 0], 1.0 + 0.25 * np.arange(ny), atol=1e-14)
    assert np.allclose(rec["m2"][:, 0, 0], A * A / 2, atol=1e-14)
    assert np.allclose(rec["m3"][:, 0, 0, 0], 0.0, atol=1e-14)


def test_online_merge_equals_one_record_of_all_samples():
    """Merging frame records one by one (Pebay-type pairwise update) equals the
    record of all frames' samples taken together (frames stacked along z)."""
    rng = np.random.default_rng(1)
    res = (4, 3, 2)
    frames = [rng.standard_normal((3, 24)) * (1 + f) + f for f in range(5)]
    acc = OS.accumulate([OS.frame_record(q, res) for q in frames])
    stacked = np.concatenate([q.reshape(3, 2, 3, 4) for q in frames], axis=1).reshape(3, -1)
    whole = OS.frame_record(stacked, (4, 3, 2 * len(frames)))
    for key in ("mean", "m2", "m3"):
        assert np.allclose(acc[key], whole[key], rtol=0, atol=1e-12), key
    assert np.all(acc["n"] == whole["n"])


def test_merge_order_does_not_matter():
    rng = np.random.default_rng(2)
    res = (5, 2, 1)
    recs = [OS.frame_record(rng.standard_normal((2, 10)) + i, res) for i in range(4)]
    a = OS.accumulate(recs)
    b = OS.merge(OS.merge(recs[3], recs[1]), OS.merge(recs[0], recs[2]))
    for key in ("mean", "m2", "m3"):
        assert np.allclose(a[key], b[key], rtol=0, atol=1e-13)


def test_record_adjoint_matches_finite_differences():
    rng = np.random.default_rng(3)
    res = (3, 3, 2)
    q = rng.standard_normal((3, 18))
    rec = OS.frame_record(q, res)
    gm = rng.standard_normal(rec["mean"].shape)
    g2 = rng.standard_normal(rec["m2"].shape)
    g3 = rng.standard_normal(rec["m3"].shape)

    def L(qq):
        r = OS.frame_record(qq, res)
        return np.sum(gm * r["mean"]) + np.sum(g2 * r["m2"]) + np.sum(g3 * r["m3"])

    dq = OS.frame_record_adjoint(q, res, rec, gm, g2, g3)
    h = 1e-5
    fd = np.zeros_like(q)
    for i in range(q.shape[0]):
        for c in range(q.shape[1]):
            e = np.zeros_like(q)
            e[i, c] = h
            fd[i, c] = (-L(q + 2 * e) + 8 * L(q + e) - 8 * L(q - e) + L(q - 2 * e)) / (12 * h)
    assert np.allclose(dq, fd, rtol=1e-8, atol=1e-9)


def test_accumulated_record_adjoint_matches_finite_differences():
    """The same adjoint applied with an accumulated record (time average over
    frames) is the derivative of the accumulated statistics with respect to one
    frame's samples: central differences through ``accumulate``."""
    rng = np.random.default_rng(4)
    res = (3, 2, 2)
    frames = [rng.standard_normal((2, 12)) + f for f in range(3)]
    acc = OS.accumulate([OS.frame_record(q, res) for q in frames])
    gm = rng.standard_normal(acc["mean"].shape)
    g2 = rng.standard_normal(acc["m2"].shape)
    g3 = rng.standard_normal(acc["m3"].shape)

    def L(q1):
        r = OS.accumulate([OS.frame_record(q, res) for q in (frames[0], q1, frames[2])])
        return np.sum(gm * r["mean"]) + np.sum(g2 * r["m2"]) + np.sum(g3 * r["m3"])

    dq = OS.frame_record_adjoint(frames[1], res, acc, gm, g2, g3)
    h = 1e-5
    fd = np.zeros_like(frames[1])
    for i in range(2):
        for c in range(12):
            e = np.zeros_like(frames[1])
            e[i, c] = h
            fd[i, c] = (-L(frames[1] + 2 * e) + 8 * L(frames[1] + e) - 8 * L(frames[1] - e) +
                        L(frames[1] - 2 * e)) / (12 * h)
    assert np.allclose(dq, fd, rtol=1e-8, atol=1e-9)


def _channel(nx=8, ny=6, nz=4, gamma=1.5):
    c = W.channel3d(nx, ny, nz, gamma=gamma)
    return c, O.mesh_from_case(c)


def _uniform_channel(nx=8, ny=6, nz=4):
    """The 64x48x32 channel with uniform spacing in y (same sides)."""
    c = W.channel3d(nx, ny, nz)
    b = W.rect_block(W.uniform_vertices(nx, 0.0, 2 * math.pi), W.uniform_vertices(ny, -1.0, 1.0),
                     W.uniform_vertices(nz, 0.0, math.pi))
    c.blocks[0] = b
    c.dirichlet = [(0, s, W.wall(b, s, 3)) for s in (2, 3)]
    return c, O.mesh_from_case(c)


def test_cell_gradients_exact_on_linear_fields():
    """On a uniform grid the central differences mapped with T are exact for
    linear fields, also in the wall cells when the wall values continue the
    linear field (ghost 2 u_b - u_P); x and z are periodic, so their
    derivatives are checked away from the seams.  Pressure: exact in the
    interior, p_P at the walls (0-Neumann)."""
    c, m = _uniform_channel()
    b = c.blocks[0]
    nx, ny, nz = b.res
    xc = W.cell_centres(b)
    a = np.array([[0.3, -1.2, 0.5], [2.0, 0.7, -0.4], [-0.6, 0.1, 1.1]])
    u = a @ xc                                   # u_i = a_ik x_k
    bval = np.zeros_like(m.bval)
    for s, yw in ((2, -1.0), (3, 1.0)):
        fc = xc.copy()
        fc[1] = yw                               # face centres of the wall faces
        bval[s] = np.where(m.is_bface[s][None, :], a @ fc, 0.0)
    gu, _ = OS.cell_gradients(m, u, np.zeros(m.N), bval)
    idx = np.arange(m.N)
    xi, yi, zi = idx % nx, (idx // nx) % ny, idx // (nx * ny)
    away = (xi > 0) & (xi < nx - 1) & (zi > 0) & (zi < nz - 1)
    for i in range(3):
        assert np.allclose(gu[i, 1], a[i, 1], atol=1e-12), i            # y: every cell, walls included
        for k in (0, 2):
            assert np.allclose(gu[i, k][away], a[i, k], atol=1e-12), (i, k)
    p = -0.9 * xc[1]
    _, gp = OS.cell_gradients(m, u, p, bval)
    inner = (yi > 0) & (yi < ny - 1)
    assert np.allclose(gp[1][inner], -0.9, atol=1e-12)
    assert np.allclose(gp[0], 0.0) and np.allclose(gp[2], 0.0)
    assert np.allclose(gp[1][yi == 0], -0.9 / 2, atol=1e-12)       # (p_1 - p_0) / 2 / dy with dy = 2/ny


def test_cell_gradients_map_computational_derivatives_with_T():
    """On the stretched grid a field linear in the computational coordinate
    (q = the y index) has d q / d xi = 1 by central differences (walls: the
    ghost of the face value q_b = -1/2 or ny - 1/2), so d q / d y = T_yy."""
    c, m = _channel(gamma=1.5)
    b = c.blocks[0]
    nx, ny, nz = b.res
    yi = (np.arange(m.N) // nx) % ny
    q = np.stack([yi.astype(float)] * 3)
    bval = np.zeros_like(m.bval)
    bval[2] = np.where(m.is_bface[2][None, :], -0.5, 0.0)
    bval[3] = np.where(m.is_bface[3][None, :], ny - 0.5, 0.0)
    gu, _ = OS.cell_gradients(m, q, np.zeros(m.N), bval)
    for i in range(3):
        assert np.allclose(gu[i, 1], m.T[:, 1, 1], atol=1e-12)
        assert np.allclose(gu[i, 0], 0.0) and np.allclose(gu[i, 2], 0.0)


def test_wall_profile_derivatives_exact_for_quadratics():
    yc = np.array([-0.9, -0.55, -0.1, 0.3, 0.8])
    y0, y1 = -1.0, 1.0
    f = (yc - y0) * (y1 - yc)
    d1, d2 = OS.wall_profile_derivatives(f, yc, y0, y1)
    assert np.allclose(d1, y0 + y1 - 2 * yc, atol=1e-13)
    assert np.allclose(d2, -2.0, atol=1e-12)


def test_budget_closed_forms_on_synthetic_fluctuations():
    """u = U(y) + a cos(k x), v = b cos(k x), w = 0, p = pc sin(k x) on the
    periodic-x channel grid: R_uv = a b / 2, P_11 = -2 R_uv dU/dy, P_12 = -R_vv
    dU/dy; eps_11 = 2 nu <(d_x u')^2> with the central difference's
    d_x cos = -sin(k dx)/dx sin; Pi_11 = -2 <u' d_x p>; T and D of profiles
    that vanish at the walls are their exact derivatives (quadratics)."""
    nx, ny, nz = 12, 7, 2
    c, m = _channel(nx, ny, nz)
    b = c.blocks[0]
    xc = W.cell_centres(b)
    yv = np.unique(b.vertices.reshape(-1, 3)[:, 1])
    y0, y1 = yv.min(), yv.max()
    Lx = 2 * math.pi
    dx = Lx / nx
    kx = 2 * math.pi * 2 / Lx
    yy = xc[1]
    U = (yy - y0) * (y1 - yy)
    aa, bb, pc, nu = 0.3, 0.2, 0.5, 0.01
    cosx = np.cos(kx * xc[0])
    sinx = np.sin(kx * xc[0])
    u = np.stack([U + aa * cosx, bb * cosx, np.zeros_like(U)])
    p = pc * sinx
    gu, gp = OS.cell_gradients(m, u, p)
    rec_u = OS.frame_record(u, b.res)
    rec_gu = OS.frame_record(gu.reshape(9, -1), b.res, order=2)
    rec_up = OS.frame_record(np.concatenate([u, gp]), b.res, order=2)
    yc = rec_u["mean"][:, 0] * 0 + np.array([xc[1][y * nx] for y in range(ny)])
    B = OS.budget(rec_u, rec_gu, rec_up, yc, y0, y1, nu)
    dU = y0 + y1 - 2 * yc
    Ruv = aa * bb / 2
    assert np.allclose(rec_u["m2"][:, 0, 1], Ruv, atol=1e-14)
    assert np.allclose(B["P"][:, 0, 0], -2 * Ruv * dU, atol=1e-12)
    assert np.allclose(B["P"][:, 0, 1], -(bb * bb / 2) * dU, atol=1e-12)
    s = math.sin(kx * dx) / dx
    # interior planes: only d_x u' (the wall planes add d_y u' through the
    # no-slip ghost value -u_P of the fluctuation)
    assert np.allclose(B["eps"][1:-1, 0, 0], 2 * nu * (aa * s) ** 2 / 2, atol=1e-12)
    assert np.allclose(B["Pi"][:, 0, 0], -2 * (aa * pc * s / 2), atol=1e-12)
    assert np.allclose(B["Pi"][:, 0, 1], -(bb * pc * s / 2), atol=1e-12)   # -(<u' d_y p> + <v' d_x p>)
    assert np.allclose(B["Pi"][:, 1, 1], 0.0, atol=1e-14)                  # p does not vary in y
    # third moments of a single cosine vanish; D of a constant R with zero wall
    # values follows the three-point formula (checked above), here R_uu is
    # constant in y
    assert np.allclose(B["T"], 0.0, atol=1e-13)


def test_stats_loss_is_zero_at_the_reference():
    rng = np.random.default_rng(5)
    res = (4, 3, 2)
    frames = [rng.standard_normal((3, 24)) for _ in range(3)]
    recs = [OS.frame_record(q, res) for q in frames]
    acc = OS.accumulate(recs)
    # per-frame terms are not zero, the averaged ones are
    L0 = OS.stats_loss(recs, acc["mean"], acc["m2"], lam_frame=0.0)
    assert L0 == pytest.approx(0.0, abs=1e-28)
