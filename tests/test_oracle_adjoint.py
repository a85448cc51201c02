"""Pins of the oracle's discrete adjoint (arXiv:2505.16992, Sec. 2.3, App. A.4):
central finite differences of the full PISO step along random directions, and
the direct-optimisation task of Sec. 4.2 (loss falls below 1e-5)."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2505_16992_b300 import workloads as W


def fd4(L, eps):
    """Fourth-order central difference of a scalar function at 0."""
    return (8.0 * (L(eps) - L(-eps)) - (L(2 * eps) - L(-2 * eps))) / (12.0 * eps)


def _fd_check(case, seed, eps=1e-4, rtol=1e-6):
    m = O.mesh_from_case(case)
    d, N = m.ndim, m.N
    rng = np.random.default_rng(seed)
    u0 = case.u0 + 0.3 * rng.standard_normal((d, N))
    p0 = rng.standard_normal(N)
    S0 = rng.standard_normal((d, N)) if case.S is None else case.S + 0.1 * rng.standard_normal((d, N))
    nu0 = case.nu
    ubar = rng.standard_normal((d, N))
    pbar = rng.standard_normal(N)
    du, dp, dS = rng.standard_normal((d, N)), rng.standard_normal(N), rng.standard_normal((d, N))
    dnu = 0.3 * nu0
    # boundary values (incl. the advective outflow faces, whose update the
    # adjoint differentiates) perturbed on their faces only
    bval = [b.copy() for b in m.bval]
    dbv = [np.where(m.is_bface[s][None, :], rng.standard_normal((d, N)), 0.0) for s in range(m.nsides)]

    def L(t):
        bv = [b + t * db for b, db in zip(bval, dbv)]
        u1, p1, _ = O.piso_step(m, u0 + t * du, p0 + t * dp, case.dt, nu0 + t * dnu, S0 + t * dS, bv)
        return float(np.sum(ubar * u1) + np.sum(pbar * p1))

    _, _, tape = O.piso_step(m, u0, p0, case.dt, nu0, S0, bval)
    gu, gp, gS, gnu, gbv = O.piso_step_adjoint(m, tape, ubar, pbar, want_bval=True)
    adj = float(np.sum(gu * du) + np.sum(gp * dp) + np.sum(gS * dS) + gnu * dnu +
                sum(np.sum(g * db) for g, db in zip(gbv, dbv)))
    fd = fd4(L, eps)
    assert abs(adj - fd) <= rtol * max(abs(fd), 1e-12), (adj, fd)
    return adj, fd


@pytest.mark.parametrize("name", ["cavity", "periodic", "bfs", "channel3d"])
def test_adjoint_matches_central_fd(name):
    """All inputs at once, boundary values included (through the Dirichlet
    fluxes, the divergence and, on the step, the advective outflow update)."""
    if name == "cavity":
        c = W.cavity2d(6, nu=0.05, dt=0.05)
    elif name == "periodic":
        c = W.turbulence2d(8, nu=0.02, dt=0.05)
    elif name == "bfs":
        c = W.bfs2d(n_in=(4, 3), n_ch=6, n_out=3, half=3, nu=0.01, dt=0.05)
    else:
        c = W.channel3d(5, 4, 3, nu=0.02, dt=0.02)
    _fd_check(c, seed=11)


@pytest.mark.parametrize("pred_grad_p", [False, True])
def test_adjoint_each_input_separately(pred_grad_p):
    """Per-input directional derivatives (u^n, p^n, S, nu) each match FD, with
    and without the predictor pressure gradient (reading R4)."""
    c = W.cavity2d(5, nu=0.05, dt=0.05)
    opts = O.Options(pred_grad_p=pred_grad_p)
    m = O.mesh_from_case(c)
    d, N = 2, m.N
    rng = np.random.default_rng(5)
    u0 = 0.5 * rng.standard_normal((d, N))
    p0 = rng.standard_normal(N)
    S0 = rng.standard_normal((d, N))
    ubar, pbar = rng.standard_normal((d, N)), rng.standard_normal(N)
    _, _, tape = O.piso_step(m, u0, p0, c.dt, c.nu, S0, None, opts)
    g = O.piso_step_adjoint(m, tape, ubar, pbar, opts)
    if not pred_grad_p:
        assert np.all(g[1] == 0.0)
    eps = 1e-4
    dirs = [rng.standard_normal((d, N)), rng.standard_normal(N), rng.standard_normal((d, N)), 0.01]
    for k in range(4):
        def L(t):
            args = [u0, p0, S0, c.nu]
            args[k] = args[k] + t * dirs[k]
            u1, p1, _ = O.piso_step(m, args[0], args[1], c.dt, args[3], args[2], None, opts)
            return float(np.sum(ubar * u1) + np.sum(pbar * p1))
        fd = fd4(L, eps)
        adj = float(np.sum(g[k] * dirs[k])) if k < 3 else g[3] * dirs[3]
        assert abs(adj - fd) <= 1e-6 * max(abs(fd), 1e-12), (k, adj, fd)


def test_direct_optimisation_initial_scale():
    """Sec. 4.2: an 18x16 periodic box with a Gaussian u-profile whose unknown
    scale is recovered by gradient descent on an L2 velocity loss after n
    steps; the loss must fall below 1e-5."""
    nx, ny = 18, 16
    c = W.periodic2d(nx, L=2 * math.pi, ny=ny, Ly=2 * math.pi * ny / nx, nu=0.05, dt=0.1)
    m = O.mesh_from_case(c)
    xc, yc = W.cell_centres(c.blocks[0])
    prof = np.exp(-((yc - yc.mean()) ** 2) / 0.8)
    base = np.zeros((2, m.N))
    base[0] = prof * (1.0 + 0.3 * np.sin(xc))
    n_steps, target_scale = 3, 1.7

    def rollout(scale, keep=False):
        u, p = scale * base, np.zeros(m.N)
        tapes = []
        for _ in range(n_steps):
            u, p, t = O.piso_step(m, u, p, c.dt, c.nu, None)
            tapes.append(t)
        return u, p, tapes

    ref, _, _ = rollout(target_scale)
    scale, lr = 1.0, 0.5
    for it in range(40):
        u, p, tapes = rollout(scale)
        loss = float(np.mean((u - ref) ** 2))
        if loss < 1e-5:
            break
        gu = 2.0 * (u - ref) / u.size
        gp = np.zeros(m.N)
        for t in reversed(tapes):
            gu, gp, _, _ = O.piso_step_adjoint(m, t, gu, gp)
        grad = float(np.sum(gu * base))
        scale -= lr * grad / max(float(np.mean(base ** 2)), 1e-12)
    assert loss < 1e-5, (it, loss, scale)


def test_outflow_update_adjoint_alone():
    """The transpose of the advective outflow update (Eq. advOut with the
    inflow/outflow rescaling, R10) against central differences of the update."""
    c = W.bfs2d(n_in=(4, 3), n_ch=6, n_out=3, half=3, nu=0.01, dt=0.05)
    m = O.mesh_from_case(c)
    d, N = m.ndim, m.N
    rng = np.random.default_rng(21)
    u0 = 0.5 + 0.3 * rng.standard_normal((d, N))
    bval = [b + np.where(m.is_bface[s][None, :], 0.1 * rng.standard_normal((d, N)), 0.0)
            for s, b in enumerate(m.bval)]
    g_used = [np.where(m.is_bface[s][None, :], rng.standard_normal((d, N)), 0.0) for s in range(m.nsides)]
    dbv = [np.where(m.is_bface[s][None, :], rng.standard_normal((d, N)), 0.0) for s in range(m.nsides)]
    du = rng.standard_normal((d, N))

    def L(t):
        out = O.outflow_update(m, u0 + t * du, [b + t * db for b, db in zip(bval, dbv)], c.dt)
        return float(sum(np.sum(g * o) for g, o in zip(g_used, out)))

    g_in, gu = O.piso.outflow_update_adjoint(m, u0, bval, c.dt, g_used)
    adj = float(np.sum(gu * du) + sum(np.sum(g * db) for g, db in zip(g_in, dbv)))
    fd = fd4(L, 1e-5)
    assert abs(adj - fd) <= 1e-8 * max(abs(fd), 1e-12), (adj, fd)
    assert np.abs(gu).max() > 0          # the update does depend on the cell values
