"""Non-orthogonal meshes on the GPU (App. A.2 "Non-Orthogonal Grids": the
cross derivatives of the viscous term, their direct-neighbour part in the
matrix and the rest deferred, and of the pressure operator, deferred, to the
right-hand sides with the previous iterate over n_nonortho corrector steps;
with App. A.4 the adjoint of that step) against the FP64 oracle, element by
element through the C ABI, on sheared 2D and 3D blocks with Dirichlet sides,
curved (wavy) blocks and sheared periodic boxes."""
import math
import types

import numpy as np
import pytest

import oracle as O
from oracle import piso as OP
from paper_2505_16992_b300 import capi
from paper_2505_16992_b300.solver import Batch
from gpu_util import FP32_REL, FP64_REL, bval_faces, gpu_domain, gpu_step, host, rel_err, to_dev

pytestmark = pytest.mark.gpu


def _verts(res, h, shear):
    nd = len(res)
    axes = [np.arange(r + 1) * hh for r, hh in zip(res, h)]
    if nd == 2:
        Y, X = np.meshgrid(axes[1], axes[0], indexing="ij")
        return np.stack([X + shear[0] * Y, Y], axis=-1)
    Z, Y, X = np.meshgrid(axes[2], axes[1], axes[0], indexing="ij")
    return np.stack([X + shear[0] * Y + shear[1] * Z, Y + shear[2] * Z, Z], axis=-1)


def _case(res, h, shear, periodic=(), seed=0, nu=0.05, dt=0.02, source=True):
    """One sheared block: periodic axes joined to themselves, Dirichlet values
    (seeded) on the other sides; seeded u0, p0 and source."""
    nd = len(res)
    rng = np.random.default_rng(seed)
    r3 = tuple(res) + ((1,) if nd == 2 else ())
    blk = types.SimpleNamespace(res=r3, vertices=_verts(res, h, shear))
    conns, dirichlet = [], []
    for ax in range(nd):
        if ax in periodic:
            conns.append((0, 2 * ax, 0, 2 * ax + 1))
            continue
        nf = int(np.prod([r3[a] for a in range(3) if a != ax]))
        for s in (2 * ax, 2 * ax + 1):
            dirichlet.append((0, s, 0.5 * rng.standard_normal((nf, nd))))
    N = int(np.prod(r3))
    return types.SimpleNamespace(ndim=nd, blocks=[blk], connections=conns, dirichlet=dirichlet, outflow=[],
                                 ncells=N, u0=rng.standard_normal((nd, N)), p0=rng.standard_normal(N),
                                 S=rng.standard_normal((nd, N)) if source else None, nu=nu, dt=dt)


def _parity(c, n_no, precision="fp64", tol=FP64_REL, **opts):
    m = O.mesh_from_case(c, allow_nonorthogonal=True)
    assert m.has_cross
    dom = gpu_domain(c, precision, n_nonortho=n_no, **opts)
    ug, pg, st = gpu_step(dom, c, c.u0, c.p0, c.S)
    assert st["status"] == "PISO_OK", st
    uo, po, _ = O.piso_step(m, c.u0, c.p0, c.dt, c.nu, c.S, None, OP.Options(n_nonortho=n_no))
    assert rel_err(ug, uo) <= tol, rel_err(ug, uo)
    assert rel_err(pg, po) <= 10 * tol, rel_err(pg, po)
    return st


@pytest.mark.parametrize("n_no", [1, 3])
def test_sheared_2d_walls(n_no):
    _parity(_case((12, 10), (0.1, 0.1), (0.6,)), n_no)


def test_sheared_2d_periodic_x():
    _parity(_case((16, 10), (0.1, 0.1), (0.5,), periodic=(0,), seed=1), 2)


@pytest.mark.parametrize("n_no", [1, 2])
def test_sheared_3d(n_no):
    _parity(_case((7, 8, 6), (0.1, 0.12, 0.09), (0.5, -0.3, 0.4), periodic=(2,), seed=2), n_no)


@pytest.mark.parametrize("ctas,threads", [(1, 256), (3, 256), (5, 768)])
def test_sheared_cta_splits(ctas, threads):
    """Neighbours of neighbours cross CTA ranges (contiguous or interleaved)."""
    _parity(_case((24, 20), (0.05, 0.05), (0.7,), periodic=(0,), seed=3), 2, ctas=ctas, block_threads=threads)


def test_sheared_fp32():
    _parity(_case((12, 10), (0.1, 0.1), (0.6,), seed=4), 2, "fp32", tol=FP32_REL, adv_rtol=1e-7, p_rtol=1e-7)


def test_sheared_with_ilu_and_line_preconditioners():
    c = _case((12, 10), (0.1, 0.1), (0.6,), seed=5)
    st = _parity(c, 2, adv_precond=capi.PISO_ADV_PRECOND_ILU, p_precond=capi.PISO_PRECOND_LINE)
    assert st["adv_precond_used"] == 1


def test_taylor_green_sheared_periodic_box():
    """The 45-degree sheared doubly periodic box of the oracle's Taylor-Green
    pin: one step on the GPU equals the oracle's."""
    n = 32
    h = 2 * math.pi / n
    c = _case((n, n), (h, h), (1.0,), periodic=(0, 1), seed=6, nu=0.1, dt=0.0125, source=False)
    _parity(c, 2)


def test_nonorthogonal_refusals():
    c = _case((8, 6), (0.1, 0.1), (0.6,), seed=7)
    with pytest.raises(capi.PisoError):
        gpu_domain(c)                                   # n_nonortho = 0 (default): rejected
    with pytest.raises(capi.PisoError):
        gpu_domain(c, n_nonortho=1, pred_grad_p=1)
    with pytest.raises(capi.PisoError):
        gpu_domain(c, n_nonortho=5)                     # the step record holds up to 4 iterates


def test_batch_with_nonorthogonal_members():
    """A batch holding sheared, curved and orthogonal members (each with its own
    n_nonortho) in one launch: every member's forward and adjoint equal the
    oracle's."""
    from paper_2505_16992_b300 import workloads as W
    cases = [(_case((12, 10), (0.1, 0.1), (0.6,), seed=20), 1), (_wavy(seed=21), 2),
             (W.cavity2d(16), 0), (_case((16, 10), (0.1, 0.1), (0.5,), periodic=(0,), seed=22), 3)]
    doms = [gpu_domain(c, n_nonortho=n) for c, n in cases]
    b = Batch(doms, capi.default_options(adv_rtol=1e-13, p_rtol=1e-13))
    rng = np.random.default_rng(23)
    us = [to_dev(d, c.u0, 2) for d, (c, _) in zip(doms, cases)]
    ps = [to_dev(d, c.p0, None) for d, (c, _) in zip(doms, cases)]
    Ss = [None if c.S is None else to_dev(d, c.S, 2) for d, (c, _) in zip(doms, cases)]
    uo, po, sts = b.step(us, ps, [c.dt for c, _ in cases], [c.nu for c, _ in cases], Ss)
    assert all(st["status"] == "PISO_OK" for st in sts), sts
    gus = [rng.standard_normal((2, c.ncells)) for c, _ in cases]
    du, dp, dS, dnu, asts = b.step_adjoint([to_dev(d, g, 2) for d, g in zip(doms, gus)])
    assert all(st["status"] == "PISO_OK" for st in asts), asts
    for i, ((c, n), d) in enumerate(zip(cases, doms)):
        m = O.mesh_from_case(c, allow_nonorthogonal=True)
        o = OP.Options(n_nonortho=max(n, 1))
        u1, p1, tape = O.piso_step(m, c.u0, c.p0, c.dt, c.nu, c.S, None, o)
        assert rel_err(host(uo[i]), u1) <= FP64_REL, (i, rel_err(host(uo[i]), u1))
        assert rel_err(host(po[i]), p1) <= 10 * FP64_REL, i
        gu, gp, gS, gnu = O.piso_step_adjoint(m, tape, gus[i], np.zeros(c.ncells), o)
        assert rel_err(host(du[i]), gu) <= ADJ_REL, (i, rel_err(host(du[i]), gu))
        assert abs(dnu[i] - gnu) <= ADJ_REL * abs(gnu), i
        if n:
            assert rel_err(host(dp[i]), gp) <= ADJ_REL, (i, rel_err(host(dp[i]), gp))


def _wavy(n=(12, 10), periodic_y=False, seed=8, nu=0.05, dt=0.02):
    """A curved block: x = xi + a sin(eta), y = eta + a sin(xi) on a 2 pi box,
    periodic in x (and in y when asked; walls otherwise): alpha_jk varies from
    cell to cell, so the direct-neighbour cross entries of C do not cancel."""
    L = 2 * math.pi
    xi = np.arange(n[0] + 1) * L / n[0]
    eta = np.arange(n[1] + 1) * L / n[1]
    E, X = np.meshgrid(eta, xi, indexing="ij")
    V = np.stack([X + 0.3 * np.sin(E), E + 0.3 * np.sin(X)], axis=-1)
    c = _case(n, (1.0, 1.0), (0.0,), periodic=(0, 1) if periodic_y else (0,), seed=seed, nu=nu, dt=dt)
    c.blocks[0].vertices = V
    return c


@pytest.mark.parametrize("periodic_y", [False, True])
def test_wavy_block_forward(periodic_y):
    _parity(_wavy(periodic_y=periodic_y), 2)


# ---------------------------------------------------------------------------
# the adjoint of the non-orthogonal step (App. A.4 with App. A.2)
# ---------------------------------------------------------------------------

ADJ_REL = 1e-8


def _adj_parity(c, n_no, precision="fp64", tol=ADJ_REL, grad_paths=3, seed=0, **opts):
    """Forward + adjoint on the GPU and in the oracle from the same state:
    dL/du^n, dL/dp^n (which the pressure cross terms make non-zero), dL/dS,
    dL/dnu and dL/d(boundary values) for seeded dL/du^{n+1}, dL/dp^{n+1}."""
    m = O.mesh_from_case(c, allow_nonorthogonal=True)
    dom = gpu_domain(c, precision, n_nonortho=n_no, grad_paths=grad_paths, **opts)
    d, N = c.ndim, c.ncells
    rng = np.random.default_rng(seed)
    ubar, pbar = rng.standard_normal((d, N)), rng.standard_normal(N)
    S = c.S
    u1, p1, st = dom.step(to_dev(dom, c.u0, d), to_dev(dom, c.p0), c.dt, c.nu,
                          None if S is None else to_dev(dom, S, d))
    assert st["status"] == "PISO_OK", st
    oo = OP.Options(n_nonortho=n_no)
    _, _, tape = O.piso_step(m, c.u0, c.p0, c.dt, c.nu, S, None, oo)
    du, dp, dS, dnu, ast = dom.step_adjoint(to_dev(dom, ubar, d), to_dev(dom, pbar))
    assert ast["status"] == "PISO_OK", ast
    oa = OP.Options(n_nonortho=n_no, grad_adv=bool(grad_paths & 1), grad_p=bool(grad_paths & 2))
    gu, gp, gS, gnu, gbv = O.piso_step_adjoint(m, tape, ubar, pbar, oa, want_bval=True)
    assert (sum(ast["adv_iters"]) > 0) == bool(grad_paths & 1), ast
    assert (sum(ast["p_iters"]) > 0) == bool(grad_paths & 2), ast
    errs = dict(u=rel_err(host(du), gu), S=rel_err(host(dS), gS), nu=abs(dnu - gnu) / max(abs(gnu), 1e-300))
    if grad_paths & 2:
        errs["p"] = rel_err(host(dp), gp)
    else:
        assert np.all(host(dp) == 0.0)
    if np.any(m.is_bface):
        errs["bval"] = rel_err(dom.boundary_adjoint(), bval_faces(m, gbv))
    for k, v in errs.items():
        assert v <= tol, (k, errs, ast)
    return errs


@pytest.mark.parametrize("n_no", [1, 2, 3])
def test_adjoint_sheared_2d_walls(n_no):
    _adj_parity(_case((12, 10), (0.1, 0.1), (0.6,)), n_no)


def test_adjoint_sheared_2d_periodic_x():
    _adj_parity(_case((16, 10), (0.1, 0.1), (0.5,), periodic=(0,), seed=1), 2)


@pytest.mark.parametrize("n_no", [1, 2])
def test_adjoint_sheared_3d(n_no):
    _adj_parity(_case((7, 8, 6), (0.1, 0.12, 0.09), (0.5, -0.3, 0.4), periodic=(2,), seed=2), n_no)


@pytest.mark.parametrize("periodic_y", [False, True])
def test_adjoint_wavy_block(periodic_y):
    _adj_parity(_wavy(periodic_y=periodic_y), 2)


@pytest.mark.parametrize("ctas,threads", [(1, 256), (3, 256), (5, 768)])
def test_adjoint_sheared_cta_splits(ctas, threads):
    _adj_parity(_case((24, 20), (0.05, 0.05), (0.7,), periodic=(0,), seed=3), 2, ctas=ctas, block_threads=threads)


@pytest.mark.parametrize("paths", [0, capi.PISO_GRAD_ADV, capi.PISO_GRAD_P])
def test_adjoint_nonorthogonal_gradient_paths(paths):
    _adj_parity(_case((12, 10), (0.1, 0.1), (0.6,), seed=9), 2, grad_paths=paths)


def test_adjoint_nonorthogonal_with_ilu_and_line_preconditioners():
    _adj_parity(_case((12, 10), (0.1, 0.1), (0.6,), seed=5), 2, adv_precond=capi.PISO_ADV_PRECOND_ILU,
                p_precond=capi.PISO_PRECOND_LINE)


def test_adjoint_nonorthogonal_fp32():
    _adj_parity(_case((12, 10), (0.1, 0.1), (0.6,), seed=4), 2, "fp32", tol=2e-3, adv_rtol=1e-7, p_rtol=1e-7)


def test_adjoint_sheared_multiblock_step_with_outflow():
    """Cross terms across block connections and the advective outflow update
    (Eq. advOut) differentiated together."""
    from paper_2505_16992_b300 import workloads as W
    c = W.bfs2d(n_in=(8, 4), n_ch=16, n_out=8, half=4, dt=0.02)
    for b in c.blocks:
        b.vertices[..., 0] += 0.3 * b.vertices[..., 1]
    _adj_parity(c, 2, p_rtol=1e-12)


def test_adjoint_sheared_channel_matches_gpu_finite_difference():
    """GPU alone: <ubar, u^{n+1}> + <pbar, p^{n+1}> along directions in u^n and
    p^n equals the adjoint's directional derivatives (4th-order central
    differences of the GPU forward) on the forced channel with slanted cells."""
    from paper_2505_16992_b300 import workloads as W
    import torch
    c = W.channel3d(10, 8, 6, shear=0.5)
    dom = gpu_domain(c, n_nonortho=2)
    d, N = c.ndim, c.ncells
    rng = np.random.default_rng(11)
    u0, p0, S0 = to_dev(dom, c.u0, d), to_dev(dom, rng.standard_normal(N)), to_dev(dom, c.S, d)
    ubar, pbar = to_dev(dom, rng.standard_normal((d, N)), d), to_dev(dom, rng.standard_normal(N))
    du_dir, dp_dir = to_dev(dom, rng.standard_normal((d, N)), d), to_dev(dom, rng.standard_normal(N))

    def L(t):
        u1, p1, _ = dom.step(u0 + t * du_dir, p0 + t * dp_dir, c.dt, c.nu, S0)
        return float((ubar * u1).sum() + (pbar * p1).sum())

    dom.step(u0, p0, c.dt, c.nu, S0)
    gu, gp, _, _, _ = dom.step_adjoint(ubar, pbar)
    adj = float((gu * du_dir).sum() + (gp * dp_dir).sum())
    e = 1e-4
    fd = (8 * (L(e) - L(-e)) - (L(2 * e) - L(-2 * e))) / (12 * e)
    assert abs(adj - fd) <= 1e-6 * abs(fd), (adj, fd)


def test_sheared_channel_fp32_after_n_steps():
    """The forced channel with slanted cells (the bench's non-orthogonal
    workload at a small size): FP32 against the FP64 oracle after 10 steps."""
    from paper_2505_16992_b300 import workloads as W
    c = W.channel3d(12, 10, 6, shear=0.5)
    m = O.mesh_from_case(c, allow_nonorthogonal=True)
    assert m.has_cross
    dom = gpu_domain(c, "fp32", n_nonortho=1, adv_rtol=1e-6, p_rtol=1e-6)
    u, p, S = to_dev(dom, c.u0, 3), to_dev(dom, c.p0), to_dev(dom, c.S, 3)
    for _ in range(10):
        u, p, st = dom.step(u, p, c.dt, c.nu, S)
        assert st["status"] == "PISO_OK", st
    uo, po, _ = O.rollout(m, c.u0, c.p0, c.dt, c.nu, c.S, 10, OP.Options(n_nonortho=1))
    assert rel_err(host(u), uo) <= FP32_REL, rel_err(host(u), uo)


def test_sheared_multiblock_step_with_outflow():
    """The 5-block backward-facing step under one affine shear x += 0.3 y (the
    blocks stay conformal): cross terms across block connections (neighbours
    of neighbours in other blocks) and at the advective-outflow faces."""
    from paper_2505_16992_b300 import workloads as W
    c = W.bfs2d(n_in=(8, 4), n_ch=16, n_out=8, half=4, dt=0.02)
    for b in c.blocks:
        b.vertices[..., 0] += 0.3 * b.vertices[..., 1]
    m = O.mesh_from_case(c, allow_nonorthogonal=True)
    assert m.has_cross and m.has_outflow
    dom = gpu_domain(c, n_nonortho=2, p_rtol=1e-12)
    ug, pg, st = gpu_step(dom, c, c.u0, c.p0, c.S)
    assert st["status"] == "PISO_OK", st
    uo, po, _ = O.piso_step(m, c.u0, c.p0, c.dt, c.nu, c.S, None, OP.Options(n_nonortho=2))
    assert rel_err(ug, uo) <= FP64_REL, rel_err(ug, uo)
    assert rel_err(pg, po) <= 10 * FP64_REL, rel_err(pg, po)
