"""Non-orthogonal meshes on the GPU (App. A.2 "Non-Orthogonal Grids": the
cross derivatives of the viscous term and of the pressure operator, deferred
to the right-hand sides with the previous iterate over n_nonortho corrector
steps) against the FP64 oracle, element by element through the C ABI, on
sheared 2D and 3D blocks with Dirichlet sides and on a sheared periodic box."""
import math
import types

import numpy as np
import pytest

import oracle as O
from oracle import piso as OP
from paper_2505_16992_b300 import capi
from paper_2505_16992_b300.solver import Batch
from gpu_util import FP32_REL, FP64_REL, gpu_domain, gpu_step, host, rel_err, to_dev

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
    dom = gpu_domain(c, n_nonortho=1)
    dom.step(to_dev(dom, c.u0, 2), to_dev(dom, c.p0), c.dt, c.nu, to_dev(dom, c.S, 2))
    with pytest.raises(capi.PisoError) as e:
        dom.step_adjoint(to_dev(dom, np.ones((2, c.ncells)), 2), to_dev(dom, np.zeros(c.ncells)))
    assert e.value.status == 7
    with pytest.raises(capi.PisoError):
        Batch([dom])


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
