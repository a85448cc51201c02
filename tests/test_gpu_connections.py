"""Block joints with exchanged or reversed axes on the GPU (Sec. 2.2, App. A.3;
the cuts of App. B's O-/C-grids): forward and adjoint steps against the FP64
oracle through the C ABI, on blocks with turned index frames (2D: 90, 180,
270 degrees; 3D: a turn that exchanges the joint's tangential axes), on
orthogonal and slanted cells, and on a C-grid whose cut is a side folded
onto itself."""
import numpy as np
import pytest

import oracle as O
from oracle import piso as OP
from paper_2505_16992_b300 import capi
from paper_2505_16992_b300 import workloads as W
from paper_2505_16992_b300.solver import Batch
from gpu_util import FP32_REL, FP64_REL, bval_faces, gpu_domain, host, rel_err, to_dev

pytestmark = pytest.mark.gpu

ADJ_REL = 1e-8


def _parity(c, precision="fp64", tol=FP64_REL, adj_tol=ADJ_REL, n_no=2, seed=0, **opts):
    m = O.mesh_from_case(c, allow_nonorthogonal=True)
    assert m.twisted
    n_use = n_no if m.has_cross else 0
    dom = gpu_domain(c, precision, n_nonortho=n_use, **opts)
    d, N = c.ndim, c.ncells
    S = None if c.S is None else to_dev(dom, c.S, d)
    u1, p1, st = dom.step(to_dev(dom, c.u0, d), to_dev(dom, c.p0), c.dt, c.nu, S)
    assert st["status"] == "PISO_OK", st
    oo = OP.Options(n_nonortho=max(n_use, 1))
    uo, po, tape = O.piso_step(m, c.u0, c.p0, c.dt, c.nu, c.S, None, oo)
    assert rel_err(host(u1), uo) <= tol, rel_err(host(u1), uo)
    assert rel_err(host(p1), po) <= 10 * tol, rel_err(host(p1), po)
    rng = np.random.default_rng(seed)
    ubar, pbar = rng.standard_normal((d, N)), rng.standard_normal(N)
    du, dp, dS, dnu, ast = dom.step_adjoint(to_dev(dom, ubar, d), to_dev(dom, pbar))
    assert ast["status"] == "PISO_OK", ast
    gu, gp, gS, gnu, gbv = O.piso_step_adjoint(m, tape, ubar, pbar, oo, want_bval=True)
    errs = dict(u=rel_err(host(du), gu), S=rel_err(host(dS), gS), nu=abs(dnu - gnu) / abs(gnu),
                bval=rel_err(dom.boundary_adjoint(), bval_faces(m, gbv)))
    if m.has_cross:
        errs["p"] = rel_err(host(dp), gp)
    for k, v in errs.items():
        assert v <= adj_tol, (k, errs)
    return st


@pytest.mark.parametrize("shear", [0.0, 0.4])
@pytest.mark.parametrize("rot", [1, 2, 3])
def test_turned_block_2d(rot, shear):
    _parity(W.two_block_cavity2d(8, 6, rot=rot, shear=shear)[0])


@pytest.mark.parametrize("shear", [0.0, 0.4])
def test_turned_block_3d_exchanged_axes(shear):
    _parity(W.two_block_channel3d(turned=True, shear=shear)[0])


def test_cgrid_folded_cut():
    _parity(W.slit_cgrid2d(16, 8))


def test_turned_block_matches_plain_layout_on_the_gpu():
    """GPU alone: the turned layout reproduces the plain layout's step."""
    c, idx = W.two_block_cavity2d(10, 8, rot=3, shear=0.3)
    c0, _ = W.two_block_cavity2d(10, 8, rot=0, shear=0.3)
    out = []
    for cc in (c, c0):
        dom = gpu_domain(cc, n_nonortho=2)
        u1, p1, st = dom.step(to_dev(dom, cc.u0, 2), to_dev(dom, cc.p0), cc.dt, cc.nu, to_dev(dom, cc.S, 2))
        assert st["status"] == "PISO_OK", st
        out.append((host(u1), host(p1)))
    assert rel_err(out[0][0], out[1][0][:, idx]) <= FP64_REL
    assert rel_err(out[0][1], out[1][1][idx]) <= 10 * FP64_REL


@pytest.mark.parametrize("ctas,threads", [(1, 256), (3, 256), (5, 768)])
def test_joints_across_cta_splits(ctas, threads):
    _parity(W.slit_cgrid2d(24, 12), ctas=ctas, block_threads=threads)


def test_joints_fp32():
    _parity(W.two_block_cavity2d(12, 8, rot=2, shear=0.4)[0], "fp32", tol=FP32_REL, adj_tol=2e-3,
            adv_rtol=1e-7, p_rtol=1e-7)


def test_joints_with_ilu_predictor():
    st = _parity(W.two_block_channel3d(turned=True, shear=0.4)[0], adv_precond=capi.PISO_ADV_PRECOND_ILU)
    assert st["adv_precond_used"] == 1


def test_joints_use_jacobi_pressure_preconditioner():
    """The y-line factors read the plain face layout, so domains with such
    joints run the Jacobi-preconditioned CG even when the line form is asked
    for."""
    c = W.two_block_channel3d(turned=True)[0]
    dom = gpu_domain(c, p_precond=capi.PISO_PRECOND_LINE)
    assert not dom.uses_line_precond()


def test_batch_with_turned_members():
    cases = [W.two_block_cavity2d(8, 6, rot=1)[0], W.slit_cgrid2d(12, 6), W.cavity2d(12)]
    doms = [gpu_domain(c, n_nonortho=2 if i == 1 else 0) for i, c in enumerate(cases)]
    b = Batch(doms, capi.default_options(adv_rtol=1e-13, p_rtol=1e-13))
    us = [to_dev(d, c.u0, 2) for d, c in zip(doms, cases)]
    ps = [to_dev(d, c.p0) for d, c in zip(doms, cases)]
    Ss = [None if c.S is None else to_dev(d, c.S, 2) for d, c in zip(doms, cases)]
    uo, po, sts = b.step(us, ps, [c.dt for c in cases], [c.nu for c in cases], Ss)
    assert all(st["status"] == "PISO_OK" for st in sts), sts
    for i, c in enumerate(cases):
        m = O.mesh_from_case(c, allow_nonorthogonal=True)
        u1, p1, _ = O.piso_step(m, c.u0, c.p0, c.dt, c.nu, c.S, None, OP.Options(n_nonortho=2))
        assert rel_err(host(uo[i]), u1) <= FP64_REL, (i, rel_err(host(uo[i]), u1))
