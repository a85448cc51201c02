"""Degenerate meshes against the FP64 oracle, through the C ABI: a single
cell, 2x2 and 2x2x2 boxes, one-cell-thick periodic directions, a column one
cell wide, a 2x2 periodic box whose pressure vanishes; forward and adjoint
step (Sec. 2.3, 2.4; App. A.1, A.4), narrowest CTAs (32 and 64 threads), one
and two CTAs, FP64 and FP32; and a block with no cells refused at creation."""
import numpy as np
import pytest

import oracle as O
from paper_2505_16992_b300 import capi
from paper_2505_16992_b300 import workloads as W
from gpu_util import FP32_REL, FP64_REL, bval_faces, gpu_domain, host, rel_err, to_dev

pytestmark = pytest.mark.gpu

CASES = {
    "cavity_1x1": lambda: W.cavity2d(1),
    "cavity_2x2": lambda: W.cavity2d(2),
    "channel_4x3x1": lambda: W.channel3d(4, 3, 1),
    "channel_1x5x1": lambda: W.channel3d(1, 5, 1),
    "cavity3d_2x2x2": lambda: W.cavity3d(2),
    "poiseuille_1x4": lambda: W.channel2d(1, 4),
    "taylor_green_2x2": lambda: W.taylor_green2d(2),
    "cavity3d_3x3x1_periodic_z": lambda: W.cavity3d(3, periodic_z=True, nz=1),
}


def _err(a, b, scale):
    """relative error, or absolute against `scale` where the oracle's field is
    zero (the single cell's and the 2x2 periodic box's pressure)"""
    return rel_err(a, b) if np.abs(b).max() > 0 else float(np.abs(a).max() / scale)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("threads", [32, 64])
@pytest.mark.parametrize("name", sorted(CASES))
def test_degenerate_mesh_against_oracle(name, threads, precision):
    c = CASES[name]()
    m = O.mesh_from_case(c)
    d, N = c.ndim, c.ncells
    rng = np.random.default_rng(sorted(CASES).index(name))
    u0 = c.u0 + 0.2 * rng.standard_normal((d, N))
    S0 = (c.S if c.S is not None else 0.0) + 0.1 * rng.standard_normal((d, N))
    fp32 = precision == "fp32"
    rt = 1e-7 if fp32 else 1e-12
    # two CTAs only where each holds several cells and the Jacobi CG runs
    for ctas, pc in ((1, capi.PISO_PRECOND_AUTO), (2 if N >= 8 else 1, capi.PISO_PRECOND_JACOBI)):
        dom = gpu_domain(c, precision, block_threads=threads, ctas=ctas, p_precond=pc, adv_rtol=rt, p_rtol=rt)
        u1, p1, st = dom.step(to_dev(dom, u0, d), to_dev(dom, c.p0), c.dt, c.nu, to_dev(dom, S0, d))
        assert st["status"] == "PISO_OK", (name, ctas, st)
        uo, po, tape = O.piso_step(m, u0, c.p0, c.dt, c.nu, S0)
        tol = FP32_REL if fp32 else FP64_REL
        us = max(np.abs(uo).max(), 1e-300)
        assert rel_err(host(u1), uo) <= tol, (name, ctas, rel_err(host(u1), uo))
        assert _err(host(p1), po, us) <= 10 * tol, (name, ctas, _err(host(p1), po, us))
        ubar, pbar = rng.standard_normal((d, N)), rng.standard_normal(N)
        du, dp, dS, dnu, ast = dom.step_adjoint(to_dev(dom, ubar, d), to_dev(dom, pbar))
        assert ast["status"] == "PISO_OK", (name, ctas, ast)
        gu, gp, gS, gnu, gbv = O.piso_step_adjoint(m, tape, ubar, pbar, want_bval=True)
        atol = 2e-3 if fp32 else 1e-8
        assert rel_err(host(du), gu) <= atol, (name, ctas, rel_err(host(du), gu))
        assert rel_err(host(dS), gS) <= atol, (name, ctas, rel_err(host(dS), gS))
        assert abs(dnu - gnu) <= (1e-2 if fp32 else 1e-8) * max(abs(gnu), 1e-3), (name, ctas, dnu, gnu)
        if np.any(m.is_bface):
            assert rel_err(dom.boundary_adjoint(), bval_faces(m, gbv)) <= atol, name


def test_block_without_cells_is_refused():
    """A block of zero cells along an axis is an argument error at block
    creation, not a launch."""
    import ctypes as C
    lib = capi.load()
    h = C.c_void_p()
    capi.check(lib.piso_domain_create(2, capi.PISO_FP64, C.byref(h)))
    einval = {v: k for k, v in capi.STATUS.items()}["PISO_EINVAL"]
    try:
        verts = (C.c_double * 64)()
        for res in ((0, 4, 1), (4, 0, 1), (3, 3, 2)):   # an empty axis; a 2D block with nz != 1
            assert lib.piso_block_add(h, (C.c_int32 * 3)(*res), verts, None) == einval, res
    finally:
        lib.piso_domain_destroy(h)
