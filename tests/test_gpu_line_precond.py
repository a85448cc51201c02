"""Pressure CG with the y-line preconditioner vs Jacobi, both against the FP64
oracle (element-wise parity through the C ABI).  The preconditioner changes
how the pressure systems of App. A.1 (Eq. pressure) are solved, not their
solutions, so both must reproduce the oracle's direct solves; the line form
must also need fewer iterations on wall-refined grids."""
import numpy as np
import pytest

import oracle as O
from paper_2505_16992_b300 import capi
from paper_2505_16992_b300 import workloads as W
from gpu_util import FP32_REL, FP64_REL, gpu_domain, gpu_step, host, oracle_step, rel_err, to_dev

pytestmark = pytest.mark.gpu

LINE, JACOBI = capi.PISO_PRECOND_LINE, capi.PISO_PRECOND_JACOBI


def _step_parity(case, precond, precision="fp64", tol=FP64_REL, **opts):
    m = O.mesh_from_case(case)
    dom = gpu_domain(case, precision, p_precond=precond, **opts)
    ug, pg, st = gpu_step(dom, case, case.u0, case.p0, case.S)
    assert st["status"] == "PISO_OK", st
    uo, po, tape = oracle_step(m, case, case.u0, case.p0, case.S)
    assert rel_err(ug, uo) <= tol, rel_err(ug, uo)
    assert rel_err(pg, po) <= 10 * tol, rel_err(pg, po)
    return st


def _ragged_channel():
    c = W.channel3d(13, 7, 5)
    return c


@pytest.mark.parametrize("make", [
    lambda: W.channel3d(16, 12, 8),
    _ragged_channel,
    lambda: W.cavity2d(33),
    lambda: W.cavity3d(5, nz=3),
    lambda: W.turbulence2d(64),
], ids=["channel3d-16x12x8", "channel3d-13x7x5", "cavity2d-33", "cavity3d-5x5x3", "periodic2d-64"])
@pytest.mark.parametrize("precond", [LINE, JACOBI], ids=["line", "jacobi"])
def test_forced_preconditioner_parity(make, precond):
    _step_parity(make(), precond)


def test_line_multiblock_bfs_with_outflow():
    """Lines stop at block sides (the step's upper/lower channel blocks are
    joined in y): the preconditioner drops those couplings, the solve does not."""
    c = W.bfs2d(n_in=(16, 8), n_ch=64, n_out=16, half=8, dt=0.02)
    _step_parity(c, LINE, p_rtol=1e-12)


def test_line_full_size_channel_fewer_iterations():
    """The 64x48x32 channel (tanh walls): parity with the oracle and
    fewer CG iterations than Jacobi for the same tolerance."""
    c = W.channel3d()
    st_l = _step_parity(c, LINE)
    st_j = _step_parity(c, JACOBI)
    for k in range(2):
        assert st_l["p_iters"][k] < 0.6 * st_j["p_iters"][k], (st_l["p_iters"], st_j["p_iters"])


def test_auto_picks_line_on_wall_refined_grids_only():
    c = W.channel3d(16, 12, 8)
    d_auto = gpu_domain(c, p_precond=capi.PISO_PRECOND_AUTO)
    d_line = gpu_domain(c, p_precond=LINE)
    assert d_auto.uses_line_precond() and d_line.uses_line_precond()
    a = gpu_step(d_auto, c, c.u0, c.p0, c.S)
    b = gpu_step(d_line, c, c.u0, c.p0, c.S)
    assert a[2]["p_iters"] == b[2]["p_iters"]
    cav = W.cavity2d(32)
    assert not gpu_domain(cav, p_precond=capi.PISO_PRECOND_AUTO).uses_line_precond()
    e = gpu_step(gpu_domain(cav, p_precond=capi.PISO_PRECOND_AUTO), cav, cav.u0, cav.p0)
    f = gpu_step(gpu_domain(cav, p_precond=JACOBI), cav, cav.u0, cav.p0)
    assert e[2]["p_iters"] == f[2]["p_iters"]


@pytest.mark.parametrize("ctas", [1, 3, 7])
def test_line_batches_and_cta_splits(ctas):
    """Few CTAs own many lines each: the lines are staged in several batches
    (1024 lines at most, bounded by shared memory), and a CTA's cell range no
    longer fits the shared neighbour table."""
    c = W.channel3d(32, 24, 32)
    _step_parity(c, LINE, ctas=ctas, block_threads=256)


def test_line_fp32_mixed_precision():
    c = W.channel3d(16, 12, 8)
    _step_parity(c, LINE, "fp32", tol=FP32_REL, adv_rtol=1e-6, p_rtol=1e-6)


def test_line_fp32_refined():
    c = W.channel3d(16, 12, 8)
    st = _step_parity(c, LINE, "fp32", tol=2e-6, adv_rtol=1e-6, p_refine_rtol=1e-10, p_inner_rtol=1e-4)
    assert min(st["p_rounds"][:2]) >= 1


def test_line_bitwise_deterministic():
    c = W.channel3d(16, 12, 8)
    dom = gpu_domain(c, p_precond=LINE)
    a = gpu_step(dom, c, c.u0, c.p0, c.S)
    b = gpu_step(dom, c, c.u0, c.p0, c.S)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


@pytest.mark.parametrize("make", [lambda: W.channel3d(16, 12, 8),
                                  lambda: W.bfs2d(n_in=(16, 8), n_ch=64, n_out=16, half=8, dt=0.02)],
                         ids=["channel3d", "bfs2d"])
def test_line_adjoint_matches_oracle(make):
    """The transposed pressure solves of the adjoint (P is symmetric) run the
    same line-preconditioned CG, with the factors rebuilt from the tape."""
    c = make()
    m = O.mesh_from_case(c)
    dom = gpu_domain(c, p_precond=LINE, p_rtol=1e-13 if c.ndim == 3 else 1e-12)
    rng = np.random.default_rng(11)
    gu = rng.standard_normal((c.ndim, c.ncells))
    gp = rng.standard_normal(c.ncells)
    d = c.ndim
    S = None if c.S is None else to_dev(dom, c.S, d)
    dom.step(to_dev(dom, c.u0, d), to_dev(dom, c.p0), c.dt, c.nu, S)
    du, dp, dS, dnu, st = dom.step_adjoint(to_dev(dom, gu, d), to_dev(dom, gp))
    assert st["status"] == "PISO_OK", st
    _, _, tape = oracle_step(m, c, c.u0, c.p0, c.S)
    ou, op, oS, onu = O.piso_step_adjoint(m, tape, gu, gp)
    assert rel_err(host(du), ou) <= 1e-8
    if dS is not None:
        assert rel_err(host(dS), oS) <= 1e-8
    assert abs(dnu - onu) <= 1e-8 * max(abs(onu), 1e-30) + 1e-12
