"""ILU(0)-preconditioned BiCGStab on the GPU (App. A.5: incomplete-LU
preconditioning of the advection-diffusion solve, throughout or only after the
plain solve failed) against the FP64 oracle, element by element through the C
ABI.  The preconditioner changes how the predictor systems are solved, not
their solutions: the steps must match the oracle's direct solves.  With one
CTA the GPU factors the whole matrix, so its iteration counts must also match
the oracle's ILU(0)-preconditioned BiCGStab on the same system."""
import numpy as np
import pytest

import oracle as O
from oracle import piso as OP
from paper_2505_16992_b300 import capi
from paper_2505_16992_b300 import workloads as W
from paper_2505_16992_b300.solver import Batch
from gpu_util import FP32_REL, FP64_REL, gpu_domain, gpu_step, host, oracle_step, rel_err, to_dev

pytestmark = pytest.mark.gpu

ILU, ON_FAIL, NONE = capi.PISO_ADV_PRECOND_ILU, capi.PISO_ADV_PRECOND_ILU_ON_FAILURE, capi.PISO_ADV_PRECOND_NONE


def _stretched():
    """Wall-refined channel with a large time step: cell sizes vary strongly
    and the unpreconditioned BiCGStab needs ~140 iterations."""
    return W.channel3d(10, 16, 4, gamma=3.0, dt=0.5)


def _parity(case, precision="fp64", tol=FP64_REL, **opts):
    m = O.mesh_from_case(case)
    dom = gpu_domain(case, precision, **opts)
    ug, pg, st = gpu_step(dom, case, case.u0, case.p0, case.S)
    assert st["status"] == "PISO_OK", st
    uo, po, _ = oracle_step(m, case, case.u0, case.p0, case.S)
    assert rel_err(ug, uo) <= tol, rel_err(ug, uo)
    assert rel_err(pg, po) <= 10 * tol, rel_err(pg, po)
    return st


@pytest.mark.parametrize("make", [
    _stretched,
    lambda: W.channel3d(16, 12, 8),
    lambda: W.channel3d(13, 7, 5),
    lambda: W.cavity2d(33),
    lambda: W.bfs2d(n_in=(16, 8), n_ch=64, n_out=16, half=8, dt=0.02),
    lambda: W.turbulence2d(64),
], ids=["channel3d-stretched", "channel3d-16x12x8", "channel3d-13x7x5", "cavity2d-33", "bfs2d", "periodic2d-64"])
def test_ilu_step_parity(make):
    st = _parity(make(), adv_precond=ILU)
    assert st["adv_precond_used"] == 1


@pytest.mark.parametrize("nz", [2, 1])
def test_ilu_periodic_direction_of_one_or_two_cells(nz):
    """Two cells in a periodic direction: both sides of a cell face the same
    neighbour (the matrix entry is the sum of the two faces); one cell: the
    cell is its own neighbour.  The block factors stay a valid preconditioner
    (not exactly ILU(0) with two cells, where the neighbour graph has a
    2-cycle), so the solution still matches the oracle's."""
    st = _parity(W.channel3d(8, 10, nz, gamma=3.0, dt=0.5), adv_precond=ILU)
    assert st["adv_precond_used"] == 1 and max(st["adv_iters"]) < 30


def test_ilu_cuts_iterations_on_the_stretched_channel():
    c = _stretched()
    plain = _parity(c)
    ilu = _parity(c, adv_precond=ILU)
    assert plain["adv_precond_used"] == 0
    assert max(ilu["adv_iters"]) * 3 < min(plain["adv_iters"]), (ilu["adv_iters"], plain["adv_iters"])


@pytest.mark.parametrize("ctas,threads", [(1, 256), (3, 256), (7, 256), (0, 512)])
def test_ilu_cta_blocks_and_ownership(ctas, threads):
    """Contiguous CTA ranges (neighbour table in shared memory) and
    round-robin chunks (the table does not fit: one CTA, or three CTAs on this
    24,576-cell grid) give different blocks, never a different solution."""
    c = W.channel3d(32, 24, 32, gamma=3.0, dt=0.2)
    _parity(c, adv_precond=ILU, ctas=ctas, block_threads=threads)


@pytest.mark.parametrize("threads", [256, 768], ids=["global-sweep", "shared-sweep"])
def test_one_cta_iterations_match_the_oracle_ilu0(threads):
    """One CTA: the block is the whole matrix, so the GPU runs ILU(0) in cell
    order exactly as the oracle does; the iteration counts of the
    preconditioned BiCGStab agree (up to one, for rounding at the stopping
    test).  256 threads for 640 cells take the global-memory sweeps, 768 the
    shared-memory ones (one cell per thread).  The plain BiCGStab takes ~150
    irregular iterations here, over which the summation order of the dot
    products already moves the count by a few: it is only checked to be of the
    same size."""
    c = _stretched()
    m = O.mesh_from_case(c)
    _, _, tape = oracle_step(m, c, c.u0, c.p0, c.S)
    for pc, name in ((ILU, "ilu"), (NONE, "none")):
        st = _parity(c, adv_precond=pc, ctas=1, block_threads=threads)
        _, infos = OP.solve_C(m, tape["C"], tape["rhs"], c.u0,
                              OP.Options(solver="krylov", adv_rtol=1e-13, adv_precond=name))
        for k in range(3):
            want, got = infos[k].iters, st["adv_iters"][k]
            if name == "ilu":
                assert abs(got - want) <= 1, (name, st["adv_iters"], [i.iters for i in infos])
            else:
                assert 0.7 * want <= got <= 1.4 * want, (name, st["adv_iters"], [i.iters for i in infos])


def test_ilu_on_failure_restarts_preconditioned():
    c = _stretched()
    full = _parity(c, adv_precond=ILU)
    lim = max(full["adv_iters"]) + 4
    st = _parity(c, adv_precond=ON_FAIL, adv_maxit=lim)
    assert st["adv_precond_used"] == 2
    for k in range(3):
        assert lim < st["adv_iters"][k] <= 2 * lim
    # without the fallback the same limit fails, and it is reported
    dom = gpu_domain(c, adv_maxit=lim)
    with pytest.raises(capi.PisoError) as e:
        gpu_step(dom, c, c.u0, c.p0, c.S)
    assert e.value.status == 3
    # a plain solve that converges is kept: no fallback
    easy = W.channel3d(16, 12, 8)
    assert _parity(easy, adv_precond=ON_FAIL)["adv_precond_used"] == 0


def test_ilu_fp32():
    st = _parity(_stretched(), "fp32", tol=FP32_REL, adv_precond=ILU, adv_rtol=1e-6, p_rtol=1e-6)
    assert st["adv_precond_used"] == 1


@pytest.mark.parametrize("mode", [ILU, ON_FAIL])
@pytest.mark.parametrize("make", [_stretched, lambda: W.bfs2d(n_in=(16, 8), n_ch=64, n_out=16, half=8, dt=0.02)],
                         ids=["channel3d-stretched", "bfs2d"])
def test_ilu_adjoint_matches_oracle(make, mode):
    """The transposed predictor solve runs with the transposed factors (same
    pivots, rebuilt from the recorded C)."""
    c = make()
    m = O.mesh_from_case(c)
    d = c.ndim
    opts = dict(adv_precond=mode, p_rtol=1e-13 if d == 3 else 1e-12)
    if mode == ON_FAIL:
        opts["adv_maxit"] = 12
    dom = gpu_domain(c, **opts)
    rng = np.random.default_rng(11)
    gu = rng.standard_normal((d, c.ncells))
    gp = rng.standard_normal(c.ncells)
    S = None if c.S is None else to_dev(dom, c.S, d)
    _, _, fst = dom.step(to_dev(dom, c.u0, d), to_dev(dom, c.p0), c.dt, c.nu, S)
    du, dp, dS, dnu, st = dom.step_adjoint(to_dev(dom, gu, d), to_dev(dom, gp))
    assert st["status"] == "PISO_OK", st
    if mode == ILU:
        assert st["adv_precond_used"] == 1
    _, _, tape = oracle_step(m, c, c.u0, c.p0, c.S)
    ou, op, oS, onu = O.piso_step_adjoint(m, tape, gu, gp)
    assert rel_err(host(du), ou) <= 1e-8
    if dS is not None:
        assert rel_err(host(dS), oS) <= 1e-8
    assert abs(dnu - onu) <= 1e-8 * max(abs(onu), 1e-30) + 1e-12


def test_ilu_bitwise_deterministic_and_autotuned():
    c = W.channel3d(32, 24, 32, gamma=3.0, dt=0.2)
    dom = gpu_domain(c, adv_precond=ILU)
    a = gpu_step(dom, c, c.u0, c.p0, c.S)
    b = gpu_step(dom, c, c.u0, c.p0, c.S)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    # the autotuner's layouts each get their own level tables
    d = c.ndim
    dom.autotune(to_dev(dom, c.u0, d), to_dev(dom, c.p0), c.dt, c.nu, to_dev(dom, c.S, d))
    assert dom.get_options().adv_precond == ILU
    m = O.mesh_from_case(c)
    uo, po, _ = oracle_step(m, c, c.u0, c.p0, c.S)
    ug, pg, st = gpu_step(dom, c, c.u0, c.p0, c.S)
    assert st["adv_precond_used"] == 1 and rel_err(ug, uo) <= FP64_REL


def test_batch_rejects_ilu():
    c = W.cavity2d(16)
    doms = [gpu_domain(c)]
    with pytest.raises(capi.PisoError):
        Batch(doms, capi.default_options(adv_precond=ILU))
