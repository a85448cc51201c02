"""The Jacobi-preconditioned pressure CG and the predictor's BiCGStab sweeping
four consecutive cells per thread (vector loads and stores; domains whose CTA
ranges are walked in interleaved passes and whose blocks all have nx a
multiple of 4) against the FP64 oracle and against the one-cell-per-thread
sweeps, through the C ABI.  The form changes how the systems of App. A.1
(Eqs. implEuler1 and pressure) and their transposes in the adjoint are
swept, not the recurrences, so the solves must reproduce the oracle's and
agree with the scalar sweeps up to the summation order of the dot products."""
import numpy as np
import pytest

import oracle as O
from paper_2505_16992_b300 import capi
from paper_2505_16992_b300 import workloads as W
from gpu_util import FP32_REL, FP64_REL, gpu_domain, gpu_step, host, oracle_step, rel_err, to_dev

pytestmark = pytest.mark.gpu

JAC = capi.PISO_PRECOND_JACOBI

# (case, CTAs, CTA width): few CTAs, so a CTA's cells exceed its shared
# neighbour table and the interleaved passes (the four-cell sweep) run
CASES = {
    # x, z periodic (the quad at x = 0 wraps to x = nx - 1), tanh walls in y;
    # 2688 quads over 512 threads: the last pass is ragged
    "channel3d-28x24x16": (lambda: W.channel3d(28, 24, 16), 1, 512),
    # walls on every side, lid on +y
    "cavity2d-128": (lambda: W.cavity2d(128), 1, 768),
    # five blocks joined in x and in y, inflow, advective outflow
    "bfs2d": (lambda: W.bfs2d(), 2, 768),
    # doubly periodic
    "periodic2d-128": (lambda: W.turbulence2d(128), 1, 256),
    # three CTAs sweeping the same passes
    "channel3d-32x24x28-3cta": (lambda: W.channel3d(32, 24, 28), 3, 128),
}


def c_is_3d(name):
    return name.startswith("channel3d")


def _dom(name, precision="fp64", **opts):
    make, ctas, threads = CASES[name]
    c = make()
    dom = gpu_domain(c, precision, p_precond=JAC, ctas=ctas, block_threads=threads, **opts)
    assert dom.uses_cg_vec4(), "four-cell sweep not taken"
    return c, dom


@pytest.mark.parametrize("name", list(CASES))
def test_vec4_forward_parity(name):
    c, dom = _dom(name, p_rtol=1e-12 if name == "bfs2d" else 1e-13)
    ug, pg, st = gpu_step(dom, c, c.u0, c.p0, c.S)
    assert st["status"] == "PISO_OK", st
    uo, po, _ = oracle_step(O.mesh_from_case(c), c, c.u0, c.p0, c.S)
    assert rel_err(ug, uo) <= FP64_REL, rel_err(ug, uo)
    assert rel_err(pg, po) <= 10 * FP64_REL, rel_err(pg, po)


@pytest.mark.parametrize("name", ["channel3d-28x24x16", "bfs2d"])
def test_vec4_matches_scalar_sweep(name):
    """Same recurrences: the four-cell sweep (few CTAs) and the one-cell sweep
    (enough CTAs for the shared neighbour table) agree to rounding and take the
    same number of iterations up to one at the tolerance boundary."""
    c, dom = _dom(name, p_rtol=1e-12)
    uv, pv, sv = gpu_step(dom, c, c.u0, c.p0, c.S)
    ds = gpu_domain(c, p_precond=JAC, p_rtol=1e-12, ctas=148, block_threads=768)
    assert not ds.uses_cg_vec4()
    us, ps, ss = gpu_step(ds, c, c.u0, c.p0, c.S)
    assert rel_err(uv, us) <= 1e-11 and rel_err(pv, ps) <= 1e-9, (rel_err(uv, us), rel_err(pv, ps))
    for k in range(2):
        assert abs(sv["p_iters"][k] - ss["p_iters"][k]) <= 1, (sv["p_iters"], ss["p_iters"])
    for k in range(c.ndim):
        assert abs(sv["adv_iters"][k] - ss["adv_iters"][k]) <= 1, (sv["adv_iters"], ss["adv_iters"])


def test_vec4_fp32_after_n_steps():
    """FP32 bulk with float-pair reductions, 10 steps against the FP64 oracle."""
    c, dom = _dom("channel3d-28x24x16", "fp32", adv_rtol=1e-7, p_rtol=1e-7)
    m = O.mesh_from_case(c)
    d = c.ndim
    u, p = to_dev(dom, c.u0, d), to_dev(dom, c.p0)
    S = to_dev(dom, c.S, d)
    uo, po = c.u0, c.p0
    for _ in range(10):
        u, p, st = dom.step(u, p, c.dt, c.nu, S)
        assert st["status"] == "PISO_OK", st
        uo, po, _ = oracle_step(m, c, uo, po, c.S)
    assert rel_err(host(u), uo) <= FP32_REL, rel_err(host(u), uo)
    assert rel_err(host(p), po) <= 10 * FP32_REL, rel_err(host(p), po)


@pytest.mark.parametrize("name", ["channel3d-32x24x28-3cta", "bfs2d"])
def test_vec4_adjoint_matches_oracle(name):
    """The adjoint's transposed pressure solves (P is symmetric) run the same
    sweep."""
    c, dom = _dom(name, p_rtol=1e-13 if c_is_3d(name) else 1e-12)
    m = O.mesh_from_case(c)
    rng = np.random.default_rng(21)
    d = c.ndim
    gu, gp = rng.standard_normal((d, c.ncells)), rng.standard_normal(c.ncells)
    S = None if c.S is None else to_dev(dom, c.S, d)
    dom.step(to_dev(dom, c.u0, d), to_dev(dom, c.p0), c.dt, c.nu, S)
    du, dp, dS, dnu, st = dom.step_adjoint(to_dev(dom, gu, d), to_dev(dom, gp))
    assert st["status"] == "PISO_OK", st
    _, _, tape = oracle_step(m, c, c.u0, c.p0, c.S)
    ou, op, oS, onu = O.piso_step_adjoint(m, tape, gu, gp)
    assert rel_err(host(du), ou) <= 1e-8, rel_err(host(du), ou)
    if dS is not None:
        assert rel_err(host(dS), oS) <= 1e-8
    assert abs(dnu - onu) <= 1e-8 * max(abs(onu), 1e-30) + 1e-12


def test_vec4_bitwise_deterministic():
    c, dom = _dom("channel3d-32x24x28-3cta", "fp32", adv_rtol=1e-6, p_rtol=1e-6)
    a = gpu_step(dom, c, c.u0, c.p0, c.S)
    b = gpu_step(dom, c, c.u0, c.p0, c.S)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_where_the_vec4_sweep_runs():
    big = W.channel3d(28, 24, 16)
    assert gpu_domain(big, p_precond=JAC, ctas=1, block_threads=512).uses_cg_vec4()
    # nx not a multiple of 4: one cell per thread
    assert not gpu_domain(W.channel3d(30, 24, 16), p_precond=JAC, ctas=1, block_threads=512).uses_cg_vec4()
    # the CTA ranges fit their neighbour tables: one cell per thread
    assert not gpu_domain(big, p_precond=JAC, ctas=64, block_threads=128).uses_cg_vec4()
    # the y-line preconditioner sweeps lines instead
    assert not gpu_domain(big, p_precond=capi.PISO_PRECOND_LINE, ctas=1, block_threads=512).uses_cg_vec4()
    # a joint that reverses an axis (block 1 turned by two quarter turns)
    c, _ = W.two_block_cavity2d(nx=96, ny=64, rot=2)
    assert not gpu_domain(c, p_precond=JAC, ctas=1, block_threads=128).uses_cg_vec4()
    c0, _ = W.two_block_cavity2d(nx=96, ny=64, rot=0)
    assert gpu_domain(c0, p_precond=JAC, ctas=1, block_threads=128).uses_cg_vec4()
