"""GPU forward PISO step vs the FP64 oracle (element-wise parity), through the
C ABI.  Cases follow the paper's scenarios at the benchmark configurations'
sizes plus small ragged ones (arXiv:2505.16992, App. A-B)."""
import math

import numpy as np
import pytest
import torch

import oracle as O
from paper_2505_16992_b300 import capi
from paper_2505_16992_b300 import workloads as W
from gpu_util import FP32_REL, FP64_REL, gpu_domain, gpu_step, host, oracle_step, rel_err, to_dev

pytestmark = pytest.mark.gpu


def _per_step_parity(case, steps, precision="fp64", tol=FP64_REL, **opts):
    """Advance the oracle; at each step run the GPU step from the oracle's
    state and compare u, p (and outflow boundary values)."""
    m = O.mesh_from_case(case)
    dom = gpu_domain(case, precision, **opts)
    u, p, bval = case.u0, case.p0, m.bval
    worst = 0.0
    for n in range(steps):
        ug, pg, st = gpu_step(dom, case, u, p, case.S)
        assert st["status"] == "PISO_OK", st
        u1, p1, tape = oracle_step(m, case, u, p, case.S, bval)
        eu, ep = rel_err(ug, u1), rel_err(pg, p1)
        worst = max(worst, eu, ep)
        assert eu <= tol and ep <= tol * 10, (n, eu, ep, st)
        u, p, bval = u1, p1, tape["bval"]
        # keep the domain's boundary state in step with the oracle's
        if m.has_outflow:
            dom.set_boundary(_bval_faces(m, bval))
    return worst


def _bval_faces(m, bval):
    """Oracle boundary values (per cell side) -> the library's face order."""
    faces = []
    # library order: blocks in order, sides in order, faces in side order
    for bi in range(len(m.res)):
        for s in range(m.nsides):
            cells = m.side_cells(bi, s)
            if m.is_bface[s, cells[0]]:
                faces.append(bval[s][:, cells])
    return np.concatenate(faces, axis=1)


def test_cavity_32_per_step():
    c = W.cavity2d(32)
    _per_step_parity(c, 4)


def test_cavity_32_rollout():
    """The 32x32 cavity (Re 100, dt 0.005) over 50 steps."""
    c = W.cavity2d(32)
    m = O.mesh_from_case(c)
    dom = gpu_domain(c)
    u, p = to_dev(dom, c.u0, 2), to_dev(dom, c.p0)
    for _ in range(50):
        u, p, st = dom.step(u, p, c.dt, c.nu)
        assert st["status"] == "PISO_OK"
    uo, po, _ = O.rollout(m, c.u0, c.p0, c.dt, c.nu, None, 50)
    assert rel_err(host(u), uo) <= 1e-9
    assert rel_err(host(p), po) <= 1e-8


@pytest.mark.parametrize("n", [(5, 3), (13, 7), (33, 17)])
def test_ragged_cavity(n):
    c = W.cavity2d(n[0])
    v = np.linspace(0, 1, n[0] + 1)
    c.blocks[0] = W.rect_block(v, np.linspace(0, 0.6, n[1] + 1))
    N = n[0] * n[1]
    c.dirichlet = []
    for s in range(4):
        val = W.wall(c.blocks[0], s, 2)
        if s == 3:
            val[:, 0] = 1.0
        c.dirichlet.append((0, s, val))
    c.u0, c.p0 = np.zeros((2, N)), np.zeros(N)
    _per_step_parity(c, 2)


def test_bfs_multiblock_outflow_small():
    c = W.bfs2d(n_in=(16, 8), n_ch=64, n_out=16, half=8, dt=0.02)
    _per_step_parity(c, 3, p_rtol=1e-12)


def test_bfs_22528_cells_full_size():
    c = W.bfs2d()
    assert c.ncells == 22528
    _per_step_parity(c, 2, p_rtol=1e-12)


def test_channel3d_small():
    c = W.channel3d(16, 12, 8)
    _per_step_parity(c, 3)


def test_channel3d_64x48x32_full_size():
    c = W.channel3d()
    assert c.ncells == 64 * 48 * 32
    _per_step_parity(c, 1)


def test_turbulence2d_periodic():
    c = W.turbulence2d(64)
    _per_step_parity(c, 2)


def test_cavity3d_ragged():
    c = W.cavity3d(5, nz=3)
    _per_step_parity(c, 2)


@pytest.mark.parametrize("ctas", [1, 3, 7, 64])
def test_cta_counts_agree(ctas):
    """The result does not depend on how the cells are split over CTAs beyond
    summation order."""
    c = W.channel3d(12, 10, 6)
    m = O.mesh_from_case(c)
    u1, p1, _ = oracle_step(m, c, c.u0, c.p0, c.S)
    dom = gpu_domain(c, ctas=ctas, block_threads=128)
    ug, pg, st = gpu_step(dom, c, c.u0, c.p0, c.S)
    assert rel_err(ug, u1) <= FP64_REL
    assert rel_err(pg, p1) <= 10 * FP64_REL


def test_bitwise_deterministic():
    c = W.channel3d(16, 12, 8)
    dom = gpu_domain(c)
    a = gpu_step(dom, c, c.u0, c.p0, c.S)
    b = gpu_step(dom, c, c.u0, c.p0, c.S)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_in_place_aliasing():
    c = W.cavity2d(16)
    m = O.mesh_from_case(c)
    dom = gpu_domain(c)
    u, p = to_dev(dom, c.u0, 2), to_dev(dom, c.p0)
    u1, p1, _ = dom.step(u, p, c.dt, c.nu, u_out=u, p_out=p)
    uo, po, _ = oracle_step(m, c, c.u0, c.p0)
    assert u1.data_ptr() == u.data_ptr()
    assert rel_err(host(u), uo) <= FP64_REL


def test_fp32_mixed_laminar_cavity():
    """Mixed precision against the FP64 oracle on a laminar flow after N steps."""
    c = W.cavity2d(32)
    m = O.mesh_from_case(c)
    dom = gpu_domain(c, "fp32", adv_rtol=1e-6, p_rtol=1e-6)
    u, p = to_dev(dom, c.u0, 2), to_dev(dom, c.p0)
    for _ in range(50):
        u, p, st = dom.step(u, p, c.dt, c.nu)
        assert st["status"] == "PISO_OK", st
    uo, po, _ = O.rollout(m, c.u0, c.p0, c.dt, c.nu, None, 50)
    assert rel_err(host(u), uo) <= FP32_REL


@pytest.mark.parametrize("make,steps", [
    (lambda: W.bfs2d(n_in=(16, 8), n_ch=64, n_out=16, half=8, dt=0.02), 20),
    (lambda: W.channel3d(16, 12, 8), 20),
], ids=["bfs2d-outflow", "channel3d-16x12x8"])
def test_fp32_mixed_laminar_after_n_steps(make, steps):
    """Mixed precision against the FP64 oracle after N steps on the laminar
    multi-block step (with its advective outflow) and the forced channel."""
    c = make()
    m = O.mesh_from_case(c)
    dom = gpu_domain(c, "fp32", adv_rtol=1e-6, p_rtol=1e-6)
    d = c.ndim
    S = None if c.S is None else to_dev(dom, c.S, d)
    u, p = to_dev(dom, c.u0, d), to_dev(dom, c.p0)
    for _ in range(steps):
        u, p, st = dom.step(u, p, c.dt, c.nu, S)
        assert st["status"] == "PISO_OK", st
    uo, po, _ = O.rollout(m, c.u0, c.p0, c.dt, c.nu, c.S, steps)
    assert rel_err(host(u), uo) <= FP32_REL, rel_err(host(u), uo)


def test_fp32_mixed_channel3d():
    c = W.channel3d(16, 12, 8)
    m = O.mesh_from_case(c)
    dom = gpu_domain(c, "fp32", adv_rtol=1e-6, p_rtol=1e-6)
    ug, pg, st = gpu_step(dom, c, c.u0, c.p0, c.S)
    uo, po, _ = oracle_step(m, c, c.u0, c.p0, c.S)
    assert st["status"] == "PISO_OK"
    assert rel_err(ug, uo) <= FP32_REL


def test_errors_reported_not_trapped():
    c = W.cavity2d(16)
    dom = gpu_domain(c, p_maxit=1)
    u, p = to_dev(dom, c.u0, 2), to_dev(dom, c.p0)
    with pytest.raises(capi.PisoError) as e:
        dom.step(u, p, c.dt, c.nu)
    assert e.value.status == 3          # PISO_ENOCONV
    with pytest.raises(capi.PisoError) as e:
        dom.step(u, p, -1.0, c.nu)
    assert e.value.status == 1          # PISO_EINVAL
    dom.set_options(capi.default_options())
    S = to_dev(dom, np.full((2, dom.N), np.nan), 2)
    with pytest.raises(capi.PisoError) as e:
        dom.step(u, p, c.dt, c.nu, S)
    assert e.value.status == 5          # PISO_ENAN
    # the context is still usable afterwards
    u1, p1, st = dom.step(u, p, c.dt, c.nu)
    assert st["status"] == "PISO_OK"


def test_barrier_timeout_is_reported_and_context_survives():
    """Failure detection without a GPU fault: one CTA withholds its first
    barrier arrival (fault injection); every bounded wait runs out after
    timeout_s, the step returns PISO_ETIMEOUT, and the next step succeeds."""
    c = W.cavity2d(32)
    dom = gpu_domain(c, ctas=4, block_threads=128, timeout_s=0.2, fault_withhold_cta=2)
    u, p = to_dev(dom, c.u0, 2), to_dev(dom, c.p0)
    with pytest.raises(capi.PisoError) as e:
        dom.step(u, p, c.dt, c.nu)
    assert e.value.status == 6          # PISO_ETIMEOUT
    dom.set_options(capi.default_options(ctas=4, block_threads=128))
    u1, p1, st = dom.step(u, p, c.dt, c.nu)
    assert st["status"] == "PISO_OK"


def test_autotuned_shape_keeps_parity():
    c = W.channel3d(16, 12, 8)
    m = O.mesh_from_case(c)
    dom = gpu_domain(c)
    u, p, S = to_dev(dom, c.u0, 3), to_dev(dom, c.p0), to_dev(dom, c.S, 3)
    threads, ctas, ms = dom.autotune(u, p, c.dt, c.nu, S)
    assert threads in (512, 768) and ctas >= 1
    u1, p1, st = dom.step(u, p, c.dt, c.nu, S)
    uo, po, _ = oracle_step(m, c, c.u0, c.p0, c.S)
    assert rel_err(host(u1), uo) <= FP64_REL
    assert np.array_equal(host(u), c.u0)          # inputs untouched by the trials


@pytest.mark.parametrize("threads", [768])
def test_wide_cta_variant(threads):
    c = W.channel3d(16, 12, 8)
    _per_step_parity(c, 2, block_threads=threads)


def test_fp32_refined_pressure_reaches_fp64_residual():
    """FP32 mode with FP64 iterative refinement of the pressure solves: the FP64
    residual of the pressure system drops below 1e-10 ||b|| and the velocity
    matches the FP64 oracle to FP32 rounding."""
    c = W.channel3d(16, 12, 8)
    m = O.mesh_from_case(c)
    dom = gpu_domain(c, "fp32", adv_rtol=1e-6, p_refine_rtol=1e-10, p_inner_rtol=1e-4)
    ug, pg, st = gpu_step(dom, c, c.u0, c.p0, c.S)
    uo, po, tape = oracle_step(m, c, c.u0, c.p0, c.S)
    assert st["status"] == "PISO_OK", st
    assert min(st["p_rounds"][:2]) >= 1
    for k in range(2):
        bn = np.linalg.norm(tape["corr"][k]["b"])
        assert st["p_resid"][k] <= 1e-10 * bn * 1.01, (k, st["p_resid"][k], bn)
    assert rel_err(ug, uo) <= 2e-6
    assert rel_err(pg, po) <= 2e-5


def test_fp32_refined_adjoint():
    c = W.cavity2d(24, nu=0.01, dt=0.01)
    m = O.mesh_from_case(c)
    dom = gpu_domain(c, "fp32", adv_rtol=1e-7, p_refine_rtol=1e-10)
    rng = np.random.default_rng(4)
    u0 = 0.2 * rng.standard_normal((2, c.ncells))
    ubar = rng.standard_normal((2, c.ncells))
    dom.step(to_dev(dom, u0, 2), to_dev(dom, c.p0), c.dt, c.nu)
    du, dp, dS, dnu, st = dom.step_adjoint(to_dev(dom, ubar, 2))
    assert st["status"] == "PISO_OK"
    _, _, tape = oracle_step(m, c, u0, c.p0)
    gu, gp, gS, gnu = O.piso_step_adjoint(m, tape, ubar, np.zeros(c.ncells))
    assert rel_err(host(du), gu) <= 1e-4


def test_fp32_pressure_cg_stall_is_finished_by_refinement():
    """An FP32 pressure CG asked for more than FP32 vectors can deliver
    (rtol 1e-11; at 1e-9 whether it stalls depends on the rounding of the
    build) stalls; the step then finishes the solve with FP64-residual
    refinement rounds to the same tolerance instead of running to the
    iteration limit."""
    c = W.cavity2d(32)
    dom = gpu_domain(c, "fp32", adv_rtol=1e-6, p_rtol=1e-11)
    u1, p1, st = gpu_step(dom, c, c.u0, c.p0)
    assert st["status"] == "PISO_OK", st
    assert all(r >= 1 for r in st["p_rounds"][:2]), st
    assert all(res <= 1e-11 * rhs * 1.0000001 for res, rhs in zip(st["p_resid"][:2], st["p_rhs_norm"][:2])), st
    m = O.mesh_from_case(c)
    u_o, p_o, _ = O.piso_step(m, c.u0, c.p0, c.dt, c.nu)
    assert rel_err(u1, u_o) <= FP32_REL


def test_headline_channel_fp32_50_steps_against_fp64_oracle():
    """The benchmarked configuration end to end: the full 64x48x32 channel
    (tanh walls gamma 2, nu 1/180, dt 0.01, seeded perturbation) in the FP32
    mode at Krylov rtol 1e-6 with the autotuned launch shape and pressure
    preconditioner, advanced 50 steps, against the FP64 oracle (Krylov to
    1e-13) advanced the same 50 steps: every velocity component within 1e-4
    of its own largest magnitude (the mixed-precision bar for laminar fields),
    the pressure within 1e-3 of its largest magnitude."""
    c = W.channel3d(64, 48, 32)
    m = O.mesh_from_case(c)
    dom = gpu_domain(c, "fp32", adv_rtol=1e-6, p_rtol=1e-6, p_maxit=20000, adv_maxit=2000)
    u, p, S = to_dev(dom, c.u0, 3), to_dev(dom, c.p0), to_dev(dom, c.S, 3)
    dom.autotune(u, p, c.dt, c.nu, S)
    steps = 50
    for _ in range(steps):
        u, p, st = dom.step(u, p, c.dt, c.nu, S)
        assert st["status"] == "PISO_OK", st
    uo, po, _ = O.rollout(m, c.u0, c.p0, c.dt, c.nu, c.S, steps)
    eu, ep = rel_err(host(u), uo), rel_err(host(p), po)
    assert eu <= FP32_REL, eu
    assert ep <= 10 * FP32_REL, ep
