"""Batched persistent launch: independent simulations of uneven size stepped in
one cooperative launch (one CTA group per domain), checked member by member
against the FP64 oracle; adjoint; CUDA-graph capture of a batched step."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2505_16992_b300 import capi
from paper_2505_16992_b300 import workloads as W
from paper_2505_16992_b300.solver import Batch
from gpu_util import gpu_domain, host, rel_err, to_dev

pytestmark = pytest.mark.gpu


def _members(cases, precision="fp64", **opts):
    doms = [gpu_domain(c, precision, **opts) for c in cases]
    us = [to_dev(d, c.u0, c.ndim) for d, c in zip(doms, cases)]
    ps = [to_dev(d, c.p0) for d, c in zip(doms, cases)]
    Ss = [None if c.S is None else to_dev(d, c.S, c.ndim) for d, c in zip(doms, cases)]
    return doms, us, ps, Ss


def test_batch_forward_matches_oracle_per_member():
    cases = W.batch2d(count=7, seed=5, nmin=6, nmax=40)
    doms, us, ps, Ss = _members(cases)
    b = Batch(doms, capi.default_options(adv_rtol=1e-13, p_rtol=1e-13))
    uo, po, st = b.step(us, ps, [c.dt for c in cases], [c.nu for c in cases], Ss)
    for i, c in enumerate(cases):
        assert st[i]["status"] == "PISO_OK", (i, st[i])
        m = O.mesh_from_case(c)
        u1, p1, _ = O.piso_step(m, c.u0, c.p0, c.dt, c.nu, c.S)
        assert rel_err(host(uo[i]), u1) <= 1e-10, i
        assert rel_err(host(po[i]), p1) <= 1e-9, i


def test_batch_equals_single_domain_launches():
    """A member's result in the batch equals its own single-domain launch up to
    the summation order of its reductions (different CTA split)."""
    cases = W.batch2d(count=5, seed=6, nmin=8, nmax=48)
    doms, us, ps, Ss = _members(cases)
    b = Batch(doms, capi.default_options(adv_rtol=1e-13, p_rtol=1e-13))
    uo, po, _ = b.step(us, ps, [c.dt for c in cases], [c.nu for c in cases], Ss)
    for i, (d, c) in enumerate(zip(doms, cases)):
        u1, p1, _ = d.step(us[i], ps[i], c.dt, c.nu, Ss[i])
        assert rel_err(host(uo[i]), host(u1)) <= 1e-11


def test_batch_adjoint_matches_oracle():
    cases = W.batch2d(count=4, seed=8, nmin=6, nmax=24)
    doms, us, ps, Ss = _members(cases)
    b = Batch(doms, capi.default_options(adv_rtol=1e-13, p_rtol=1e-13))
    b.step(us, ps, [c.dt for c in cases], [c.nu for c in cases], Ss)
    rng = np.random.default_rng(1)
    gus = [rng.standard_normal((2, c.ncells)) for c in cases]
    du, dp, dS, dnu, st = b.step_adjoint([to_dev(d, g, 2) for d, g in zip(doms, gus)])
    for i, c in enumerate(cases):
        assert st[i]["status"] == "PISO_OK"
        m = O.mesh_from_case(c)
        _, _, tape = O.piso_step(m, c.u0, c.p0, c.dt, c.nu, c.S)
        gu, gp, gS, gnu = O.piso_step_adjoint(m, tape, gus[i], np.zeros(c.ncells))
        assert rel_err(host(du[i]), gu) <= 1e-8, i
        assert abs(dnu[i] - gnu) <= 1e-8 * abs(gnu), i


def test_batch_adjoint_gradient_path_variant():
    """The batched adjoint honours the gradient-path selection (Sec. 2.4)."""
    cases = W.batch2d(count=3, seed=10, nmin=6, nmax=24)
    doms, us, ps, Ss = _members(cases)
    b = Batch(doms, capi.default_options(adv_rtol=1e-13, p_rtol=1e-13, grad_paths=capi.PISO_GRAD_ADV))
    b.step(us, ps, [c.dt for c in cases], [c.nu for c in cases], Ss)
    rng = np.random.default_rng(2)
    gus = [rng.standard_normal((2, c.ncells)) for c in cases]
    du, dp, dS, dnu, st = b.step_adjoint([to_dev(d, g, 2) for d, g in zip(doms, gus)])
    for i, c in enumerate(cases):
        assert st[i]["status"] == "PISO_OK" and sum(st[i]["p_iters"]) == 0, st[i]
        m = O.mesh_from_case(c)
        _, _, tape = O.piso_step(m, c.u0, c.p0, c.dt, c.nu, c.S)
        gu, gp, gS, gnu = O.piso_step_adjoint(m, tape, gus[i], np.zeros(c.ncells), O.Options(grad_p=False))
        assert rel_err(host(du[i]), gu) <= 1e-8, i
        assert abs(dnu[i] - gnu) <= 1e-8 * abs(gnu), i


def test_batch_of_64_simulations_full_size_sampled_parity():
    """The batch of 64 independent 2D cavity/channel simulations, sides uniform in
    32..256, Re in [100, 2000], FP32 bulk; sampled members against the oracle."""
    cases = W.batch2d()
    assert len(cases) == 64
    doms, us, ps, Ss = _members(cases, "fp32", adv_rtol=1e-6, p_rtol=1e-6)
    b = Batch(doms, capi.default_options(adv_rtol=1e-6, p_rtol=1e-6))
    uo, po, st = b.step(us, ps, [c.dt for c in cases], [c.nu for c in cases], Ss)
    assert all(s["status"] == "PISO_OK" for s in st)
    sizes = [c.ncells for c in cases]
    pick = sorted({int(np.argmin(sizes)), int(np.argmax(sizes)), 1, 10})
    for i in pick:
        c = cases[i]
        m = O.mesh_from_case(c)
        u1, p1, _ = O.piso_step(m, c.u0, c.p0, c.dt, c.nu, c.S)
        assert rel_err(host(uo[i]), u1) <= 1e-4, (i, c.ncells)


def test_batch_step_in_cuda_graph():
    """The batched forward step captured in a CUDA graph replays bit-identically
    to the eager launch."""
    cases = W.batch2d(count=6, seed=9, nmin=16, nmax=64)
    doms, us, ps, Ss = _members(cases, "fp32", adv_rtol=1e-6, p_rtol=1e-6)
    b = Batch(doms, capi.default_options(adv_rtol=1e-6, p_rtol=1e-6))
    dts, nus = [c.dt for c in cases], [c.nu for c in cases]
    uo = [torch.empty_like(u) for u in us]
    po = [torch.empty_like(p) for p in ps]
    ref_u, ref_p, _ = b.step(us, ps, dts, nus, Ss)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        b.step(us, ps, dts, nus, Ss, u_out=uo, p_out=po, sync=False)     # warm-up on the side stream
    torch.cuda.current_stream().wait_stream(s)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        b.step(us, ps, dts, nus, Ss, u_out=uo, p_out=po, sync=False)
    for t in uo + po:
        t.zero_()
    g.replay()
    torch.cuda.synchronize()
    for i in range(len(cases)):
        assert torch.equal(uo[i], ref_u[i]) and torch.equal(po[i], ref_p[i]), i


def test_batch_forward_and_adjoint_graph_and_back_to_back_enqueues():
    """Forward and adjoint of a step captured together in one CUDA graph replay
    bit-identically to eager launches; and forward/adjoint enqueued back to
    back without synchronising, with the argument sets changing every step,
    give the same results as synchronised calls (each direction stages its
    per-domain arguments in its own buffers)."""
    cases = W.batch2d(count=5, seed=11, nmin=16, nmax=48)
    doms, us, ps, Ss = _members(cases, "fp32", adv_rtol=1e-6, p_rtol=1e-6)
    b = Batch(doms, capi.default_options(adv_rtol=1e-6, p_rtol=1e-6))
    dts, nus = [c.dt for c in cases], [c.nu for c in cases]
    g0 = torch.Generator(device="cpu").manual_seed(3)
    gs = [torch.randn(u.shape, generator=g0).to(u.dtype).cuda() for u in us]
    # eager reference, synchronised
    ref_u, ref_p, _ = b.step(us, ps, dts, nus, Ss)
    ref_du, ref_dp, ref_dS, _, _ = b.step_adjoint(gs)
    # back to back, alternating output buffers, no synchronisation in between
    outs = [([torch.empty_like(u) for u in us], [torch.empty_like(p) for p in ps]) for _ in range(2)]
    adj = [([torch.empty_like(g) for g in gs], [torch.empty_like(p) for p in ps], [torch.empty_like(g) for g in gs])
           for _ in range(2)]
    for k in range(4):
        uo, po = outs[k % 2]
        du, dp, dS = adj[k % 2]
        b.step(us, ps, dts, nus, Ss, u_out=uo, p_out=po, sync=False)
        b.step_adjoint(gs, sync=False, du_in=du, dp_in=dp, dS=dS)
    torch.cuda.synchronize()
    for k in range(2):
        for i in range(len(cases)):
            assert torch.equal(outs[k][0][i], ref_u[i]) and torch.equal(outs[k][1][i], ref_p[i]), (k, i)
            assert torch.equal(adj[k][0][i], ref_du[i]) and torch.equal(adj[k][2][i], ref_dS[i]), (k, i)
    # one graph holding both launches
    uo, po = outs[0]
    du, dp, dS = adj[0]
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        b.step(us, ps, dts, nus, Ss, u_out=uo, p_out=po, sync=False)
        b.step_adjoint(gs, sync=False, du_in=du, dp_in=dp, dS=dS)
    torch.cuda.current_stream().wait_stream(s)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        b.step(us, ps, dts, nus, Ss, u_out=uo, p_out=po, sync=False)
        b.step_adjoint(gs, sync=False, du_in=du, dp_in=dp, dS=dS)
    for t in uo + po + du + dS:
        t.zero_()
    g.replay()
    g.replay()
    torch.cuda.synchronize()
    for i in range(len(cases)):
        assert torch.equal(uo[i], ref_u[i]) and torch.equal(po[i], ref_p[i]), i
        assert torch.equal(du[i], ref_du[i]) and torch.equal(dS[i], ref_dS[i]), i


def test_batch_autotune_keeps_parity_and_inputs():
    """The batch autotuner times the forward step with 512- and 768-thread
    CTAs and two CTA totals, restores the state, and the chosen layout steps
    every member as the oracle does (forward and adjoint)."""
    cases = W.batch2d(count=6, seed=9, nmin=8, nmax=40)
    doms, us, ps, Ss = _members(cases)
    b = Batch(doms, capi.default_options(adv_rtol=1e-13, p_rtol=1e-13))
    u_before = [host(u).copy() for u in us]
    dts, nus = [c.dt for c in cases], [c.nu for c in cases]
    threads, ctas, ms = b.autotune(us, ps, dts, nus, Ss)
    assert threads in (512, 768) and ctas >= len(cases) and ms > 0
    assert all(np.array_equal(host(u), u0) for u, u0 in zip(us, u_before))
    with pytest.raises(capi.PisoError):
        b.step_adjoint([torch.ones_like(u) for u in us])        # the trials are not a step to differentiate
    uo, po, st = b.step(us, ps, dts, nus, Ss)
    rng = np.random.default_rng(2)
    gus = [rng.standard_normal((2, c.ncells)) for c in cases]
    du, dp, dS, dnu, ast = b.step_adjoint([to_dev(d, g, 2) for d, g in zip(doms, gus)])
    for i, c in enumerate(cases):
        assert st[i]["status"] == "PISO_OK" and ast[i]["status"] == "PISO_OK", (i, st[i], ast[i])
        m = O.mesh_from_case(c)
        u1, p1, tape = O.piso_step(m, c.u0, c.p0, c.dt, c.nu, c.S)
        assert rel_err(host(uo[i]), u1) <= 1e-10, i
        gu, gp, gS, gnu = O.piso_step_adjoint(m, tape, gus[i], np.zeros(c.ncells))
        assert rel_err(host(du[i]), gu) <= 1e-8, i


def test_batch_fp32_refined_pressure_reaches_fp64_tolerance():
    """The mixed-precision batch with FP64-refined pressure solves reaches the
    same relative residual as the FP64 batch (1e-10 of each right-hand side)
    and the FP64 oracle's velocity to FP32 rounding."""
    cases = W.batch2d(count=5, seed=10, nmin=16, nmax=48)
    doms, us, ps, Ss = _members(cases, "fp32", adv_rtol=1e-7, p_rtol=1e-6, p_refine_rtol=1e-10)
    b = Batch(doms, capi.default_options(adv_rtol=1e-7, p_rtol=1e-6, p_refine_rtol=1e-10))
    uo, po, st = b.step(us, ps, [c.dt for c in cases], [c.nu for c in cases], Ss)
    for i, c in enumerate(cases):
        assert st[i]["status"] == "PISO_OK", (i, st[i])
        assert all(res <= 1e-10 * rhs * 1.01 for res, rhs in zip(st[i]["p_resid"][:2], st[i]["p_rhs_norm"][:2])), st[i]
        m = O.mesh_from_case(c)
        u1, p1, _ = O.piso_step(m, c.u0, c.p0, c.dt, c.nu, c.S)
        assert rel_err(host(uo[i]), u1) <= 2e-5, (i, rel_err(host(uo[i]), u1))


def test_batch_members_keep_the_y_line_preconditioner_they_ask_for():
    """Wall-refined members (tanh channels: alpha_yy >> alpha_xx near the walls)
    whose options ask for the y-line preconditioned CG run it inside the batch,
    as they do alone (the same iteration counts); a member that got it only
    from PISO_PRECOND_AUTO runs Jacobi there (more iterations); every member
    reproduces the oracle's step."""
    cases = [W.channel2d(16, 24, gamma=2.0, nu=0.05, dt=0.05), W.cavity2d(20),
             W.channel2d(24, 32, gamma=2.5, nu=0.02, dt=0.05)]
    asked = [capi.PISO_PRECOND_LINE, capi.PISO_PRECOND_AUTO, capi.PISO_PRECOND_AUTO]
    doms = [gpu_domain(c, p_precond=pc) for c, pc in zip(cases, asked)]
    us = [to_dev(d, c.u0, c.ndim) for d, c in zip(doms, cases)]
    ps = [to_dev(d, c.p0) for d, c in zip(doms, cases)]
    Ss = [None if c.S is None else to_dev(d, c.S, c.ndim) for d, c in zip(doms, cases)]
    assert [d.uses_line_precond() for d in doms] == [True, False, True]
    alone = [d.step(us[i], ps[i], cases[i].dt, cases[i].nu, Ss[i])[2] for i, d in enumerate(doms)]
    b = Batch(doms, capi.default_options(adv_rtol=1e-13, p_rtol=1e-13))
    uo, po, st = b.step(us, ps, [c.dt for c in cases], [c.nu for c in cases], Ss)
    for i, c in enumerate(cases):
        assert st[i]["status"] == "PISO_OK", (i, st[i])
        m = O.mesh_from_case(c)
        u1, p1, _ = O.piso_step(m, c.u0, c.p0, c.dt, c.nu, c.S)
        assert rel_err(host(uo[i]), u1) <= 1e-10, (i, rel_err(host(uo[i]), u1))
    assert abs(st[0]["p_iters"][0] - alone[0]["p_iters"][0]) <= 2, (st[0]["p_iters"], alone[0]["p_iters"])
    assert st[2]["p_iters"][0] > alone[2]["p_iters"][0] + 2, (st[2]["p_iters"], alone[2]["p_iters"])
