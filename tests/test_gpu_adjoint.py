"""GPU adjoint PISO step vs the oracle's adjoint (arXiv:2505.16992, Sec. 2.3,
App. A.4), through the C ABI; the autograd wrapper and a checkpointed rollout."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2505_16992_b300 import capi
from paper_2505_16992_b300 import workloads as W
from paper_2505_16992_b300.solver import piso_step, rollout
from gpu_util import bval_faces, gpu_domain, host, rel_err, to_dev

pytestmark = pytest.mark.gpu

ADJ_REL = 1e-8


def _adjoint_parity(case, seed=0, tol=ADJ_REL, precision="fp64", pred_grad_p=0, grad_paths=3, **opts):
    m = O.mesh_from_case(case)
    dom = gpu_domain(case, precision, pred_grad_p=pred_grad_p, grad_paths=grad_paths, **opts)
    d, N = case.ndim, case.ncells
    rng = np.random.default_rng(seed)
    u0 = case.u0 + 0.2 * rng.standard_normal((d, N))
    p0 = rng.standard_normal(N)
    S0 = (case.S if case.S is not None else 0.0) + 0.1 * rng.standard_normal((d, N))
    ubar = rng.standard_normal((d, N))
    pbar = rng.standard_normal(N)
    # forward on both sides from the same state
    u1, p1, st = dom.step(to_dev(dom, u0, d), to_dev(dom, p0), case.dt, case.nu, to_dev(dom, S0, d))
    assert st["status"] == "PISO_OK"
    oo = O.Options(pred_grad_p=bool(pred_grad_p))
    uo, po, tape = O.piso_step(m, u0, p0, case.dt, case.nu, S0, None, oo)
    du, dp, dS, dnu, ast = dom.step_adjoint(to_dev(dom, ubar, d), to_dev(dom, pbar))
    assert ast["status"] == "PISO_OK", ast
    oa = O.Options(pred_grad_p=bool(pred_grad_p), grad_adv=bool(grad_paths & 1), grad_p=bool(grad_paths & 2))
    gu, gp, gS, gnu, gbv = O.piso_step_adjoint(m, tape, ubar, pbar, oa, want_bval=True)
    # a solve left out of the backward pass (Sec. 2.4) does not run at all
    assert (sum(ast["adv_iters"]) > 0) == bool(grad_paths & 1), ast
    assert (sum(ast["p_iters"]) > 0) == bool(grad_paths & 2), ast
    errs = dict(u=rel_err(host(du), gu), S=rel_err(host(dS), gS), nu=abs(dnu - gnu) / max(abs(gnu), 1e-300))
    if np.any(m.is_bface):
        errs["bval"] = rel_err(dom.boundary_adjoint(), bval_faces(m, gbv))
    if pred_grad_p:
        errs["p"] = rel_err(host(dp), gp)
    else:
        assert np.all(host(dp) == 0.0)
    for k, v in errs.items():
        assert v <= tol, (k, errs, ast)
    return errs


def test_adjoint_cavity():
    _adjoint_parity(W.cavity2d(32, nu=0.01, dt=0.01))


def test_adjoint_cavity_pred_grad_p():
    _adjoint_parity(W.cavity2d(16, nu=0.05, dt=0.05), pred_grad_p=1)


def test_adjoint_turbulence2d_128_squared():
    _adjoint_parity(W.turbulence2d(128))


def test_adjoint_channel3d_small():
    _adjoint_parity(W.channel3d(16, 12, 8))


def test_adjoint_channel3d_full_size():
    _adjoint_parity(W.channel3d(), tol=1e-7)


def test_adjoint_bfs_multiblock():
    _adjoint_parity(W.bfs2d(n_in=(16, 8), n_ch=64, n_out=16, half=8, dt=0.02), p_rtol=1e-12)


@pytest.mark.parametrize("ctas", [1, 5])
def test_adjoint_ragged_ctas(ctas):
    c = W.cavity3d(5, nz=3)
    _adjoint_parity(c, ctas=ctas, block_threads=64)


def test_adjoint_fp32_mixed():
    _adjoint_parity(W.cavity2d(32, nu=0.01, dt=0.01), tol=2e-3, precision="fp32", adv_rtol=1e-6, p_rtol=1e-6)


@pytest.mark.parametrize("paths", [0, capi.PISO_GRAD_ADV, capi.PISO_GRAD_P])
@pytest.mark.parametrize("name", ["cavity", "bfs", "channel3d"])
def test_adjoint_gradient_path_variants(name, paths):
    """Sec. 2.4 gradient paths: adjoints with the advection and/or pressure
    solves left out equal the oracle's variants (pinned there by FD of the step
    with frozen solve outputs)."""
    if name == "cavity":
        c, kw = W.cavity2d(32, nu=0.01, dt=0.01), {}
    elif name == "bfs":
        c, kw = W.bfs2d(n_in=(16, 8), n_ch=64, n_out=16, half=8, dt=0.02), dict(p_rtol=1e-12)
    else:
        c, kw = W.channel3d(16, 12, 8), {}
    _adjoint_parity(c, grad_paths=paths, **kw)


@pytest.mark.parametrize("paths", [0, capi.PISO_GRAD_P])
def test_adjoint_gradient_paths_with_predictor_pressure_gradient(paths):
    """With -grad p^n in the predictor (reading R4), dL/dp^n flows only through
    the advection solve: it must vanish when that path is left out."""
    _adjoint_parity(W.cavity2d(16, nu=0.05, dt=0.05), pred_grad_p=1, grad_paths=paths)


@pytest.mark.parametrize("precision,tol", [("fp64", ADJ_REL), ("fp32", 2e-3)])
def test_adjoint_with_ilu_preconditioned_solves(precision, tol):
    """Every gradient of the step (u, S, nu, boundary values) with the
    ILU(0)-preconditioned predictor and transposed predictor solves, on the
    strongly stretched channel they are meant for."""
    kw = dict(adv_rtol=1e-6, p_rtol=1e-6) if precision == "fp32" else {}
    _adjoint_parity(W.channel3d(10, 16, 4, gamma=3.0, dt=0.5), tol=tol, precision=precision,
                    adv_precond=capi.PISO_ADV_PRECOND_ILU, **kw)


def test_adjoint_gradient_paths_fp32_full_channel():
    _adjoint_parity(W.channel3d(), tol=2e-3, precision="fp32", adv_rtol=1e-6, p_rtol=1e-6,
                    grad_paths=capi.PISO_GRAD_ADV)


def test_adjoint_matches_gpu_finite_difference():
    """Self-consistency on the GPU alone: <ubar, du1> along a direction equals
    the adjoint's directional derivative (4th-order central differences)."""
    c = W.channel3d(12, 10, 6)
    dom = gpu_domain(c)
    d, N = c.ndim, c.ncells
    rng = np.random.default_rng(3)
    u0 = to_dev(dom, c.u0, d)
    p0 = to_dev(dom, c.p0)
    S0 = to_dev(dom, c.S, d)
    ubar = to_dev(dom, rng.standard_normal((d, N)), d)
    du = to_dev(dom, rng.standard_normal((d, N)), d)

    def L(t):
        u1, p1, _ = dom.step(u0 + t * du, p0, c.dt, c.nu, S0)
        return float((ubar * u1).sum())

    dom.step(u0, p0, c.dt, c.nu, S0)
    gu, _, _, _, _ = dom.step_adjoint(ubar, None)
    adj = float((gu * du).sum())
    e = 1e-4
    fd = (8 * (L(e) - L(-e)) - (L(2 * e) - L(-2 * e))) / (12 * e)
    assert abs(adj - fd) <= 1e-6 * abs(fd), (adj, fd)


def test_autograd_rollout_checkpointed():
    """Gradient of a loss after 4 steps w.r.t. u^0, S and nu through the
    autograd wrapper (checkpointed recompute) vs the oracle chained adjoint."""
    c = W.turbulence2d(32, nu=0.01, dt=0.02)
    m = O.mesh_from_case(c)
    dom = gpu_domain(c)
    d, N = c.ndim, c.ncells
    rng = np.random.default_rng(7)
    target = rng.standard_normal((d, N))
    u0 = to_dev(dom, c.u0, d).requires_grad_(True)
    S = to_dev(dom, c.S, d).requires_grad_(True)
    nu = torch.tensor(c.nu, dtype=torch.float64, device="cuda", requires_grad=True)
    p0 = to_dev(dom, c.p0)
    u, p = u0, p0
    for _ in range(4):
        u, p = piso_step(dom, u, p, c.dt, nu, S)
    loss = ((u - to_dev(dom, target, d)) ** 2).sum()
    loss.backward()
    # oracle
    uo, po, tapes = c.u0, c.p0, []
    for _ in range(4):
        uo, po, t = O.piso_step(m, uo, po, c.dt, c.nu, c.S)
        tapes.append(t)
    gu, gp = 2 * (uo - target), np.zeros(N)
    gS, gnu = np.zeros((d, N)), 0.0
    for t in reversed(tapes):
        gu, gp, gs, gn = O.piso_step_adjoint(m, t, gu, gp)
        gS += gs
        gnu += gn
    assert rel_err(host(u0.grad), gu) <= 1e-7
    assert rel_err(host(S.grad), gS) <= 1e-7
    assert abs(float(nu.grad) - gnu) <= 1e-7 * abs(gnu)


def test_boundary_adjoint_matches_gpu_finite_difference():
    """dL/d(boundary values) on the multi-block step with inflow and advective
    outflow (App. A.4: boundary velocities are differentiable; the outflow
    update, Eq. advOut, is differentiated): <ubar, du1> along a perturbation
    of every boundary-face value, 4th-order central differences of the GPU
    forward, against the adjoint's directional derivative."""
    c = W.bfs2d(n_in=(16, 8), n_ch=32, n_out=16, half=8, dt=0.02)
    dom = gpu_domain(c, p_rtol=1e-12)
    d, N = c.ndim, c.ncells
    rng = np.random.default_rng(12)
    u0 = to_dev(dom, c.u0 + 0.2 * rng.standard_normal((d, N)), d)
    p0 = to_dev(dom, c.p0)
    ubar = to_dev(dom, rng.standard_normal((d, N)), d)
    b0 = dom.get_boundary()
    db = rng.standard_normal(b0.shape)

    def L(t):
        dom.set_boundary(b0 + t * db)
        u1, _, _ = dom.step(u0, p0, c.dt, c.nu)
        return float((ubar * u1).sum())

    dom.set_boundary(b0)
    dom.step(u0, p0, c.dt, c.nu)
    dom.step_adjoint(ubar, None)
    adj = float(np.sum(dom.boundary_adjoint() * db))
    e = 1e-4
    fd = (8 * (L(e) - L(-e)) - (L(2 * e) - L(-2 * e))) / (12 * e)
    assert abs(adj - fd) <= 1e-6 * abs(fd), (adj, fd)


def test_adjoint_without_a_recorded_step_is_refused():
    """A NULL tape means the domain's own record of its last forward step: it
    must exist, else the call is out of order (PISO_ESTATE) instead of
    differentiating a stale or empty record."""
    c = W.cavity2d(16)
    dom = gpu_domain(c)
    d = c.ndim
    u, p = to_dev(dom, c.u0, d), to_dev(dom, c.p0)
    g = torch.ones_like(u)
    with pytest.raises(capi.PisoError) as e:          # no step yet
        dom.step_adjoint(g)
    assert e.value.status == 7               # PISO_ESTATE
    tape = dom.new_tape()
    dom.step(u, p, c.dt, c.nu, tape=tape)             # recorded into a caller tape only
    with pytest.raises(capi.PisoError) as e:
        dom.step_adjoint(g)
    assert e.value.status == 7               # PISO_ESTATE
    du_t = dom.step_adjoint(g, tape=tape)[0]          # the caller's tape works
    dom.step(u, p, c.dt, c.nu)                        # same step into the domain's own record
    du_w = dom.step_adjoint(g)[0]
    assert torch.equal(du_t, du_w)
