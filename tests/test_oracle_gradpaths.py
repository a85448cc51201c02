"""Pins of the oracle's gradient-path variants (arXiv:2505.16992, Sec. 2.4 and
Sec. 4.3, Eq. jnone).

Leaving the advection path out treats u* as a constant of the backward pass;
leaving the pressure path out treats every corrector's pressure as one.  A
variant's adjoint must therefore be the exact adjoint of a *different forward
function*: the PISO step whose solves return their base-point results whatever
their inputs.  That function is built here by replacing the oracle's solvers
(not its adjoint), and its central finite differences pin the variants."""
import numpy as np
import pytest

import oracle as O
import oracle.piso as OP
from paper_2505_16992_b300 import workloads as W
from test_oracle_adjoint import fd4


def _case(name):
    if name == "cavity":
        return W.cavity2d(6, nu=0.05, dt=0.05)
    if name == "bfs":
        return W.bfs2d(n_in=(4, 3), n_ch=6, n_out=3, half=3, nu=0.01, dt=0.05)
    return W.channel3d(5, 4, 3, nu=0.02, dt=0.02)


def _frozen_solvers(monkeypatch, tape, freeze_adv, freeze_p):
    """Make the oracle's forward solves return the base point's solutions."""
    ustar = tape["ustar"].copy()
    xs = [cr["x"].copy() for cr in tape["corr"]]
    state = {"k": 0}
    real_C, real_P = OP.solve_C, OP.solve_P

    def solve_C(mesh, C, rhs, x0, opts):
        state["k"] = 0                     # the predictor starts each step
        if freeze_adv:
            return ustar.copy(), None
        return real_C(mesh, C, rhs, x0, opts)

    def solve_P(mesh, Pm, b, x0, opts):
        k = state["k"]
        state["k"] += 1
        if freeze_p:
            return xs[k].copy(), None
        return real_P(mesh, Pm, b, x0, opts)

    monkeypatch.setattr(OP, "solve_C", solve_C)
    monkeypatch.setattr(OP, "solve_P", solve_P)


@pytest.mark.parametrize("name", ["cavity", "bfs", "channel3d"])
@pytest.mark.parametrize("grad_adv,grad_p", [(False, True), (True, False), (False, False)])
def test_variant_adjoint_is_the_adjoint_of_the_frozen_step(monkeypatch, name, grad_adv, grad_p):
    c = _case(name)
    m = O.mesh_from_case(c)
    d, N = m.ndim, m.N
    rng = np.random.default_rng(21)
    u0 = c.u0 + 0.3 * rng.standard_normal((d, N))
    p0 = rng.standard_normal(N)
    S0 = rng.standard_normal((d, N)) if c.S is None else c.S + 0.1 * rng.standard_normal((d, N))
    ubar, pbar = rng.standard_normal((d, N)), rng.standard_normal(N)
    du, dS = rng.standard_normal((d, N)), rng.standard_normal((d, N))
    dnu = 0.3 * c.nu
    bval = O.outflow_update(m, u0, m.bval, c.dt)          # boundary values held fixed (R16)
    opts = O.Options(update_outflow=False)
    _, _, tape = O.piso_step(m, u0, p0, c.dt, c.nu, S0, bval, opts)
    vopts = O.Options(update_outflow=False, grad_adv=grad_adv, grad_p=grad_p)
    gu, gp, gS, gnu = O.piso_step_adjoint(m, tape, ubar, pbar, vopts)
    adj = float(np.sum(gu * du) + np.sum(gS * dS) + gnu * dnu)
    full = O.piso_step_adjoint(m, tape, ubar, pbar, opts)

    _frozen_solvers(monkeypatch, tape, freeze_adv=not grad_adv, freeze_p=not grad_p)

    def L(t):
        u1, p1, _ = O.piso_step(m, u0 + t * du, p0, c.dt, c.nu + t * dnu, S0 + t * dS, bval, opts)
        return float(np.sum(ubar * u1) + np.sum(pbar * p1))

    assert L(0.0) == pytest.approx(float(np.sum(ubar * tape["u_out"]) + np.sum(pbar * tape["p_out"])),
                                   rel=1e-12)
    fd = fd4(L, 1e-4)
    assert abs(adj - fd) <= 1e-6 * max(abs(fd), 1e-12), (adj, fd)
    # the variant really differs from the full adjoint (the dropped paths carry gradient)
    assert np.max(np.abs(full[0] - gu)) > 1e-6 * np.max(np.abs(full[0]))


def test_pressure_path_with_predictor_gradient_reading(monkeypatch):
    """With -grad p^n in the predictor (reading R4) p^n reaches u^{n+1} only
    through the advection solve: without that path dL/dp^n vanishes, and with
    it the frozen-pressure FD still pins dL/dp^n."""
    c = _case("cavity")
    m = O.mesh_from_case(c)
    rng = np.random.default_rng(3)
    u0 = 0.5 * rng.standard_normal((2, m.N))
    p0 = rng.standard_normal(m.N)
    ubar, pbar = rng.standard_normal((2, m.N)), rng.standard_normal(m.N)
    opts = O.Options(pred_grad_p=True)
    _, _, tape = O.piso_step(m, u0, p0, c.dt, c.nu, None, None, opts)
    g_none = O.piso_step_adjoint(m, tape, ubar, pbar, O.Options(pred_grad_p=True, grad_adv=False))
    assert np.all(g_none[1] == 0.0)
    g_adv = O.piso_step_adjoint(m, tape, ubar, pbar, O.Options(pred_grad_p=True, grad_p=False))
    _frozen_solvers(monkeypatch, tape, freeze_adv=False, freeze_p=True)
    dp = rng.standard_normal(m.N)

    def L(t):
        u1, p1, _ = O.piso_step(m, u0, p0 + t * dp, c.dt, c.nu, None, None, opts)
        return float(np.sum(ubar * u1) + np.sum(pbar * p1))

    fd = fd4(L, 1e-4)
    adj = float(np.sum(g_adv[1] * dp))
    assert abs(adj - fd) <= 1e-6 * max(abs(fd), 1e-12), (adj, fd)


def test_bypass_only_variant_runs_no_solve(monkeypatch):
    """With both paths left out the backward pass is linear work only (Eq.
    jnone): no transposed solve may run."""
    c = _case("bfs")
    m = O.mesh_from_case(c)
    rng = np.random.default_rng(4)
    _, _, tape = O.piso_step(m, c.u0, c.p0, c.dt, c.nu, c.S)

    def boom(*a, **k):
        raise AssertionError("a transposed solve ran")

    monkeypatch.setattr(OP, "solve_C_T", boom)
    monkeypatch.setattr(OP, "solve_P", boom)
    gu, gp, gS, gnu = O.piso_step_adjoint(m, tape, rng.standard_normal((2, m.N)), rng.standard_normal(m.N),
                                          O.Options(grad_adv=False, grad_p=False))
    assert np.all(np.isfinite(gu)) and np.any(gu != 0)
