"""The step at the above-L2 size the benchmark times (channel 256x192x128,
6.3 M cells, FP32, autotuned launch: four cells per thread in the Jacobi CG
and BiCGStab sweeps), through the C ABI.  The FP64 oracle cannot run this
size, so the checks are properties the discretisation of App. A has at any
size: a field that does not vary along a periodic direction stays so (the
translation invariance of the uniform periodic directions, which exercises
every wrap-around and quad boundary of the vectorised sweeps), and the
solves of the forward and adjoint steps reach their tolerances."""
import numpy as np
import pytest

from paper_2505_16992_b300 import capi
from paper_2505_16992_b300 import workloads as W
from gpu_util import gpu_domain, host, to_dev

pytestmark = pytest.mark.gpu

NX, NY, NZ = 256, 192, 128


def _case():
    return W.channel3d(NX, NY, NZ)


def _grid(c):
    xc, yc, zc = W.cell_centres(c.blocks[0])
    return xc, yc, zc


def _step(c, u0, p0, **opts):
    dom = gpu_domain(c, "fp32", adv_rtol=1e-6, p_rtol=1e-6, p_maxit=20000, adv_maxit=2000, **opts)
    dom.autotune(to_dev(dom, u0, 3), to_dev(dom, p0), c.dt, c.nu, to_dev(dom, c.S, 3))
    u1, p1, st = dom.step(to_dev(dom, u0, 3), to_dev(dom, p0), c.dt, c.nu, to_dev(dom, c.S, 3))
    assert st["status"] == "PISO_OK", st
    for k in range(2):
        assert st["p_resid"][k] <= 1e-6 * st["p_rhs_norm"][k] * 1.001, st
    return dom, host(u1).reshape(3, NZ, NY, NX), host(p1).reshape(NZ, NY, NX), st


def _spread(a, axis):
    """largest deviation along `axis` from the mean along it, relative to the
    field's largest magnitude"""
    return float(np.abs(a - a.mean(axis=axis, keepdims=True)).max() / max(np.abs(a).max(), 1e-30))


def test_large_channel_z_invariant_flow_stays_z_invariant():
    """A perturbation that varies in x and y but not in z: the step keeps
    every component z-invariant (w stays zero)."""
    c = _case()
    xc, yc, zc = _grid(c)
    u0 = np.zeros((3, c.ncells))
    u0[0] = 1.0 - yc ** 2 + 0.1 * np.sin(xc) * (1.0 - yc ** 2)
    u0[1] = 0.05 * np.cos(xc) * (1.0 - yc ** 2) ** 2
    dom, u1, p1, st = _step(c, u0, np.zeros(c.ncells), p_precond=capi.PISO_PRECOND_JACOBI)
    assert dom.uses_cg_vec4()
    for k in range(2):
        assert _spread(u1[k], 0) <= 1e-5, (k, _spread(u1[k], 0))
    assert np.abs(u1[2]).max() <= 1e-5 * np.abs(u1[0]).max()
    assert _spread(p1, 0) <= 1e-4, _spread(p1, 0)


def test_large_channel_x_invariant_flow_stays_x_invariant():
    """A perturbation that varies in y and z but not in x (the quads' left and
    right neighbours wrap around the periodic x direction): every component
    stays x-invariant."""
    c = _case()
    xc, yc, zc = _grid(c)
    u0 = np.zeros((3, c.ncells))
    u0[0] = 1.0 - yc ** 2 + 0.1 * np.sin(2.0 * zc) * (1.0 - yc ** 2)
    u0[2] = 0.05 * np.cos(2.0 * zc) * (1.0 - yc ** 2) ** 2
    dom, u1, p1, st = _step(c, u0, np.zeros(c.ncells), p_precond=capi.PISO_PRECOND_JACOBI)
    assert dom.uses_cg_vec4()
    for k in range(3):
        assert _spread(u1[k], 2) <= 1e-5, (k, _spread(u1[k], 2))
    assert _spread(p1, 2) <= 1e-4, _spread(p1, 2)


def test_large_channel_bench_state_solves_converge():
    """The benchmark's own initial state (laminar profile plus seeded noise):
    every solve of the step converges in the autotuned launch, and the adjoint
    step too."""
    c = _case()
    dom, u1, p1, st = _step(c, c.u0, c.p0)
    assert max(st["adv_iters"][:3]) > 0 and min(st["p_iters"][:2]) > 0
    import torch
    du, dp, dS, dnu, ast = dom.step_adjoint(torch.ones((3, c.ncells), dtype=torch.float32, device="cuda"), None)
    assert ast["status"] == "PISO_OK", ast
    assert np.isfinite(host(du)).all() and np.isfinite(dnu)
