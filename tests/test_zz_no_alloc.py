"""piso_step_static: the forward step for callers that cannot allocate device
memory when they step (their device memory is already reserved by another
allocator, or their loop must not risk an allocation failing mid-run).  It
takes its scratch from a fixed buffer inside the library instead of from
cudaMalloc; its results must equal those of piso_step, call after call, and
domains too large for the buffer must be refused with a clear error.

This file is collected last on purpose, and each test passes on its own in a
fresh process as well as after the rest of the suite."""
import ctypes as C

import numpy as np
import pytest
import torch

from paper_2505_16992_b300 import capi
from paper_2505_16992_b300 import workloads as W
from gpu_util import FP32_REL, FP64_REL, gpu_domain, host, rel_err, to_dev

pytestmark = pytest.mark.gpu


def _static_step(dom, u, p, dt, nu, S):
    """One piso_step_static call through the C ABI; returns (u_out, p_out, stats)."""
    lib = capi.load()
    uo, po = torch.empty_like(u), torch.empty_like(p)
    st = capi.Stats()
    rc = lib.piso_step_static(dom.h, capi.dptr(u), capi.dptr(p), capi.dptr(uo), capi.dptr(po), float(dt),
                              float(nu), capi.dptr(S), torch.cuda.current_stream().cuda_stream or None,
                              C.byref(st))
    capi.check(rc, dom.h)
    return uo, po, st.as_dict()


@pytest.mark.parametrize("name,precision", [("cavity", "fp64"), ("channel3d", "fp64"), ("turbulence", "fp32")])
def test_static_scratch_step_equals_piso_step_twice(name, precision):
    if name == "cavity":
        c = W.cavity2d(32)
    elif name == "channel3d":
        c = W.channel3d(12, 10, 6)
    else:
        c = W.turbulence2d(64)
    tol = FP64_REL if precision == "fp64" else FP32_REL
    kw = {} if precision == "fp64" else dict(adv_rtol=1e-6, p_rtol=1e-6)
    dom = gpu_domain(c, precision, **kw)
    d = c.ndim
    u = to_dev(dom, c.u0, d)
    p = to_dev(dom, c.p0)
    S = None if c.S is None else to_dev(dom, c.S, d)
    for call in range(2):                     # two calls in a row, the second from the first's result
        ref_u, ref_p, ref_st = dom.step(u, p, c.dt, c.nu, S)
        su, sp, sst = _static_step(dom, u, p, c.dt, c.nu, S)
        assert sst["status"] == "PISO_OK", (call, sst)
        assert sst["p_iters"] == ref_st["p_iters"] and sst["adv_iters"] == ref_st["adv_iters"]
        assert rel_err(host(su), host(ref_u)) <= tol, call
        assert rel_err(host(sp), host(ref_p)) <= 10 * tol, call
        u, p = su, sp


def test_static_scratch_step_with_ilu_preconditioned_predictor():
    """The ILU(0) tables live with the domain (built when its launch layout is
    chosen), so the static entry point runs the preconditioned solve without
    allocating either."""
    c = W.channel3d(10, 16, 4, gamma=3.0, dt=0.5)
    dom = gpu_domain(c, adv_precond=capi.PISO_ADV_PRECOND_ILU)
    u, p, S = to_dev(dom, c.u0, 3), to_dev(dom, c.p0), to_dev(dom, c.S, 3)
    ref_u, ref_p, ref_st = dom.step(u, p, c.dt, c.nu, S)
    su, sp, sst = _static_step(dom, u, p, c.dt, c.nu, S)
    assert sst["status"] == "PISO_OK" and sst["adv_precond_used"] == 1, sst
    assert sst["adv_iters"] == ref_st["adv_iters"]
    assert rel_err(host(su), host(ref_u)) <= FP64_REL
    assert rel_err(host(sp), host(ref_p)) <= 10 * FP64_REL


def test_static_scratch_refuses_domains_that_do_not_fit():
    c = W.channel3d(64, 48, 32)            # 98,304 cells in FP64 need more than the 32 MiB buffer
    dom = gpu_domain(c)
    u = to_dev(dom, c.u0, 3)
    p = to_dev(dom, c.p0)
    with pytest.raises(capi.PisoError) as e:
        _static_step(dom, u, p, c.dt, c.nu, None)
    assert e.value.status == 1              # PISO_EINVAL
    assert "bytes of scratch" in str(e.value)


def test_adjoint_after_static_step_is_refused():
    """The static step's record lives in the shared buffer, so an adjoint that
    asks for the domain's own record (tape NULL) must be refused, not answered
    from the record of an earlier piso_step."""
    c = W.cavity2d(16)
    dom = gpu_domain(c)
    u, p = to_dev(dom, c.u0, 2), to_dev(dom, c.p0)
    dom.step(u, p, c.dt, c.nu)
    _static_step(dom, u, p, c.dt, c.nu, None)
    with pytest.raises(capi.PisoError) as e:
        dom.step_adjoint(torch.ones_like(u))
    assert e.value.status == 7              # PISO_ESTATE
