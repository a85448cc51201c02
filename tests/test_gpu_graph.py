"""A single domain's forward and adjoint steps captured in one CUDA graph and
replayed (the launch-bound inner loop of a training rollout without a
per-step host round trip), through the C ABI: the replays equal the eager
launches bit for bit, and a graph of several chained steps equals the same
steps launched one by one."""
import pytest
import torch

from paper_2505_16992_b300 import capi
from paper_2505_16992_b300 import workloads as W
from gpu_util import gpu_domain, to_dev

pytestmark = pytest.mark.gpu


def _setup(precond):
    c = W.channel3d(16, 12, 8)
    dom = gpu_domain(c, "fp32", adv_rtol=1e-6, p_rtol=1e-6, p_precond=precond)
    u, p, S = to_dev(dom, c.u0, 3), to_dev(dom, c.p0), to_dev(dom, c.S, 3)
    g = torch.randn(u.shape, generator=torch.Generator().manual_seed(3), dtype=u.dtype).cuda()
    return c, dom, u, p, S, g


@pytest.mark.parametrize("precond", [capi.PISO_PRECOND_LINE, capi.PISO_PRECOND_JACOBI])
def test_step_and_adjoint_in_cuda_graph(precond):
    c, dom, u, p, S, g = _setup(precond)
    uo, po = torch.empty_like(u), torch.empty_like(p)
    du, dS = torch.empty_like(u), torch.empty_like(u)
    # eager reference
    ru, rp, _ = dom.step(u, p, c.dt, c.nu, S)
    rdu, _, rdS, _, _ = dom.step_adjoint(g, None)
    ru, rp, rdu, rdS = ru.clone(), rp.clone(), rdu.clone(), rdS.clone()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):      # warm the side stream outside the capture
        dom.step(u, p, c.dt, c.nu, S, u_out=uo, p_out=po, sync=False)
        dom.step_adjoint(g, None, sync=False, du_in=du, dS=dS)
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        dom.step(u, p, c.dt, c.nu, S, u_out=uo, p_out=po, sync=False)
        dom.step_adjoint(g, None, sync=False, du_in=du, dS=dS)
    for _ in range(2):
        for t in (uo, po, du, dS):
            t.zero_()
        graph.replay()
        torch.cuda.synchronize()
        assert torch.equal(uo, ru) and torch.equal(po, rp)
        assert torch.equal(du, rdu) and torch.equal(dS, rdS)


def test_graph_of_chained_steps_equals_eager_rollout():
    """Three forward steps chained inside one graph (each reads the previous
    step's output buffers) equal three eager steps."""
    c, dom, u, p, S, _ = _setup(capi.PISO_PRECOND_AUTO)
    bufs = [(torch.empty_like(u), torch.empty_like(p)) for _ in range(3)]
    eu, ep = u, p
    for _ in range(3):
        eu, ep, st = dom.step(eu, ep, c.dt, c.nu, S)
        assert st["status"] == "PISO_OK"
    eu, ep = eu.clone(), ep.clone()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        dom.step(u, p, c.dt, c.nu, S, u_out=bufs[0][0], p_out=bufs[0][1], sync=False)
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        prev = (u, p)
        for k in range(3):
            dom.step(prev[0], prev[1], c.dt, c.nu, S, u_out=bufs[k][0], p_out=bufs[k][1], sync=False)
            prev = bufs[k]
    graph.replay()
    torch.cuda.synchronize()
    assert torch.equal(bufs[2][0], eu) and torch.equal(bufs[2][1], ep)
