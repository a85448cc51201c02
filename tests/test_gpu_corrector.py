"""The 128^2 periodic box with a learned corrector: a 3-layer 3x3-conv corrector produces the source S of every step
of a differentiable rollout on 2D forced turbulence (Sec. 3: learned
corrections enter as the source term; Sec. 2.3: gradients through the solver).
Gradients w.r.t. the network parameters are checked against finite
differences, and the FP32 configuration-size loop trains."""
import numpy as np
import pytest
import torch
import torch.nn as nn
import torch.nn.functional as F

from paper_2505_16992_b300 import workloads as W
from paper_2505_16992_b300.solver import rollout
from gpu_util import gpu_domain, to_dev

pytestmark = pytest.mark.gpu


class Corrector(nn.Module):
    """2 -> ch -> ch -> 2 channels, 3x3 kernels, circular padding, ReLU (tanh
    for the finite-difference check, which needs a smooth network)."""

    def __init__(self, ch, dtype, act=torch.relu):
        super().__init__()
        self.act = act
        self.c1 = nn.Conv2d(2, ch, 3, dtype=dtype)
        self.c2 = nn.Conv2d(ch, ch, 3, dtype=dtype)
        self.c3 = nn.Conv2d(ch, 2, 3, dtype=dtype)

    def forward(self, u, n):
        x = u.reshape(1, 2, n, n)
        for k, c in enumerate((self.c1, self.c2, self.c3)):
            x = c(F.pad(x, (1, 1, 1, 1), mode="circular"))
            if k < 2:
                x = self.act(x)
        return 0.1 * x.reshape(2, n * n)


def _loss(dom, case, net, n, steps, target):
    u = to_dev(dom, case.u0, 2)
    p = to_dev(dom, case.p0)
    S0 = to_dev(dom, case.S, 2)
    u, p = rollout(dom, u, p, case.dt, case.nu, steps, source_fn=lambda v: S0 + net(v, n))
    return ((u - target) ** 2).mean()


def test_corrector_gradients_match_finite_differences():
    n, steps = 24, 4
    case = W.turbulence2d(n, nu=0.01, dt=0.02)
    dom = gpu_domain(case)
    torch.manual_seed(2)
    net = Corrector(6, torch.float64, act=torch.tanh).cuda()
    rng = np.random.default_rng(3)
    target = to_dev(dom, rng.standard_normal((2, n * n)), 2)
    loss = _loss(dom, case, net, n, steps, target)
    grads = torch.autograd.grad(loss, list(net.parameters()))
    dirs = [torch.randn_like(q) for q in net.parameters()]
    adj = sum(float((g * d).sum()) for g, d in zip(grads, dirs))

    def L(t):
        with torch.no_grad():
            for q, d in zip(net.parameters(), dirs):
                q.add_(t * d)
            v = float(_loss(dom, case, net, n, steps, target))
            for q, d in zip(net.parameters(), dirs):
                q.sub_(t * d)
        return v

    e = 1e-4
    fd = (8 * (L(e) - L(-e)) - (L(2 * e) - L(-2 * e))) / (12 * e)
    assert abs(adj - fd) <= 1e-6 * abs(fd), (adj, fd)


def test_corrector_training_periodic_box_fp32():
    """128x128 periodic forced turbulence, 16-step rollout, 32-channel FP32
    corrector, MSE to a seeded target: a few Adam steps reduce the loss."""
    n, steps = 128, 16
    case = W.turbulence2d(n)
    dom = gpu_domain(case, "fp32", adv_rtol=1e-6, p_rtol=1e-6)
    torch.manual_seed(2)
    net = Corrector(32, torch.float32).cuda()
    rng = np.random.default_rng(3)
    target = to_dev(dom, W.turbulence2d(n, seed=3).u0, 2)
    opt = torch.optim.Adam(net.parameters(), lr=1e-3)
    losses = []
    for _ in range(4):
        opt.zero_grad()
        loss = _loss(dom, case, net, n, steps, target)
        loss.backward()
        opt.step()
        losses.append(float(loss))
    assert all(np.isfinite(losses))
    assert losses[-1] < losses[0]
