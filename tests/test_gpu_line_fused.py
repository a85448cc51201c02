"""The y-line preconditioned pressure CG in its fused form (one group barrier
per iteration: each CTA also solves the halo lines next to its own) against the
FP64 oracle and against the split form (two barriers per iteration), through
the C ABI.  The form changes how the pressure systems of App. A.1
(Eq. pressure) are iterated, not the recurrences, so both forms must reproduce
the oracle's solves and agree with each other up to rounding."""
import numpy as np
import pytest

import oracle as O
from paper_2505_16992_b300 import capi
from paper_2505_16992_b300 import workloads as W
from gpu_util import FP32_REL, FP64_REL, gpu_domain, gpu_step, host, oracle_step, rel_err, to_dev

pytestmark = pytest.mark.gpu

LINE = capi.PISO_PRECOND_LINE

CASES = {
    "channel3d-16x12x8": lambda: W.channel3d(16, 12, 8),
    "channel3d-13x7x5": lambda: W.channel3d(13, 7, 5),
    "cavity2d-33": lambda: W.cavity2d(33),
    "cavity3d-5x5x3": lambda: W.cavity3d(5, nz=3),
    "periodic2d-64": lambda: W.turbulence2d(64),
    "bfs2d": lambda: W.bfs2d(n_in=(16, 8), n_ch=64, n_out=16, half=8, dt=0.02),
}


def _forward(case, split, precision="fp64", **opts):
    dom = gpu_domain(case, precision, p_precond=LINE, p_line_split=split, **opts)
    assert dom.uses_fused_lines() == (not split), "fused plan not taken"
    return dom, gpu_step(dom, case, case.u0, case.p0, case.S)


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("ctas", [0, 5, 12])
def test_fused_forward_parity(name, ctas):
    """Own lines cut from strips of columns, halo lines across block joints
    (the step's blocks meet in x and in y), periodic wraps in x, y and z."""
    c = CASES[name]()
    _, (ug, pg, st) = _forward(c, 0, ctas=ctas, p_rtol=1e-12 if name == "bfs2d" else 1e-13)
    assert st["status"] == "PISO_OK", st
    uo, po, _ = oracle_step(O.mesh_from_case(c), c, c.u0, c.p0, c.S)
    assert rel_err(ug, uo) <= FP64_REL, rel_err(ug, uo)
    assert rel_err(pg, po) <= 10 * FP64_REL, rel_err(pg, po)


def test_one_line_per_cta():
    """As many CTAs as lines: every CTA owns one line and solves its four
    neighbours' lines as halo."""
    c = W.channel3d(8, 12, 4)
    _, (ug, pg, st) = _forward(c, 0, ctas=32, block_threads=128)
    assert st["status"] == "PISO_OK", st
    uo, po, _ = oracle_step(O.mesh_from_case(c), c, c.u0, c.p0, c.S)
    assert rel_err(ug, uo) <= FP64_REL and rel_err(pg, po) <= 10 * FP64_REL


@pytest.mark.parametrize("name", ["channel3d-16x12x8", "bfs2d", "periodic2d-64"])
def test_fused_matches_split(name):
    """Same recurrences: the two forms agree to rounding and take the same
    number of iterations (up to one at the tolerance boundary)."""
    c = CASES[name]()
    _, (uf, pf, sf) = _forward(c, 0, p_rtol=1e-12)
    _, (us, ps, ss) = _forward(c, 1, p_rtol=1e-12)
    assert rel_err(uf, us) <= 1e-12 and rel_err(pf, ps) <= 1e-10
    for k in range(2):
        assert abs(sf["p_iters"][k] - ss["p_iters"][k]) <= 1, (sf["p_iters"], ss["p_iters"])


def test_full_size_channel_fused():
    """The 64x48x32 channel, FP64 and FP32 (the mixed-precision arm), as the
    bench runs it: parity with the oracle and the split form's iteration
    counts."""
    c = W.channel3d()
    uo, po, _ = oracle_step(O.mesh_from_case(c), c, c.u0, c.p0, c.S)
    # 128 CTAs of 16 lines (the autotuned shape)
    _, (ug, pg, st) = _forward(c, 0, ctas=128)
    assert rel_err(ug, uo) <= FP64_REL and rel_err(pg, po) <= 10 * FP64_REL
    _, (u2, p2, s2) = _forward(c, 1, ctas=128)
    for k in range(2):
        assert abs(st["p_iters"][k] - s2["p_iters"][k]) <= 1, (st["p_iters"], s2["p_iters"])
    _, (u3, p3, s3) = _forward(c, 0, "fp32", block_threads=768, ctas=128, adv_rtol=1e-6, p_rtol=1e-6)
    assert s3["status"] == "PISO_OK", s3
    assert rel_err(u3, uo) <= FP32_REL, rel_err(u3, uo)


def test_fused_fp32_refined():
    c = W.channel3d(16, 12, 8)
    _, (ug, pg, st) = _forward(c, 0, "fp32", adv_rtol=1e-6, p_refine_rtol=1e-10, p_inner_rtol=1e-4)
    assert st["status"] == "PISO_OK" and min(st["p_rounds"][:2]) >= 1, st
    uo, po, _ = oracle_step(O.mesh_from_case(c), c, c.u0, c.p0, c.S)
    assert rel_err(ug, uo) <= 2e-6 and rel_err(pg, po) <= 2e-5


def test_fused_bitwise_deterministic():
    c = W.channel3d(16, 12, 8)
    dom, a = _forward(c, 0)
    b = gpu_step(dom, c, c.u0, c.p0, c.S)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


@pytest.mark.parametrize("name", ["channel3d-16x12x8", "bfs2d"])
def test_fused_adjoint_matches_oracle(name):
    """The adjoint's transposed pressure solves (P is symmetric) run the fused
    CG too."""
    c = CASES[name]()
    m = O.mesh_from_case(c)
    dom = gpu_domain(c, p_precond=LINE, p_rtol=1e-13 if c.ndim == 3 else 1e-12)
    assert dom.uses_fused_lines()
    rng = np.random.default_rng(12)
    d = c.ndim
    gu, gp = rng.standard_normal((d, c.ncells)), rng.standard_normal(c.ncells)
    S = None if c.S is None else to_dev(dom, c.S, d)
    dom.step(to_dev(dom, c.u0, d), to_dev(dom, c.p0), c.dt, c.nu, S)
    du, dp, dS, dnu, st = dom.step_adjoint(to_dev(dom, gu, d), to_dev(dom, gp))
    assert st["status"] == "PISO_OK", st
    _, _, tape = oracle_step(m, c, c.u0, c.p0, c.S)
    ou, op, oS, onu = O.piso_step_adjoint(m, tape, gu, gp)
    assert rel_err(host(du), ou) <= 1e-8
    if dS is not None:
        assert rel_err(host(dS), oS) <= 1e-8
    assert abs(dnu - onu) <= 1e-8 * max(abs(onu), 1e-30) + 1e-12


def test_where_the_fused_form_runs():
    c = W.channel3d(16, 12, 8)
    assert gpu_domain(c, p_precond=LINE).uses_fused_lines()
    assert not gpu_domain(c, p_precond=LINE, p_line_split=1).uses_fused_lines()
    assert not gpu_domain(c, p_precond=capi.PISO_PRECOND_JACOBI).uses_fused_lines()
    # one CTA holding all 1,024 lines of a 32x24x32 channel: no room, split form
    big = W.channel3d(32, 24, 32)
    dom = gpu_domain(big, p_precond=LINE, ctas=1, block_threads=256)
    assert dom.uses_line_precond() and not dom.uses_fused_lines()
