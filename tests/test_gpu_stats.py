"""Turbulence-statistics operators on the GPU vs the FP64 oracle (Sec. 2.5 and
Sec. 3.3 of arXiv:2505.16992), through the C ABI: plane records, their online
merge and adjoint, cell gradients, budget terms, the statistics loss and its
gradient through a PISO rollout."""
import math

import numpy as np
import pytest
import torch

import oracle as O
from oracle import stats as OS
from paper_2505_16992_b300 import capi
from paper_2505_16992_b300 import losses as LS
from paper_2505_16992_b300 import solver as SV
from paper_2505_16992_b300 import workloads as W
from gpu_util import gpu_domain, host, rel_err, to_dev

pytestmark = pytest.mark.gpu


def _rec_dict(stats, rec):
    n, mean, m2, m3 = stats.split(rec)
    return dict(n=host(n), mean=host(mean), m2=host(m2), m3=None if m3 is None else host(m3))


def _assert_rec(stats, rec, ref, tol):
    g = _rec_dict(stats, rec)
    assert np.array_equal(g["n"], ref["n"])
    for key in ("mean", "m2", "m3"):
        if ref.get(key) is None or g.get(key) is None:
            continue
        scale = max(np.abs(ref[key]).max(), 1e-300)
        assert np.abs(g[key] - ref[key]).max() <= tol * scale, (key, np.abs(g[key] - ref[key]).max() / scale)


def _fields(c, nq, seed, scale=1.0):
    rng = np.random.default_rng(seed)
    return scale * rng.standard_normal((nq, c.ncells)) + np.arange(nq)[:, None] * 0.5


@pytest.mark.parametrize("nq,order", [(3, 3), (9, 2), (6, 2), (1, 3), (4, 3), (12, 2)])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_frame_record_matches_oracle(nq, order, precision):
    c = W.channel3d(16, 12, 8)
    dom = gpu_domain(c, precision)
    st = SV.PlaneStats(dom, nq, order)
    q = _fields(c, nq, 1)
    qd = to_dev(dom, q, nq)
    ref = OS.frame_record(host(qd), c.blocks[0].res, order)     # the oracle on the same stored values
    _assert_rec(st, st.frame(qd), ref, 1e-12)


def test_frame_record_2d_and_ragged():
    c = W.cavity2d(13)
    dom = gpu_domain(c)
    st = SV.PlaneStats(dom, 2, 3)
    q = _fields(c, 2, 2)
    _assert_rec(st, st.frame(to_dev(dom, q, 2)), OS.frame_record(q, c.blocks[0].res, 3), 1e-12)


def test_online_accumulation_matches_oracle():
    c = W.channel3d(12, 10, 6)
    dom = gpu_domain(c)
    st = SV.PlaneStats(dom, 3, 3)
    frames = [_fields(c, 3, 10 + f, scale=1 + f) for f in range(6)]
    acc = st.empty()
    for q in frames:
        st.frame(to_dev(dom, q, 3), acc)
    ref = OS.accumulate([OS.frame_record(q, c.blocks[0].res) for q in frames])
    _assert_rec(st, acc, ref, 1e-12)
    # merging two partial accumulations equals the accumulation of all
    a, b = st.empty(), st.empty()
    for q in frames[:2]:
        st.frame(to_dev(dom, q, 3), a)
    for q in frames[2:]:
        st.frame(to_dev(dom, q, 3), b)
    st.merge(a, b)
    _assert_rec(st, a, ref, 1e-12)


@pytest.mark.parametrize("which", ["frame", "accumulated"])
def test_record_adjoint_matches_oracle(which):
    c = W.channel3d(12, 10, 6)
    dom = gpu_domain(c)
    st = SV.PlaneStats(dom, 3, 3)
    res = c.blocks[0].res
    frames = [_fields(c, 3, 20 + f) for f in range(3)]
    recs = [OS.frame_record(q, res) for q in frames]
    rec = recs[0] if which == "frame" else OS.accumulate(recs)
    rng = np.random.default_rng(5)
    gm, g2, g3 = (rng.standard_normal(rec["mean"].shape), rng.standard_normal(rec["m2"].shape),
                  rng.standard_normal(rec["m3"].shape))
    ref = OS.frame_record_adjoint(frames[0], res, rec, gm, g2, g3)
    ny = rec["mean"].shape[0]
    rec_t = torch.tensor(np.concatenate([rec["n"][:, None], rec["mean"], rec["m2"].reshape(ny, -1),
                                         rec["m3"].reshape(ny, -1)], axis=1), device="cuda")
    g_t = torch.tensor(np.concatenate([np.zeros((ny, 1)), gm, g2.reshape(ny, -1), g3.reshape(ny, -1)], axis=1),
                       device="cuda")
    dq = st.frame_adjoint(to_dev(dom, frames[0], 3), rec_t, g_t)
    assert rel_err(host(dq), ref) <= 1e-12


def test_cell_gradients_match_oracle():
    c = W.channel3d(12, 10, 6)
    m = O.mesh_from_case(c)
    dom = gpu_domain(c)
    rng = np.random.default_rng(6)
    u = rng.standard_normal((3, c.ncells))
    p = rng.standard_normal(c.ncells)
    gu, gp = SV.cell_gradients(dom, to_dev(dom, u, 3), to_dev(dom, p))
    ou, op = OS.cell_gradients(m, u, p)
    assert rel_err(host(gu), ou) <= 1e-12
    assert rel_err(host(gp), op) <= 1e-12
    # 2D multi-block with inflow values at Dirichlet faces
    c2 = W.bfs2d(n_in=(8, 4), n_ch=16, n_out=8, half=4)
    m2 = O.mesh_from_case(c2)
    d2 = gpu_domain(c2)
    u2 = rng.standard_normal((2, c2.ncells))
    gu2, _ = SV.cell_gradients(d2, to_dev(d2, u2, 2))
    ou2, _ = OS.cell_gradients(m2, u2, np.zeros(c2.ncells))
    assert rel_err(host(gu2), ou2) <= 1e-12


def test_budget_matches_oracle():
    c = W.channel3d(16, 12, 8)
    m = O.mesh_from_case(c)
    dom = gpu_domain(c)
    res = c.blocks[0].res
    rng = np.random.default_rng(7)
    frames = [(c.u0 + 0.1 * rng.standard_normal(c.u0.shape), rng.standard_normal(c.ncells)) for _ in range(3)]
    su, sg, sp = SV.PlaneStats(dom, 3, 3), SV.PlaneStats(dom, 9, 2), SV.PlaneStats(dom, 6, 2)
    au, ag, ap = su.empty(), sg.empty(), sp.empty()
    ru, rg, rp = [], [], []
    for u, p in frames:
        ut, pt = to_dev(dom, u, 3), to_dev(dom, p)
        gu, gp = SV.cell_gradients(dom, ut, pt)
        su.frame(ut, au)
        sg.frame(gu.reshape(9, -1), ag)
        sp.frame(torch.cat([ut, gp]), ap)
        ou, op = OS.cell_gradients(m, u, p)
        ru.append(OS.frame_record(u, res))
        rg.append(OS.frame_record(ou.reshape(9, -1), res, 2))
        rp.append(OS.frame_record(np.concatenate([u, op]), res, 2))
    b = c.blocks[0]
    yv = np.unique(b.vertices.reshape(-1, 3)[:, 1])
    xc = W.cell_centres(b)
    yc = np.array([xc[1][y * res[0]] for y in range(res[1])])
    ref = OS.budget(OS.accumulate(ru), OS.accumulate(rg), OS.accumulate(rp), yc, yv.min(), yv.max(), c.nu)
    got = SV.budget(su, au, sg, ag, sp, ap, c.nu)
    for key in ("P", "eps", "T", "D", "Pi"):
        assert rel_err(host(got[key]), ref[key]) <= 1e-10, key


def test_stats_loss_gradient_matches_oracle():
    """dL/dq of the statistics loss (time-averaged + per-frame terms) through
    the torch autograd functions vs the oracle's adjoint chain."""
    c = W.channel3d(12, 10, 6)
    dom = gpu_domain(c)
    st = SV.PlaneStats(dom, 3, 3)
    res = c.blocks[0].res
    frames = [_fields(c, 3, 30 + f) for f in range(3)]
    rng = np.random.default_rng(8)
    ref_mean = rng.standard_normal((res[1], 3))
    ref_m2 = rng.standard_normal((res[1], 3, 3))
    qs = [to_dev(dom, q, 3).requires_grad_(True) for q in frames]
    L = LS.stats_loss(st, qs, torch.tensor(ref_mean, device="cuda"), torch.tensor(ref_m2, device="cuda"),
                      lam_U=1.0, lam_uu=0.5, lam_frame=0.25)
    L.backward()
    recs = [OS.frame_record(q, res) for q in frames]
    L_ref = OS.stats_loss(recs, ref_mean, ref_m2, 1.0, 0.5, 0.25)
    assert abs(float(L) - L_ref) <= 1e-12 * abs(L_ref)
    ny = res[1]
    acc = OS.accumulate(recs)

    def g_of(rec, w):
        return (w * 2.0 * (rec["mean"] - ref_mean) / ny, w * 0.5 * 2.0 * (rec["m2"] - ref_m2) / ny)

    for f, q in enumerate(frames):
        gm, g2 = g_of(acc, 1.0)
        want = OS.frame_record_adjoint(q, res, acc, gm, g2, np.zeros_like(acc["m3"]))
        gm, g2 = g_of(recs[f], 0.25)
        want = want + OS.frame_record_adjoint(q, res, recs[f], gm, g2, np.zeros_like(acc["m3"]))
        assert rel_err(host(qs[f].grad), want) <= 1e-11


def test_stats_loss_through_rollout_matches_finite_differences():
    """L_stats of the frames of a 3-step PISO rollout (FP64): the gradient with
    respect to the initial velocity through the step adjoints and the record
    adjoints equals 4th-order central differences of the GPU forward."""
    c = W.channel3d(8, 8, 4)
    dom = gpu_domain(c)
    st = SV.PlaneStats(dom, 3, 3)
    S = to_dev(dom, c.S, 3)
    ny = c.blocks[0].res[1]
    rng = np.random.default_rng(9)
    ref_mean = torch.tensor(rng.standard_normal((ny, 3)) * 0.1, device="cuda")
    ref_m2 = torch.tensor(rng.standard_normal((ny, 3, 3)) * 0.01, device="cuda")

    def loss(u0, grad=False):
        u, p = u0, to_dev(dom, c.p0)
        frames = []
        for _ in range(3):
            u, p = SV.piso_step(dom, u, p, c.dt, c.nu, S)
            frames.append(u)
        return LS.stats_loss(st, frames, ref_mean, ref_m2, lam_frame=0.5)

    u0 = to_dev(dom, c.u0, 3).requires_grad_(True)
    L = loss(u0)
    L.backward()
    g = host(u0.grad)
    h = 1e-4
    for (comp, cell) in [(0, 5), (1, 77), (2, 130), (0, 200)]:
        vals = []
        for k in (2, 1, -1, -2):
            v = c.u0.copy()
            v[comp, cell] += k * h
            with torch.no_grad():
                vals.append(float(loss(to_dev(dom, v, 3))))
        fd = (-vals[0] + 8 * vals[1] - 8 * vals[2] + vals[3]) / (12 * h)
        assert abs(g[comp, cell] - fd) <= 1e-6 * max(abs(fd), 1e-8) + 1e-10, (comp, cell, g[comp, cell], fd)


def test_statistics_reject_bad_arguments():
    c = W.bfs2d(n_in=(8, 4), n_ch=16, n_out=8, half=4)
    dom = gpu_domain(c)
    with pytest.raises(capi.PisoError):
        SV.PlaneStats(dom, 2, 3)                    # multi-block
    c3 = W.channel3d(8, 6, 4)
    d3 = gpu_domain(c3)
    with pytest.raises(capi.PisoError):
        SV.PlaneStats(d3, 5, 3)                     # order 3 needs nq <= 4
    with pytest.raises(capi.PisoError):
        SV.PlaneStats(d3, 13, 2)
