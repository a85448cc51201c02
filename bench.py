"""Benchmark: PISO steps/s on the 3D periodic channel 64x48x32 (tanh walls,
gamma 2, nu = 1/180, dt = 0.01, laminar profile + seeded perturbation 0.1).

One bench step = one forward PISO step followed by its adjoint (the whole hot
path).  Prints one JSON line (see the repository's design notes for every key).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision fp32|fp64]
                  [--mode fwd|fwdadj] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

L2_FLUSH_BYTES = 256 << 20          # > 126 MB L2


# ---------------------------------------------------------------------------
# algorithmic traffic model: every array a phase touches, counted once per
# phase (neighbour re-reads are cache hits), in words per cell
# ---------------------------------------------------------------------------
def cg_words_per_cell(d: int, it_p: int, line: bool, fused: bool = False) -> float:
    """Stored-array words per cell of one pressure CG solve (start + iterations).
    Jacobi (one phase per iteration): r, w, s, 1/diag, p, x, P faces read; p, x,
    s, r, w written.  y-line, split form (two phases): phase A reads u, w, r, x,
    p, s and the three line factors and writes p, s, x, r, u; phase B reads u and
    the P faces and writes w.  y-line, fused form (one phase; u, p, x, the line
    factors, the P faces, and r and s of the own and halo lines stay in shared
    memory for the whole solve): w written by its owner and read back by the
    halo lines; its start reads x, b, the P faces and the three factors and
    writes r0, then reads r0 and writes w0; x is written every iteration."""
    if line and fused:
        return (d + 7) + 2 + it_p * 3
    if line:
        return (d + 7) + (d + 2) + it_p * (14 + d + 2)
    return (d + 4) + (d + 3) + it_p * (d + 11)


def bicg_words_per_cell(d: int, it_a: int, ilu: bool) -> float:
    """Stored-array words per cell of one BiCGStab solve.  Plain: BA 8d+1, BB
    5d+1, BC 8d per iteration.  ILU(0)-preconditioned (five phases): PA r, p, v
    in, p out, then the two triangular sweeps (level order, mask and pivot
    1.5 + 1 words, the C row 2d+1, y written, read and rewritten) 11d+7; PB C,
    y, rhat -> v 5d+1; PC r, v in and the sweeps 9d+7; PD C, z, r, v -> t 6d+1;
    PE r, v, y, z, t, rhat, x -> x, r 9d; plus the factorisation once per solve
    (level order, mask, C row and the transposed entries, pivot out) 4d+3.5."""
    if ilu:
        return (4 * d + 3.5) + it_a * (40 * d + 16)
    return it_a * (21 * d + 2)


def fwd_words_per_cell(d: int, adv_iters, p_iters, line: bool = False, ilu: bool = False,
                       fused: bool = False) -> float:
    """Stored-array words per cell one forward launch touches (each array once
    per phase; neighbour re-reads are cache hits).  One line per kernel phase."""
    it_a = max(adv_iters) if adv_iters else 0
    w = 0.0
    w += d * d + 3 * d + 1            # F1: u, T, J -> u^n copy, U
    w += 11 * d + 3                   # F2: u, S, U, alpha, J -> C (2d+1), 1/A, alpha/A, rhs0, r, rhat, u*
    w += bicg_words_per_cell(d, it_a, ilu)   # predictor BiCGStab
    for k, it_p in enumerate(p_iters):
        w += (d * d + 8 * d + 4) if k == 0 else (d * d + 6 * d + 4)   # C1: (P), h, J T.h
        w += d + 3                    # C2: divergence, x0
        if line and k == 0:
            w += 5                    # line factors: diag P, +y faces -> fa, fm, fc
        w += cg_words_per_cell(d, it_p, line, fused)
        w += d * d + 2 * d + 2        # C4: correction
    w += 3                            # final pressure
    return w


def adj_words_per_cell(d: int, adv_iters, p_iters, line: bool = False, ilu: bool = False,
                       fused: bool = False) -> float:
    it_a = max(adv_iters) if adv_iters else 0
    w = 6 * d + 3                     # R0 extra on the first pass: rebuild P, clear accumulators
    if line and any(p_iters):
        w += 5                        # line factors of the rebuilt P
    for it_p in p_iters:
        w += d * d + 2 * d + 4        # R0: W = T gu / A, dL/dA
        w += d + 3                    # R1: -G^T W
        w += cg_words_per_cell(d, it_p, line, fused)   # CG on P
        w += d * d + 7 * d + 6        # R3: d(alpha/A), div^T y, gg, dL/dA, dL/drhs0
        w += 9 * d                    # R4: -H^T gg, dL/dH
    w += 6 * d + 3                    # R5: start of the C^T solve
    w += bicg_words_per_cell(d, it_a, ilu)   # BiCGStab on C^T
    w += 9 * d + 3                    # R6: dL/dC from the predictor, dS, du (1/dt part)
    w += d * d + 5 * d + 3            # R7: assembly adjoint
    return w


# ---------------------------------------------------------------------------
def clocks_sampler_start(path):
    q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    try:
        f = open(path, "w")
        return subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                 "-lms", "20"], stdout=f, stderr=subprocess.DEVNULL), f
    except Exception:
        return None, None


def clocks_sampler_stop(proc, f, path, gpu_index=0):
    if proc is None:
        return None
    proc.terminate()
    try:
        proc.wait(timeout=5)
    except Exception:
        proc.kill()
    f.close()
    sm, mx, reasons = [], None, set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for line in open(path):
        parts = [x.strip() for x in line.split(",")]
        if len(parts) < 9 or parts[0] != str(gpu_index):
            continue
        try:
            sm.append(float(parts[1]))
            mx = float(parts[2])
        except ValueError:
            continue
        for n, v in zip(names, parts[5:9]):
            if v.lower().startswith("active"):
                reasons.add(n)
    if not sm:
        return None
    return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
            "samples": len(sm)}


def whole_job_value(total_s: float, steps: int, world: int, dist=None, device="cuda") -> float:
    """Replicas: every rank times its own K steps; the job's throughput is the
    units all ranks processed over the slowest rank's time."""
    if dist is not None and world > 1:
        import torch
        t = torch.tensor([total_s], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_s = float(t.item())
    return world * steps / total_s


# the headers fwd_kernel and adj_kernel are compiled from (the statistics
# kernels' header is not among them)
STEP_KERNEL_HEADERS = ("piso_device.cuh", "piso_krylov.cuh", "piso_lines.cuh", "piso_ilu.cuh", "piso_nonortho.cuh",
                       "piso_forward.cuh",
                       "piso_adjoint.cuh")


def kernel_sources_hash() -> str:
    """Hash of the step kernels' sources: a recorded ncu traffic figure is used
    only while it matches."""
    import hashlib
    h = hashlib.sha256()
    for name in STEP_KERNEL_HEADERS:
        h.update(open(os.path.join(ROOT, "paper_2505_16992_b300", "csrc", name), "rb").read())
    return h.hexdigest()[:16]


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        j = json.load(open(p))
        return float(j["hbm_gbs"]), "measured"
    return 6400.0, "fallback"


# ---------------------------------------------------------------------------
# the CPU oracle: single-core and all-core timings, and the fields the GPU
# path is compared with (the oracle is test infrastructure; this leg is the
# only place the benchmark runs it)
# ---------------------------------------------------------------------------
def _oracle_worker(job):
    """Run the FP64 oracle, as it stands, on a bounded sample of the channel:
    fwd+adjoint steps (adjoint seeds dL/du^{n+1} = 1, dL/dp^{n+1} = 0) along the
    rollout from the seeded initial state (each step from the previous one's
    output), first `warmup` untimed steps, then until the step cap or the time
    budget; Krylov solves to `rtol` (None: the oracle's default 1e-13).
    Returns (steps, seconds of the step loop, fields of the last step or None,
    per-step seconds)."""
    seconds_budget, steps_cap, want_fields, size, rtol, warmup = job
    import numpy as np
    import oracle as O
    from paper_2505_16992_b300 import workloads as W
    case = W.channel3d(*size)
    m = O.mesh_from_case(case)
    oo = O.Options(adv_rtol=rtol, p_rtol=rtol) if rtol else O.Options()
    u, p = case.u0, case.p0
    n = 0
    fields = None
    times = []

    def one(u, p):
        u1, p1, tape = O.piso_step(m, u, p, case.dt, case.nu, case.S, None, oo)
        gu, gp, gS, gnu = O.piso_step_adjoint(m, tape, np.ones_like(u1), np.zeros_like(p1), oo)
        return u1, p1, dict(u=u1, p=p1, du=gu, dS=gS, dnu=gnu)

    for _ in range(warmup):
        u, p, _ = one(u, p)
    t0 = time.perf_counter()
    while n < steps_cap:
        ts = time.perf_counter()
        u, p, f = one(u, p)
        times.append(time.perf_counter() - ts)
        n += 1
        if want_fields:
            fields = f
        if time.perf_counter() - t0 > seconds_budget:
            break
    return n, time.perf_counter() - t0, fields, times


def _oracle_pool(workers, job):
    """Run ``workers`` copies of _oracle_worker(job) in fresh (spawned)
    processes with single-threaded numerical libraries; returns the results."""
    import multiprocessing as mp
    env_keys = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")
    saved = {k: os.environ.get(k) for k in env_keys}
    for k in env_keys:
        os.environ[k] = "1"
    try:
        ctx = mp.get_context("spawn")
        with ctx.Pool(workers) as pool:
            return pool.map(_oracle_worker, [job] * workers)
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v


def cpu_baseline(seconds_budget=20.0, steps_cap=3, size=(64, 48, 32), rtol=None, want_fields=True):
    """The oracle on one host core (steps/s) and its fields after the last step."""
    n, dt, fields, _ = _oracle_pool(1, (seconds_budget, steps_cap, want_fields, size, rtol, 0))[0]
    return n / dt, n, dt, fields


def cpu_baseline_all_cores(seconds_budget=15.0, max_workers=64, size=(64, 48, 32), rtol=None):
    """Independent copies of the oracle on every host core (one process each,
    capped at max_workers), one or more fwd+adjoint steps each: aggregate
    steps/s = all steps / the slowest copy's step-loop time."""
    nproc = os.cpu_count() or 1
    workers = max(1, min(nproc, max_workers))
    res = _oracle_pool(workers, (seconds_budget, 1, False, size, rtol, 0))
    steps = sum(r[0] for r in res)
    slowest = max(r[1] for r in res)
    return steps / slowest, workers, nproc, steps, slowest


HEADLINE_RTOL = 1e-6     # relative residual of every Krylov solve of the timed workload
HEADLINE_WORKLOAD = ("channel3d 64x48x32, x/z periodic, tanh walls gamma 2, nu 1/180, dt 0.01, "
                     "laminar + N(0,0.1^2) perturbation (seed 0)")
ROLLOUT_STATE = "advances: each timed step starts from the previous step's output"


def run_reference(args):
    """The CPU oracle as the reference arm (rank 0 only): the headline workload
    at its Krylov tolerance, advanced along the rollout as the timed GPU steps
    are, one untimed step first, then up to --steps timed steps within a
    bounded budget (about two minutes of one host core)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    from paper_2505_16992_b300 import workloads as W
    case = W.channel3d()
    n, _, _, times = _oracle_pool(1, (120.0, max(args.steps, 1), False, (64, 48, 32), HEADLINE_RTOL, 1))[0]
    value = n / sum(times)
    line = {"metric": "PISO steps/s (fwd+adjoint), 64x48x32 channel", "value": value,
            "unit": "steps/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * sum(times) / n, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": HEADLINE_WORKLOAD, "cells": case.ncells, "precision": "fp64",
                       "krylov_rtol": HEADLINE_RTOL, "state": ROLLOUT_STATE, "parallelism": "single"},
            "cpu_baseline": {"value": value, "unit": "steps/s", "cores": 1, "kind": "oracle",
                             "sample": f"{n} timed fwd+adjoint steps along the rollout after one untimed "
                                       f"step (budget 120 s of one core; --steps {args.steps} asked)"},
            "e2e": {"value": value, "unit": "steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


class Arm:
    """One configuration of the step on one workload: its domain (launch shape
    and pressure preconditioner autotuned unless a CTA width is given), the
    seeded fields, and timing along the rollout."""

    def __init__(self, case, prec, opts_kw, threads=0):
        import torch
        from paper_2505_16992_b300 import capi
        from paper_2505_16992_b300.solver import Domain
        self.case, self.prec = case, prec
        kw = dict(p_maxit=20000, adv_maxit=2000, block_threads=threads)
        kw.update(opts_kw)
        self.dom = dom = Domain.from_case(case, prec, capi.default_options(**kw))
        d = case.ndim
        self.u0, self.p0 = dom.field(case.u0, d), dom.field(case.p0)
        self.S = None if case.S is None else dom.field(case.S, d)
        if threads == 0:
            self.shape = dom.autotune(self.u0, self.p0, case.dt, case.nu, self.S)
        else:
            self.shape = (threads, opts_kw.get("ctas") or None, None)
        pc = dom.get_options().p_precond
        if pc == capi.PISO_PRECOND_AUTO:
            pc = capi.PISO_PRECOND_LINE if dom.uses_line_precond() else capi.PISO_PRECOND_JACOBI
        self.pc_used = "y-line" if pc == capi.PISO_PRECOND_LINE else "jacobi"
        # y-line CG iteration form: one group barrier per iteration (fused) or two
        self.line_form = None if self.pc_used != "y-line" else ("fused" if dom.uses_fused_lines() else "split")
        self.g = torch.ones_like(self.u0)          # adjoint seed dL/du^{n+1} = 1
        self.w = 4 if prec == "fp32" else 8

    def _step(self, u, p, uo, po, with_adj, sync):
        st = self.dom.step(u, p, self.case.dt, self.case.nu, self.S, u_out=uo, p_out=po, sync=sync)[2]
        ast = self.dom.step_adjoint(self.g, None, sync=sync)[4] if with_adj else None
        return st, ast

    def run(self, steps, warmup, flush, with_adj, on_start=None, on_end=None):
        """Warm-up steps, then ``steps`` timed steps, each starting from the
        previous step's output (the flow advances as in a rollout), each
        bracketed by CUDA events on the launching stream with an untimed L2
        flush before it; then the same steps replayed untimed from the same
        state with statistics read back (the kernels are deterministic, so the
        replay has the timed steps' iteration counts)."""
        import torch
        stream = torch.cuda.current_stream()
        u, p = self.u0.clone(), self.p0.clone()
        uo, po = torch.empty_like(u), torch.empty_like(p)
        for _ in range(warmup):
            self._step(u, p, uo, po, with_adj, False)
            u, uo, p, po = uo, u, po, p
        start = (u.clone(), p.clone())
        torch.cuda.synchronize()
        ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(steps)]
        if on_start:
            on_start()
        torch.cuda.synchronize()
        for k in range(steps):
            flush.fill_(float(k))                       # L2 flush between timed steps (not timed)
            ev[k][0].record(stream)
            self.dom.step(u, p, self.case.dt, self.case.nu, self.S, u_out=uo, p_out=po, sync=False)
            ev[k][1].record(stream)
            if with_adj:
                self.dom.step_adjoint(self.g, None, sync=False)
            ev[k][2].record(stream)
            u, uo, p, po = uo, u, po, p
        torch.cuda.synchronize()
        if on_end:
            on_end()
        fwd_ms = [e[0].elapsed_time(e[1]) for e in ev]
        step_ms = [e[0].elapsed_time(e[2]) for e in ev]
        u, p = start
        uo, po = torch.empty_like(u), torch.empty_like(p)
        sts, asts = [], []
        for k in range(steps):
            st, ast = self._step(u, p, uo, po, with_adj, True)
            sts.append(st)
            asts.append(ast)
            u, uo, p, po = uo, u, po, p
        return dict(fwd_ms=fwd_ms, step_ms=step_ms, stats=sts, adj_stats=asts)

    def rollout_fields(self, n):
        """n fwd+adjoint steps from the seeded state (untimed): host u, p after
        the last step and dL/du^n, dL/dS, dL/dnu of its adjoint."""
        import torch
        u, p = self.u0.clone(), self.p0.clone()
        out = None
        for _ in range(n):
            u1, p1, st = self.dom.step(u, p, self.case.dt, self.case.nu, self.S)
            du, dp, dS, dnu, ast = self.dom.step_adjoint(self.g, None)
            assert st["status"] == "PISO_OK" and ast["status"] == "PISO_OK", (st, ast)
            out = (u1, p1, du, dS, dnu)
            u, p = u1, p1
        host = lambda t: t.detach().double().cpu().numpy()
        return dict(u=host(out[0]), p=host(out[1]), du=host(out[2]), dS=host(out[3]), dnu=out[4])


def iter_summary(stats, adj_stats, d):
    """min / median / max over the timed steps of the Krylov iteration counts:
    the BiCGStab (largest over the velocity components) and each corrector's
    pressure CG, forward and adjoint."""
    def mmm(v):
        return [min(v), statistics.median(v), max(v)]
    out = {"adv": mmm([max(s["adv_iters"][:d]) for s in stats]),
           "p": [mmm([s["p_iters"][k] for s in stats]) for k in range(2)]}
    if adj_stats and adj_stats[0] is not None:
        out["adj_adv"] = mmm([max(s["adv_iters"][:d]) for s in adj_stats])
        out["adj_p"] = [mmm([s["p_iters"][k] for s in adj_stats]) for k in range(2)]
    return out


def arm_summary(arm, res, with_adj):
    d = arm.case.ndim
    out = {"fwd_steps_per_s": 1e3 * len(res["fwd_ms"]) / sum(res["fwd_ms"]),
           "fwd_ms": statistics.mean(res["fwd_ms"]),
           "launch": {"threads": arm.shape[0], "ctas": arm.shape[1]}, "pressure_precond": arm.pc_used,
           "line_form": arm.line_form,
           "iterations": iter_summary(res["stats"], res["adj_stats"], d)}
    if with_adj:
        out["fwdadj_steps_per_s"] = 1e3 * len(res["step_ms"]) / sum(res["step_ms"])
        out["adj_ms"] = statistics.mean([t - f for t, f in zip(res["step_ms"], res["fwd_ms"])])
    return out


def fwd_roofline(arm, res, peak, peak_kind, traffic=None, extra_words=0.0):
    """Roofline of the forward-step kernel: algorithmic bytes (the words-per-cell
    model at each timed step's iteration counts, x cells x word size) over the
    summed launch times."""
    d, N = arm.case.ndim, arm.case.ncells
    byts = 0.0
    for st in res["stats"]:
        words = fwd_words_per_cell(d, st["adv_iters"][:d], st["p_iters"][:2], line=arm.pc_used == "y-line",
                                   ilu=st["adv_precond_used"] == 1, fused=arm.line_form == "fused") + extra_words
        byts += words * N * arm.w
    achieved = byts / (sum(res["fwd_ms"]) / 1e3) / 1e9
    words_mean = byts / len(res["stats"]) / (N * arm.w)
    return {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": traffic, "peak_kind": peak_kind, "kernel": "fwd_kernel", "words_per_cell": words_mean,
            "alg_bytes_per_launch": words_mean * N * arm.w}


def time_variant(case, prec, kw, steps, with_adj, flush):
    """Steps/s of one precision/tolerance/preconditioner variant on a workload."""
    arm = Arm(case, prec, kw)
    res = arm.run(steps, 3, flush, with_adj)
    st = res["stats"][-1]
    d = case.ndim
    out = arm_summary(arm, res, with_adj)
    out["steps_per_s"] = out["fwdadj_steps_per_s"] if with_adj else out["fwd_steps_per_s"]
    out.update({"p_rounds": st["p_rounds"][:2], "p_resid": st["p_resid"][:2],
                "adv_precond_used": st["adv_precond_used"]})
    del arm
    return out


def time_statistics(dom, u, p, nu, steps, flush, peak):
    """Turbulence statistics of the step's fields (Sec. 2.5): per frame the
    cell gradients and the records of u (order 3), grad u and (u, grad p)
    (order 2) merged into their accumulators; the adjoint of the u record.
    Returns per-frame times and the roofline of the u-record kernel
    (algorithmic bytes: one read of the d fields)."""
    import torch
    from paper_2505_16992_b300 import solver as SV
    d, N = dom.ndim, dom.N
    w = 4 if dom.dtype == torch.float32 else 8
    su, sg, sp = SV.PlaneStats(dom, d, 3), SV.PlaneStats(dom, d * d, 2), SV.PlaneStats(dom, 2 * d, 2)
    au, ag, ap = su.empty(), sg.empty(), sp.empty()
    up = torch.empty((2 * d, N), dtype=dom.dtype, device="cuda")
    grad = torch.randn_like(au)
    dq = torch.zeros_like(u)
    stream = torch.cuda.current_stream()

    def frame():
        gu, gp = SV.cell_gradients(dom, u, p)
        su.frame(u, au)
        sg.frame(gu.reshape(d * d, N), ag)
        up[:d].copy_(u)
        up[d:].copy_(gp)
        sp.frame(up, ap)

    for _ in range(3):
        frame()
        su.frame_adjoint(u, au, grad, dq)
    t_frame = t_rec = t_adj = 0.0
    for k in range(steps):
        flush.fill_(float(k))
        e = [torch.cuda.Event(enable_timing=True) for _ in range(6)]
        e[0].record(stream)
        frame()
        e[1].record(stream)
        flush.fill_(float(k) + 0.5)
        e[2].record(stream)
        su.frame(u)
        e[3].record(stream)
        flush.fill_(float(k) + 0.25)
        e[4].record(stream)
        su.frame_adjoint(u, au, grad, dq)
        e[5].record(stream)
        e[5].synchronize()
        t_frame += e[0].elapsed_time(e[1])
        t_rec += e[2].elapsed_time(e[3])
        t_adj += e[4].elapsed_time(e[5])
    B = SV.budget(su, au, sg, ag, sp, ap, nu)
    torch.cuda.synchronize()
    rec_ms = t_rec / steps
    achieved = d * N * w / (rec_ms / 1e3) / 1e9
    return {"frame_ms": t_frame / steps, "u_record_ms": rec_ms, "u_record_adjoint_ms": t_adj / steps,
            "budget_finite": bool(all(torch.isfinite(v).all() for v in B.values())),
            "roofline_u_record": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                                  "frac": achieved / peak, "bytes_per_launch": d * N * w}}


def time_batch(prec, kw, steps, warmup, with_adj, flush, threads=0, clocks=False):
    """The batch of 64 independent 2D cavity/channel simulations (sides 32..256,
    Re 100..2000, seed 4) advanced together: one persistent launch for the
    forward step of all members and one for their adjoint, captured once in a
    CUDA graph and replayed; the launch shape autotuned for the batch unless a
    CTA width is given.  Returns sim-steps/s and the details."""
    import torch
    from paper_2505_16992_b300 import capi, workloads as W
    from paper_2505_16992_b300.solver import Batch, Domain
    cases = W.batch2d()
    opts = capi.default_options(p_maxit=20000, adv_maxit=2000, block_threads=threads or 768, **kw)
    doms = [Domain.from_case(c, prec, opts) for c in cases]
    us = [d.field(c.u0, 2) for d, c in zip(doms, cases)]
    ps = [d.field(c.p0) for d, c in zip(doms, cases)]
    Ss = [None if c.S is None else d.field(c.S, 2) for d, c in zip(doms, cases)]
    uo = [torch.empty_like(u) for u in us]
    po = [torch.empty_like(p) for p in ps]
    g0 = torch.Generator(device="cpu").manual_seed(7)
    gs = [torch.randn(u.shape, generator=g0, dtype=u.dtype).cuda() for u in us]   # seeded adjoint seeds
    b = Batch(doms, opts)
    dts, nus = [c.dt for c in cases], [c.nu for c in cases]
    shape = b.autotune(us, ps, dts, nus, Ss) if not threads else (threads, None, None)
    gdu = [torch.empty_like(g) for g in gs]
    gdp = [torch.empty((d.N,), dtype=d.dtype, device="cuda") for d in doms]
    gdS = [torch.empty_like(g) for g in gs]

    def one():
        b.step(us, ps, dts, nus, Ss, u_out=uo, p_out=po, sync=False)
        if with_adj:
            b.step_adjoint(gs, sync=False, du_in=gdu, dp_in=gdp, dS=gdS)

    for _ in range(warmup):
        one()
    _, _, st = b.step(us, ps, dts, nus, Ss, u_out=uo, p_out=po)
    if with_adj:
        b.step_adjoint(gs, du_in=gdu, dp_in=gdp, dS=gdS)
    torch.cuda.synchronize()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(side):
        one()                          # warm the side stream once outside the capture
        torch.cuda.current_stream().synchronize()
        with torch.cuda.graph(graph, stream=side):
            one()
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    graph.replay()
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    tot = 0.0
    clk_path = os.path.join(tempfile.gettempdir(), f"piso_clocks_{os.getpid()}.csv")
    proc, fh = clocks_sampler_start(clk_path) if clocks else (None, None)
    for _ in range(steps):
        flush.fill_(0.0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        graph.replay()
        e1.record(stream)
        e1.synchronize()
        tot += e0.elapsed_time(e1) / 1e3
    clk = clocks_sampler_stop(proc, fh, clk_path, 0) if clocks else None
    _, _, st_after = b.step(us, ps, dts, nus, Ss, u_out=uo, p_out=po)     # replayed steps still converge
    assert all(x["status"] == "PISO_OK" for x in st_after), "batch step failed after graph replays"
    cells = sum(c.ncells for c in cases)
    out = {"sim_steps_per_s": len(cases) * steps / tot, "ms_per_step": 1e3 * tot / steps,
           "cell_updates_per_s": cells * steps / tot, "cells": cells, "members": len(cases),
           "launch": {"threads": shape[0], "ctas": shape[1], "autotuned": not threads},
           "p_iters_max": max(max(x["p_iters"][:2]) for x in st),
           "p_iters_min": min(min(x["p_iters"][:2]) for x in st),
           "p_rounds_max": max(max(x["p_rounds"][:2]) for x in st), "clocks": clk}
    if with_adj:
        # algorithmic bytes of one replayed step (every replay runs the same
        # forward and adjoint from the same inputs): the words-per-cell models
        # at each member's iteration counts, over the measured step time
        ast = b.step_adjoint(gs, du_in=gdu, dp_in=gdp, dS=gdS)[4]
        w = 4 if prec == "fp32" else 8
        byts = 0.0
        for c, f, a in zip(cases, st_after, ast):
            d = c.ndim
            byts += c.ncells * w * (fwd_words_per_cell(d, f["adv_iters"][:d], f["p_iters"][:2])
                                    + adj_words_per_cell(d, a["adv_iters"][:d], a["p_iters"][:2]))
        peak, peak_kind = measured_peaks()
        achieved = byts / (tot / steps) / 1e9
        out["roofline"] = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                           "frac": achieved / peak, "peak_kind": peak_kind, "alg_bytes_per_step": byts,
                           "what": "forward + adjoint launches of one batch step, algorithmic bytes (the "
                                   "words-per-cell models at each member's iteration counts) over the step time"}
    return out


def run_batch(args):
    """The batch workload as its own JSON line."""
    import torch
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    prec = args.precision
    rtol = 1e-6 if prec == "fp32" else 1e-10
    with_adj = args.mode == "fwdadj"
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    r = time_batch(prec, dict(adv_rtol=rtol, p_rtol=rtol), args.steps, args.warmup, with_adj, flush,
                   threads=args.threads, clocks=True)
    line = {"metric": "batched PISO sim-steps/s (64 independent 2D sims, fwd+adjoint)" if with_adj else
                      "batched PISO sim-steps/s (64 independent 2D sims, fwd)",
            "value": r["sim_steps_per_s"], "unit": "sim-steps/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": r["ms_per_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32" if prec == "fp32" else "f64", "data": "synthetic",
            "config": {"workload": "batch64: 2D cavities/channels, side U{32..256}, Re U[100,2000], seed 4",
                       "cells": r["cells"], "krylov_rtol": rtol, "launch": r["launch"],
                       "l2": "flushed between timed steps (256 MB write, untimed)",
                       "cuda_graph": "forward + adjoint launches of a step captured once, replayed per step"},
            "cell_updates_per_s": r["cell_updates_per_s"], "p_iters_max": r["p_iters_max"],
            "p_iters_min": r["p_iters_min"], "gpu_launches": args.steps * (2 if with_adj else 1),
            "clocks": r["clocks"]}
    if "roofline" in r:
        line["roofline"] = r["roofline"]
    print(json.dumps(line))
    return 0


ADV_PRECOND = {"none": 0, "ilu": 1, "ilu_on_failure": 2}     # piso_options.adv_precond


def ilu_compare(prec, rtol, steps, with_adj, flush):
    """Steps/s of the three BiCGStab preconditioner settings on a channel whose
    cell sizes vary strongly (steeper tanh walls, gamma 3, and a 20x larger
    time step than the headline channel), the case the incomplete-LU
    preconditioner is meant for."""
    from paper_2505_16992_b300 import workloads as W
    case = W.channel3d(64, 48, 32, gamma=3.0, dt=0.2)
    out = {"workload": "channel3d 64x48x32, tanh walls gamma 3, dt 0.2 (otherwise as the headline)"}
    for name, code in ADV_PRECOND.items():
        out[name] = time_variant(case, prec, dict(adv_rtol=rtol, p_rtol=rtol, adv_precond=code), steps, with_adj,
                                 flush)
    return out


def nonortho_compare(prec, rtol, steps, flush):
    """Forward and fwd+adjoint steps/s of the 64x48x32 channel with slanted
    cells (x += 0.5 y, a non-orthogonal grid, App. A.2) at one and two
    non-orthogonal corrector steps, beside the same channel with rectangular
    cells."""
    from paper_2505_16992_b300 import workloads as W
    out = {"workload": "channel3d 64x48x32 with cells slanted x += 0.5 y"}
    kw = dict(adv_rtol=rtol, p_rtol=rtol)
    r = time_variant(W.channel3d(64, 48, 32), prec, kw, steps, True, flush)
    out["orthogonal"] = {"fwd_steps_per_s": r["fwd_steps_per_s"], "fwdadj_steps_per_s": r["fwdadj_steps_per_s"]}
    for n in (1, 2):
        r = time_variant(W.channel3d(64, 48, 32, shear=0.5), prec, dict(kw, n_nonortho=n), steps, True, flush)
        out[f"n_nonortho_{n}"] = {"fwd_steps_per_s": r["fwd_steps_per_s"], "fwdadj_steps_per_s": r["fwdadj_steps_per_s"],
                                  "iterations": r["iterations"]}
    return out


def rel_err_per_component(a, b):
    """max over components of max|a_c - b_c| / max|b_c| (a scalar field: one
    component)."""
    import numpy as np
    a = np.asarray(a, dtype=np.float64).reshape(-1, np.asarray(b).shape[-1])
    b = np.asarray(b, dtype=np.float64).reshape(a.shape)
    return float(max(np.abs(a[c] - b[c]).max() / max(np.abs(b[c]).max(), 1e-300) for c in range(a.shape[0])))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--mode", default="fwdadj", choices=["fwd", "fwdadj"])
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-stats", action="store_true", help="skip the turbulence-statistics timing")
    ap.add_argument("--threads", type=int, default=0, help="CTA width; 0 = autotune")
    ap.add_argument("--ctas", type=int, default=0, help="CTA count with --threads (0: one per SM)")
    ap.add_argument("--refine", type=float, default=0.0, help="FP32: FP64-refined pressure tolerance")
    ap.add_argument("--precond", default="auto", choices=["auto", "jacobi", "line"],
                    help="pressure CG preconditioner (auto: the autotuner times both on anisotropic grids)")
    ap.add_argument("--line-split", action="store_true",
                    help="y-line CG with two group barriers per iteration even where the fused form fits")
    ap.add_argument("--adv-precond", default="none", choices=["none", "ilu", "ilu_on_failure"],
                    help="BiCGStab preconditioner of the predictor solve (ILU(0), or ILU(0) after a failed plain solve)")
    ap.add_argument("--nonortho", type=int, default=1,
                    help="non-orthogonal corrector steps on the sheared channel (piso_options.n_nonortho)")
    ap.add_argument("--no-nonortho", action="store_true",
                    help="skip timing the forward step on the channel with slanted (non-orthogonal) cells")
    ap.add_argument("--no-ilu-compare", action="store_true",
                    help="skip timing the BiCGStab preconditioners on the strongly stretched channel")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched-form timing in the default run")
    ap.add_argument("--size", type=int, nargs=3, default=None, metavar=("NX", "NY", "NZ"),
                    help="channel resolution in place of the workload's (same recipe)")
    ap.add_argument("--no-extras", action="store_true",
                    help="headline arm only: skip the other precision arms, the above-L2 channel, the gradient "
                         "paths, statistics and preconditioner comparisons")
    ap.add_argument("--workload", default="channel3d",
                    choices=["channel3d", "channel3d-mid", "channel3d-large", "channel3d-stretched",
                             "channel3d-sheared", "batch64"],
                    help="channel3d: 64x48x32 (default); channel3d-large: 256x192x128 (HBM-bound sizes); "
                         "channel3d-stretched: 64x48x32 with tanh gamma 3 and dt 0.2 (for --adv-precond); "
                         "channel3d-sheared: 64x48x32 with cells slanted by x += 0.5 y (non-orthogonal); "
                         "batch64: 64 independent 2D simulations in one launch")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batch64":
        return run_batch(args)

    import torch

    from paper_2505_16992_b300 import capi, workloads as W

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    sizes = {"channel3d": (64, 48, 32), "channel3d-mid": (160, 120, 80), "channel3d-large": (256, 192, 128),
             "channel3d-stretched": (64, 48, 32), "channel3d-sheared": (64, 48, 32)}
    headline = args.workload == "channel3d"
    stretched = args.workload == "channel3d-stretched"      # the case for the ILU(0) BiCGStab (App. A.5)
    sheared = args.workload == "channel3d-sheared"          # a non-orthogonal grid (App. A.2)
    extra = dict(gamma=3.0, dt=0.2) if stretched else (dict(shear=0.5) if sheared else {})
    if args.size:
        sizes[args.workload] = tuple(args.size)
    headline = headline and sizes[args.workload] == (64, 48, 32)
    case = W.channel3d(*sizes[args.workload], **extra)
    prec = args.precision
    rtol = HEADLINE_RTOL if prec == "fp32" else 1e-10
    pc_code = {"auto": capi.PISO_PRECOND_AUTO, "jacobi": capi.PISO_PRECOND_JACOBI, "line": capi.PISO_PRECOND_LINE}
    opts_kw = dict(adv_rtol=rtol, p_rtol=rtol, p_refine_rtol=args.refine, p_precond=pc_code[args.precond],
                   adv_precond=ADV_PRECOND[args.adv_precond], n_nonortho=args.nonortho if sheared else 0,
                   p_line_split=1 if args.line_split else 0, ctas=args.ctas if args.threads else 0)
    d, N = case.ndim, case.ncells
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    with_adj = args.mode == "fwdadj"
    extras = headline and not args.no_extras

    # ---- the headline arm: timed region with clocks sampled, barrier + max over ranks
    arm = Arm(case, prec, opts_kw, threads=args.threads)
    clk_path = os.path.join(tempfile.gettempdir(), f"piso_clocks_{os.getpid()}.csv")
    clk = {}

    def on_start():
        clk["proc"], clk["fh"] = clocks_sampler_start(clk_path)
        if dist is not None:
            dist.barrier()

    def on_end():
        if dist is not None:
            dist.barrier()
        clk["clocks"] = clocks_sampler_stop(clk["proc"], clk["fh"], clk_path, local)

    res = arm.run(args.steps, args.warmup, flush, with_adj, on_start, on_end)
    step_ms = res["step_ms"] if with_adj else res["fwd_ms"]
    total_s = sum(step_ms) / 1e3
    value = whole_job_value(total_s, args.steps, world, dist)
    total_s = world * args.steps / value
    summ = arm_summary(arm, res, with_adj)

    # ---- end to end through the public API with host buffers: every step copies
    # its inputs from pinned host memory and its outputs back (the outputs feed
    # the next step's inputs)
    dom = arm.dom
    stream = torch.cuda.current_stream()
    hu = torch.empty((d, N), dtype=dom.dtype, pin_memory=True)
    hp = torch.empty((N,), dtype=dom.dtype, pin_memory=True)
    hu.copy_(arm.u0.cpu())
    hp.copy_(arm.p0.cpu())
    u, p = torch.empty_like(arm.u0), torch.empty_like(arm.p0)
    uo, po = torch.empty_like(u), torch.empty_like(p)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for k in range(args.steps):
        u.copy_(hu, non_blocking=True)
        p.copy_(hp, non_blocking=True)
        arm._step(u, p, uo, po, with_adj, False)
        hu.copy_(uo, non_blocking=True)
        hp.copy_(po, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e = whole_job_value(e0.elapsed_time(e1) / 1e3, args.steps, world, dist)
    io_bytes = (d + 1) * N * arm.w

    # ---- roofline of the dominant kernel (the persistent forward-step kernel)
    peak, peak_kind = measured_peaks()
    extra_words = 0.0
    if sheared:
        # cross terms: each viscous evaluation reads u, the cross metrics and J
        # (predictor loops + each corrector's h); each pressure one reads x, the
        # cross metrics and 1/A, reads b and writes the right-hand side; every
        # further predictor solve restarts (rhs0, C, u* in, r, rhat out)
        nx_ = d * (d - 1) // 2
        extra_words += (d + nx_ + 1) * (args.nonortho + 2) + (nx_ + 4) * 2 * args.nonortho
        extra_words += (args.nonortho - 1) * (4 * d + 2 * d + 1)
    traffic = None
    prof = os.path.join(ROOT, "profiles", f"traffic_fwd_kernel_channel3d_{prec}.json")
    if os.path.exists(prof) and headline:
        try:
            tj = json.load(open(prof))
            # counters are valid only for the kernel sources they were taken on
            if tj.get("kernel_sources_sha256_16") == kernel_sources_hash():
                traffic = tj.get("dram_bytes_per_launch")
        except Exception:
            traffic = None
    roof = fwd_roofline(arm, res, peak, peak_kind, traffic, extra_words)
    if headline:
        roof["working_set"] = "L2-resident (about 60 MB in FP32 against a 126 MB L2): the achieved figure is " \
                              "algorithmic bytes over time, mostly served from L2; roofline_above_l2 is the HBM case"
        if traffic:
            roof["dram_gbs"] = traffic / (summ["fwd_ms"] / 1e3) / 1e9

    # ---- gradient-path variants of the adjoint (Sec. 2.4): the same fwd+adjoint
    # step with the advection and/or pressure solves left out of the backward pass
    paths = None
    if with_adj and extras:
        paths = {"adv+p": {"steps_per_s": value, "adj_ms": summ.get("adj_ms")}}
        nvar = max(5, args.steps // 3)
        tuned = dom.get_options()          # launch shape and pressure preconditioner as tuned
        for name, bits in (("adv", capi.PISO_GRAD_ADV), ("p", capi.PISO_GRAD_P), ("none", 0)):
            tuned.grad_paths = bits
            dom.set_options(tuned)
            r = arm.run(nvar, 3, flush, True)
            paths[name] = {"steps_per_s": 1e3 * nvar / sum(r["step_ms"]),
                           "adj_ms": statistics.mean([t - f for t, f in zip(r["step_ms"], r["fwd_ms"])]),
                           "adj_iters": {"adv": r["adj_stats"][-1]["adv_iters"][:d],
                                         "p": r["adj_stats"][-1]["p_iters"][:2]}}
        tuned.grad_paths = capi.PISO_GRAD_ADV | capi.PISO_GRAD_P
        dom.set_options(tuned)

    # ---- the metric's other arms: forward and fwd+adjoint in FP32 and FP64, and
    # the two precisions at matched pressure (divergence) tolerances
    arms = compare = None
    nsub = max(5, args.steps // 2)
    if extras:
        other = "fp64" if prec == "fp32" else "fp32"
        orr = 1e-10 if other == "fp64" else 1e-6
        oarm = Arm(case, other, dict(opts_kw, adv_rtol=orr, p_rtol=orr))
        osum = arm_summary(oarm, oarm.run(nsub, 3, flush, True), True)
        del oarm
        arms = {prec: dict(summ, krylov_rtol=rtol), other: dict(osum, krylov_rtol=orr)}
        compare = {"what": "fwd+adjoint steps/s at the same relative residual of every pressure solve (the "
                           "Rhie-Chow divergence left by the correctors) and of the BiCGStab"}
        for name, pr, kw in (("fp64_rtol1e-6", "fp64", dict(adv_rtol=1e-6, p_rtol=1e-6)),
                             ("fp32_refined1e-10", "fp32", dict(adv_rtol=1e-6, p_rtol=1e-6, p_refine_rtol=1e-10))):
            compare[name] = time_variant(case, pr, kw, nsub, True, flush)
        compare["fp32_rtol1e-6"] = {"steps_per_s": arms["fp32"]["fwdadj_steps_per_s"]}
        compare["fp64_rtol1e-10"] = {"steps_per_s": arms["fp64"]["fwdadj_steps_per_s"]}

    # ---- the same step above L2: 256x192x128 (6.3 M cells, ~2.5 GB of FP32
    # fields and workspace), where the forward kernel is bound by HBM
    large = None
    if extras:
        lcase = W.channel3d(256, 192, 128)
        larm = Arm(lcase, "fp32", dict(opts_kw, adv_rtol=1e-6, p_rtol=1e-6))
        lres = larm.run(3, 3, flush, True)
        ltraffic = None
        lprof = os.path.join(ROOT, "profiles", "traffic_fwd_kernel_channel3d_256x192x128_fp32.json")
        if os.path.exists(lprof):
            try:
                tj = json.load(open(lprof))
                if tj.get("kernel_sources_sha256_16") == kernel_sources_hash():
                    ltraffic = tj.get("dram_bytes_per_launch")
            except Exception:
                ltraffic = None
        large = arm_summary(larm, lres, True)
        large["workload"] = "channel3d 256x192x128 (same recipe), FP32, Krylov rtol 1e-6, autotuned"
        large["cells"] = lcase.ncells
        large["roofline"] = fwd_roofline(larm, lres, peak, peak_kind, ltraffic)
        del larm

    # ---- the batched form (64 independent 2D simulations in one launch, CUDA
    # graph, autotuned launch shape) in both precisions, at matched relative
    # residuals of the Krylov solves (the divergence left by the correctors)
    batch = None
    if extras and not args.no_batch:
        bsteps = max(5, args.steps // 4)
        batch = {"workload": "batch64: 64 independent 2D cavities/channels, side U{32..256}, Re U[100,2000], "
                             "seed 4; forward + adjoint per step, one CUDA graph replay",
                 "fp32_rtol1e-6": time_batch("fp32", dict(adv_rtol=1e-6, p_rtol=1e-6), bsteps, 3, True, flush),
                 "fp64_rtol1e-6": time_batch("fp64", dict(adv_rtol=1e-6, p_rtol=1e-6), bsteps, 3, True, flush),
                 "fp32_refined1e-10": time_batch("fp32", dict(adv_rtol=1e-6, p_rtol=1e-6, p_refine_rtol=1e-10),
                                                 bsteps, 3, True, flush),
                 "fp64_rtol1e-10": time_batch("fp64", dict(adv_rtol=1e-10, p_rtol=1e-10), bsteps, 3, True, flush)}

    statistics_obj = None
    if not args.no_stats and extras:
        statistics_obj = time_statistics(dom, arm.u0, arm.p0, case.nu, max(5, args.steps // 3), flush, peak)

    ilu_cmp = None
    if not args.no_ilu_compare and extras:
        ilu_cmp = ilu_compare(prec, rtol, max(5, args.steps // 3), with_adj, flush)
    no_cmp = None
    if not args.no_nonortho and extras:
        no_cmp = nonortho_compare(prec, rtol, max(5, args.steps // 3), flush)

    # ---- the oracle on the host cores, and the GPU path's error against it on
    # the same steps (computed outside every timed region)
    cpu = cpu_all = parity = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and headline:
        v, n, dt, _ = cpu_baseline(seconds_budget=20.0, steps_cap=10, rtol=rtol, want_fields=False)
        cpu = {"value": v, "unit": "steps/s", "cores": 1, "kind": "oracle",
               "sample": f"{n} fwd+adjoint steps of the same workload (Krylov rtol {rtol:g}) along the rollout "
                         f"from its seeded state in {dt:.1f} s"}
        va, workers, nproc, steps_all, slow = cpu_baseline_all_cores(rtol=rtol)
        cpu_all = {"value": va, "unit": "steps/s", "cores": workers, "nproc": nproc, "kind": "oracle",
                   "sample": f"{workers} independent copies, {steps_all} fwd+adjoint steps in total (Krylov rtol "
                             f"{rtol:g}), slowest copy {slow:.1f} s"}
        _, n, _, of = cpu_baseline(seconds_budget=60.0, steps_cap=3)      # the precise oracle for the parity
        gf = arm.rollout_fields(n)
        parity = {"against": f"FP64 oracle (Krylov rtol 1e-13), after {n} fwd+adjoint steps from the seeded state",
                  "gpu": f"{prec}, Krylov rtol {rtol:g}, the timed launch shape",
                  "u": rel_err_per_component(gf["u"], of["u"]), "p": rel_err_per_component(gf["p"], of["p"]),
                  "du": rel_err_per_component(gf["du"], of["du"]), "dS": rel_err_per_component(gf["dS"], of["dS"]),
                  "dnu": abs(gf["dnu"] - of["dnu"]) / max(abs(of["dnu"]), 1e-300),
                  "norm": "per component: max|gpu - oracle| / max|oracle|"}

    if rank == 0:
        line = {
            "metric": "PISO steps/s (fwd+adjoint), 64x48x32 channel" if with_adj else
                      "PISO steps/s (fwd), 64x48x32 channel",
            "value": value, "unit": "steps/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * total_s / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32" if prec == "fp32" else "f64", "data": "synthetic",
            "config": {"workload": HEADLINE_WORKLOAD,
                       "cells": N, "precision": prec, "krylov_rtol": rtol,
                       "l2": "flushed between timed steps (256 MB write, untimed)",
                       "state": ROLLOUT_STATE,
                       "parallelism": "replicas" if world > 1 else "single",
                       "launch": {"threads": arm.shape[0], "ctas": arm.shape[1], "autotuned": args.threads == 0},
                       "pressure_precond": arm.pc_used, "line_form": arm.line_form,
                       "adv_precond": args.adv_precond},
            "iterations": summ["iterations"],
            "fwd_ms": summ["fwd_ms"],
            "cell_updates_per_s": value * N,
            "e2e": {"value": e2e, "unit": "steps/s", "h2d_bytes_per_step": io_bytes,
                    "d2h_bytes_per_step": io_bytes},
            "gpu_launches": args.steps * (2 if with_adj else 1),
            "roofline": roof,
            "clocks": clk.get("clocks"),
        }
        if arms is not None:
            line["arms"] = arms
        if compare is not None:
            line["precision_compare"] = compare
        if large is not None:
            line["roofline_above_l2"] = dict(large["roofline"], workload=large["workload"],
                                             fwd_steps_per_s=large["fwd_steps_per_s"],
                                             fwdadj_steps_per_s=large["fwdadj_steps_per_s"],
                                             iterations=large["iterations"], launch=large["launch"],
                                             pressure_precond=large["pressure_precond"])
        if parity is not None:
            line["parity"] = parity
        if batch is not None:
            line["batch"] = batch
        if ilu_cmp is not None:
            line["adv_precond_compare"] = ilu_cmp
        if no_cmp is not None:
            line["nonortho"] = no_cmp
        if paths is not None:
            line["grad_paths"] = paths
        if statistics_obj is not None:
            line["statistics"] = statistics_obj
        if stretched:
            line["config"]["workload"] = line["config"]["workload"].replace("gamma 2", "gamma 3").replace(
                "dt 0.01", "dt 0.2")
            line["metric"] = line["metric"].replace("channel", "channel (tanh gamma 3, dt 0.2)")
        elif sheared:
            line["config"]["workload"] += ", cells slanted x += 0.5 y (non-orthogonal)"
            line["config"]["n_nonortho"] = args.nonortho
            line["metric"] = line["metric"].replace("channel", "sheared channel")
        elif not headline:
            tag = "x".join(str(v) for v in sizes[args.workload])
            line["config"]["workload"] = line["config"]["workload"].replace("64x48x32", tag)
            line["metric"] = line["metric"].replace("64x48x32", tag)
        if cpu is not None:
            line["cpu_baseline"] = cpu
            line["cpu_baseline_all_cores"] = cpu_all
        print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
