"""PyTorch-facing wrapper of the C ABI: domains, steps, adjoints, batches and a
differentiable rollout (arXiv:2505.16992, Sec. 2.3: discretise-then-optimise
through the PISO step with solve adjoints; App. A.5: fields are PyTorch
tensors).  Every numerical step runs in the CUDA library; this module only
marshals arguments.
"""
from __future__ import annotations

import ctypes as C
from typing import List, Optional, Sequence

import numpy as np
import torch

from . import capi

_DT = {capi.PISO_FP64: torch.float64, capi.PISO_FP32: torch.float32}


def _prec(precision) -> int:
    if precision in (capi.PISO_FP64, "fp64", torch.float64):
        return capi.PISO_FP64
    if precision in (capi.PISO_FP32, "fp32", torch.float32):
        return capi.PISO_FP32
    raise ValueError(f"unknown precision {precision}")


def _stream_ptr(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream or None


class Domain:
    """A multi-block domain (App. A.5 Domain/Block/Boundary) living on cuda:0."""

    def __init__(self, ndim: int, precision="fp64"):
        self.lib = capi.load()
        self.ndim = ndim
        self.prec = _prec(precision)
        self.dtype = _DT[self.prec]
        h = C.c_void_p()
        capi.check(self.lib.piso_domain_create(ndim, self.prec, C.byref(h)))
        self.h = h
        self.finalized = False

    # -- description -----------------------------------------------------------
    def add_block(self, res, vertices) -> int:
        r = (C.c_int32 * 3)(*[int(v) for v in res])
        _, vp = capi.dbuf(vertices)
        bid = C.c_int32()
        capi.check(self.lib.piso_block_add(self.h, r, vp, C.byref(bid)), self.h)
        return bid.value

    def connect(self, a, sa, b, sb, axis_perm=0, flip_mask=0):
        capi.check(self.lib.piso_connect(self.h, a, sa, b, sb, axis_perm, flip_mask), self.h)

    def set_dirichlet(self, blk, side, values):
        _, vp = capi.dbuf(values)
        capi.check(self.lib.piso_set_dirichlet(self.h, blk, side, vp), self.h)

    def set_advective_outflow(self, blk, side, u_m, values):
        _, up = capi.dbuf(u_m)
        _, vp = capi.dbuf(values)
        capi.check(self.lib.piso_set_advective_outflow(self.h, blk, side, up, vp), self.h)

    def finalize(self, options: Optional[capi.Options] = None, **kw):
        o = options if options is not None else capi.default_options(**kw)
        capi.check(self.lib.piso_finalize(self.h, C.byref(o)), self.h)
        self.finalized = True
        self.N = int(self.lib.piso_num_cells(self.h))
        self.nbf = int(self.lib.piso_num_boundary_faces(self.h))
        self.tape_bytes = int(self.lib.piso_tape_bytes(self.h))
        return self

    def set_options(self, options: Optional[capi.Options] = None, **kw):
        o = options if options is not None else capi.default_options(**kw)
        capi.check(self.lib.piso_set_options(self.h, C.byref(o)), self.h)

    def get_options(self) -> capi.Options:
        o = capi.Options()
        capi.check(self.lib.piso_get_options(self.h, C.byref(o)), self.h)
        return o

    def uses_line_precond(self) -> bool:
        """True when the pressure CG of the next step uses the y-line preconditioner."""
        return int(self.lib.piso_pressure_precond(self.h)) == capi.PISO_PRECOND_LINE

    def uses_fused_lines(self) -> bool:
        """True when that y-line CG runs with one group barrier per iteration."""
        return int(self.lib.piso_pressure_line_fused(self.h)) == 1

    def uses_cg_vec4(self) -> bool:
        """True when the next step's Jacobi CG sweeps four cells per thread."""
        return int(self.lib.piso_pressure_cg_vec4(self.h)) == 1

    @classmethod
    def from_case(cls, case, precision="fp64", options=None, **kw) -> "Domain":
        """Build from an object with ndim/blocks/connections/dirichlet/outflow
        (the seeded input generators produce such objects)."""
        d = cls(case.ndim, precision)
        for b in case.blocks:
            d.add_block(b.res, b.vertices)
        for conn in case.connections:
            d.connect(*conn)
        for (blk, s, vals) in case.dirichlet:
            d.set_dirichlet(blk, s, vals)
        for (blk, s, um, vals) in case.outflow:
            d.set_advective_outflow(blk, s, um, vals)
        return d.finalize(options, **kw)

    def __del__(self):
        try:
            if getattr(self, "h", None):
                self.lib.piso_domain_destroy(self.h)
                self.h = None
        except Exception:
            pass

    # -- fields -----------------------------------------------------------------
    def field(self, values=None, components: Optional[int] = None) -> torch.Tensor:
        shape = (self.N,) if components is None else (components, self.N)
        if values is None:
            return torch.zeros(shape, dtype=self.dtype, device="cuda")
        t = torch.as_tensor(np.asarray(values), dtype=self.dtype)
        return t.reshape(shape).contiguous().cuda()

    def new_tape(self) -> torch.Tensor:
        return torch.empty(self.tape_bytes, dtype=torch.uint8, device="cuda")

    def _check_field(self, t, comps, name):
        if t is None:
            return
        want = (self.N,) if comps is None else (comps, self.N)
        if t.dtype != self.dtype or not t.is_cuda or not t.is_contiguous() or tuple(t.shape) != want:
            raise ValueError(f"{name} must be a contiguous cuda {self.dtype} tensor of shape {want}")

    # -- step ---------------------------------------------------------------------
    def step(self, u, p, dt, nu, S=None, tape=None, u_out=None, p_out=None, stream=None, sync=True):
        """One PISO step; returns (u_new, p_new, stats-dict or None)."""
        d = self.ndim
        self._check_field(u, d, "u")
        self._check_field(p, None, "p")
        self._check_field(S, d, "S")
        u_out = torch.empty_like(u) if u_out is None else u_out
        p_out = torch.empty_like(p) if p_out is None else p_out
        st = capi.Stats() if sync else None
        rc = self.lib.piso_step(self.h, capi.dptr(u), capi.dptr(p), capi.dptr(u_out), capi.dptr(p_out),
                                float(dt), float(nu), capi.dptr(S), capi.dptr(tape), _stream_ptr(stream),
                                C.byref(st) if st is not None else None)
        capi.check(rc, self.h)
        return u_out, p_out, (st.as_dict() if st is not None else None)

    def autotune(self, u, p, dt, nu, S=None, stream=None):
        """Pick the fastest launch shape on this state; returns (threads, ctas, ms)."""
        t, c, ms = C.c_int32(), C.c_int32(), C.c_double()
        rc = self.lib.piso_autotune(self.h, capi.dptr(u), capi.dptr(p), float(dt), float(nu), capi.dptr(S),
                                    _stream_ptr(stream), C.byref(t), C.byref(c), C.byref(ms))
        capi.check(rc, self.h)
        return t.value, c.value, ms.value

    def last_stats(self):
        st = capi.Stats()
        rc = self.lib.piso_last_stats(self.h, C.byref(st))
        capi.check(rc, self.h)
        return st.as_dict()

    def step_adjoint(self, du_out, dp_out=None, tape=None, stream=None, want=("u", "p", "S", "nu"), sync=True,
                     du_in=None, dp_in=None, dS=None):
        """Adjoint of the last (or taped) step: returns (du_in, dp_in, dS, dnu,
        stats).  sync=False only enqueues (no dnu or statistics read back; they
        come back as None)."""
        d = self.ndim
        if du_in is None and "u" in want:
            du_in = torch.empty((d, self.N), dtype=self.dtype, device="cuda")
        if dp_in is None and "p" in want:
            dp_in = torch.empty((self.N,), dtype=self.dtype, device="cuda")
        if dS is None and "S" in want:
            dS = torch.empty((d, self.N), dtype=self.dtype, device="cuda")
        dnu = C.c_double(0.0)
        st = capi.Stats() if sync else None
        rc = self.lib.piso_step_adjoint(self.h, capi.dptr(tape), capi.dptr(du_out), capi.dptr(dp_out),
                                        capi.dptr(du_in), capi.dptr(dp_in), capi.dptr(dS),
                                        C.byref(dnu) if ("nu" in want and sync) else None, _stream_ptr(stream),
                                        C.byref(st) if sync else None)
        capi.check(rc, self.h)
        if not sync:
            return du_in, dp_in, dS, None, None
        return du_in, dp_in, dS, dnu.value, st.as_dict()

    def get_boundary(self) -> np.ndarray:
        out = np.zeros((self.ndim, max(self.nbf, 0)))
        capi.check(self.lib.piso_get_boundary(self.h, out.ctypes.data_as(C.POINTER(C.c_double))), self.h)
        return out

    def set_boundary(self, values):
        a, vp = capi.dbuf(values)
        capi.check(self.lib.piso_set_boundary(self.h, vp), self.h)

    def boundary_adjoint(self) -> np.ndarray:
        """dL/d(boundary-face values) of the last adjoint, [ndim][nbf] (App. A.4:
        boundary velocities are differentiable)."""
        out = np.zeros((self.ndim, max(self.nbf, 0)))
        capi.check(self.lib.piso_get_boundary_adjoint(self.h, out.ctypes.data_as(C.POINTER(C.c_double))),
                   self.h)
        return out


class Batch:
    """Independent domains stepped together in one persistent launch."""

    def __init__(self, domains: Sequence[Domain], options: Optional[capi.Options] = None, **kw):
        self.lib = capi.load()
        self.domains = list(domains)
        arr = (C.c_void_p * len(domains))(*[d.h.value for d in domains])
        o = options if options is not None else capi.default_options(**kw)
        h = C.c_void_p()
        capi.check(self.lib.piso_batch_create(arr, len(domains), C.byref(o), C.byref(h)))
        self.h = h

    def __del__(self):
        try:
            if getattr(self, "h", None):
                self.lib.piso_batch_destroy(self.h)
                self.h = None
        except Exception:
            pass

    @staticmethod
    def _ptrs(ts):
        return (C.c_void_p * len(ts))(*[capi.dptr(t) for t in ts])

    def step(self, us, ps, dts, nus, Ss=None, u_out=None, p_out=None, stream=None, sync=True):
        n = len(self.domains)
        u_out = [torch.empty_like(u) for u in us] if u_out is None else u_out
        p_out = [torch.empty_like(p) for p in ps] if p_out is None else p_out
        Ss = [None] * n if Ss is None else Ss
        dt = (C.c_double * n)(*dts)
        nu = (C.c_double * n)(*nus)
        st = (capi.Stats * n)() if sync else None
        rc = self.lib.piso_batch_step(self.h, self._ptrs(us), self._ptrs(ps), self._ptrs(u_out),
                                      self._ptrs(p_out), dt, nu, self._ptrs(Ss), _stream_ptr(stream),
                                      st if st is not None else None)
        capi.check(rc, None)
        return u_out, p_out, ([s.as_dict() for s in st] if st is not None else None)

    def autotune(self, us, ps, dts, nus, Ss=None, stream=None):
        """Pick the fastest CTA width and count for this batch on this state;
        returns (threads, ctas, ms)."""
        n = len(self.domains)
        Ss = [None] * n if Ss is None else Ss
        t, c, ms = C.c_int32(), C.c_int32(), C.c_double()
        rc = self.lib.piso_batch_autotune(self.h, self._ptrs(us), self._ptrs(ps), (C.c_double * n)(*dts),
                                          (C.c_double * n)(*nus), self._ptrs(Ss), _stream_ptr(stream), C.byref(t),
                                          C.byref(c), C.byref(ms))
        capi.check(rc, None)
        return t.value, c.value, ms.value

    def step_adjoint(self, du_out, dp_out=None, stream=None, sync=True, du_in=None, dp_in=None, dS=None):
        """Adjoint of every member's last step.  sync=False enqueues only (no
        statistics or dnu read back; usable inside CUDA-graph capture)."""
        n = len(self.domains)
        dp_out = [None] * n if dp_out is None else dp_out
        du_in = [torch.empty_like(g) for g in du_out] if du_in is None else du_in
        dp_in = [torch.empty((d.N,), dtype=d.dtype, device="cuda") for d in self.domains] if dp_in is None else dp_in
        dS = [torch.empty_like(g) for g in du_out] if dS is None else dS
        dnu = (C.c_double * n)() if sync else None
        st = (capi.Stats * n)() if sync else None
        rc = self.lib.piso_batch_step_adjoint(self.h, self._ptrs(du_out), self._ptrs(dp_out),
                                              self._ptrs(du_in), self._ptrs(dp_in), self._ptrs(dS), dnu,
                                              _stream_ptr(stream), st)
        capi.check(rc, None)
        if not sync:
            return du_in, dp_in, dS, None, None
        return du_in, dp_in, dS, list(dnu), [s.as_dict() for s in st]


class PisoStepFunction(torch.autograd.Function):
    """u^{n+1}, p^{n+1} = PISO(u^n, p^n, S, nu) with the hand-written adjoint.

    The forward keeps only (u^n, p^n, S, nu) (checkpoint); backward recomputes
    the step into the domain's own tape and runs the adjoint kernel on it."""

    @staticmethod
    def forward(ctx, u, p, S, nu, domain: Domain, dt: float):
        nu_f = float(nu)
        u1, p1, _ = domain.step(u.detach().contiguous(), p.detach().contiguous(), dt, nu_f,
                                None if S is None else S.detach().contiguous(), sync=False)
        ctx.domain, ctx.dt, ctx.nu = domain, dt, nu_f
        ctx.has_S = S is not None
        ctx.nu_is_tensor = torch.is_tensor(nu)
        ctx.save_for_backward(u.detach(), p.detach(), S.detach() if S is not None else None)
        return u1, p1

    @staticmethod
    def backward(ctx, gu, gp):
        u, p, S = ctx.saved_tensors
        dom = ctx.domain
        # recompute the step internals into the domain's workspace tape
        dom.step(u.contiguous(), p.contiguous(), ctx.dt, ctx.nu, S, sync=False)
        gu = torch.zeros_like(u) if gu is None else gu.contiguous()
        gp = None if gp is None else gp.contiguous()
        du, dp, dS, dnu, _ = dom.step_adjoint(gu, gp)
        gnu = torch.tensor(dnu, dtype=u.dtype, device=u.device) if ctx.nu_is_tensor else None
        return du, dp, (dS if ctx.has_S else None), gnu, None, None


def piso_step(domain: Domain, u, p, dt, nu, S=None):
    """Differentiable PISO step (checkpointed: internals recomputed in backward)."""
    return PisoStepFunction.apply(u, p, S, nu, domain, dt)


def rollout(domain: Domain, u, p, dt, nu, steps: int, source_fn=None):
    """Differentiable rollout of ``steps`` PISO steps.  source_fn(u) -> S lets a
    learned corrector enter as the source term (Sec. 3)."""
    for _ in range(steps):
        S = source_fn(u) if source_fn is not None else None
        u, p = piso_step(domain, u, p, dt, nu, S)
    return u, p


# ---------------------------------------------------------------------------
# turbulence statistics (Sec. 2.5 "Operators for Turbulence Statistics";
# Sec. 3.3 "Losses from Turbulence Statistics")
# ---------------------------------------------------------------------------

class PlaneStats:
    """Plane records of nq per-cell fields of a single-block domain: count,
    means and central moments up to ``order`` per plane y (homogeneous x, z),
    as float64 tensors [ny][record_size] = [n, mean, m2, m3]."""

    def __init__(self, domain: Domain, nq: int, order: int = 3):
        self.lib = capi.load()
        self.domain, self.nq, self.order = domain, nq, order
        h = C.c_void_p()
        capi.check(self.lib.piso_stats_create(domain.h, nq, order, C.byref(h)), domain.h)
        self.h = h
        self.rsize = int(self.lib.piso_stats_record_size(h))
        self.ny = int(self.lib.piso_stats_planes(h))

    def __del__(self):
        try:
            if getattr(self, "h", None):
                self.lib.piso_stats_destroy(self.h)
                self.h = None
        except Exception:
            pass

    def empty(self) -> torch.Tensor:
        """An accumulator with no samples (n = 0 in every plane)."""
        return torch.zeros((self.ny, self.rsize), dtype=torch.float64, device="cuda")

    def _q(self, q):
        q = q.detach().contiguous()
        if q.dtype != self.domain.dtype or q.numel() != self.nq * self.domain.N:
            raise ValueError(f"q must hold {self.nq} x {self.domain.N} {self.domain.dtype} values")
        return q

    def frame(self, q, acc: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
        rec = torch.empty((self.ny, self.rsize), dtype=torch.float64, device="cuda")
        capi.check(self.lib.piso_stats_frame(self.h, capi.dptr(self._q(q)), capi.dptr(rec), capi.dptr(acc),
                                             _stream_ptr(stream)), self.domain.h)
        return rec

    def merge(self, a: torch.Tensor, b: torch.Tensor, stream=None) -> torch.Tensor:
        capi.check(self.lib.piso_stats_merge(self.h, capi.dptr(a), capi.dptr(b), _stream_ptr(stream)),
                   self.domain.h)
        return a

    def frame_adjoint(self, q, rec, grad, dq=None, stream=None) -> torch.Tensor:
        q = self._q(q)
        dq = torch.zeros_like(q) if dq is None else dq
        capi.check(self.lib.piso_stats_frame_adjoint(self.h, capi.dptr(q), capi.dptr(rec.contiguous()),
                                                     capi.dptr(grad.contiguous()), capi.dptr(dq),
                                                     _stream_ptr(stream)), self.domain.h)
        return dq

    def split(self, rec: torch.Tensor):
        """(n [ny], mean [ny][nq], m2 [ny][nq][nq], m3 [ny][nq][nq][nq] or None) views of a record."""
        nq = self.nq
        n = rec[:, 0]
        mean = rec[:, 1:1 + nq]
        m2 = rec[:, 1 + nq:1 + nq + nq * nq].reshape(-1, nq, nq)
        m3 = rec[:, 1 + nq + nq * nq:].reshape(-1, nq, nq, nq) if self.order == 3 else None
        return n, mean, m2, m3


class FrameRecordFunction(torch.autograd.Function):
    """record = plane statistics of one frame q (differentiable in q)."""

    @staticmethod
    def forward(ctx, q, stats: PlaneStats):
        rec = stats.frame(q)
        ctx.stats = stats
        ctx.save_for_backward(q.detach(), rec)
        return rec

    @staticmethod
    def backward(ctx, g):
        q, rec = ctx.saved_tensors
        return ctx.stats.frame_adjoint(q, rec, g.contiguous()), None


class TimeAveragedRecordFunction(torch.autograd.Function):
    """record of all samples of the frames qs (averaging over time and the
    homogeneous directions), accumulated online; the derivative with respect
    to each frame uses the accumulated record."""

    @staticmethod
    def forward(ctx, stats: PlaneStats, *qs):
        acc = stats.empty()
        tmp = torch.empty_like(acc)
        for q in qs:
            capi.check(stats.lib.piso_stats_frame(stats.h, capi.dptr(stats._q(q)), capi.dptr(tmp), capi.dptr(acc),
                                                  _stream_ptr(None)), stats.domain.h)
        ctx.stats = stats
        ctx.save_for_backward(acc, *[q.detach() for q in qs])
        return acc

    @staticmethod
    def backward(ctx, g):
        acc, *qs = ctx.saved_tensors
        g = g.contiguous()
        return (None,) + tuple(ctx.stats.frame_adjoint(q, acc, g) for q in qs)


def frame_record(stats: PlaneStats, q):
    return FrameRecordFunction.apply(q, stats)


def time_averaged_record(stats: PlaneStats, qs):
    return TimeAveragedRecordFunction.apply(stats, *qs)


def cell_gradients(domain: Domain, u, p=None, stream=None):
    """(grad_u [d][d][N] with grad_u[i, k] = d u_i / d x_k, grad_p [d][N] or None)."""
    d, N = domain.ndim, domain.N
    gu = torch.empty((d, d, N), dtype=domain.dtype, device="cuda")
    gp = torch.empty((d, N), dtype=domain.dtype, device="cuda") if p is not None else None
    capi.check(domain.lib.piso_cell_gradients(domain.h, capi.dptr(u.contiguous()),
                                              capi.dptr(None if p is None else p.contiguous()), capi.dptr(gu),
                                              capi.dptr(gp), _stream_ptr(stream)), domain.h)
    return gu, gp


def budget(su: PlaneStats, rec_u, sg: PlaneStats, rec_g, sp: PlaneStats, rec_p, nu: float, stream=None):
    """Budget terms per plane: dict of [ny][d][d] tensors P, eps, T, D, Pi."""
    d = su.domain.ndim
    out = torch.empty((5, su.ny, d, d), dtype=torch.float64, device="cuda")
    capi.check(su.lib.piso_stats_budget(su.h, capi.dptr(rec_u), sg.h, capi.dptr(rec_g), sp.h, capi.dptr(rec_p),
                                        float(nu), capi.dptr(out), _stream_ptr(stream)), su.domain.h)
    return dict(P=out[0], eps=out[1], T=out[2], D=out[3], Pi=out[4])
