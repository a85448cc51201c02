"""Helpers shared by the GPU parity tests (CUDA path vs the FP64 oracle)."""
import numpy as np
import torch

import oracle as O
from paper_2505_16992_b300 import capi
from paper_2505_16992_b300.solver import Domain

FP64_REL = 1e-10     # per-step FP64 parity bar (relative to the field's max)
FP32_REL = 1e-4      # mixed precision on laminar fields


def rel_err(a, b):
    """Largest error relative to the reference, per component: a field of
    shape (d, N) is judged component by component, each against its own
    largest magnitude (floored at 1e-3 of the whole field's, so a component
    that is identically zero up to round-off is judged at that scale); a
    scalar field against its own largest magnitude."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    if b.ndim < 2:
        return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)) if b.size else 0.0
    a2 = a.reshape(b.shape[0], -1)
    b2 = b.reshape(b.shape[0], -1)
    if not b2.size:
        return 0.0
    floor = max(1e-3 * np.abs(b2).max(), 1e-300)
    return float(max(np.abs(a2[c] - b2[c]).max() / max(np.abs(b2[c]).max(), floor) for c in range(b2.shape[0])))


def gpu_domain(case, precision="fp64", **opts):
    if precision == "fp64":
        opts.setdefault("adv_rtol", 1e-13)
        opts.setdefault("p_rtol", 1e-13)
    o = capi.default_options(**opts)
    return Domain.from_case(case, precision, o)


def to_dev(dom, arr, comps=None):
    return dom.field(arr, comps)


def host(t):
    return t.detach().double().cpu().numpy()


def gpu_step(dom, case, u, p, S=None, **kw):
    d = case.ndim
    ut = to_dev(dom, u, d)
    pt = to_dev(dom, p)
    St = None if S is None else to_dev(dom, S, d)
    u1, p1, st = dom.step(ut, pt, case.dt, case.nu, St, **kw)
    return host(u1), host(p1), st


def oracle_step(mesh, case, u, p, S=None, bval=None, opts=None):
    return O.piso_step(mesh, u, p, case.dt, case.nu, S, bval, opts)


def sync():
    torch.cuda.synchronize()


def bval_faces(m, bval):
    """Oracle boundary values (per cell side, [nsides][d][N]) -> the library's
    face order [d][nbf] (blocks in order, sides in order, faces in side order)."""
    faces = []
    for bi in range(len(m.res)):
        for s in range(m.nsides):
            cells = m.side_cells(bi, s)
            if m.is_bface[s, cells[0]]:
                faces.append(bval[s][:, cells])
    return np.concatenate(faces, axis=1) if faces else np.zeros((m.ndim, 0))
