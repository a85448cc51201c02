"""FP64 CPU oracle of the per-time-step PISO update and its discrete adjoint.

TEST INFRASTRUCTURE ONLY.  This module is the slow, plain reference that the
CUDA path is checked against.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import it; the product path never does.

It restates, in the paper's order and notation, the collocated first-order
finite-volume PISO scheme of arXiv:2505.16992:

* Sec. 2.1 and App. A.1 (Eqs. advection, advectionMat, pressureRHS, pressure,
  correction): one implicit-Euler predictor solve C u* = u^n/dt - grad p + S,
  then two correctors h = A^-1(u^n/dt + S - H u), div(A^-1 grad p) = div h,
  u = h - A^-1 grad p.
* App. A.2 "Grid Transformations": metrics T_ji = d xi^j / d x_i and
  J = det(dx/dxi) at cell centres; contravariant flux U^j = J T_j . u.
* App. A.2 Eq. advMatDiscrete (central advection entries 0.5 N_f U_f),
  Eq. difMatDiscrete (orthogonal diffusion, alpha_jj = J T_j . T_j),
  Eq. velRHSdiscrete (Dirichlet boundary fluxes on the right-hand side),
  Eq. pMatDiscrete (pressure matrix from alpha_jj / A),
  Eqs. pressureRHSdiscrete / pressureRHSdivDiscrete (divergence of h),
  Eq. velCorrDiscrete (cell-centred central pressure gradient).
* App. A.3 (boundaries): block connections only change the neighbour lookup;
  Dirichlet velocity faces carry their own values and imply 0-Neumann pressure;
  the advective outflow Eq. advOut updates its face values before each step and
  is rescaled to balance the in- and outflow.
* Sec. 2.3 and App. A.4 (gradients): linear solves are differentiated by the
  transposed solve  A^T db = dx,  dA = -db (x) x  on the sparsity pattern; every
  other operation by its exact transpose.
* App. A.5 (solvers): the advection-diffusion BiCGStab may be ILU(0)-
  preconditioned, from the start or only after the plain solve failed; the
  transposed solve of the adjoint uses the factorisation of C^T.
* Sec. 2.4 (gradient paths, Eq. jnone): the paths through the advection solve
  and through the pressure solves can each be left out of the backward pass
  (that solve's output is then a constant of the backward pass), leaving the
  bypass paths when both are left out.

Readings of points the paper leaves open (the same readings the CUDA path
implements; each is listed in the design notes):

* R1 every momentum row is taken per unit volume: C_P = 1/dt + (1/J_P)(...),
  C_F = (1/J_P)(0.5 N_f U_f - nu mean(alpha_jj)), matching the 1/J_P of the
  velocity right-hand side.
* R2 face interpolation is the arithmetic mean of the two cells.
* R3 boundary faces use the adjacent cell's metrics.
* R4 the predictor right-hand side is the discrete Eq. velRHSdiscrete, without
  a pressure gradient (the -grad p of Eq. advectionMat is an option: with the
  compact pressure matrix and the wide central gradient it makes the pressure
  iteration unstable on anisotropic cells); h never contains it.
* R5 at a Dirichlet face the missing pressure neighbour is p_P.
* R6 the divergence b includes the prescribed boundary flux N_b J_P T_j . u_b.
* R7 the pressure system is singular (constants); b is projected to zero mean
  and each solution is returned with zero mean.
* R10 the outflow update uses the stable factor c/(1+c), c = 2 dt |T_j . u_m|.
* App. A.2 "Non-Orthogonal Grids" (Eqs. difNonOrthoMatDiscrete,
  velRHSnonOrtho, pressureRHSnonOrtho): on meshes whose cross metrics
  alpha_jk (j != k) do not vanish (``allow_nonorthogonal=True``), the cross
  derivatives of the diffusion are split as the paper does: the terms on P's
  direct neighbours join the matrix C (Eq. difNonOrthoMatDiscrete), those on
  its diagonal neighbours go to the right-hand side with the previous iterate
  (Eq. velRHSnonOrtho); the cross derivatives of the pressure Laplacian are
  deferred to the right-hand side whole (Eq. pressureRHSnonOrtho; their
  direct-neighbour part would make P unsymmetric for the CG).  The solves are
  repeated ``n_nonortho`` times (non-orthogonal corrector steps) and the
  adjoint runs those loops in reverse (the starting pressure p^n now matters
  through the pressure cross terms).  ``nonortho_split="deferred"`` defers
  the viscous terms whole as well.  Without the flag such meshes are rejected.
* Block connections join a side to the opposite side of the same axis with the
  same tangential ordering (no axis permutation).
"""
from __future__ import annotations

import dataclasses
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np
import scipy.sparse as sp

from . import krylov


# ----------------------------------------------------------------------------
# mesh: metrics, neighbours, boundary faces
# ----------------------------------------------------------------------------

@dataclasses.dataclass
class Options:
    pred_grad_p: bool = False    # R4: predictor rhs of Eq. velRHSdiscrete (no grad p^n) by default
    n_correctors: int = 2        # App. A.1: two corrector rounds
    n_nonortho: int = 1          # App. A.2: solves per predictor / pressure solve on non-orthogonal meshes
    adv_rtol: float = 1e-13
    p_rtol: float = 1e-13
    atol: float = 0.0
    maxit: int = 20000
    solver: str = "auto"         # "krylov" | "direct" | "auto" (direct where a sparse LU is cheap)
    update_outflow: bool = True  # App. A.3 advective outflow update before the step
    grad_adv: bool = True        # Sec. 2.4: keep the gradient paths through the advection solve
    grad_p: bool = True          # Sec. 2.4: keep the gradient paths through the pressure solves
    adv_precond: str = "none"    # App. A.5: BiCGStab preconditioner "none" | "ilu" (ILU(0)) |
                                 # "ilu_on_failure" (ILU(0) only after the plain solve failed)
    nonortho_split: str = "paper"  # App. A.2: "paper" keeps the direct-neighbour part of the viscous cross
                                 # terms in C (Eq. difNonOrthoMatDiscrete) and defers the diagonal-neighbour
                                 # part (Eq. velRHSnonOrtho); "deferred" moves every cross term to the
                                 # right-hand side.  The pressure cross terms are deferred in both.


class Mesh:
    """Multi-block structured mesh (Sec. 2.2; App. A.5 Domain/Block/Boundary).

    blocks: sequence of (res, vertices); connections: (blk_a, side_a, blk_b, side_b)
    or (blk_a, side_a, blk_b, side_b, axis_perm, flip_mask); dirichlet: (blk, side,
    values (nfaces, ndim)); outflow: (blk, side, u_m, values).

    A connection joins side_a of block a to side_b of block b, cell to cell
    (Sec. 2.2: conformal, matching resolution; App. A.3: it only changes the
    neighbour lookup): the i-th tangential axis of side_a (ascending axis
    order) runs along tangential axis (i if axis_perm == 0 else 1 - i) of
    side_b, reversed when bit i of flip_mask is set; any two sides may be
    joined, a side to itself as a fold.  The neighbour across a side then has
    its own frame: nbax[s, P, a] is the neighbour's axis for P's axis a and
    nbsg[s, P, a] = +1 / -1 its orientation (the normal's orientation follows
    from the two sides), nbret[s, P] the neighbour's side that faces P.  Every
    per-axis quantity of a neighbour (contravariant fluxes, alpha_jj, the cross
    metrics, its central differences) is read through that frame.
    """

    def __init__(self, ndim: int, blocks: Sequence, connections: Sequence = (),
                 dirichlet: Sequence = (), outflow: Sequence = (), allow_nonorthogonal: bool = False):
        self.ndim = d = ndim
        self.nsides = 2 * d
        self.res = [tuple(int(v) for v in (b[0] if isinstance(b, tuple) else b.res)) for b in blocks]
        verts = [np.asarray(b[1] if isinstance(b, tuple) else b.vertices, dtype=np.float64) for b in blocks]
        self.offsets = np.cumsum([0] + [r[0] * r[1] * r[2] for r in self.res])
        self.N = N = int(self.offsets[-1])

        # --- metrics at cell centres (App. A.2): M_ik = d x_i / d xi^k from
        # differences of opposite face centres, T = M^-1, J = det M.
        M = np.zeros((N, d, d))
        for bi, (r, V) in enumerate(zip(self.res, verts)):
            o = self.offsets[bi]
            M[o:o + r[0] * r[1] * r[2]] = _block_jacobian(V, d)
        self.J = np.linalg.det(M)
        if np.any(self.J <= 0):
            raise ValueError("mesh has cells with non-positive volume")
        self.T = np.linalg.inv(M)                     # T[i, j, k] = d xi^j / d x_k at cell i
        G = np.einsum("njk,nlk->njl", self.T, self.T) * self.J[:, None, None]
        self.alpha = np.stack([G[:, j, j] for j in range(d)])   # (d, N): alpha_jj
        self.G = G                                    # (N, d, d): alpha_jk = J T_j . T_k
        off = np.abs(G - np.einsum("nj,jk->njk", self.alpha.T, np.eye(d)))
        self.has_cross = bool(off.max() > 1e-9 * np.abs(G).max())
        if self.has_cross and not allow_nonorthogonal:
            raise ValueError("non-orthogonal mesh: cross-diffusion terms are not supported")

        # --- neighbours and boundary faces
        self.nb = -np.ones((self.nsides, N), dtype=np.int64)
        self.nbax = np.broadcast_to(np.arange(3), (self.nsides, N, 3)).copy()
        self.nbsg = np.ones((self.nsides, N, 3))
        self.nbret = np.repeat(np.array([s ^ 1 for s in range(self.nsides)])[:, None], N, axis=1)
        self.bval = np.zeros((self.nsides, d, N))
        self.is_bface = np.zeros((self.nsides, N), dtype=bool)
        self.is_outflow = np.zeros((self.nsides, N), dtype=bool)
        self.u_m = np.zeros((self.nsides, d, N))
        assigned = {}
        for conn in connections:
            a, sa, b, sb = conn[:4]
            perm, flip = (int(conn[4]), int(conn[5])) if len(conn) > 4 else (0, 0)
            for key in {(a, sa), (b, sb)}:
                if key in assigned:
                    raise ValueError(f"side {key} has two boundaries")
                assigned[key] = "conn"
            self._connect(a, sa, b, sb, perm, flip)
            if (a, sa) != (b, sb):
                # the inverse map: the swap is its own inverse, the flip bits follow the axes
                iflip = (((flip & 1) << 1) | ((flip >> 1) & 1)) if perm else flip
                self._connect(b, sb, a, sa, perm, iflip)
            else:
                ca = self.side_cells(a, sa)
                cb = self.nb[sa, ca]
                if np.any(cb == ca) or np.any(self.nb[sa, cb] != ca):
                    raise ValueError("a side joined to itself must pair distinct cells")
        for (blk, s, vals) in dirichlet:
            if (blk, s) in assigned:
                raise ValueError(f"side {(blk, s)} has two boundaries")
            assigned[(blk, s)] = "dir"
            self._set_faces(blk, s, np.asarray(vals, dtype=np.float64), None)
        for (blk, s, um, vals) in outflow:
            if (blk, s) in assigned:
                raise ValueError(f"side {(blk, s)} has two boundaries")
            assigned[(blk, s)] = "out"
            self._set_faces(blk, s, np.asarray(vals, dtype=np.float64), np.asarray(um, dtype=np.float64))
        # interior neighbours inside each block
        for bi, r in enumerate(self.res):
            o = self.offsets[bi]
            idx, coords = _block_index(r)
            strides = (1, r[0], r[0] * r[1])
            for s in range(self.nsides):
                ax, hi = s // 2, s % 2
                c = coords[ax]
                inner = (c < r[ax] - 1) if hi else (c > 0)
                step = strides[ax] if hi else -strides[ax]
                self.nb[s, o + idx[inner]] = o + idx[inner] + step
                if not np.all(inner) and (bi, s) not in assigned:
                    raise ValueError(f"block {bi} side {s} has no boundary")
        self.safe_nb = np.where(self.nb >= 0, self.nb, np.arange(N)[None, :])
        self.inner = self.nb >= 0
        self.has_outflow = bool(self.is_outflow.any())
        self.twisted = bool(np.any(self.nbax != np.arange(3)) or np.any(self.nbsg != 1.0))

    # -- boundary helpers ------------------------------------------------------
    def side_cells(self, blk: int, s: int) -> np.ndarray:
        """Global indices of the cells on a block side, in boundary-face order."""
        r = self.res[blk]
        o = self.offsets[blk]
        ax, hi = s // 2, s % 2
        idx, coords = _block_index(r)
        m = coords[ax] == (r[ax] - 1 if hi else 0)
        cells = idx[m]
        t = [a for a in range(3) if a != ax][: 2 if self.ndim == 3 else 1]
        # face order: lower tangential axis fastest
        keys = [coords[a][m] for a in t]
        if len(keys) == 2:
            order = np.lexsort((keys[0], keys[1]))
        else:
            order = np.argsort(keys[0], kind="stable")
        return o + cells[order]

    def _connect(self, a, sa, b, sb, perm=0, flip=0):
        d = self.ndim
        ra, rb = self.res[a], self.res[b]
        ja, jb = sa // 2, sb // 2
        ta = [x for x in range(3) if x != ja][: d - 1]
        tb = [x for x in range(3) if x != jb][: d - 1]
        pt = [1, 0] if perm else [0, 1]
        if (d == 2 and perm) or perm not in (0, 1) or flip >> (d - 1):
            raise ValueError("axis_perm / flip_mask out of range")
        for i in range(d - 1):
            if ra[ta[i]] != rb[tb[pt[i]]]:
                raise ValueError("connected sides must have matching resolution")
        ca = self.side_cells(a, sa)
        _, coords = _block_index(ra)
        la = ca - self.offsets[a]
        cc = [np.zeros(len(ca), dtype=np.int64) for _ in range(3)]
        cc[jb][:] = rb[jb] - 1 if sb % 2 else 0
        for i in range(d - 1):
            v = coords[ta[i]][la]
            if (flip >> i) & 1:
                v = ra[ta[i]] - 1 - v
            cc[tb[pt[i]]] = v
        self.nb[sa, ca] = self.offsets[b] + cc[0] + rb[0] * (cc[1] + rb[1] * cc[2])
        ax = list(range(3))
        sg = [1.0, 1.0, 1.0]
        ax[ja] = jb
        sg[ja] = -sign(sa) * sign(sb)       # P's outward normal is the neighbour's inward one
        for i in range(d - 1):
            ax[ta[i]] = tb[pt[i]]
            sg[ta[i]] = -1.0 if (flip >> i) & 1 else 1.0
        self.nbax[sa, ca] = ax
        self.nbsg[sa, ca] = sg
        self.nbret[sa, ca] = sb

    def frame(self, s: int, P: np.ndarray, a):
        """(the neighbour's axis, its orientation) for P's axis a (an int or an
        array over P) across side s of the cells P."""
        if np.isscalar(a):
            return self.nbax[s, P, a], self.nbsg[s, P, a]
        return self.nbax[s, P, a], self.nbsg[s, P, a]

    def _set_faces(self, blk, s, vals, um):
        cells = self.side_cells(blk, s)
        if vals.shape != (len(cells), self.ndim):
            raise ValueError(f"boundary values for block {blk} side {s} must be ({len(cells)}, {self.ndim})")
        self.is_bface[s, cells] = True
        self.bval[s, :, cells] = vals
        if um is not None:
            self.is_outflow[s, cells] = True
            self.u_m[s, :, cells] = um[None, :]

    def side_values(self, bval, blk, s):
        return bval[s, :, self.side_cells(blk, s)]

    # -- elementary per-cell quantities ---------------------------------------
    def contravariant(self, v: np.ndarray) -> np.ndarray:
        """U^j = J T_j . v at each cell (App. A.2), shape (d, N)."""
        return np.einsum("n,njk,kn->jn", self.J, self.T, v)

    def face_flux_b(self, s: int, vb: np.ndarray) -> np.ndarray:
        """J_P T_j,P . v_b for the boundary face on side s of every cell (R3)."""
        j = s // 2
        return self.J * np.einsum("nk,kn->n", self.T[:, j, :], vb)


def _block_index(r):
    nx, ny, nz = r
    idx = np.arange(nx * ny * nz)
    x = idx % nx
    y = (idx // nx) % ny
    z = idx // (nx * ny)
    return idx, (x, y, z)


def _block_jacobian(V: np.ndarray, d: int) -> np.ndarray:
    """d x / d xi at cell centres from opposite face-centre differences."""
    if d == 2:                                    # V[y, x, 2]
        fxm = 0.5 * (V[:-1, :-1] + V[1:, :-1])
        fxp = 0.5 * (V[:-1, 1:] + V[1:, 1:])
        fym = 0.5 * (V[:-1, :-1] + V[:-1, 1:])
        fyp = 0.5 * (V[1:, :-1] + V[1:, 1:])
        cols = [fxp - fxm, fyp - fym]             # each (ny, nx, 2)
        M = np.stack(cols, axis=-1)               # (ny, nx, 2[i], 2[k])
        return M.reshape(-1, 2, 2)
    def face(a, b, c, e):
        return 0.25 * (a + b + c + e)
    v = V                                         # V[z, y, x, 3]
    fxm = face(v[:-1, :-1, :-1], v[:-1, 1:, :-1], v[1:, :-1, :-1], v[1:, 1:, :-1])
    fxp = face(v[:-1, :-1, 1:], v[:-1, 1:, 1:], v[1:, :-1, 1:], v[1:, 1:, 1:])
    fym = face(v[:-1, :-1, :-1], v[:-1, :-1, 1:], v[1:, :-1, :-1], v[1:, :-1, 1:])
    fyp = face(v[:-1, 1:, :-1], v[:-1, 1:, 1:], v[1:, 1:, :-1], v[1:, 1:, 1:])
    fzm = face(v[:-1, :-1, :-1], v[:-1, :-1, 1:], v[:-1, 1:, :-1], v[:-1, 1:, 1:])
    fzp = face(v[1:, :-1, :-1], v[1:, :-1, 1:], v[1:, 1:, :-1], v[1:, 1:, 1:])
    M = np.stack([fxp - fxm, fyp - fym, fzp - fzm], axis=-1)
    return M.reshape(-1, 3, 3)


def sign(s: int) -> float:
    """Face sign N_f: +1 on the + side of an axis, -1 on the - side."""
    return 1.0 if s % 2 else -1.0


def opp(s: int) -> int:
    return s ^ 1


# ----------------------------------------------------------------------------
# forward operators (App. A.2)
# ----------------------------------------------------------------------------

@dataclasses.dataclass
class Matrix:
    """Stencil matrix: row P = diag[P] x_P + sum_s off[s, P] x_{nb(P,s)}."""
    diag: np.ndarray
    off: np.ndarray


def assemble_C(mesh: Mesh, u, nu, dt, S, bval):
    """Advection-diffusion matrix C = C^t + C^adv + C^nu and the velocity
    right-hand side without the pressure gradient (Eqs. advMatDiscrete,
    difMatDiscrete, velRHSdiscrete; per-unit-volume rows, R1)."""
    d, N = mesh.ndim, mesh.N
    U = mesh.contravariant(u)
    diag = np.full(N, 1.0 / dt)
    off = np.zeros((mesh.nsides, N))
    rhs0 = u / dt
    if S is not None:
        rhs0 = rhs0 + S
    for s in range(mesh.nsides):
        j, n = s // 2, sign(s)
        P = np.nonzero(mesh.inner[s])[0]
        F = mesh.nb[s, P]
        jF, eF = mesh.frame(s, P, j)               # the neighbour's flux in P's frame
        Uf = 0.5 * (U[j, P] + eF * U[jF, F])
        Df = nu * 0.5 * (mesh.alpha[j, P] + mesh.alpha[jF, F])
        off[s, P] = (0.5 * n * Uf - Df) / mesh.J[P]
        diag[P] += (0.5 * n * Uf + Df) / mesh.J[P]
        B = np.nonzero(mesh.is_bface[s])[0]
        ub = bval[s][:, B]
        Ub = mesh.face_flux_b(s, bval[s])[B]
        diag[B] += 2.0 * mesh.alpha[j, B] * nu / mesh.J[B]
        rhs0[:, B] += ub * ((2.0 * mesh.alpha[j, B] * nu - n * Ub) / mesh.J[B])[None, :]
    return Matrix(diag, off), rhs0


def matvec(mesh: Mesh, M: Matrix, x: np.ndarray) -> np.ndarray:
    """y = M x for a scalar field (N,) or each component of (d, N)."""
    y = M.diag * x
    for s in range(mesh.nsides):
        y = y + M.off[s] * x[..., mesh.safe_nb[s]]
    return y


def matvec_T(mesh: Mesh, M: Matrix, y: np.ndarray) -> np.ndarray:
    """x = M^T y, gathered: the entry of row F = nb(P,s) that points back at P
    is F's coefficient on its side facing P (the opposite side within a
    block)."""
    x = M.diag * y
    for s in range(mesh.nsides):
        F = mesh.safe_nb[s]
        coef = np.where(mesh.inner[s], M.off[mesh.nbret[s], F], 0.0)
        x = x + coef * y[..., F]
    return x


def offdiag_matvec(mesh: Mesh, M: Matrix, x):
    return matvec(mesh, Matrix(np.zeros(mesh.N), M.off), x)


def to_sparse(mesh: Mesh, M: Matrix) -> sp.csr_matrix:
    rows = [np.arange(mesh.N)]
    cols = [np.arange(mesh.N)]
    vals = [M.diag]
    for s in range(mesh.nsides):
        P = np.nonzero(mesh.inner[s])[0]
        rows.append(P)
        cols.append(mesh.nb[s, P])
        vals.append(M.off[s, P])
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(mesh.N, mesh.N))


def grad_p(mesh: Mesh, p: np.ndarray) -> np.ndarray:
    """(grad p)_i = sum_j T_ji (p_{j+1} - p_{j-1}) / 2 (Eq. velCorrDiscrete), with
    p_P standing in for a missing neighbour at Dirichlet faces (R5)."""
    d = mesh.ndim
    g = np.zeros((d, mesh.N))
    for j in range(d):
        dp = 0.5 * (p[mesh.safe_nb[2 * j + 1]] - p[mesh.safe_nb[2 * j]])
        g += mesh.T[:, j, :].T * dp[None, :]
    return g


def grad_p_T(mesh: Mesh, g: np.ndarray) -> np.ndarray:
    """Transpose of grad_p: p_bar = sum over the stencil of T_ji g_i (+-0.5)."""
    d = mesh.ndim
    out = np.zeros(mesh.N)
    for j in range(d):
        w = 0.5 * np.einsum("nk,kn->n", mesh.T[:, j, :], g)   # per-cell 0.5 T_j . g
        np.add.at(out, mesh.safe_nb[2 * j + 1], w)
        np.add.at(out, mesh.safe_nb[2 * j], -w)
    return out


def assemble_P(mesh: Mesh, A: np.ndarray) -> Matrix:
    """Pressure matrix: P_F = mean(alpha_jj / A) over the face, P_P = -sum P_F
    (Eq. pMatDiscrete); Dirichlet faces contribute nothing (0-Neumann)."""
    w = mesh.alpha / A[None, :]
    off = np.zeros((mesh.nsides, mesh.N))
    for s in range(mesh.nsides):
        j = s // 2
        P = np.nonzero(mesh.inner[s])[0]
        jF, _ = mesh.frame(s, P, j)
        off[s, P] = 0.5 * (w[j, P] + w[jF, mesh.nb[s, P]])
    return Matrix(-off.sum(axis=0), off)


def pressure_rhs_vec(mesh: Mesh, C: Matrix, rhs0: np.ndarray, u: np.ndarray) -> np.ndarray:
    """h = A^-1 (u^n/dt + boundary terms + S - H u)  (Eq. pressureRHSdiscrete)."""
    return (rhs0 - offdiag_matvec(mesh, C, u)) / C.diag[None, :]


def divergence(mesh: Mesh, h: np.ndarray, bval) -> np.ndarray:
    """b_P = sum_f N_f mean(J T_j . h) over inner faces (Eq. pressureRHSdivDiscrete)
    plus the prescribed flux N_b J_P T_j . u_b over Dirichlet faces (R6)."""
    F = mesh.contravariant(h)
    b = np.zeros(mesh.N)
    for s in range(mesh.nsides):
        j, n = s // 2, sign(s)
        P = np.nonzero(mesh.inner[s])[0]
        jF, eF = mesh.frame(s, P, j)
        b[P] += n * 0.5 * (F[j, P] + eF * F[jF, mesh.nb[s, P]])
        B = np.nonzero(mesh.is_bface[s])[0]
        b[B] += n * mesh.face_flux_b(s, bval[s])[B]
    return b


def divergence_T(mesh: Mesh, gb: np.ndarray) -> np.ndarray:
    """Transpose of the inner-face part of ``divergence``:
    h_bar_P = sum_f 0.5 N_f J_P T_j,P (b_bar_P - b_bar_F)  (the neighbour's row
    sees the same face with the opposite sign: across a permuted or flipped
    connection both its face sign and its flux's orientation change, and the
    two signs cancel)."""
    d = mesh.ndim
    gF = np.zeros((d, mesh.N))
    for s in range(mesh.nsides):
        j, n = s // 2, sign(s)
        P = np.nonzero(mesh.inner[s])[0]
        gF[j, P] += n * 0.5 * (gb[P] - gb[mesh.nb[s, P]])
    # F^j = J T_j . h  ->  h_bar_k = J sum_j T_jk F_bar^j
    return np.einsum("n,njk,jn->kn", mesh.J, mesh.T, gF)


def correct(mesh: Mesh, h, A, p):
    """u = h - A^-1 grad p (Eq. velCorrDiscrete)."""
    return h - grad_p(mesh, p) / A[None, :]


# ----------------------------------------------------------------------------
# non-orthogonal cross terms (App. A.2 "Non-Orthogonal Grids")
# ----------------------------------------------------------------------------

def _cell_diff(mesh: Mesh, q: np.ndarray, k: int, ghost) -> np.ndarray:
    """Central difference of the cell values q (N,) along computational axis k:
    (q_{k+} - q_{k-}) / 2, a missing neighbour (a boundary face on side s)
    replaced by ghost(s) (N,)."""
    hi = np.where(mesh.inner[2 * k + 1], q[mesh.safe_nb[2 * k + 1]], ghost(2 * k + 1))
    lo = np.where(mesh.inner[2 * k], q[mesh.safe_nb[2 * k]], ghost(2 * k))
    return 0.5 * (hi - lo)


def _nb_metric(mesh: Mesh, coef: np.ndarray, s: int, P, F, j: int, k: int):
    """coef_jk of the neighbours F = nb(P, s) in P's frame (coef (N, d, d))."""
    jF, ej = mesh.frame(s, P, j)
    kF, ek = mesh.frame(s, P, k)
    return ej * ek * coef[F, jF, kF]


def _nb_diff(mesh: Mesh, dq, s: int, P, F, k: int):
    """The central difference along P's axis k of the neighbours F = nb(P, s),
    from their own differences (dq (d, N), each cell's own axes)."""
    kF, ek = mesh.frame(s, P, k)
    return ek * dq[kF, F]


def _nb_side(mesh: Mesh, s_conn: int, P, s: int):
    """The side of the neighbours across s_conn of the cells P that corresponds
    to P's side s (its axis and orientation through the frame)."""
    jF, ej = mesh.frame(s_conn, P, s // 2)
    return 2 * jF + ((sign(s) * ej) > 0).astype(np.int64)


def _cross_flux_sum(mesh: Mesh, coef: np.ndarray, dq, bface_grad, part: str = "all") -> np.ndarray:
    """sum_j sum_{k != j} sum_{faces f of P on axis j} N_f c_jk,f g_k,f for one
    scalar field: c_jk,f the face mean of coef (N, d, d) over P and its
    neighbour, g_k,f the mean of the two cells' central differences dq[k] (d, N)
    along P's axis k (the neighbour's values read through its frame).
    Boundary faces: c_jk of P and g_k = bface_grad(s, k) (N,), or no flux when
    bface_grad is None.  part selects the terms: "all"; "own", the halves with
    P's own differences dq[k][P] (its direct neighbours) and the boundary
    faces; "nbr", the halves with the neighbour's differences dq[k][F] (P's
    diagonal neighbours).  "own" + "nbr" = "all"."""
    d = mesh.ndim
    dq = np.asarray(dq)
    out = np.zeros(mesh.N)
    for s in range(mesh.nsides):
        j, n = s // 2, sign(s)
        P = np.nonzero(mesh.inner[s])[0]
        F = mesh.nb[s, P]
        B = np.nonzero(mesh.is_bface[s])[0]
        for k in range(d):
            if k == j:
                continue
            cf = 0.5 * (coef[P, j, k] + _nb_metric(mesh, coef, s, P, F, j, k))
            dF = _nb_diff(mesh, dq, s, P, F, k)
            if part == "all":
                out[P] += n * cf * 0.5 * (dq[k][P] + dF)
            elif part == "own":
                out[P] += n * cf * 0.5 * dq[k][P]
            else:
                out[P] += n * cf * 0.5 * dF
            if bface_grad is not None and len(B) and part != "nbr":
                out[B] += n * coef[B, j, k] * bface_grad(s, k)[B]
    return out


def cross_diffusion(mesh: Mesh, u: np.ndarray, nu: float, bval, part: str = "all") -> np.ndarray:
    """Cross-derivative part of the viscous term per unit volume, (nu / J_P)
    sum_j sum_{k != j} sum_f N_f mean(alpha_jk) (d_k u)_f, for every velocity
    component (the part of Eqs. difNonOrthoMatDiscrete / velRHSnonOrtho that
    the orthogonal matrix C leaves out).  Cell differences use the ghost value
    2 u_b - u_P at Dirichlet faces (linear through the face value); on a
    Dirichlet face the tangential derivative is the central difference of the
    boundary values of the neighbouring faces on the same side (a face whose
    neighbour has none uses its own value in its place)."""
    d = mesh.ndim
    out = np.zeros((d, mesh.N))
    bval = np.asarray(bval)
    for c in range(d):
        q = u[c]
        ghost = lambda s, c=c, q=q: 2.0 * bval[s][c] - q
        dq = np.array([_cell_diff(mesh, q, k, ghost) for k in range(d)])

        def bgrad(s, k, c=c):
            fb = bval[s][c]
            allc = np.arange(mesh.N)
            vals = []
            for sk in (2 * k + 1, 2 * k):
                Q = mesh.safe_nb[sk]
                sq = _nb_side(mesh, sk, allc, s)          # the k-neighbour's side matching s
                ok = mesh.inner[sk] & mesh.is_bface[sq, Q]
                vals.append(np.where(ok, bval[sq, c, Q], fb))
            return 0.5 * (vals[0] - vals[1])
        out[c] = nu * _cross_flux_sum(mesh, mesh.G, dq, bgrad, part) / mesh.J
    return out


def cross_matrix(mesh: Mesh, nu: float) -> Matrix:
    """The direct-neighbour part of the viscous cross terms as matrix entries
    (Eq. difNonOrthoMatDiscrete): in part "own" of cross_diffusion every face
    tangential derivative uses P's own central difference (q_{k+} - q_{k-})/2,
    so that part is W_k(P) (q_{k+} - q_{k-})/2 with W_k(P) = sum over P's inner
    faces on the axes j != k of N_f mean(alpha_jk) / 2, times nu / J_P; a
    missing k-neighbour's ghost 2 u_b - q_P puts -/+ W_k / 2 on the diagonal
    (its 2 u_b part is a constant).  Returns M with cross_diffusion(u, "own") =
    M u + cross_diffusion(0, "own") for each velocity component; the matrix of
    the paper's split is C - M."""
    d, N = mesh.ndim, mesh.N
    W = np.zeros((d, N))
    for s in range(mesh.nsides):
        j, n = s // 2, sign(s)
        P = np.nonzero(mesh.inner[s])[0]
        F = mesh.nb[s, P]
        for k in range(d):
            if k != j:
                W[k][P] += n * 0.5 * (mesh.G[P, j, k] + _nb_metric(mesh, mesh.G, s, P, F, j, k)) * 0.5
    diag = np.zeros(N)
    off = np.zeros((mesh.nsides, N))
    for k in range(d):
        for s, w in ((2 * k + 1, 0.5), (2 * k, -0.5)):
            inn = mesh.inner[s]
            off[s, inn] += w * W[k][inn]
            diag[~inn] -= w * W[k][~inn]
    f = nu / mesh.J
    return Matrix(f * diag, f[None, :] * off)


def cross_pressure(mesh: Mesh, p: np.ndarray, A: np.ndarray) -> np.ndarray:
    """Cross-derivative part of the pressure operator, sum_j sum_{k != j} sum_f
    N_f mean(alpha_jk / A) (d_k p)_f (cell-integrated like the matrix P of Eq.
    pMatDiscrete; the part Eq. pressureRHSnonOrtho moves to the right-hand
    side).  Cell differences take p_P for a missing neighbour and no cross flux
    crosses a Dirichlet-velocity face (zero-Neumann pressure, App. A.3)."""
    d = mesh.ndim
    ghost = lambda s: p
    dq = np.array([_cell_diff(mesh, p, k, ghost) for k in range(d)])
    return _cross_flux_sum(mesh, mesh.G / A[:, None, None], dq, None)


def _cell_diff_T(mesh: Mesh, gd: np.ndarray, k: int, gq: np.ndarray, ghost_coef: float, gghost=None):
    """Transpose of _cell_diff along k: add to gq (N,) the gradient of
    sum_Q gd_Q dq_k(Q).  A missing neighbour's ghost is ghost_coef * q_Q + 2 q_b
    (velocity: -1, pressure: +1 with no boundary term); gghost(s) receives the
    boundary-value part (velocity only)."""
    for s, w in ((2 * k + 1, 0.5), (2 * k, -0.5)):
        inn = mesh.inner[s]
        np.add.at(gq, mesh.nb[s, inn], w * gd[inn])
        out = ~inn
        gq[out] += w * ghost_coef * gd[out]
        if gghost is not None:
            gghost(s)[out] += w * 2.0 * gd[out]


def cross_diffusion_T(mesh: Mesh, g: np.ndarray, nu: float, part: str = "all"):
    """Transpose of cross_diffusion (the same part) in u and in the boundary
    values: returns (dL/du (d, N), dL/dbval per side [nsides](d, N)) for
    dL/dX = g."""
    d, N = mesh.ndim, mesh.N
    gu = np.zeros((d, N))
    gb = np.zeros((mesh.nsides, d, N))
    for c in range(d):
        w = nu * g[c] / mesh.J
        gdk = np.zeros((d, N))                      # per cell, along its own axes
        for s in range(mesh.nsides):
            j, n = s // 2, sign(s)
            P = np.nonzero(mesh.inner[s])[0]
            F = mesh.nb[s, P]
            B = np.nonzero(mesh.is_bface[s])[0]
            for k in range(d):
                if k == j:
                    continue
                t = n * 0.5 * (mesh.G[P, j, k] + _nb_metric(mesh, mesh.G, s, P, F, j, k)) * 0.5 * w[P]
                if part != "nbr":
                    np.add.at(gdk[k], P, t)
                if part != "own":
                    kF, ek = mesh.frame(s, P, k)
                    np.add.at(gdk, (kF, F), ek * t)
                if len(B) and part != "nbr":
                    tb = n * mesh.G[B, j, k] * w[B] * 0.5
                    for sk, sg_ in ((2 * k + 1, 1.0), (2 * k, -1.0)):
                        Q = mesh.safe_nb[sk][B]
                        sq = _nb_side(mesh, sk, B, s)
                        ok = mesh.inner[sk][B] & mesh.is_bface[sq, Q]
                        np.add.at(gb, (np.where(ok, sq, s), c, np.where(ok, Q, B)), sg_ * tb)
        for k in range(d):
            _cell_diff_T(mesh, gdk[k], k, gu[c], -1.0, lambda s, c=c: gb[s][c])
    return gu, list(gb)


def cross_pressure_T(mesh: Mesh, g: np.ndarray, p: np.ndarray, A: np.ndarray):
    """Transpose of cross_pressure: (dL/dp (N,), dL/dA (N,)) at (p, A) for
    dL/dY = g."""
    d, N = mesh.ndim, mesh.N
    gp = np.zeros(N)
    gA = np.zeros(N)
    dq = np.array([_cell_diff(mesh, p, k, lambda s: p) for k in range(d)])
    gdk = np.zeros((d, N))
    for s in range(mesh.nsides):
        j, n = s // 2, sign(s)
        P = np.nonzero(mesh.inner[s])[0]
        F = mesh.nb[s, P]
        for k in range(d):
            if k == j:
                continue
            GF = _nb_metric(mesh, mesh.G, s, P, F, j, k)
            cf = 0.5 * (mesh.G[P, j, k] / A[P] + GF / A[F])
            t = n * cf * 0.5 * g[P]
            np.add.at(gdk[k], P, t)
            kF, ek = mesh.frame(s, P, k)
            np.add.at(gdk, (kF, F), ek * t)
            gk = 0.5 * (dq[k][P] + _nb_diff(mesh, dq, s, P, F, k))
            np.add.at(gA, P, -n * 0.5 * mesh.G[P, j, k] / A[P] ** 2 * gk * g[P])
            np.add.at(gA, F, -n * 0.5 * GF / A[F] ** 2 * gk * g[P])
    for k in range(d):
        _cell_diff_T(mesh, gdk[k], k, gp, 1.0)
    return gp, gA


def outflow_update(mesh: Mesh, u, bval, dt):
    """Advective outflow (App. A.3, Eq. advOut, reading R10): each outflow face
    moves towards its cell value with factor c/(1+c), c = 2 dt |T_j . u_m|; then
    all outflow faces are scaled so the outflow balances the inflow through the
    other Dirichlet faces."""
    if not mesh.has_outflow:
        return bval
    bval = bval.copy()
    q_in = 0.0
    q_out = 0.0
    for s in range(mesh.nsides):
        j, n = s // 2, sign(s)
        O = np.nonzero(mesh.is_outflow[s])[0]
        if len(O):
            c = 2.0 * dt * np.abs(np.einsum("nk,kn->n", mesh.T[O, j, :], mesh.u_m[s][:, O]))
            f = c / (1.0 + c)
            bval[s][:, O] = bval[s][:, O] - f[None, :] * (bval[s][:, O] - u[:, O])
            q_out += float(np.sum(n * mesh.face_flux_b(s, bval[s])[O]))
        D = np.nonzero(mesh.is_bface[s] & ~mesh.is_outflow[s])[0]
        q_in -= float(np.sum(n * mesh.face_flux_b(s, bval[s])[D]))
    if q_out != 0.0:
        scale = q_in / q_out
        for s in range(mesh.nsides):
            O = np.nonzero(mesh.is_outflow[s])[0]
            bval[s][:, O] *= scale
    return bval


# ----------------------------------------------------------------------------
# linear solves
# ----------------------------------------------------------------------------

def use_direct(mesh, opts: Options) -> bool:
    """The linear systems of App. A.1 define u* and p* as their exact solutions;
    the oracle solves them by sparse LU where that is cheap (all 2D grids here,
    small 3D grids) and by Krylov iteration otherwise."""
    if opts.solver == "auto":
        return mesh.N <= (250000 if mesh.ndim == 2 else 8192)
    return opts.solver == "direct"


def bicgstab_adv(A, matvec, b, x0, opts: Options):
    """One advection-diffusion solve by BiCGStab with the preconditioning of
    App. A.5: none, ILU(0) of the assembled matrix A throughout, or ILU(0) only
    when the unpreconditioned solve did not converge (it then restarts from
    x0).  info.precond is "none", "ilu" or "ilu_after_failure"; info.iters
    counts the iterations of every attempt."""
    if opts.adv_precond not in ("none", "ilu", "ilu_on_failure"):
        raise ValueError(f"unknown adv_precond {opts.adv_precond!r}")
    if opts.adv_precond == "ilu":
        x, info = krylov.bicgstab(matvec, b, x0, opts.adv_rtol, opts.atol, opts.maxit,
                                  precond=krylov.ilu0_preconditioner(A))
        info.precond = "ilu"
        return x, info
    x, info = krylov.bicgstab(matvec, b, x0, opts.adv_rtol, opts.atol, opts.maxit)
    info.precond = "none"
    if info.converged or opts.adv_precond == "none":
        return x, info
    first = info.iters
    x, info = krylov.bicgstab(matvec, b, x0, opts.adv_rtol, opts.atol, opts.maxit,
                              precond=krylov.ilu0_preconditioner(A))
    info.iters += first
    info.precond = "ilu_after_failure"
    return x, info


def solve_C(mesh, C, rhs, x0, opts: Options):
    out = np.empty_like(rhs)
    infos = []
    if use_direct(mesh, opts):
        Cs = to_sparse(mesh, C)
        for c in range(rhs.shape[0]):
            out[c] = krylov.direct_solve(Cs, rhs[c])
        return out, infos
    Cs = to_sparse(mesh, C) if opts.adv_precond != "none" else None
    for c in range(rhs.shape[0]):
        out[c], info = bicgstab_adv(Cs, lambda v: matvec(mesh, C, v), rhs[c], x0[c], opts)
        infos.append(info)
    return out, infos


def solve_C_T(mesh, C, rhs, opts: Options):
    out = np.empty_like(rhs)
    if use_direct(mesh, opts):
        CsT = to_sparse(mesh, C).T
        for c in range(rhs.shape[0]):
            out[c] = krylov.direct_solve(CsT, rhs[c])
        return out
    CsT = to_sparse(mesh, C).T.tocsr() if opts.adv_precond != "none" else None
    for c in range(rhs.shape[0]):
        out[c], _ = bicgstab_adv(CsT, lambda v: matvec_T(mesh, C, v), rhs[c], np.zeros(mesh.N), opts)
    return out


def solve_P(mesh, Pm: Matrix, b, x0, opts: Options):
    """Solve P x = b for mean-free b; returns mean-free x (R7).  CG runs on the
    positive semi-definite -P."""
    if use_direct(mesh, opts):
        return krylov.direct_solve_singular(to_sparse(mesh, Pm), b), None
    neg = Matrix(-Pm.diag, -Pm.off)
    x, info = krylov.pcg(lambda v: matvec(mesh, neg, v), neg.diag, -b, x0, opts.p_rtol,
                         opts.atol, opts.maxit)
    return x - x.mean(), info


# ----------------------------------------------------------------------------
# the PISO step (App. A.1) and its adjoint (Sec. 2.3, App. A.4)
# ----------------------------------------------------------------------------

def piso_step(mesh: Mesh, u, p, dt, nu, S=None, bval=None, opts: Optional[Options] = None):
    """One PISO step.  Returns (u_new, p_new, tape); tape['bval'] holds the
    boundary values after the outflow update (they carry over to the next step)."""
    opts = opts or Options()
    bval = mesh.bval if bval is None else bval
    bval_in = bval
    updated = bool(opts.update_outflow and mesh.has_outflow)
    if opts.update_outflow:
        bval = outflow_update(mesh, u, bval, dt)
    C, rhs0 = assemble_C(mesh, u, nu, dt, S, bval)
    X = mesh.has_cross
    if opts.nonortho_split not in ("paper", "deferred"):
        raise ValueError(f"unknown nonortho_split {opts.nonortho_split!r}")
    paper = X and opts.nonortho_split == "paper"
    xpart = "nbr" if paper else "all"
    if paper:
        # App. A.2: the direct-neighbour cross entries join the matrix (Eq.
        # difNonOrthoMatDiscrete), their boundary-value constants the rhs
        Mx = cross_matrix(mesh, nu)
        C = Matrix(C.diag - Mx.diag, C.off - Mx.off)
        rhs0 = rhs0 + cross_diffusion(mesh, np.zeros_like(u), nu, bval, part="own")
    rhs = rhs0 - grad_p(mesh, p) if opts.pred_grad_p else rhs0
    # non-orthogonal meshes: the remaining cross-derivative terms are deferred
    # to the right-hand side with the previous iterate, n_nonortho solves each
    ustar = u
    ustar_it = [u]
    for _ in range(opts.n_nonortho if X else 1):
        rhs_m = rhs + cross_diffusion(mesh, ustar, nu, bval, xpart) if X else rhs
        ustar, adv_info = solve_C(mesh, C, rhs_m, ustar, opts)
        ustar_it.append(ustar)
    A = C.diag
    Pm = assemble_P(mesh, A)
    uk, pk = ustar, p
    corr = []
    p_infos = []
    for _ in range(opts.n_correctors):
        rhs0_k = rhs0 + cross_diffusion(mesh, uk, nu, bval, xpart) if X else rhs0
        h = pressure_rhs_vec(mesh, C, rhs0_k, uk)
        b = divergence(mesh, h, bval)
        b = b - b.mean()
        x = pk
        x_it = [pk]
        for _ in range(opts.n_nonortho if X else 1):
            bm = b - cross_pressure(mesh, x, A) if X else b
            x, info = solve_P(mesh, Pm, bm - bm.mean() if X else bm, x, opts)
            x_it.append(x)
        p_infos.append(info)
        unew = correct(mesh, h, A, x)
        corr.append(dict(u_in=uk, h=h, b=b, x=x, x_it=x_it))
        uk, pk = unew, x
    tape = dict(u=u, p=p, S=S, nu=nu, dt=dt, bval=bval, bval_in=bval_in, outflow_updated=updated, C=C,
                rhs0=rhs0, rhs=rhs, ustar=ustar, ustar_it=ustar_it, Pm=Pm, corr=corr, u_out=uk, p_out=pk,
                adv_info=adv_info, p_infos=p_infos, xpart=xpart)
    return uk, pk, tape


def outflow_update_adjoint(mesh: Mesh, u, bval_in, dt, g_used):
    """Transpose of ``outflow_update`` at (u, bval_in): given dL/d(bval after
    the update) per side, return (dL/d bval_in per side, dL/du).  Forward:
    b1 = (1 - f) b + f u_O on outflow faces (f = c/(1+c)); q_out = sum of the
    outflow faces' fluxes N J T_j . b1, q_in = -sum of the other Dirichlet
    faces' fluxes of b; outflow faces become (q_in / q_out) b1 (when q_out is
    not 0), the others are unchanged."""
    d, N = mesh.ndim, mesh.N
    g_in = [g.copy() for g in g_used]
    gu = np.zeros((d, N))
    if not mesh.has_outflow:
        return g_in, gu
    # forward quantities
    b1 = [b.copy() for b in bval_in]
    fac = [np.zeros(N) for _ in range(mesh.nsides)]
    q_in = q_out = 0.0
    for s in range(mesh.nsides):
        j, n = s // 2, sign(s)
        O = np.nonzero(mesh.is_outflow[s])[0]
        if len(O):
            c = 2.0 * dt * np.abs(np.einsum("nk,kn->n", mesh.T[O, j, :], mesh.u_m[s][:, O]))
            fac[s][O] = c / (1.0 + c)
            b1[s][:, O] = bval_in[s][:, O] - fac[s][O][None, :] * (bval_in[s][:, O] - u[:, O])
            q_out += float(np.sum(n * mesh.face_flux_b(s, b1[s])[O]))
        D = np.nonzero(mesh.is_bface[s] & ~mesh.is_outflow[s])[0]
        q_in -= float(np.sum(n * mesh.face_flux_b(s, bval_in[s])[D]))
    scaled = q_out != 0.0
    scale = q_in / q_out if scaled else 1.0
    # dL/dscale = sum over outflow faces of g_used . b1
    gscale = 0.0
    for s in range(mesh.nsides):
        O = np.nonzero(mesh.is_outflow[s])[0]
        gscale += float(np.sum(g_used[s][:, O] * b1[s][:, O]))
    for s in range(mesh.nsides):
        j, n = s // 2, sign(s)
        O = np.nonzero(mesh.is_outflow[s])[0]
        D = np.nonzero(mesh.is_bface[s] & ~mesh.is_outflow[s])[0]
        JT = mesh.J[:, None] * mesh.T[:, j, :]          # d(flux)/d(face value): J T_j
        g_in[s][:, O] = 0.0
        if len(O):
            gb1 = scale * g_used[s][:, O]
            if scaled:
                gb1 = gb1 - gscale * q_in / q_out ** 2 * n * JT[O].T
            g_in[s][:, O] = (1.0 - fac[s][O])[None, :] * gb1
            np.add.at(gu.T, O, (fac[s][O][None, :] * gb1).T)
        if scaled and len(D):
            g_in[s][:, D] += gscale / q_out * (-n) * JT[D].T
    return g_in, gu


def piso_step_adjoint(mesh: Mesh, tape: Dict, du_out, dp_out, opts: Optional[Options] = None,
                      want_bval: bool = False):
    """Reverse of ``piso_step``: given dL/du^{n+1} and dL/dp^{n+1}, return
    dL/du^n, dL/dp^n, dL/dS and dL/dnu, and with ``want_bval`` also dL/d(the
    boundary values before the step's outflow update), per side [nsides][d][N].
    The boundary values enter the momentum right-hand side (Dirichlet fluxes,
    Eq. velRHSdiscrete: u_b (2 alpha nu - N_f U_b)/J with U_b = J T_j . u_b)
    and every corrector's divergence (R6: N_f J T_j . u_b); the advective
    outflow update (Eq. advOut) is differentiated too, contributing to dL/du^n
    through the cell values it moves towards.

    ``opts.grad_adv`` / ``opts.grad_p`` select the gradient paths of Sec. 2.4:
    the full adjoint is J^Adv + J^P + J^none, and dropping a path treats that
    solve's output (u*, or every corrector's pressure) as a constant of the
    backward pass, i.e. its transposed solve contributes zero.  With both off
    only the bypass paths of Eq. jnone remain."""
    opts = opts or Options()
    X = mesh.has_cross
    xpart = tape.get("xpart", "all")
    d, N = mesh.ndim, mesh.N
    C, Pm = tape["C"], tape["Pm"]
    A = C.diag
    nu, dt, bval = tape["nu"], tape["dt"], tape["bval"]
    gA = np.zeros(N)                  # dL/dA (A = diag C)
    gCoff = np.zeros((mesh.nsides, N))
    grhs0 = np.zeros((d, N))
    gw = np.zeros((d, N))             # dL/d(alpha_jj / A)
    gu = np.array(du_out, dtype=np.float64, copy=True)
    gp_last = np.array(dp_out, dtype=np.float64, copy=True)
    gbs = []                          # dL/db of every corrector (divergence right-hand sides)
    gbX = [np.zeros((d, N)) for _ in range(mesh.nsides)]   # non-orthogonal: dL/dbval via the cross terms
    gx_carry = np.zeros(N)            # non-orthogonal: dL/d(the next corrector's starting pressure)
    gnu_x = 0.0                       # non-orthogonal: dL/dnu through the cross terms (linear in nu)
    gp_in_x = np.zeros(N)
    ncorr = len(tape["corr"])
    for k in reversed(range(ncorr)):
        cr = tape["corr"][k]
        x, h, uin = cr["x"], cr["h"], cr["u_in"]
        # u_{k+1} = h - grad(x) / A
        gh = gu.copy()
        gx = -grad_p_T(mesh, gu / A[None, :])
        gA += np.sum(gu * grad_p(mesh, x), axis=0) / A ** 2
        if k == ncorr - 1:
            gx = gx + gp_last
        if X:
            gx = gx + gx_carry
        if X and opts.grad_p:
            # x_m = Pi P^+ Pi (b - Y(x_{m-1})), m = 1..n, x_0 = this corrector's
            # starting pressure: transposed solves in reverse order
            gb = np.zeros(N)
            gxm = gx
            xs = cr["x_it"]
            for m in range(len(xs) - 1, 0, -1):
                g0 = gxm - gxm.mean()
                y, _ = solve_P(mesh, Pm, g0, np.zeros(N), opts)
                y = y - y.mean()
                for s in range(mesh.nsides):
                    j = s // 2
                    P = np.nonzero(mesh.inner[s])[0]
                    F = mesh.nb[s, P]
                    gw[j, P] += 0.5 * (y[P] - y[F]) * (xs[m][P] - xs[m][F])
                gb += y
                gyx, gyA = cross_pressure_T(mesh, -y, xs[m - 1], A)
                gA += gyA
                gxm = gyx
            gx_carry = gxm
            gh += divergence_T(mesh, gb)
            gbs.append(gb)
        elif X:
            gx_carry = np.zeros(N)
        if opts.grad_p and not X:
            # x = Pi(P^+ Pi b): transposed (symmetric) solve
            gx = gx - gx.mean()
            y, _ = solve_P(mesh, Pm, gx, np.zeros(N), opts)
            gb = y - y.mean()
            # dP = -y (x) x on the pattern -> d(alpha/A): 0.5 (y_P - y_F)(x_P - x_F) per inner face
            for s in range(mesh.nsides):
                j = s // 2
                P = np.nonzero(mesh.inner[s])[0]
                F = mesh.nb[s, P]
                gw[j, P] += 0.5 * (y[P] - y[F]) * (x[P] - x[F])
            # b = div(h) + boundary flux
            gh += divergence_T(mesh, gb)
            gbs.append(gb)
        # without the pressure path (Sec. 2.4) x is a constant of the backward
        # pass: gx is dropped and neither b nor P receives a gradient
        # h = (rhs0 (+ X(u_in)) - H u_in) / A
        gg = gh / A[None, :]
        gA -= np.sum(gh * h, axis=0) / A
        grhs0 += gg
        gu = -offdiag_matvec_T(mesh, C, gg)
        for s in range(mesh.nsides):
            gCoff[s] -= np.sum(gg * uin[:, mesh.safe_nb[s]], axis=0) * mesh.inner[s]
        if X:
            gxu, gxb = cross_diffusion_T(mesh, gg, nu, xpart)
            gu = gu + gxu
            for s in range(mesh.nsides):
                gbX[s] += gxb[s]
            if nu:
                gnu_x += float(np.sum(gg * cross_diffusion(mesh, uin, nu, bval, xpart))) / nu
    if X:
        gp_in_x = gx_carry
    # pressure matrix built from w = alpha / A
    gA -= np.sum(gw * mesh.alpha, axis=0) / A ** 2
    # predictor: u* = C^-1 rhs
    ustar = tape["ustar"]
    # without the advection path (Sec. 2.4) u* is a constant of the backward
    # pass: the transposed solve is skipped and C, rhs receive nothing from it
    gu_pred = np.zeros((d, N))
    if X and opts.grad_adv:
        # u*_m = C^-1 (rhs + X(u*_{m-1})), m = 1..n, u*_0 = u^n
        its = tape["ustar_it"]
        grhs = np.zeros((d, N))
        gm = gu
        for m in range(len(its) - 1, 0, -1):
            z = solve_C_T(mesh, C, gm, opts)
            grhs += z
            gA -= np.sum(z * its[m], axis=0)
            for s in range(mesh.nsides):
                gCoff[s] -= np.sum(z * its[m][:, mesh.safe_nb[s]], axis=0) * mesh.inner[s]
            gxu, gxb = cross_diffusion_T(mesh, z, nu, xpart)
            for s in range(mesh.nsides):
                gbX[s] += gxb[s]
            if nu:
                gnu_x += float(np.sum(z * cross_diffusion(mesh, its[m - 1], nu, bval, xpart))) / nu
            gm = gxu
        gu_pred = gm
    else:
        z = solve_C_T(mesh, C, gu, opts) if opts.grad_adv else np.zeros_like(gu)
        grhs = z
        gA -= np.sum(z * ustar, axis=0)
        for s in range(mesh.nsides):
            gCoff[s] -= np.sum(z * ustar[:, mesh.safe_nb[s]], axis=0) * mesh.inner[s]
    grhs0 += grhs
    if xpart == "nbr":
        # the paper's split: C holds -M (linear in nu) and rhs0 the constant
        # part of the direct-neighbour cross terms (linear in nu and in the
        # boundary values)
        M1 = cross_matrix(mesh, 1.0)
        gnu_x -= float(np.sum(gA * M1.diag)) + float(np.sum(gCoff * M1.off))
        gnu_x += float(np.sum(grhs0 * cross_diffusion(mesh, np.zeros((d, N)), 1.0, bval, part="own")))
        _, gxb = cross_diffusion_T(mesh, grhs0, nu, part="own")
        for s in range(mesh.nsides):
            gbX[s] += gxb[s]
    gp_in = -grad_p_T(mesh, grhs) if opts.pred_grad_p else np.zeros(N)
    if X:
        gp_in = gp_in + gp_in_x
    # assembly
    gu_in = grhs0 / dt + gu_pred
    gS = grhs0.copy()
    gnu = gnu_x if X else 0.0
    gU = np.zeros((d, N))
    for s in range(mesh.nsides):
        j, n = s // 2, sign(s)
        P = np.nonzero(mesh.inner[s])[0]
        F = mesh.nb[s, P]
        # off[s,P] = (0.5 n Uf - nu Df)/J_P,  diag[P] += (0.5 n Uf + nu Df)/J_P
        gUf = 0.5 * n * (gCoff[s, P] + gA[P]) / mesh.J[P]
        np.add.at(gU[j], P, 0.5 * gUf)
        jF, eF = mesh.frame(s, P, j)
        np.add.at(gU, (jF, F), eF * 0.5 * gUf)
        Df = 0.5 * (mesh.alpha[j, P] + mesh.alpha[jF, F])
        gnu += float(np.sum((gA[P] - gCoff[s, P]) * Df / mesh.J[P]))
        B = np.nonzero(mesh.is_bface[s])[0]
        gnu += float(np.sum(gA[B] * 2.0 * mesh.alpha[j, B] / mesh.J[B]))
        ub = bval[s][:, B]
        gnu += float(np.sum(grhs0[:, B] * ub * (2.0 * mesh.alpha[j, B] / mesh.J[B])[None, :]))
    gu_in += np.einsum("n,njk,jn->kn", mesh.J, mesh.T, gU)
    # boundary values used by the step: rhs0 (assembly) and the divergences
    gbu = [np.zeros((d, N)) for _ in range(mesh.nsides)]
    for s in range(mesh.nsides):
        j, n = s // 2, sign(s)
        B = np.nonzero(mesh.is_bface[s])[0]
        if not len(B):
            continue
        ub = bval[s][:, B]
        TjB = mesh.T[B, j, :].T                                    # [d][nB]
        tu = np.sum(TjB * ub, axis=0)                             # T_j . u_b
        a = 2.0 * mesh.alpha[j, B] * nu / mesh.J[B] - n * tu
        g = grhs0[:, B]
        gbu[s][:, B] = g * a[None, :] - n * TjB * np.sum(g * ub, axis=0)[None, :]
        for gbk in gbs:
            gbu[s][:, B] += n * (mesh.J[B] * gbk[B])[None, :] * TjB
    if X:
        for s in range(mesh.nsides):
            gbu[s] = gbu[s] + gbX[s]
    if tape.get("outflow_updated", False):
        g_in, gu_o = outflow_update_adjoint(mesh, tape["u"], tape["bval_in"], dt, gbu)
        gu_in = gu_in + gu_o
    else:
        g_in = gbu
    if want_bval:
        return gu_in, gp_in, gS, gnu, g_in
    return gu_in, gp_in, gS, gnu


def offdiag_matvec_T(mesh: Mesh, M: Matrix, y):
    return matvec_T(mesh, Matrix(np.zeros(mesh.N), M.off), y)


# ----------------------------------------------------------------------------
# convenience
# ----------------------------------------------------------------------------

def mesh_from_case(case, allow_nonorthogonal: bool = False) -> Mesh:
    """Build a Mesh from any object with ndim/blocks/connections/dirichlet/outflow
    attributes (the seeded input generators produce such objects)."""
    return Mesh(case.ndim, [(b.res, b.vertices) for b in case.blocks], case.connections,
                case.dirichlet, case.outflow, allow_nonorthogonal)


def rollout(mesh: Mesh, u, p, dt, nu, S, steps, opts=None, bval=None):
    bval = mesh.bval if bval is None else bval
    for _ in range(steps):
        u, p, tape = piso_step(mesh, u, p, dt, nu, S, bval, opts)
        bval = tape["bval"]
    return u, p, bval


def rhie_chow_residual(mesh: Mesh, tape: Dict, k: int = -1) -> np.ndarray:
    """Face-flux divergence of corrector k in the compact (Rhie-Chow) form:
    sum_f N_f [mean(J T_j . h) - P_F (p_F - p_P)] + boundary flux = b - P x."""
    cr = tape["corr"][k]
    return cr["b"] - matvec(mesh, tape["Pm"], cr["x"])
