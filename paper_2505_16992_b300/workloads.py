"""Seeded synthetic inputs shaped like the paper's flow cases.

This module only builds *inputs*: block vertex coordinates, block connections,
boundary values, initial fields, sources and scalar parameters.  It holds none
of the solver's arithmetic (no metrics, no fluxes, no matrices, no solves), so
both the CUDA path and the CPU oracle can be fed from it.

Layout conventions shared by every consumer:

* Sides are numbered 0..5 = -x, +x, -y, +y, -z, +z (2D uses 0..3).
* A block of resolution (nx, ny, nz) owns cells with local index
  ``x + nx*(y + ny*z)``; global cell index = block offset + local index, blocks
  in the order they were added.
* Vertex arrays have shape ``(nz+1, ny+1, nx+1, ndim)`` in 3D and
  ``(ny+1, nx+1, 2)`` in 2D (x fastest).
* Fields are structure-of-arrays: velocity ``u[c, i]`` has shape (ndim, N),
  pressure ``p[i]`` shape (N,).
* Values on a block side are listed per boundary face, ordered by the two
  tangential cell indices with the lower axis fastest: x-sides (y, z), y-sides
  (x, z), z-sides (x, y).

Case parameters follow the paper's scenarios (lid-driven cavity, backward-facing
step channel, periodic turbulent channel, forced 2D turbulence; Sec. 4-5 and
App. B) at the sizes of the paper's workloads.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Tuple

import numpy as np

SIDE_XM, SIDE_XP, SIDE_YM, SIDE_YP, SIDE_ZM, SIDE_ZP = range(6)


@dataclasses.dataclass
class Block:
    res: Tuple[int, int, int]          # (nx, ny, nz); nz == 1 in 2D
    vertices: np.ndarray               # see module docstring

    @property
    def ncells(self) -> int:
        return self.res[0] * self.res[1] * self.res[2]


@dataclasses.dataclass
class Case:
    name: str
    ndim: int
    blocks: List[Block]
    connections: List[Tuple[int, int, int, int]]            # (blk_a, side_a, blk_b, side_b)
    dirichlet: List[Tuple[int, int, np.ndarray]]            # (blk, side, values (nfaces, ndim))
    outflow: List[Tuple[int, int, np.ndarray, np.ndarray]]  # (blk, side, u_m (ndim,), initial values)
    u0: np.ndarray                                          # (ndim, N)
    p0: np.ndarray                                          # (N,)
    S: Optional[np.ndarray]                                 # (ndim, N) or None
    nu: float
    dt: float
    steps: int

    @property
    def ncells(self) -> int:
        return sum(b.ncells for b in self.blocks)

    def block_offsets(self) -> List[int]:
        off, out = 0, []
        for b in self.blocks:
            out.append(off)
            off += b.ncells
        return out


# ----------------------------------------------------------------------------
# vertex coordinates
# ----------------------------------------------------------------------------

def uniform_vertices(n: int, lo: float, hi: float) -> np.ndarray:
    return np.linspace(lo, hi, n + 1)


def tanh_vertices(n: int, lo: float, hi: float, gamma: float) -> np.ndarray:
    """Vertices refined towards both ends: s_k = tanh(gamma(2k/n - 1))/tanh(gamma)."""
    k = np.arange(n + 1, dtype=np.float64)
    s = np.tanh(gamma * (2.0 * k / n - 1.0)) / math.tanh(gamma)
    s[0], s[-1] = -1.0, 1.0
    return lo + (hi - lo) * 0.5 * (s + 1.0)


def tensor_vertices(xv: np.ndarray, yv: np.ndarray, zv: Optional[np.ndarray] = None) -> np.ndarray:
    if zv is None:
        Y, X = np.meshgrid(yv, xv, indexing="ij")
        return np.stack([X, Y], axis=-1).astype(np.float64)
    Z, Y, X = np.meshgrid(zv, yv, xv, indexing="ij")
    return np.stack([X, Y, Z], axis=-1).astype(np.float64)


def rect_block(xv, yv, zv=None) -> Block:
    nz = 1 if zv is None else len(zv) - 1
    return Block((len(xv) - 1, len(yv) - 1, nz), tensor_vertices(xv, yv, zv))


def side_nfaces(res, side: int, ndim: int) -> int:
    nx, ny, nz = res
    ax = side // 2
    if ndim == 2:
        return ny if ax == 0 else nx
    return (ny * nz, nx * nz, nx * ny)[ax]


def cell_centres(block: Block) -> np.ndarray:
    """Cell-centre coordinates (ndim, ncells) as the mean of the cell's vertices.
    Used only to place initial and boundary values."""
    V = block.vertices
    if V.ndim == 3:
        c = 0.25 * (V[:-1, :-1] + V[1:, :-1] + V[:-1, 1:] + V[1:, 1:])
        return c.reshape(-1, 2).T.copy()
    c = 0.125 * (V[:-1, :-1, :-1] + V[1:, :-1, :-1] + V[:-1, 1:, :-1] + V[:-1, :-1, 1:]
                 + V[1:, 1:, :-1] + V[1:, :-1, 1:] + V[:-1, 1:, 1:] + V[1:, 1:, 1:])
    return c.reshape(-1, 3).T.copy()


def side_face_centres(block: Block, side: int) -> np.ndarray:
    """Face-centre coordinates (nfaces, ndim) of the boundary faces on one side."""
    V = block.vertices
    ax, hi = side // 2, side % 2
    if V.ndim == 3:  # 2D: V[y, x]
        if ax == 0:
            col = V[:, -1 if hi else 0]           # (ny+1, 2)
            return 0.5 * (col[:-1] + col[1:])
        row = V[-1 if hi else 0, :]               # (nx+1, 2)
        return 0.5 * (row[:-1] + row[1:])
    if ax == 0:
        s = V[:, :, -1 if hi else 0]              # (nz+1, ny+1, 3): faces (y fastest, then z)
    elif ax == 1:
        s = V[:, -1 if hi else 0, :]              # (nz+1, nx+1, 3)
    else:
        s = V[-1 if hi else 0, :, :]              # (ny+1, nx+1, 3)
    f = 0.25 * (s[:-1, :-1] + s[1:, :-1] + s[:-1, 1:] + s[1:, 1:])
    return f.reshape(-1, 3)


def wall(block: Block, side: int, ndim: int) -> np.ndarray:
    return np.zeros((side_nfaces(block.res, side, ndim), ndim))


# ----------------------------------------------------------------------------
# cases
# ----------------------------------------------------------------------------

def cavity2d(n: int = 32, nu: float = 0.01, dt: float = 0.005, steps: int = 200,
             lid_side: int = SIDE_YP, lid_speed: float = 1.0, stretch: float = 0.0) -> Case:
    """2D lid-driven cavity on [0,1]^2 (App. B.2).  The lid moves tangentially
    (+x for a y-side lid, +y for an x-side lid) with ``lid_speed``."""
    v = tanh_vertices(n, 0.0, 1.0, stretch) if stretch > 0 else uniform_vertices(n, 0.0, 1.0)
    b = rect_block(v, v)
    dirichlet = []
    for s in range(4):
        val = wall(b, s, 2)
        if s == lid_side:
            val[:, 1 - s // 2] = lid_speed
        dirichlet.append((0, s, val))
    N = b.ncells
    return Case("cavity2d", 2, [b], [], dirichlet, [], np.zeros((2, N)), np.zeros(N), None,
                nu, dt, steps)


def cavity3d(n: int = 16, nu: float = 0.01, dt: float = 0.005, steps: int = 10,
             periodic_z: bool = False, nz: Optional[int] = None) -> Case:
    nz = n if nz is None else nz
    v = uniform_vertices(n, 0.0, 1.0)
    zv = uniform_vertices(nz, 0.0, 1.0 * nz / n)
    b = rect_block(v, v, zv)
    dirichlet, conns = [], []
    for s in range(6):
        if periodic_z and s >= 4:
            continue
        val = wall(b, s, 3)
        if s == SIDE_YP:
            val[:, 0] = 1.0
        dirichlet.append((0, s, val))
    if periodic_z:
        conns.append((0, SIDE_ZP, 0, SIDE_ZM))
    N = b.ncells
    return Case("cavity3d", 3, [b], conns, dirichlet, [], np.zeros((3, N)), np.zeros(N), None,
                nu, dt, steps)


def channel3d(nx: int = 64, ny: int = 48, nz: int = 32, gamma: float = 2.0,
              nu: float = 1.0 / 180.0, dt: float = 0.01, amp: float = 0.1, seed: int = 0,
              steps: int = 1000, shear: float = 0.0) -> Case:
    """3D channel, periodic in x and z, no-slip walls at y = -1, 1 with tanh
    refinement; box 2pi x 2 x pi (App. B.4 geometry).  Constant streamwise
    forcing G = 2 nu makes u = 1 - y^2 the laminar steady state; the initial field
    is that profile plus seeded Gaussian noise.  shear != 0 slants the cells
    (x += shear * y at every vertex): the same channel on a non-orthogonal grid
    (cross metric alpha_xy != 0, App. A.2 "Non-Orthogonal Grids")."""
    xv = uniform_vertices(nx, 0.0, 2.0 * math.pi)
    yv = tanh_vertices(ny, -1.0, 1.0, gamma)
    zv = uniform_vertices(nz, 0.0, math.pi)
    b = rect_block(xv, yv, zv)
    if shear:
        b.vertices[..., 0] += shear * b.vertices[..., 1]
    N = b.ncells
    yc = cell_centres(b)[1]
    rng = np.random.default_rng(seed)
    u0 = amp * rng.standard_normal((3, N))
    u0[0] += 1.0 - yc ** 2
    S = np.zeros((3, N))
    S[0] = 2.0 * nu
    return Case("channel3d", 3, [b], [(0, SIDE_XP, 0, SIDE_XM), (0, SIDE_ZP, 0, SIDE_ZM)],
                [(0, SIDE_YM, wall(b, SIDE_YM, 3)), (0, SIDE_YP, wall(b, SIDE_YP, 3))], [],
                u0, np.zeros(N), S, nu, dt, steps)


def channel2d(nx: int = 16, ny: int = 16, gamma: float = 0.0, length: float = 1.0,
              height: float = 1.0, G: float = 1.0, nu: float = 1.0, dt: float = 0.1,
              steps: int = 100) -> Case:
    """Plane Poiseuille flow (App. B.1): periodic in x, walls at y = 0 and y = height,
    constant forcing G in x.  Analytic u = G/(2 nu) y (height - y)."""
    xv = uniform_vertices(nx, 0.0, length)
    yv = tanh_vertices(ny, 0.0, height, gamma) if gamma > 0 else uniform_vertices(ny, 0.0, height)
    b = rect_block(xv, yv)
    N = b.ncells
    S = np.zeros((2, N))
    S[0] = G
    return Case("poiseuille2d", 2, [b], [(0, SIDE_XP, 0, SIDE_XM)],
                [(0, SIDE_YM, wall(b, SIDE_YM, 2)), (0, SIDE_YP, wall(b, SIDE_YP, 2))], [],
                np.zeros((2, N)), np.zeros(N), S, nu, dt, steps)


def periodic2d(n: int = 32, L: float = 2.0 * math.pi, nu: float = 0.01, dt: float = 0.01,
               steps: int = 10, u0: Optional[np.ndarray] = None, S: Optional[np.ndarray] = None,
               ny: Optional[int] = None, Ly: Optional[float] = None) -> Case:
    ny = n if ny is None else ny
    Ly = L if Ly is None else Ly
    b = rect_block(uniform_vertices(n, 0.0, L), uniform_vertices(ny, 0.0, Ly))
    N = b.ncells
    u0 = np.zeros((2, N)) if u0 is None else u0
    return Case("periodic2d", 2, [b], [(0, SIDE_XP, 0, SIDE_XM), (0, SIDE_YP, 0, SIDE_YM)], [], [],
                u0, np.zeros(N), S, nu, dt, steps)


def taylor_green2d(n: int = 32, nu: float = 0.1, dt: float = 0.01, steps: int = 10) -> Case:
    """Taylor-Green vortex on the periodic box [0, 2pi)^2 sampled at cell centres:
    u = -cos x sin y, v = sin x cos y (decays as exp(-2 nu t))."""
    c = periodic2d(n, nu=nu, dt=dt, steps=steps)
    xc, yc = cell_centres(c.blocks[0])
    c.u0 = np.stack([-np.cos(xc) * np.sin(yc), np.sin(xc) * np.cos(yc)])
    c.name = "taylor_green2d"
    return c


def turbulence2d(n: int = 128, nu: float = 2e-3, dt: float = 0.01, seed: int = 1,
                 forcing: float = 0.1, steps: int = 16) -> Case:
    """Forced 2D turbulence on [0, 2pi)^2: divergence-free random initial field
    from a streamfunction with a k^-3 energy spectrum (random phases), scaled to
    rms velocity 1, plus Kolmogorov forcing (forcing * sin 4y, 0)."""
    rng = np.random.default_rng(seed)
    k = np.fft.fftfreq(n, d=1.0 / n)
    KX, KY = np.meshgrid(k, k, indexing="xy")
    K = np.sqrt(KX ** 2 + KY ** 2)
    amp = np.zeros_like(K)
    nz = K > 0
    # E(k) ~ k^-3 -> |psi_k| ~ k^-1 * sqrt(E(k)/k) = k^-3 (2D shell density ~ k)
    amp[nz] = K[nz] ** -3.0
    psi_hat = amp * np.exp(2j * math.pi * rng.random(K.shape))
    psi = np.real(np.fft.ifft2(psi_hat))
    # velocity from the streamfunction, spectrally: u = dpsi/dy, v = -dpsi/dx
    ph = np.fft.fft2(psi)
    u = np.real(np.fft.ifft2(1j * KY * ph))
    v = np.real(np.fft.ifft2(-1j * KX * ph))
    rms = math.sqrt(np.mean(u ** 2 + v ** 2))
    u0 = np.stack([u.reshape(-1), v.reshape(-1)]) / rms
    c = periodic2d(n, nu=nu, dt=dt, steps=steps, u0=u0)
    yc = cell_centres(c.blocks[0])[1]
    S = np.zeros((2, n * n))
    S[0] = forcing * np.sin(4.0 * yc)
    c.S = S
    c.name = "turbulence2d"
    return c


def bfs2d(n_in: Tuple[int, int] = (64, 32), n_ch: int = 256, n_out: int = 64, half: int = 32,
          gamma: float = 2.0, nu: float = 1e-3, dt: float = 0.01, steps: int = 500) -> Case:
    """Backward-facing-step channel as five conformal blocks: inlet (x in [-2,0],
    y in [0,1]), channel upper/lower (x in [0,16], y in [0,1] / [-1,0]) and outlet
    upper/lower (x in [16,24]).  The channel height [-1,1] carries 2*half cells
    with tanh refinement to both walls; the inlet shares the upper half's
    vertices.  Parabolic inflow u = 4y(1-y), no-slip walls (including the step
    face), advective outflow at x = 24 whose initial value is the plug flow
    carrying the inflow rate."""
    ni, _ = n_in
    yall = tanh_vertices(2 * half, -1.0, 1.0, gamma)
    y_lo, y_hi = yall[: half + 1], yall[half:]
    x_in = uniform_vertices(ni, -2.0, 0.0)
    x_ch = uniform_vertices(n_ch, 0.0, 16.0)
    x_out = uniform_vertices(n_out, 16.0, 24.0)
    blocks = [rect_block(x_in, y_hi), rect_block(x_ch, y_hi), rect_block(x_ch, y_lo),
              rect_block(x_out, y_hi), rect_block(x_out, y_lo)]
    INL, CHU, CHL, OUU, OUL = range(5)
    conns = [(INL, SIDE_XP, CHU, SIDE_XM), (CHU, SIDE_YM, CHL, SIDE_YP),
             (CHU, SIDE_XP, OUU, SIDE_XM), (CHL, SIDE_XP, OUL, SIDE_XM),
             (OUU, SIDE_YM, OUL, SIDE_YP)]
    dirichlet = []
    inflow = wall(blocks[INL], SIDE_XM, 2)
    yf = side_face_centres(blocks[INL], SIDE_XM)[:, 1]
    inflow[:, 0] = 4.0 * yf * (1.0 - yf)
    dirichlet.append((INL, SIDE_XM, inflow))
    for blk, s in [(INL, SIDE_YM), (INL, SIDE_YP), (CHU, SIDE_YP), (CHL, SIDE_YM), (CHL, SIDE_XM),
                   (OUU, SIDE_YP), (OUL, SIDE_YM)]:
        dirichlet.append((blk, s, wall(blocks[blk], s, 2)))
    q_in = 2.0 / 3.0           # integral of 4y(1-y) over [0,1]
    plug = q_in / 2.0          # outlet height 2
    outflow = []
    for blk in (OUU, OUL):
        val = wall(blocks[blk], SIDE_XP, 2)
        val[:, 0] = plug
        outflow.append((blk, SIDE_XP, np.array([plug, 0.0]), val))
    N = sum(b.ncells for b in blocks)
    return Case("bfs2d", 2, blocks, conns, dirichlet, outflow, np.zeros((2, N)), np.zeros(N), None,
                nu, dt, steps)


def batch2d(count: int = 64, seed: int = 4, nmin: int = 32, nmax: int = 256,
            steps: int = 10) -> List[Case]:
    """Independent 2D simulations of uneven size: side n ~ U{nmin..nmax},
    Re ~ U[100, 2000], half lid-driven cavities and half x-periodic forced
    channels (walls in y)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = int(rng.integers(nmin, nmax + 1))
        re = float(rng.uniform(100.0, 2000.0))
        if i % 2 == 0:
            nu = 1.0 / re
            dt = 0.5 / n
            out.append(cavity2d(n, nu=nu, dt=dt, steps=steps))
        else:
            nu = 1.0 / re
            c = channel2d(nx=n, ny=n, length=2.0, height=1.0, G=8.0 * nu, nu=nu, dt=0.5 / n,
                          steps=steps)
            yc = cell_centres(c.blocks[0])[1]
            c.u0[0] = 4.0 * yc * (1.0 - yc) + 0.05 * rng.standard_normal(c.ncells)
            out.append(c)
    return out


# ----------------------------------------------------------------------------
# blocks joined with permuted / flipped axes (Sec. 2.2, App. A.3)
# ----------------------------------------------------------------------------

def rotate_block_2d(block: Block, quarter_turns: int):
    """The same cells with the block's index frame turned by quarter_turns x
    90 degrees (right-handed frames stay right-handed).  Returns (block,
    old_index) with old_index[new cell] = the cell's index in the input block,
    and side_map[old side] = new side."""
    V = block.vertices
    nx, ny, _ = block.res
    old = np.arange(nx * ny).reshape(ny, nx)          # old[y, x]
    side_map = [0, 1, 2, 3]
    for _ in range(quarter_turns % 4):
        # new x = old y, new y = (old nx) - old x
        V = np.transpose(V, (1, 0, 2))[::-1].copy()
        old = np.transpose(old, (1, 0))[::-1].copy()
        # old -x -> new +y, old +x -> new -y, old -y -> new -x, old +y -> new +x
        side_map = [{0: 3, 1: 2, 2: 0, 3: 1}[s] for s in side_map]
    nyn, nxn = old.shape
    return Block((nxn, nyn, 1), V), old.ravel(), side_map


def rotate_block_x_3d(block: Block):
    """The block's index frame turned about x: new y = old z, new z = (old ny) -
    old y.  Returns (block, old_index, side_map) as rotate_block_2d."""
    V = block.vertices                                  # V[z, y, x]
    nx, ny, nz = block.res
    old = np.arange(nx * ny * nz).reshape(nz, ny, nx)
    # new[z', y', x] = old[z = y', y = ny - 1 - z', x]
    Vn = np.transpose(V, (1, 0, 2, 3))[::-1].copy()     # Vn[z', y', x] = V[y', NY - z', x]
    On = np.transpose(old, (1, 0, 2))[::-1].copy()
    side_map = [0, 1, 5, 4, 2, 3]                       # old -y -> new +z, +y -> -z, -z -> -y, +z -> +y
    return Block((nx, nz, ny), Vn), On.ravel(), side_map


def _fields_from_positions(blocks, ndim, seed_shift=0.0):
    """Smooth seeded-free initial velocity, pressure and source as functions of
    the cell centres (so any block layout of the same cells gets the same
    values)."""
    xc = np.concatenate([cell_centres(b) for b in blocks], axis=1)
    x, y = xc[0], xc[1]
    z = xc[2] if ndim == 3 else 0.0 * x
    u = np.stack([np.sin(3 * x + 0.5) * np.cos(2 * y) + 0.2 * np.cos(z),
                  0.5 * np.cos(2 * x) * np.sin(3 * y + seed_shift)] +
                 ([0.3 * np.sin(x + 2 * y + z)] if ndim == 3 else []))
    p = np.cos(x + y) + 0.1 * z
    S = 0.3 * np.stack([np.cos(x - y), np.sin(2 * x)] + ([np.cos(z + x)] if ndim == 3 else []))
    return u, p, S


def two_block_cavity2d(nx: int = 8, ny: int = 6, rot: int = 0, shear: float = 0.0, gamma: float = 1.5,
                       nu: float = 0.02, dt: float = 0.02):
    """Lid-driven cavity [0, 2] x [0, 1] of two blocks joined at x = 1 (tanh
    refinement in y, optional slant x += shear y): block 1's index frame is
    turned by rot quarter turns, so the joint is an ordinary side-to-side
    connection (rot 0) or one with a flip / an axis exchange.  The lid
    (top) moves with u = sin^2(pi x / 2); the other sides are walls.  Returns
    (case, cell_index) with cell_index[cell of this layout] = the cell's index
    in the rot = 0 layout."""
    yv = tanh_vertices(ny, 0.0, 1.0, gamma)
    A = rect_block(uniform_vertices(nx, 0.0, 1.0), yv)
    B0 = rect_block(uniform_vertices(nx, 1.0, 2.0), yv)
    for b in (A, B0):
        b.vertices[..., 0] += shear * b.vertices[..., 1]
    B, old, side_map = rotate_block_2d(B0, rot)
    blocks = [A, B]
    inv_map = {v: k for k, v in enumerate(side_map)}
    # the joint: A's +x side to B's (old -x) side; its tangential axis is old y
    sb = side_map[0]
    flip = 1 if rot % 4 in (2, 3) else 0
    conns = [(0, 1, 1, sb, 0, flip)] if (rot % 4) else [(0, 1, 1, 0)]

    def bc(block, side, top):
        fc = side_face_centres(block, side)
        v = np.zeros((len(fc), 2))
        if top:
            v[:, 0] = np.sin(0.5 * math.pi * (fc[:, 0] - shear * fc[:, 1])) ** 2
        return v
    dirichlet = [(0, s, bc(A, s, s == SIDE_YP)) for s in (SIDE_XM, SIDE_YM, SIDE_YP)]
    for old_side in (SIDE_XP, SIDE_YM, SIDE_YP):
        s = side_map[old_side]
        dirichlet.append((1, s, bc(B, s, old_side == SIDE_YP)))
    u0, p0, S = _fields_from_positions(blocks, 2)
    cell_index = np.concatenate([np.arange(A.ncells), A.ncells + old])
    del inv_map
    return Case("two_block_cavity2d", 2, blocks, conns, dirichlet, [], u0, p0, S, nu, dt, 10), cell_index


def two_block_channel3d(nx: int = 5, ny: int = 6, nz: int = 4, turned: bool = False, shear: float = 0.0,
                        gamma: float = 1.5, nu: float = 0.02, dt: float = 0.02):
    """3D box [0, 2] x [0, 1] x [0, 1] of two blocks joined at x = 1, periodic
    in z (each block to itself), walls at y = 0 and y = 1 (the top one
    sliding with u = 1), an inflow profile at x = 0 and the matching outflow
    at x = 2; block 1 optionally turned about x (its y and z axes exchanged
    and one reversed), so the joint needs axis_perm = 1 with a flip.
    Returns (case, cell_index) as two_block_cavity2d."""
    yv = tanh_vertices(ny, 0.0, 1.0, gamma)
    zv = uniform_vertices(nz, 0.0, 1.0)
    A = rect_block(uniform_vertices(nx, 0.0, 1.0), yv, zv)
    B0 = rect_block(uniform_vertices(nx, 1.0, 2.0), yv, zv)
    for b in (A, B0):
        b.vertices[..., 0] += shear * b.vertices[..., 1]
    if turned:
        B, old, side_map = rotate_block_x_3d(B0)
        conns = [(0, SIDE_XP, 1, SIDE_XM, 1, 1)]
    else:
        B, old, side_map = B0, np.arange(B0.ncells), list(range(6))
        conns = [(0, SIDE_XP, 1, SIDE_XM)]
    conns += [(0, SIDE_ZP, 0, SIDE_ZM), (1, side_map[SIDE_ZP], 1, side_map[SIDE_ZM])]

    def prof(block, side, kind):
        fc = side_face_centres(block, side)
        v = np.zeros((len(fc), 3))
        if kind == "lid":
            v[:, 0] = 1.0
        elif kind == "in":
            v[:, 0] = 4.0 * fc[:, 1] * (1.0 - fc[:, 1])
        return v
    dirichlet = [(0, SIDE_XM, prof(A, SIDE_XM, "in")), (0, SIDE_YM, prof(A, SIDE_YM, "wall")),
                 (0, SIDE_YP, prof(A, SIDE_YP, "lid"))]
    for old_side, kind in ((SIDE_XP, "in"), (SIDE_YM, "wall"), (SIDE_YP, "lid")):
        s = side_map[old_side]
        dirichlet.append((1, s, prof(B, s, kind)))
    u0, p0, S = _fields_from_positions([A, B], 3)
    cell_index = np.concatenate([np.arange(A.ncells), A.ncells + old])
    return Case("two_block_channel3d", 3, [A, B], conns, dirichlet, [], u0, p0, S, nu, dt, 10), cell_index


def slit_cgrid2d(n_xi: int = 16, n_eta: int = 8, a: float = 1.4, b: float = 1.2, nu: float = 0.05,
                 dt: float = 0.02, u_inf=(1.0, 0.0), skew: float = 0.25):
    """A C-grid around a slit (App. B: O-/C-grids around obstacles): the block
    (xi, eta) in [-a, a] x [0, b] mapped by x + i y = (xi + i eta)^2, plus
    skew * xi * eta in x (which makes the cells non-orthogonal and keeps
    J = 4 (xi^2 + eta^2) > 0), so its eta = 0 side folds onto itself along the
    positive x-axis (the cut): cell xi meets cell -xi, which is a connection
    of that side to itself with its tangential axis reversed.  The other sides
    carry the free stream u_inf; smooth initial field.  n_xi must be even (no
    cell meets itself)."""
    xi = np.linspace(-a, a, n_xi + 1)
    eta = np.linspace(0.0, b, n_eta + 1)
    E, X = np.meshgrid(eta, xi, indexing="ij")
    V = np.stack([X ** 2 - E ** 2 + skew * X * E, 2.0 * X * E], axis=-1)
    blk = Block((n_xi, n_eta, 1), V)
    conns = [(0, SIDE_YM, 0, SIDE_YM, 0, 1)]
    ui = np.asarray(u_inf, dtype=np.float64)
    dirichlet = [(0, s, np.tile(ui, (side_nfaces(blk.res, s, 2), 1))) for s in (SIDE_XM, SIDE_XP, SIDE_YP)]
    u0, p0, S = _fields_from_positions([blk], 2)
    return Case("slit_cgrid2d", 2, [blk], conns, dirichlet, [], u0 * 0.3 + ui[:, None], p0, None, nu, dt, 10)
