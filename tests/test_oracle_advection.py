"""Pins of the oracle's advection operator on grids that are not uniform:
stretched, curved and rotated (arXiv:2505.16992, App. A.2 Eq. advMatDiscrete
with the contravariant flux U^j = J T_j . u of "Grid Transformations", and the
boundary fluxes of Eq. velRHSdiscrete).

Three independent pins, none of which calls the oracle's metric code:
  * a closed form in the vertex positions on a curved periodic 2D block: the
    cell Jacobian dx/dxi from face-centre differences, J T_j . u from its
    cofactors, the face flux as the mean of the two cells' fluxes, the row
    divided by the cell's own J (reading R1), walls carrying u_b with the
    adjacent cell's metric (reading R3);
  * discrete conservation: the J-weighted sum of the advective rows telescopes
    to zero over interior faces for any field and any velocity (stretched 3D
    channel, multi-block step, curved block);
  * rotation equivariance of the whole step: a grid rotated by 30 degrees with
    rotated velocities, sources and wall values gives the rotated solution.
Each plausible slip in forming the advective entries (the neighbour's J in
place of the cell's, the face flux from face-averaged velocities and metrics,
the transposed metric, a flipped face sign) is planted in a copy of the
assembly and shown to fail at least one of these pins."""
import math

import numpy as np
import pytest

import oracle as O
from oracle import piso as OP
from paper_2505_16992_b300 import workloads as W


# ---------------------------------------------------------------------------
# meshes
# ---------------------------------------------------------------------------

def _curved_block(nx=6, ny=5, L=2.0):
    """Periodic in x (period L), walls at the bottom and top: x stretched
    periodically and sheared with y, y tanh-stretched and displaced by a
    periodic wave, so J, T and J T_j vary from cell to cell and no two
    neighbours share a metric."""
    i = np.arange(nx + 1)
    xi = L * (i / nx + 0.06 * np.sin(2 * math.pi * i / nx))
    yj = np.tanh(1.2 * np.linspace(-1.0, 1.0, ny + 1)) / math.tanh(1.2)
    X, Y = np.meshgrid(xi, yj)                    # [ny+1][nx+1]
    Xs = X + 0.1 * Y
    Ys = Y + 0.15 * np.sin(2 * math.pi * Xs / L)
    return np.stack([Xs, Ys], axis=-1)


def _curved_mesh(seed=0, nx=6, ny=5):
    V = _curved_block(nx, ny)
    rng = np.random.default_rng(seed)
    walls = [(0, s, 0.3 * rng.standard_normal((nx, 2))) for s in (2, 3)]
    m = O.Mesh(2, [((nx, ny, 1), V)], [(0, 1, 0, 0)], walls, allow_nonorthogonal=True)
    return m, V


# ---------------------------------------------------------------------------
# the advective part of the assembly
# ---------------------------------------------------------------------------

def _adv_action(assemble, m, u, phi):
    """(C^adv phi, advective part of rhs0): the assembly at nu = 0, dt = 1,
    no source, minus its time-derivative part."""
    C, rhs0 = assemble(m, u, 0.0, 1.0, None, m.bval)
    return OP.matvec(m, C, phi) - phi, rhs0 - u


def _closed_form_2d(V, u, phi, bval_lo, bval_hi):
    """Pure-Python restatement on one 2D block, periodic in x, walls at y-min
    and y-max.  Cell (i, j) = vertices V[j:j+2, i:i+2]; dx/dxi from the
    differences of opposite face centres; J = det; J T_xi . u = M_y,eta u_x -
    M_x,eta u_y and J T_eta . u = -M_y,xi u_x + M_x,xi u_y (the cofactor rows).
    Interior face of P towards F with sign n: 0.5 n (U_P + U_F)/2 (phi_P +
    phi_F) / J_P; a wall face adds -n U_b u_b / J_P to the rhs, with U_b from
    the cell's own cofactors."""
    ny, nx = V.shape[0] - 1, V.shape[1] - 1
    cof = {}
    jac = {}
    for j in range(ny):
        for i in range(nx):
            a, b_, c, d = V[j, i], V[j, i + 1], V[j + 1, i], V[j + 1, i + 1]
            m_xi = 0.5 * (b_ + d) - 0.5 * (a + c)           # d x / d xi
            m_eta = 0.5 * (c + d) - 0.5 * (a + b_)          # d x / d eta
            jac[i, j] = m_xi[0] * m_eta[1] - m_eta[0] * m_xi[1]
            cof[i, j] = (np.array([m_eta[1], -m_eta[0]]), np.array([-m_xi[1], m_xi[0]]))
    idx = lambda i, j: i + nx * j
    cadv = np.zeros(nx * ny)
    radv = np.zeros((2, nx * ny))
    for j in range(ny):
        for i in range(nx):
            P = idx(i, j)
            acc = 0.0
            for axis, sgn in ((0, -1), (0, 1), (1, -1), (1, 1)):
                if axis == 0:
                    fi, fj = (i + sgn) % nx, j
                else:
                    fi, fj = i, j + sgn
                    if fj < 0 or fj >= ny:
                        ub = (bval_lo if fj < 0 else bval_hi)[:, i]
                        Ub = cof[i, j][axis] @ ub
                        radv[:, P] += -sgn * Ub * ub / jac[i, j]
                        continue
                F = idx(fi, fj)
                UP = cof[i, j][axis] @ u[:, P]
                UF = cof[fi, fj][axis] @ u[:, F]
                acc += 0.5 * sgn * 0.5 * (UP + UF) * (phi[P] + phi[F])
            cadv[P] = acc / jac[i, j]
    return cadv, radv


def _check_closed_form(assemble):
    m, V = _curved_mesh()
    rng = np.random.default_rng(1)
    u = rng.standard_normal((2, m.N))
    phi = rng.standard_normal(m.N)
    cadv, radv = _adv_action(assemble, m, u, phi)
    nx = V.shape[1] - 1
    lo = m.side_values(m.bval, 0, 2).T
    hi = m.side_values(m.bval, 0, 3).T
    ref_c, ref_r = _closed_form_2d(V, u, phi, lo, hi)
    err_c = np.abs(cadv - ref_c).max() / np.abs(ref_c).max()
    err_r = np.abs(radv - ref_r).max() / np.abs(ref_r).max()
    assert nx == 6
    return max(err_c, err_r)


def _check_conservation(assemble):
    """max over meshes of |sum_P J_P (C^adv phi)_P| / sum_P |J_P (C^adv phi)_P|."""
    worst = 0.0
    cases = [O.mesh_from_case(W.channel3d(8, 10, 6, gamma=2.0)),
             O.mesh_from_case(W.bfs2d(n_in=(6, 4), n_ch=10, n_out=6, half=4)),
             _curved_mesh(3)[0]]
    for k, m in enumerate(cases):
        rng = np.random.default_rng(10 + k)
        u = rng.standard_normal((m.ndim, m.N))
        phi = rng.standard_normal(m.N)
        cadv, _ = _adv_action(assemble, m, u, phi)
        t = m.J * cadv
        worst = max(worst, abs(t.sum()) / np.abs(t).sum())
    return worst


def _rotated(V, th):
    R = np.array([[math.cos(th), -math.sin(th)], [math.sin(th), math.cos(th)]])
    return V @ R.T, R


def _check_rotation(monkeypatch, assemble):
    """max relative difference between R (step of the original) and the step
    of the rotated problem, velocity and pressure, on a periodic box and on a
    stretched channel with moving walls, advection on."""
    monkeypatch.setattr(OP, "assemble_C", assemble)
    worst = 0.0
    th = math.radians(30.0)
    rng = np.random.default_rng(5)
    # periodic 12 x 10 box with a random velocity and source
    c1 = W.periodic2d(12, L=2.0, ny=10, Ly=1.6)
    # channel periodic in x with tanh walls; the lower wall slides
    c2 = W.channel2d(10, 12, gamma=1.5, nu=0.05, dt=0.05)
    c2.dirichlet[0][2][:, 0] = 0.7
    for c in (c1, c2):
        b = c.blocks[0]
        Vr, R = _rotated(b.vertices, th)
        d = [(blk, s, vals) for (blk, s, vals) in c.dirichlet]
        m = O.Mesh(2, [(b.res, b.vertices)], c.connections, d)
        mr = O.Mesh(2, [(b.res, Vr)], c.connections, [(blk, s, vals @ R.T) for (blk, s, vals) in d])
        u0 = rng.standard_normal((2, m.N))
        S = 0.5 * rng.standard_normal((2, m.N))
        p0 = rng.standard_normal(m.N)
        u1, p1, _ = O.piso_step(m, u0, p0, 0.05, 0.05, S)
        u1r, p1r, _ = O.piso_step(mr, R @ u0, p0, 0.05, 0.05, R @ S)
        worst = max(worst, np.abs(u1r - R @ u1).max() / np.abs(u1).max(),
                    np.abs(p1r - p1).max() / np.abs(p1).max())
    return worst


# ---------------------------------------------------------------------------
# the pins
# ---------------------------------------------------------------------------

def test_advection_closed_form_on_curved_periodic_block():
    assert _check_closed_form(O.assemble_C) <= 1e-13


def test_advection_discretely_conservative():
    assert _check_conservation(O.assemble_C) <= 1e-13


def test_step_rotation_equivariant_with_advection(monkeypatch):
    assert _check_rotation(monkeypatch, O.assemble_C) <= 1e-12


# ---------------------------------------------------------------------------
# planted slips: each must fail at least one pin
# ---------------------------------------------------------------------------

def _assemble_variant(kind):
    """A copy of the assembly with one slip in the advective entries."""
    def assemble(mesh, u, nu, dt, S, bval):
        d, N = mesh.ndim, mesh.N
        if kind == "transposed_T":
            U = np.einsum("n,nkj,kn->jn", mesh.J, mesh.T, u)
        else:
            U = mesh.contravariant(u)
        JT = mesh.J[:, None, None] * mesh.T
        diag = np.full(N, 1.0 / dt)
        off = np.zeros((mesh.nsides, N))
        rhs0 = u / dt
        if S is not None:
            rhs0 = rhs0 + S
        for s in range(mesh.nsides):
            j, n = s // 2, OP.sign(s)
            P = np.nonzero(mesh.inner[s])[0]
            F = mesh.nb[s, P]
            if kind == "face_averaged":
                Uf = np.einsum("nk,kn->n", 0.5 * (JT[P, j, :] + JT[F, j, :]), 0.5 * (u[:, P] + u[:, F]))
            else:
                Uf = 0.5 * (U[j, P] + U[j, F])
            Df = nu * 0.5 * (mesh.alpha[j, P] + mesh.alpha[j, F])
            Joff = mesh.J[F] if kind == "neighbour_J" else mesh.J[P]
            no = -n if kind == "flipped_sign" else n
            off[s, P] = (0.5 * no * Uf) / Joff - Df / mesh.J[P]
            diag[P] += (0.5 * n * Uf + Df) / mesh.J[P]
            B = np.nonzero(mesh.is_bface[s])[0]
            ub = bval[s][:, B]
            Ub = mesh.face_flux_b(s, bval[s])[B]
            diag[B] += 2.0 * mesh.alpha[j, B] * nu / mesh.J[B]
            rhs0[:, B] += ub * ((2.0 * mesh.alpha[j, B] * nu - n * Ub) / mesh.J[B])[None, :]
        return OP.Matrix(diag, off), rhs0
    return assemble


def test_variant_copy_without_slip_passes():
    """The copy used for planting is the oracle's assembly when no slip is set
    (so a failing variant fails because of its slip)."""
    m, _ = _curved_mesh(7)
    rng = np.random.default_rng(2)
    u = rng.standard_normal((2, m.N))
    nu, dt = 0.3, 0.1
    Ca, ra = O.assemble_C(m, u, nu, dt, None, m.bval)
    Cb, rb = _assemble_variant("none")(m, u, nu, dt, None, m.bval)
    np.testing.assert_allclose(Cb.diag, Ca.diag, rtol=1e-14)
    np.testing.assert_allclose(Cb.off, Ca.off, rtol=1e-14, atol=1e-15)
    np.testing.assert_allclose(rb, ra, rtol=1e-14)


@pytest.mark.parametrize("kind", ["neighbour_J", "face_averaged", "transposed_T", "flipped_sign"])
def test_planted_slip_fails_a_pin(kind, monkeypatch):
    f = _assemble_variant(kind)
    errs = {"closed_form": _check_closed_form(f), "conservation": _check_conservation(f)}
    if max(errs.values()) <= 1e-6:
        errs["rotation"] = _check_rotation(monkeypatch, f)
    assert max(errs.values()) > 1e-6, (kind, errs)
