"""FP64 CPU oracle of the turbulence-statistics operators (TEST INFRASTRUCTURE
ONLY: only ``tests/`` and the CPU-baseline leg of ``bench.py`` may import it).

arXiv:2505.16992, Sec. 2.5 (Operators for Turbulence Statistics): central
(co)moments of flow quantities averaged over time and the homogeneous
directions, accumulated online (the paper cites Pebay et al.'s pairwise
formulas), from which turbulence statistics and the terms of the turbulent
energy budget (production, dissipation, turbulent transport, viscous
diffusion, velocity pressure-gradient) are formed; Sec. 3.3 (Losses from
Turbulence Statistics) builds the training losses L_U and L_u' from the mean
profiles and second-order statistics per wall-normal position y.

Definitions used here, written out from the mathematics:

* A *record* of per-cell fields q [nq][N] on one block (nx, ny, nz) holds, for
  every plane y = const (the homogeneous directions are x and, in 3D, z):
  n (cells averaged), mean_i = (1/n) sum q_i, m2_ij = (1/n) sum a_i a_j and
  m3_ijk = (1/n) sum a_i a_j a_k with a = q - mean (central moments normalised
  by the count, two-pass definition).
* ``merge`` combines two records of the same planes into the record of the
  union of their samples (pairwise update; derived in ``merge``'s docstring),
  so averaging over time is merging the frames' records one after another.
* ``frame_record_adjoint`` is the exact derivative of one frame's record with
  respect to the frame's fields.
* ``cell_gradients`` forms d q_i / d x_k at cell centres by central
  differences in computational space mapped with T (the operator of Eq.
  velCorrDiscrete), with a ghost value at Dirichlet faces: 2 u_b - u_P for the
  velocity (linear through the face value), p_P for the pressure (0-Neumann,
  App. A.3).
* ``budget`` forms the budget terms per y from three records (reading R19):
  velocity (u_i), velocity gradient (d u_i / d x_k, q index i*d + k) and
  velocity with pressure gradient (u_i, d p / d x_j): P_ij = -(R_ik dU_j/dx_k +
  R_jk dU_i/dx_k) with only d/dy non-zero, eps_ij = 2 nu <d_k u_i' d_k u_j'>,
  T_ij = -d<u_i' u_j' v'>/dy, D_ij = nu d^2 R_ij/dy^2, Pi_ij = -(<u_i' d_j p> +
  <u_j' d_i p>).  The paper prints eps and D without nu (a non-dimensional
  form); the dimensional form with nu is used.  Profiles are differentiated
  in y on the points {wall, cell centres, wall} with the values 0 at no-slip
  walls (mean velocity and all velocity moments vanish there), by the
  three-point formulas for unequal spacing.
"""
from __future__ import annotations

from typing import Dict, Optional, Sequence

import numpy as np


# ----------------------------------------------------------------------------
# per-frame plane records (Sec. 2.5)
# ----------------------------------------------------------------------------

def plane_view(q: np.ndarray, res) -> np.ndarray:
    """[nq][N] cell fields of one block -> [nq][ny][n_plane] (x, z flattened)."""
    nx, ny = int(res[0]), int(res[1])
    nz = int(res[2]) if len(res) > 2 else 1
    q = np.asarray(q, dtype=np.float64).reshape(q.shape[0], nz, ny, nx)
    return np.transpose(q, (0, 2, 1, 3)).reshape(q.shape[0], ny, nz * nx)


def frame_record(q: np.ndarray, res, order: int = 3) -> Dict[str, np.ndarray]:
    """Plane record of one frame: the two-pass definitions above."""
    P = plane_view(q, res)                      # [nq][ny][n]
    nq, ny, n = P.shape
    mean = P.mean(axis=2).T                     # [ny][nq]
    a = P - mean.T[:, :, None]                  # central values
    m2 = np.einsum("iyc,jyc->yij", a, a) / n
    rec = dict(n=np.full(ny, float(n)), mean=mean, m2=m2)
    rec["m3"] = np.einsum("iyc,jyc,kyc->yijk", a, a, a) / n if order >= 3 else None
    return rec


def merge(A: Dict[str, np.ndarray], B: Dict[str, np.ndarray]) -> Dict[str, np.ndarray]:
    """Record of the union of the samples of A and B (per plane).

    With n = nA + nB, d = mean_B - mean_A, and central sums C2 = n m2,
    C3 = n m3, writing the combined central values as a_A - (nB/n) d and
    a_B + (nA/n) d and expanding (the first central sums of each part vanish):
      mean = mean_A + (nB/n) d
      C2   = C2A + C2B + (nA nB / n) d d
      C3   = C3A + C3B + (nA nB (nA - nB) / n^2) d d d
             + (1/n) S(nA C2B - nB C2A, d)
    where S(M, d)_ijk = M_jk d_i + M_ik d_j + M_ij d_k."""
    nA, nB = A["n"], B["n"]
    n = nA + nB
    d = B["mean"] - A["mean"]
    mean = A["mean"] + (nB / n)[:, None] * d
    C2A, C2B = nA[:, None, None] * A["m2"], nB[:, None, None] * B["m2"]
    dd = np.einsum("yi,yj->yij", d, d)
    C2 = C2A + C2B + (nA * nB / n)[:, None, None] * dd
    out = dict(n=n, mean=mean, m2=C2 / n[:, None, None], m3=None)
    if A.get("m3") is not None and B.get("m3") is not None:
        C3A, C3B = nA[:, None, None, None] * A["m3"], nB[:, None, None, None] * B["m3"]
        M = nA[:, None, None] * C2B - nB[:, None, None] * C2A
        S = (np.einsum("yjk,yi->yijk", M, d) + np.einsum("yik,yj->yijk", M, d) +
             np.einsum("yij,yk->yijk", M, d))
        C3 = (C3A + C3B + (nA * nB * (nA - nB) / n ** 2)[:, None, None, None] *
              np.einsum("yi,yj,yk->yijk", d, d, d) + S / n[:, None, None, None])
        out["m3"] = C3 / n[:, None, None, None]
    return out


def accumulate(records: Sequence[Dict[str, np.ndarray]]) -> Dict[str, np.ndarray]:
    """Time average as an online accumulation: merge the frames one by one."""
    acc = records[0]
    for r in records[1:]:
        acc = merge(acc, r)
    return acc


def frame_record_adjoint(q: np.ndarray, res, rec: Dict[str, np.ndarray], g_mean: np.ndarray,
                         g_m2: np.ndarray, g_m3: Optional[np.ndarray] = None) -> np.ndarray:
    """dL/dq [nq][N] of one frame, given dL/d(mean, m2, m3) of a record that
    contains the frame's samples: its own record, or a record accumulated over
    several frames (time average), whose count n and moments are then used.

    For a cell c of plane y with a = q(c) - mean (n samples in the record):
      d mean_i / d q_l = delta_il / n
      d m2_ij / d q_l  = (delta_il a_j + delta_jl a_i) / n        (sum of a is 0)
      d m3_ijk / d q_l = (delta_il (a_j a_k - m2_jk) + delta_jl (a_i a_k - m2_ik)
                          + delta_kl (a_i a_j - m2_ij)) / n
    contracted with the gradients."""
    P = plane_view(q, res)
    nq, ny, n = P.shape
    a = P - rec["mean"].T[:, :, None]                     # [nq][ny][n]
    g2s = g_m2 + np.transpose(g_m2, (0, 2, 1))            # g_lj + g_jl
    out = g_mean.T[:, :, None] + np.einsum("ylj,jyc->lyc", g2s, a)
    if g_m3 is not None:
        g3s = g_m3 + np.transpose(g_m3, (0, 2, 1, 3)) + np.transpose(g_m3, (0, 3, 1, 2))
        # g3s[y, l, j, k] = g_ljk + g_jlk + g_jkl
        aa = np.einsum("jyc,kyc->yjkc", a, a) - rec["m2"][:, :, :, None]
        out = out + np.einsum("yljk,yjkc->lyc", g3s, aa)
    out = out / rec["n"][None, :, None]
    # back to the cell order [nq][N]
    nx, ny_ = int(res[0]), int(res[1])
    nz = int(res[2]) if len(res) > 2 else 1
    out = out.reshape(nq, ny_, nz, nx)
    return np.transpose(out, (0, 2, 1, 3)).reshape(nq, -1)


# ----------------------------------------------------------------------------
# cell-centred gradients (Eq. velCorrDiscrete operator, ghost values at walls)
# ----------------------------------------------------------------------------

def cell_gradients(mesh, u: np.ndarray, p: np.ndarray, bval=None):
    """(grad_u [d][d][N] with grad_u[i, k] = d u_i / d x_k, grad_p [d][N])."""
    d, N = mesh.ndim, mesh.N
    bval = mesh.bval if bval is None else bval
    gu = np.zeros((d, d, N))
    gp = np.zeros((d, N))
    for j in range(d):
        sp, sm = 2 * j + 1, 2 * j
        du = np.zeros((d, N))
        for s, sign in ((sp, 1.0), (sm, -1.0)):
            inner = mesh.nb[s] >= 0
            nbv = np.where(inner[None, :], u[:, np.maximum(mesh.nb[s], 0)], 2.0 * bval[s] - u)
            du += sign * 0.5 * nbv
        pp = np.where(mesh.nb[sp] >= 0, p[np.maximum(mesh.nb[sp], 0)], p)
        pm = np.where(mesh.nb[sm] >= 0, p[np.maximum(mesh.nb[sm], 0)], p)
        dp = 0.5 * (pp - pm)
        for k in range(d):
            gu[:, k, :] += mesh.T[:, j, k][None, :] * du
            gp[k] += mesh.T[:, j, k] * dp
    return gu, gp


# ----------------------------------------------------------------------------
# budget terms per y (reading R19)
# ----------------------------------------------------------------------------

def wall_profile_derivatives(f: np.ndarray, yc: np.ndarray, y0: float, y1: float):
    """First and second y-derivatives of profiles f [ny][...] at the cell
    centres yc, on the points {y0, yc..., y1} with f = 0 at both walls
    (three-point formulas for unequal spacing)."""
    ny = f.shape[0]
    Y = np.concatenate([[y0], yc, [y1]])
    F = np.concatenate([np.zeros((1,) + f.shape[1:]), f, np.zeros((1,) + f.shape[1:])])
    d1 = np.zeros_like(f)
    d2 = np.zeros_like(f)
    for j in range(ny):
        hm = Y[j + 1] - Y[j]
        hp = Y[j + 2] - Y[j + 1]
        fm, f0, fp = F[j], F[j + 1], F[j + 2]
        d1[j] = (hm * hm * fp - hp * hp * fm + (hp * hp - hm * hm) * f0) / (hm * hp * (hm + hp))
        d2[j] = 2.0 * (hm * fp - (hm + hp) * f0 + hp * fm) / (hm * hp * (hm + hp))
    return d1, d2


def budget(rec_u, rec_gu, rec_up, yc, y0, y1, nu):
    """Budget terms [ny][d][d]: P, eps, T, D, Pi (see the module docstring)."""
    d = rec_u["mean"].shape[1]
    ny = rec_u["mean"].shape[0]
    R = rec_u["m2"]                                   # [ny][d][d]
    dU, _ = wall_profile_derivatives(rec_u["mean"], yc, y0, y1)   # dU_i/dy
    P = -(np.einsum("yi,yj->yij", R[:, :, 1], dU) + np.einsum("yj,yi->yij", R[:, :, 1], dU))
    G = rec_gu["m2"].reshape(ny, d, d, d, d)          # [(i,k),(j,l)]
    eps = 2.0 * nu * np.einsum("yikjk->yij", G)
    dT, _ = wall_profile_derivatives(rec_u["m3"][:, :, :, 1], yc, y0, y1)
    T = -dT
    _, dR2 = wall_profile_derivatives(R, yc, y0, y1)
    D = nu * dR2
    C = rec_up["m2"]                                  # [(u_i, d_j p)]
    Pi = -(C[:, :d, d:] + np.transpose(C[:, :d, d:], (0, 2, 1)))
    return dict(P=P, eps=eps, T=T, D=D, Pi=Pi)


# ----------------------------------------------------------------------------
# losses of Sec. 3.3 (for finite-difference checks of the differentiable path)
# ----------------------------------------------------------------------------

def stats_loss(frame_records, ref_mean, ref_m2, lam_U=1.0, lam_uu=1.0, lam_frame=1.0):
    """L_stats of Eq. TCFstatsLossGeneric with all weights equal per kind:
    the time-averaged terms over all frames plus lam_frame times the per-frame
    terms; each term is (1/Y) sum_y of the squared error."""
    def terms(rec):
        ny = rec["mean"].shape[0]
        lu = np.sum((rec["mean"] - ref_mean) ** 2) / ny
        luu = np.sum((rec["m2"] - ref_m2) ** 2) / ny
        return lam_U * lu + lam_uu * luu
    total = terms(accumulate(frame_records))
    for r in frame_records:
        total += lam_frame * terms(r)
    return total
