// Cross-derivative terms of non-orthogonal meshes (arXiv:2505.16992, App. A.2
// "Non-Orthogonal Grids", Eqs. difNonOrthoMatDiscrete, velRHSnonOrtho,
// pressureRHSnonOrtho).  With alpha_jk = J T_j . T_k, the flux through a face
// of cell P on axis j gets, for every k != j, N_f mean(alpha_jk) (d_k q)_f,
// where (d_k q)_f is the mean of the central differences along k of P and of
// its neighbour across the face: summed over P's faces this is the central
// d_j d_k q.
//   - velocity, (nu / J_P) times the sum: the halves with P's own
//     differences touch only P's direct neighbours and join the matrix C
//     (Eq. difNonOrthoMatDiscrete: W_k(P) = sum over P's inner faces on the
//     axes j != k of N_f mean(alpha_jk) / 2 multiplies (q_{k+} - q_{k-}) / 2);
//     their boundary-value constants and the tangential fluxes through
//     Dirichlet faces go to rhs0 once per step; the halves with the
//     neighbour's differences (P's diagonal neighbours, Eq. velRHSnonOrtho)
//     go to the right-hand sides with the previous iterate (the predictor's,
//     each corrector's input velocity).  A missing neighbour in a cell
//     difference is the ghost 2 u_b - u_Q of the Dirichlet face; on a
//     Dirichlet face of P the tangential derivative is half the difference of
//     the boundary values on the same side at P's k-neighbours (P's own value
//     where a k-neighbour has no face there);
//   - pressure: the whole cell-integrated sum with mean(alpha_jk / A) goes to
//     the right-hand side with the previous pressure iterate (its direct part
//     in P would make P unsymmetric for the CG); a missing neighbour in a cell
//     difference is p_Q, and no cross flux crosses a Dirichlet-velocity face
//     (zero-Neumann pressure, App. A.3).
// The solves are repeated n_nonortho times.  Neighbours of neighbours are
// located arithmetically (locate), so the terms can be formed for any cell.
#pragma once

namespace piso {

// alpha_jk, j != k, of cell i (pairs (0,1), (0,2), (1,2) stored at j + k - 1).
template <typename real>
__device__ __forceinline__ real cross_metric(const real* Gx, int32_t N, int j, int k, int32_t i) {
  return Gx[(size_t)(j + k - 1) * N + i];
}

// alpha_jk of the neighbour across side s of cell i, in cell i's frame (its
// own metric read through the joint's frame code; the plain reading when fr
// is null).
template <typename real>
__device__ __forceinline__ real cross_metric_nb(const real* Gx, const int16_t* fr, int32_t N, int s, int32_t i,
                                                int32_t F, int j, int k) {
  if (!fr) return cross_metric(Gx, N, j, k, F);
  const int code = fr[(size_t)s * N + i];
  const real v = cross_metric(Gx, N, fr_ax(code, j), fr_ax(code, k), F);
  return (fr_neg(code, j) ^ fr_neg(code, k)) ? -v : v;
}

// Central difference of q along axis k at cell c; bq: this component's
// boundary values [nbf] (velocity) or null (pressure: the cell's own value).
template <typename real, int ND>
__device__ __forceinline__ real cell_diff(const Cell& c, const real* q, const real* bq, int k) {
  const real qP = q[c.i];
  const int32_t hi = c.nb[2 * k + 1], lo = c.nb[2 * k];
  const real vh = hi >= 0 ? q[hi] : (bq ? real(2) * bq[-1 - hi] - qP : qP);
  const real vl = lo >= 0 ? q[lo] : (bq ? real(2) * bq[-1 - lo] - qP : qP);
  return real(0.5) * (vh - vl);
}

// Central difference along cell i's axis k of its neighbour cF across side s
// (the neighbour's own difference along the matching axis, with its
// orientation).
template <typename real, int ND>
__device__ __forceinline__ real cell_diff_nb(const Cell& cF, const real* q, const real* bq, const int16_t* fr,
                                             int32_t N, int s, int32_t i, int k) {
  if (!fr) return cell_diff<real, ND>(cF, q, bq, k);
  const int code = fr[(size_t)s * N + i];
  const real v = cell_diff<real, ND>(cF, q, bq, fr_ax(code, k));
  return fr_neg(code, k) ? -v : v;
}

// The side of cell i's neighbour across side sk that matches cell i's side s.
__device__ __forceinline__ int side_nb(const int16_t* fr, int32_t N, int sk, int32_t i, int s) {
  if (!fr) return s;
  const int code = fr[(size_t)sk * N + i];
  const int j = s >> 1;
  return 2 * fr_ax(code, j) + ((((s & 1) ? 1 : 0) ^ fr_neg(code, j)) ? 1 : 0);
}

// W_k(P) = sum over P's inner faces f on the axes j != k of N_f mean(alpha_jk)
// / 2: the coefficient of P's own central difference along k in the viscous
// cross terms (the direct-neighbour part of Eq. difNonOrthoMatDiscrete).
template <typename real, int ND>
__device__ __forceinline__ void cross_w(const Cell& c, const real* Gx, int32_t N, real (&W)[ND],
                                        const int16_t* fr = nullptr) {
  const int32_t P = c.i;
#pragma unroll
  for (int k = 0; k < ND; k++) W[k] = 0;
#pragma unroll
  for (int s = 0; s < 2 * ND; s++) {
    const int j = s >> 1;
    const int32_t F = c.nb[s];
    if (F < 0) continue;
    const real n = (s & 1) ? real(1) : real(-1);
#pragma unroll
    for (int k = 0; k < ND; k++)
      if (k != j) W[k] += n * real(0.25) * (cross_metric(Gx, N, j, k, P) + cross_metric_nb(Gx, fr, N, s, P, F, j, k));
  }
}

// Tangential cross flux through a Dirichlet face on side s (axis j) of cell c
// for every component: sum_{k != j} N_f alpha_jk,P (bq[fh] - bq[fl]) / 2, fh / fl
// the faces on side s of P's k-neighbours (P's own face where there is none).
template <typename real, int ND>
__device__ __forceinline__ void cross_bface(const DomStatic& D, const Cell& c, int s, const real* bval, int32_t nbf,
                                            const real* Gx, real (&acc)[ND]) {
  const int32_t N = D.N, P = c.i;
  const int j = s >> 1;
  const real n = (s & 1) ? real(1) : real(-1);
  const int32_t fP = -1 - c.nb[s];
  for (int k = 0; k < ND; k++) {
    if (k == j) continue;
    const real a = cross_metric(Gx, N, j, k, P);
    int32_t fh = fP, fl = fP;
    if (c.nb[2 * k + 1] >= 0) {
      const int32_t t = locate<ND>(D, c.nb[2 * k + 1]).nb[side_nb(D.nbfr, N, 2 * k + 1, P, s)];
      if (t < 0) fh = -1 - t;
    }
    if (c.nb[2 * k] >= 0) {
      const int32_t t = locate<ND>(D, c.nb[2 * k]).nb[side_nb(D.nbfr, N, 2 * k, P, s)];
      if (t < 0) fl = -1 - t;
    }
#pragma unroll
    for (int q = 0; q < ND; q++) {
      const real* bq = bval + (size_t)q * nbf;
      acc[q] += n * a * (real(0.5) * (bq[fh] - bq[fl]));
    }
  }
}

// The deferred viscous cross terms at cell c (Eq. velRHSnonOrtho): (nu / J_P)
// sum over P's inner faces f on axis j, k != j, of N_f mean(alpha_jk) times
// half the neighbour's central difference along k, for the ND components of
// u [ND][N]; bval [ND][nbf] gives the ghosts of the neighbour's differences.
template <typename real, int ND>
__device__ __forceinline__ void cross_visc(const DomStatic& D, const Cell& c, const real* u, const real* bval,
                                          int32_t nbf, const real* Gx, const real* J, real nu,
                                          real (&out)[ND]) {
  const int32_t N = D.N, P = c.i;
  real acc[ND];
#pragma unroll
  for (int q = 0; q < ND; q++) acc[q] = 0;
  for (int s = 0; s < 2 * ND; s++) {
    const int j = s >> 1;
    const real n = (s & 1) ? real(1) : real(-1);
    const int32_t F = c.nb[s];
    if (F < 0) continue;
    const Cell cF = locate<ND>(D, F);
    for (int k = 0; k < ND; k++) {
      if (k == j) continue;
      const real a = real(0.5) * (cross_metric(Gx, N, j, k, P) + cross_metric_nb(Gx, D.nbfr, N, s, P, F, j, k));
#pragma unroll
      for (int q = 0; q < ND; q++) {
        const real* uq = u + (size_t)q * N;
        const real* bq = bval + (size_t)q * nbf;
        acc[q] += n * a * (real(0.5) * cell_diff_nb<real, ND>(cF, uq, bq, D.nbfr, N, s, P, k));
      }
    }
  }
  const real f = nu / J[P];
#pragma unroll
  for (int q = 0; q < ND; q++) out[q] = f * acc[q];
}

// sum_j sum_{k != j} sum_{inner f} N_f mean(alpha_jk / A) (d_k p)_f at cell c.
template <typename real, int ND>
__device__ __forceinline__ real cross_pres(const DomStatic& D, const Cell& c, const real* p, const real* invA,
                                           const real* Gx) {
  const int32_t N = D.N, P = c.i;
  real acc = 0;
  for (int s = 0; s < 2 * ND; s++) {
    const int j = s >> 1;
    const real n = (s & 1) ? real(1) : real(-1);
    const int32_t F = c.nb[s];
    if (F < 0) continue;
    const Cell cF = locate<ND>(D, F);
    for (int k = 0; k < ND; k++) {
      if (k == j) continue;
      const real a = real(0.5) * (cross_metric(Gx, N, j, k, P) * invA[P] +
                                  cross_metric_nb(Gx, D.nbfr, N, s, P, F, j, k) * invA[F]);
      const real g = real(0.5) * (cell_diff<real, ND>(c, p, nullptr, k) +
                                  cell_diff_nb<real, ND>(cF, p, nullptr, D.nbfr, N, s, P, k));
      acc += n * a * g;
    }
  }
  return acc;
}

// ---------------------------------------------------------------------------
// Transposes of the deferred cross terms for the adjoint step, in gather form
// (each cell collects what its neighbours' terms send it, so no atomics and a
// fixed summation order).  The neighbour R across side s of Q sees Q across
// its opposite side, so the face sign from R is -N_s and the face mean is the
// same.  Two phases with a group barrier between them: phase 1 forms, per
// cell, the sensitivity gdk[k] of the cross terms to the cell's own central
// difference along k; phase 2 spreads gdk back to the cells (and boundary
// faces) those differences read.
// ---------------------------------------------------------------------------

// Pressure, phase 1 at cell c for dL/dY = sc g (Y the pressure cross terms at
// pressure p, A = 1/invA): gdk[k][Q] = sum over Q's inner faces on axes j != k
// of N_s mean(alpha_jk / A) (g_Q - g_F) / 2; returns dL/dA_Q = -sum N_s
// alpha_jk,Q / (2 A_Q^2) (d_k p)_f (g_Q - g_F).
template <typename real, int ND>
__device__ __forceinline__ real cross_pres_T1(const DomStatic& D, const Cell& c, const real* g, real sc, const real* p,
                                              const real* invA, const real* Gx, real* gdk) {
  const int32_t N = D.N, Q = c.i;
  real acc[ND];
#pragma unroll
  for (int k = 0; k < ND; k++) acc[k] = 0;
  real ga = 0;
  const real iaQ = invA[Q];
  for (int s = 0; s < 2 * ND; s++) {
    const int j = s >> 1;
    const int32_t F = c.nb[s];
    if (F < 0) continue;
    const real n = (s & 1) ? real(1) : real(-1);
    const Cell cF = locate<ND>(D, F);
    const real dg = real(0.5) * n * sc * (g[Q] - g[F]);
    for (int k = 0; k < ND; k++) {
      if (k == j) continue;
      const real GQ = cross_metric(Gx, N, j, k, Q);
      const real a = real(0.5) * (GQ * iaQ + cross_metric_nb(Gx, D.nbfr, N, s, Q, F, j, k) * invA[F]);
      acc[k] += a * dg;
      const real gk = real(0.5) * (cell_diff<real, ND>(c, p, nullptr, k) +
                                   cell_diff_nb<real, ND>(cF, p, nullptr, D.nbfr, N, s, Q, k));
      ga -= GQ * iaQ * iaQ * gk * dg;
    }
  }
#pragma unroll
  for (int k = 0; k < ND; k++) gdk[(size_t)k * N + Q] = acc[k];
  return ga;
}

// Phase 2 of both transposes: the transpose of the central differences,
// sum_k (gdk[k] at the -k neighbour - gdk[k] at the +k neighbour) / 2; a
// missing neighbour was the ghost of cell Q itself: for the pressure (p_Q) its
// own gdk[k] / 2 with the sign of that side; for the velocity (2 u_b - u_Q)
// minus that, and the face value receives gdk[k] with the sign of the side
// (gbk: the component's boundary-value gradient [nbf], or null).
template <typename real, int ND, bool VEL>
__device__ __forceinline__ real cross_diff_T2(const Cell& c, const real* gdk, int32_t N, real* gbk,
                                              const int16_t* fr = nullptr) {
  const int32_t Q = c.i;
  real v = 0;
#pragma unroll
  for (int k = 0; k < ND; k++) {
    const real* gk = gdk + (size_t)k * N;
    const int32_t hi = c.nb[2 * k + 1], lo = c.nb[2 * k];
    if (fr) {
      // the neighbour R's own difference reads this cell on R's side facing it
#pragma unroll
      for (int e = 0; e < 2; e++) {
        const int s = 2 * k + e;
        const int32_t R = c.nb[s];
        if (R < 0) continue;
        const int rs = fr_ret(fr[(size_t)s * N + Q], s);
        const real w = gdk[(size_t)(rs >> 1) * N + R];
        v += (rs & 1) ? real(0.5) * w : real(-0.5) * w;
      }
    } else {
      if (lo >= 0) v += real(0.5) * gk[lo];
      if (hi >= 0) v -= real(0.5) * gk[hi];
    }
    if (hi < 0) {
      v += (VEL ? real(-0.5) : real(0.5)) * gk[Q];
      if (VEL && gbk) gbk[-1 - hi] += gk[Q];
    }
    if (lo < 0) {
      v -= (VEL ? real(-0.5) : real(0.5)) * gk[Q];
      if (VEL && gbk) gbk[-1 - lo] -= gk[Q];
    }
  }
  return v;
}

// Velocity (the deferred halves, Eq. velRHSnonOrtho), phase 1 at cell c for
// g = dL/dX [ND][N] (X at viscosity nu): for every component q,
// gdk[q][k][Q] = sum over Q's inner faces (axis j, neighbour R) with k != j of
// -N_s mean(alpha_jk) (nu / J_R) g_q,R / 2.
template <typename real, int ND>
__device__ __forceinline__ void cross_visc_T1(const Cell& c, const real* g, const real* Gx, const real* J, real nu,
                                              int32_t N, real* gdk, const int16_t* fr = nullptr) {
  const int32_t Q = c.i;
  real acc[ND][ND];
#pragma unroll
  for (int q = 0; q < ND; q++)
#pragma unroll
    for (int k = 0; k < ND; k++) acc[q][k] = 0;
#pragma unroll
  for (int s = 0; s < 2 * ND; s++) {
    const int j = s >> 1;
    const int32_t R = c.nb[s];
    if (R < 0) continue;
    const real n = (s & 1) ? real(1) : real(-1);
    const real w = -n * real(0.5) * nu / J[R];
#pragma unroll
    for (int k = 0; k < ND; k++) {
      if (k == j) continue;
      const real a = real(0.5) * (cross_metric(Gx, N, j, k, Q) + cross_metric_nb(Gx, fr, N, s, Q, R, j, k)) * w;
#pragma unroll
      for (int q = 0; q < ND; q++) acc[q][k] += a * g[(size_t)q * N + R];
    }
  }
#pragma unroll
  for (int q = 0; q < ND; q++)
#pragma unroll
    for (int k = 0; k < ND; k++) gdk[((size_t)q * ND + k) * N + Q] = acc[q][k];
}

// Transpose, in the boundary values, of the constant part of the matrix
// (direct-neighbour) cross terms that rhs0 carries (Eq.
// difNonOrthoMatDiscrete with Dirichlet ghosts, and the tangential fluxes
// through Dirichlet faces) for g = dL/drhs0 [ND][N]: adds to the gradient of
// every Dirichlet face of cell c (gbval [ND][nbf]) what the rows of c and of
// its neighbours along that side send it.  W: cross_w of c.
template <typename real, int ND>
__device__ __forceinline__ void cross_const_T(const DomStatic& D, const Cell& c, const real (&W)[ND], const real* g,
                                              const real* Gx, const real* J, real nu, int32_t nbf, real* gbval) {
  const int32_t N = D.N, Q = c.i;
  const real fQ = nu / J[Q];
#pragma unroll
  for (int s = 0; s < 2 * ND; s++) {
    if (c.nb[s] >= 0) continue;
    const int j = s >> 1;
    const real n = (s & 1) ? real(1) : real(-1);
    const int32_t f = -1 - c.nb[s];
    real acc[ND];
#pragma unroll
    for (int q = 0; q < ND; q++) acc[q] = n * W[j] * fQ * g[(size_t)q * N + Q];   // Q's own ghost on this face
    for (int k = 0; k < ND; k++) {
      if (k == j) continue;
      const real hQ = real(0.5) * n * fQ * cross_metric(Gx, N, j, k, Q);
      bool hi_face = false, lo_face = false;
      // a k-neighbour R reads this face in its own tangential difference (the
      // face of its side matching s): with 1/2 if this cell is R's + neighbour
      // along that difference, -1/2 if its - neighbour; the term's sign N_s
      // alpha_jk of R in R's frame is the same in this cell's frame up to the
      // joint's orientation of j
#pragma unroll
      for (int e = 0; e < 2; e++) {
        const int sk = 2 * k + e;
        const int32_t R = c.nb[sk];
        if (R < 0) continue;
        const bool face = locate<ND>(D, R).nb[side_nb(D.nbfr, N, sk, Q, s)] < 0;
        if (e) hi_face = face;
        else lo_face = face;
        if (!face) continue;
        real hR;
        bool plus;
        if (D.nbfr) {
          const int code = D.nbfr[(size_t)sk * N + Q];
          const real Gr = cross_metric(Gx, N, fr_ax(code, j), fr_ax(code, k), R);
          hR = real(0.5) * n * (fr_neg(code, j) ? -Gr : Gr) * (nu / J[R]);
          plus = (fr_ret(code, sk) & 1) != 0;
        } else {
          hR = real(0.5) * n * (nu / J[R]) * cross_metric(Gx, N, j, k, R);
          plus = !e;
        }
#pragma unroll
        for (int q = 0; q < ND; q++) acc[q] += (plus ? hR : -hR) * g[(size_t)q * N + R];
      }
      // Q's own tangential difference uses its own face where a k-neighbour has none
#pragma unroll
      for (int q = 0; q < ND; q++) acc[q] += hQ * g[(size_t)q * N + Q] * (real(hi_face ? 0 : 1) - real(lo_face ? 0 : 1));
    }
#pragma unroll
    for (int q = 0; q < ND; q++) gbval[(size_t)q * nbf + f] += acc[q];
  }
}

// Per-unit-viscosity constant part of the matrix cross terms of rhs0 at cell
// c for every component: (1 / J_P) (sum over Dirichlet sides of N_s W_k u_b +
// the tangential fluxes through P's Dirichlet faces).
template <typename real, int ND>
__device__ __forceinline__ void cross_const(const DomStatic& D, const Cell& c, const real (&W)[ND], const real* bval,
                                            int32_t nbf, const real* Gx, const real* J, real (&out)[ND]) {
  real acc[ND];
#pragma unroll
  for (int q = 0; q < ND; q++) acc[q] = 0;
#pragma unroll
  for (int s = 0; s < 2 * ND; s++) {
    if (c.nb[s] >= 0) continue;
    const int j = s >> 1;
    const real n = (s & 1) ? real(1) : real(-1);
    const int32_t f = -1 - c.nb[s];
#pragma unroll
    for (int q = 0; q < ND; q++) acc[q] += n * W[j] * bval[(size_t)q * nbf + f];
    cross_bface<real, ND>(D, c, s, bval, nbf, Gx, acc);
  }
  const real f1 = real(1) / J[c.i];
#pragma unroll
  for (int q = 0; q < ND; q++) out[q] = f1 * acc[q];
}

}  // namespace piso
