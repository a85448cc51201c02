// Cross-derivative terms of non-orthogonal meshes (arXiv:2505.16992, App. A.2
// "Non-Orthogonal Grids", Eqs. difNonOrthoMatDiscrete, velRHSnonOrtho,
// pressureRHSnonOrtho).  With alpha_jk = J T_j . T_k, the flux through a face
// of cell P on axis j gets, for every k != j, N_f mean(alpha_jk) (d_k q)_f,
// where (d_k q)_f is the mean of the central differences along k of P and of
// its neighbour across the face: summed over P's faces this is the central
// d_j d_k q.  The matrices C and P keep their orthogonal stencils; these terms
// go to the right-hand sides with the previous iterate (the predictor's, each
// corrector's input velocity, the previous pressure), and the solves are
// repeated n_nonortho times.
//   - velocity: (nu / J_P) times the sum; a missing neighbour in a cell
//     difference is the ghost 2 u_b - u_Q of the Dirichlet face; on a
//     Dirichlet face of P the tangential derivative is half the difference of
//     the boundary values on the same side at P's k-neighbours (P's own value
//     where a k-neighbour has no face there);
//   - pressure: the cell-integrated sum with mean(alpha_jk / A); a missing
//     neighbour in a cell difference is p_Q, and no cross flux crosses a
//     Dirichlet-velocity face (zero-Neumann pressure, App. A.3).
// Neighbours of neighbours are located arithmetically (locate), so the terms
// can be formed for any cell of the domain.
#pragma once

namespace piso {

// alpha_jk, j != k, of cell i (pairs (0,1), (0,2), (1,2) stored at j + k - 1).
template <typename real>
__device__ __forceinline__ real cross_metric(const real* Gx, int32_t N, int j, int k, int32_t i) {
  return Gx[(size_t)(j + k - 1) * N + i];
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

// (nu / J_P) sum_j sum_{k != j} sum_f N_f mean(alpha_jk) (d_k u)_f for the ND
// components of u [ND][N] at cell c; bval [ND][nbf].
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
    if (F >= 0) {
      const Cell cF = locate<ND>(D, F);
      for (int k = 0; k < ND; k++) {
        if (k == j) continue;
        const real a = real(0.5) * (cross_metric(Gx, N, j, k, P) + cross_metric(Gx, N, j, k, F));
#pragma unroll
        for (int q = 0; q < ND; q++) {
          const real* uq = u + (size_t)q * N;
          const real* bq = bval + (size_t)q * nbf;
          const real g = real(0.5) * (cell_diff<real, ND>(c, uq, bq, k) + cell_diff<real, ND>(cF, uq, bq, k));
          acc[q] += n * a * g;
        }
      }
    } else {
      const int32_t fP = -1 - F;
      for (int k = 0; k < ND; k++) {
        if (k == j) continue;
        const real a = cross_metric(Gx, N, j, k, P);
        // faces on side s of P's k-neighbours (P's own where there is none)
        int32_t fh = fP, fl = fP;
        if (c.nb[2 * k + 1] >= 0) {
          const int32_t t = locate<ND>(D, c.nb[2 * k + 1]).nb[s];
          if (t < 0) fh = -1 - t;
        }
        if (c.nb[2 * k] >= 0) {
          const int32_t t = locate<ND>(D, c.nb[2 * k]).nb[s];
          if (t < 0) fl = -1 - t;
        }
#pragma unroll
        for (int q = 0; q < ND; q++) {
          const real* bq = bval + (size_t)q * nbf;
          acc[q] += n * a * (real(0.5) * (bq[fh] - bq[fl]));
        }
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
      const real a = real(0.5) * (cross_metric(Gx, N, j, k, P) * invA[P] + cross_metric(Gx, N, j, k, F) * invA[F]);
      const real g = real(0.5) * (cell_diff<real, ND>(c, p, nullptr, k) + cell_diff<real, ND>(cF, p, nullptr, k));
      acc += n * a * g;
    }
  }
  return acc;
}

}  // namespace piso
