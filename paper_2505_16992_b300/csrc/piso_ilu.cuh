// ILU(0)-preconditioned BiCGStab for the advection-diffusion solves
// (arXiv:2505.16992, App. A.5: an incomplete-LU preconditioner for the
// BiCGStab, for grids with strongly varying cell sizes, used throughout or only
// after the unpreconditioned solve failed).
//
// B300 layout.  A global ILU(0) couples every cell to every cell before it in
// index order, so its triangular solves advance one grid hyperplane at a time
// (nx + ny + nz steps), each needing a grid-wide barrier: ~1 ms per
// application on this path.  Here each CTA factors the diagonal block of C made
// of the cells it owns (block Jacobi with ILU(0) blocks): couplings to cells of
// other CTAs are left out of the preconditioner, never out of the matrix.  The
// CTA's triangular solves then need only CTA barriers: its cells are grouped by
// level on the host (level = longest chain of lower in-block neighbours), and
// all cells of a level are solved in parallel.  With one CTA the block is the
// whole matrix and this is exactly ILU(0) in natural order.
//
// Form of the factors.  For matrices whose neighbour graph has no triangles
// (every structured grid here: a triangle needs a periodic direction of at
// most 3 cells) zero-fill ILU changes only the diagonal: with L and U the
// strictly lower and upper parts of the block, M = (D + L) D^-1 (D + U) and
//   d_i = c_ii - sum_{k < i, k ~ i in block} c_ik c_ki / d_k.
// The products c_ik c_ki are symmetric, so C^T (the adjoint's transposed
// solve) has the same pivots and its factors are the transposes: one
// factorisation serves both directions, applied with the transposed rows.
#pragma once

namespace piso {

// Host-built tables of one launch layout (CTA count, CTA width and cell
// ownership of the launch).
struct IluTab {
  const int32_t* order;    // [N] each CTA's cells grouped by level, ascending index inside a level
  const uint16_t* mask;    // [N] bit s: nb(i, s) lies in i's CTA block with a lower index; bit 8+s: higher
  const int32_t* lstart;   // level starts of every CTA, relative to its slice of order
  const int32_t* lidx;     // [ncta + 1] CTA r's level starts are lstart[lidx[r] .. lidx[r + 1])
  const int32_t* base;     // [ncta] start of CTA r's slice of order
};

template <typename real>
struct IluPre {
  const int32_t* ord;      // this CTA's cells by level
  const int32_t* ls;       // its level starts (nlev + 1 entries)
  const uint16_t* mask;
  real* dinv;              // [N] reciprocal pivots 1 / d_i
  int32_t nlev;
};

template <typename real>
__device__ __forceinline__ IluPre<real> ilu_setup(const IluTab& t, real* dinv, int rank) {
  IluPre<real> P;
  const int32_t l0 = t.lidx[rank], l1 = t.lidx[rank + 1];
  P.ord = t.order + t.base[rank];
  P.ls = t.lstart + l0;
  P.nlev = l1 - l0 - 1;
  P.mask = t.mask;
  P.dinv = dinv;
  return P;
}

// Pivots of this CTA's block, level by level (CTA barrier between levels).
// A pivot that is not safely positive (C has a positive diagonal; ILU(0) of
// an M-matrix keeps its pivots positive) falls back to c_ii.
template <typename real, int ND>
__device__ void ilu_factor(const Ctx<real, ND>& X, const IluPre<real>& P, const real* Cdiag, const real* Coff) {
  const int32_t N = X.N;
  for (int l = 0; l < P.nlev; l++) {
    const int32_t e = P.ls[l + 1];
    for (int32_t j = P.ls[l] + (int32_t)threadIdx.x; j < e; j += (int32_t)blockDim.x) {
      const Cell c = X.cell(P.ord[j]);
      const uint32_t m = P.mask[c.i];
      real diag, cf[2 * ND], ct[2 * ND];
      c_row<real, ND, false>(c, N, Cdiag, Coff, diag, cf);
      real d = diag;
      if (m & 0xffu) {
        c_row<real, ND, true>(c, N, Cdiag, Coff, diag, ct);
#pragma unroll
        for (int s = 0; s < 2 * ND; s++)
          if ((m >> s) & 1u) d -= cf[s] * ct[s] * P.dinv[c.nb[s]];
      }
      if (!(d > real(1e-5) * diag)) d = diag;
      P.dinv[c.i] = real(1) / d;
    }
    __syncthreads();
  }
}

// z = M^-1 w for the active components, M = C's block factors (TR = false) or
// their transposes (TR = true).  Forward substitution with the lower part over
// ascending levels, q_i = (w_i - sum_{k lower} m_ik q_k) / d_i, then backward
// with the upper part over descending levels, z_i = q_i - (1/d_i) sum_{j upper}
// m_ij z_j.  src(k, i) yields w_k at own cell i; it is called exactly once per
// cell and component, in the forward pass (so it may also store w).  Only the
// CTA's own cells are read and written: no group barrier is needed.
template <typename real, int ND, bool TR, typename SRC>
__device__ __forceinline__ void ilu_apply(const Ctx<real, ND>& X, const IluPre<real>& P, const real* Cdiag,
                                          const real* Coff, const int (&act)[ND], SRC&& src, real* z) {
  const int32_t N = X.N;
  __syncthreads();   // own-cell values written by other threads of the CTA before this call
  for (int l = 0; l < P.nlev; l++) {
    const int32_t e = P.ls[l + 1];
    for (int32_t j = P.ls[l] + (int32_t)threadIdx.x; j < e; j += (int32_t)blockDim.x) {
      const Cell c = X.cell(P.ord[j]);
      const uint32_t m = P.mask[c.i] & 0xffu;
      const real di = P.dinv[c.i];
      real diag, cf[2 * ND];
      if (m) c_row<real, ND, TR>(c, N, Cdiag, Coff, diag, cf);
#pragma unroll
      for (int k = 0; k < ND; k++) {
        if (!act[k]) continue;
        const size_t o_ = (size_t)k * N;
        real w = src(k, c.i);
        if (m) {
#pragma unroll
          for (int s = 0; s < 2 * ND; s++)
            if ((m >> s) & 1u) w -= cf[s] * z[o_ + c.nb[s]];
        }
        z[o_ + c.i] = w * di;
      }
    }
    __syncthreads();
  }
  for (int l = P.nlev - 1; l >= 0; l--) {
    const int32_t e = P.ls[l + 1];
    for (int32_t j = P.ls[l] + (int32_t)threadIdx.x; j < e; j += (int32_t)blockDim.x) {
      const int32_t i = P.ord[j];
      const uint32_t m = P.mask[i] >> 8;
      if (!m) continue;
      const Cell c = X.cell(i);
      const real di = P.dinv[i];
      real diag, cf[2 * ND];
      c_row<real, ND, TR>(c, N, Cdiag, Coff, diag, cf);
#pragma unroll
      for (int k = 0; k < ND; k++) {
        if (!act[k]) continue;
        const size_t o_ = (size_t)k * N;
        real acc = 0;
#pragma unroll
        for (int s = 0; s < 2 * ND; s++)
          if ((m >> s) & 1u) acc += cf[s] * z[o_ + c.nb[s]];
        z[o_ + i] -= di * acc;
      }
    }
    __syncthreads();
  }
}

// Restart of a BiCGStab that failed: x = x0 (zero when x0 is null), r = rhat
// (the shadow residual is the initial residual b - M x0 and never changes),
// and the scalars from the saved norms.  The iterations of the failed attempt
// are kept in iters_prev.
template <typename real, int ND>
__device__ void bicg_restart(const Ctx<real, ND>& X, BiState& bs, real* x, const real* x0, real* r,
                             const real* rhat, double rtol, double atol, int32_t* status) {
  const int32_t N = X.N;
  X.own([&](int32_t i) {
#pragma unroll
    for (int k = 0; k < ND; k++) {
      const size_t o_ = (size_t)k * N + i;
      x[o_] = x0 ? x0[o_] : real(0);
      r[o_] = rhat[o_];
    }
  });
  if (threadIdx.x == 0) {
    int prev[3];
    double q[6];
    for (int k = 0; k < ND; k++) prev[k] = bs.iters[k] + bs.iters_prev[k];
    for (int k = 0; k < 2 * ND; k++) q[k] = bs.q0[k];
    bicg_start<ND>(bs, q, rtol, atol, status);
    for (int k = 0; k < ND; k++) bs.iters_prev[k] = prev[k];
  }
  __syncthreads();
}

// Right-preconditioned BiCGStab (van der Vorst 1992 with K1 = I, K2 = M) on
// Mat x = b, Mat = C or C^T, for the ND components sharing Mat.  Per iteration:
//   PA  p = r + beta (p - omega v); y = K^-1 p          (CTA-local) + barrier
//   PB  v = Mat y; (rhat, v) -> alpha                   reduction
//   PC  s = r - alpha v; z = K^-1 s                     (CTA-local) + barrier
//   PD  t = Mat z; (t, s), (t, t), (s, s) -> omega      reduction
//   PE  x += alpha y + omega z; r = s - omega t; (rhat, r), (r, r)   reduction
// On entry x = x0, r = b - Mat x0, rhat = r, bs from bicg_start, pivots formed.
template <typename real, int ND, bool TR>
__device__ bool bicgstab_ilu(const Ctx<real, ND>& X, const IluPre<real>& P, BiState& bs, int maxit,
                             const real* Cdiag, const real* Coff, real* x, real* r, const real* rhat, real* p,
                             real* v, real* y, real* z, real* t) {
  const int32_t N = X.N;
  while (bs.any && bs.it < maxit) {
    // PA
    {
      real beta[ND], om[ND];
      int act[ND];
#pragma unroll
      for (int k = 0; k < ND; k++) {
        act[k] = bs.active[k];
        beta[k] = pick<real>(bs.beta_d[k], bs.beta_f[k]);
        om[k] = pick<real>(bs.omega[k], bs.omega_f[k]);
      }
      const int first = bs.first;
      ilu_apply<real, ND, TR>(X, P, Cdiag, Coff, act, [&](int k, int32_t i) -> real {
        const size_t o_ = (size_t)k * N + i;
        const real pn = first ? r[o_] : r[o_] + beta[k] * (p[o_] - om[k] * v[o_]);
        p[o_] = pn;
        return pn;
      }, y);
      if (!plain_sync(X.g)) return false;
    }
    // PB
    {
      Acc<real> a[ND];
      int act[ND];
#pragma unroll
      for (int k = 0; k < ND; k++) {
        a[k].zero();
        act[k] = bs.active[k];
      }
      X.cells([&](const Cell& c) {
        real diag, cf[2 * ND];
        c_row<real, ND, TR>(c, N, Cdiag, Coff, diag, cf);
#pragma unroll
        for (int k = 0; k < ND; k++) {
          if (!act[k]) continue;
          const size_t o_ = (size_t)k * N;
          real vv = diag * y[o_ + c.i];
#pragma unroll
          for (int s = 0; s < 2 * ND; s++)
            if (c.nb[s] >= 0) vv += cf[s] * y[o_ + c.nb[s]];
          v[o_ + c.i] = vv;
          a[k].add_prod(rhat[o_ + c.i], vv);
        }
      });
      if (!reduce_sync<real, ND>(X.g, a, [&](const double* q) { bicg_update_alpha<ND>(bs, q); })) return false;
    }
    // PC
    {
      real al[ND];
      int act[ND];
#pragma unroll
      for (int k = 0; k < ND; k++) {
        act[k] = bs.active[k];
        al[k] = pick<real>(bs.alpha[k], bs.alpha_f[k]);
      }
      ilu_apply<real, ND, TR>(X, P, Cdiag, Coff, act, [&](int k, int32_t i) -> real {
        const size_t o_ = (size_t)k * N + i;
        return r[o_] - al[k] * v[o_];
      }, z);
      if (!plain_sync(X.g)) return false;
    }
    // PD
    {
      Acc<real> a[3 * ND];
      real al[ND];
      int act[ND];
#pragma unroll
      for (int k = 0; k < ND; k++) {
        act[k] = bs.active[k];
        al[k] = pick<real>(bs.alpha[k], bs.alpha_f[k]);
      }
#pragma unroll
      for (int k = 0; k < 3 * ND; k++) a[k].zero();
      X.cells([&](const Cell& c) {
        real diag, cf[2 * ND];
        c_row<real, ND, TR>(c, N, Cdiag, Coff, diag, cf);
#pragma unroll
        for (int k = 0; k < ND; k++) {
          if (!act[k]) continue;
          const size_t o_ = (size_t)k * N;
          real tt = diag * z[o_ + c.i];
#pragma unroll
          for (int s = 0; s < 2 * ND; s++)
            if (c.nb[s] >= 0) tt += cf[s] * z[o_ + c.nb[s]];
          const real sP = r[o_ + c.i] - al[k] * v[o_ + c.i];
          t[o_ + c.i] = tt;
          a[k].add_prod(tt, sP);
          a[ND + k].add_prod(tt, tt);
          a[2 * ND + k].add_prod(sP, sP);
        }
      });
      if (!reduce_sync<real, 3 * ND>(X.g, a, [&](const double* q) { bicg_update_omega<ND>(bs, q); })) return false;
    }
    // PE
    {
      Acc<real> a[2 * ND];
      real al[ND], om[ND];
      int act[ND], sc[ND];
#pragma unroll
      for (int k = 0; k < ND; k++) {
        act[k] = bs.active[k];
        sc[k] = bs.sconv[k];
        al[k] = pick<real>(bs.alpha[k], bs.alpha_f[k]);
        om[k] = pick<real>(bs.omega[k], bs.omega_f[k]);
        a[k].zero();
        a[ND + k].zero();
      }
      X.own([&](int32_t i) {
#pragma unroll
        for (int k = 0; k < ND; k++) {
          if (!act[k]) continue;
          const size_t o_ = (size_t)k * N + i;
          if (sc[k]) {
            x[o_] += al[k] * y[o_];
            continue;
          }
          const real sP = r[o_] - al[k] * v[o_];
          x[o_] += al[k] * y[o_] + om[k] * z[o_];
          const real rn = sP - om[k] * t[o_];
          r[o_] = rn;
          a[k].add_prod(rhat[o_], rn);
          a[ND + k].add_prod(rn, rn);
        }
      });
      if (!reduce_sync<real, 2 * ND>(X.g, a, [&](const double* q) { bicg_update_rho<ND>(bs, q); })) return false;
    }
  }
  return true;
}

}  // namespace piso
