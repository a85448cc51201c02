// Forward PISO step as one persistent cooperative launch (arXiv:2505.16992,
// Sec. 2.1 and App. A.1-A.3): outflow update, assembly of C = A + H and the
// predictor right-hand side, BiCGStab for the d velocity components sharing
// C, assembly of the pressure matrix P, and n correctors (h, div h,
// Jacobi-PCG on -P, velocity correction).  Every phase walks this CTA's cell
// range; phases are separated by the group barrier.
#pragma once
#include "piso_device.cuh"

namespace piso {

// Per-domain, per-call arguments of the forward step.  Arrays are SoA,
// [component][cell]; "real" is the storage type (float or double).
template <typename real>
struct FwdCall {
  const DomStatic* dom;
  const real* u_in;          // [d][N] u^n
  const real* p_in;          // [N]    p^n
  real* u_out;               // [d][N] u^{n+1} (may alias u_in)
  real* p_out;               // [N]    p^{n+1} (may alias p_in)
  const real* S;             // [d][N] source or nullptr
  real* bval;                // [d][nbf] boundary values (outflow faces updated)
  double dt, nu;
  // recorded intermediates (tape or internal workspace)
  real* un;                  // [d][N] copy of u^n
  real* Cdiag;               // [N]
  real* Coff;                // [2d][N]
  real* ustar;               // [d][N]
  real* h[4];                // [d][N] per corrector
  real* xk[4];               // [N]    mean-free pressure per corrector
  real* uc[4];               // [d][N] corrector outputs (last one unused)
  real* bval_rec;            // [d][nbf] boundary values used by this step
  // scratch
  real* U;                   // [d][N]
  real* rhs0;                // [d][N]
  real* r;                   // [d][N]
  real* rhat;                // [d][N]
  real* pv[2];               // [d][N]
  real* vv[2];               // [d][N]
  real* t;                   // [d][N]
  real* Poff;                // [d][N] + faces
  real* Pdiag;               // [N]
  real* Fh;                  // [d][N] J T . h
  real* b;                   // [N]
  real* cx;                  // [N]
  real* cr;                  // [N]
  real* cz;                  // [N]
  real* cd[2];               // [N]
  real* cq;                  // [N]
  // group control
  uint32_t* bar;
  double* partials;
  int32_t* status;
  int32_t* istats;           // [16]
  double* dstats;            // [16]
  int32_t cta0, ncta;
};

struct SolverOpts {
  int32_t n_corr, pred_grad_p, adv_maxit, p_maxit;
  double adv_rtol, p_rtol, atol;
  uint64_t timeout_ns;
};

// Launch arguments.  One domain: its call travels by value in call0.  A batch:
// calls[] and cta_first[] live in device memory (CTA c belongs to group g when
// cta_first[g] <= c < cta_first[g+1]).
template <typename real>
struct FwdLaunch {
  int32_t ngroups;
  SolverOpts o;
  const int32_t* cta_first;
  const FwdCall<real>* calls;
  FwdCall<real> call0;
};

// Copy a POD struct into shared memory word by word (all threads).
template <typename Tt>
__device__ __forceinline__ void copy_to_smem(Tt* dst, const Tt* src) {
  static_assert(sizeof(Tt) % 4 == 0, "word-sized struct");
  const int32_t* s = reinterpret_cast<const int32_t*>(src);
  int32_t* d = reinterpret_cast<int32_t*>(dst);
  for (int k = threadIdx.x; k < (int)(sizeof(Tt) / 4); k += blockDim.x) d[k] = s[k];
}

__device__ __forceinline__ int find_group(int ngroups, const int32_t* cta_first) {
  int gi = 0;
  if (cta_first)
    while (gi + 1 < ngroups && (int)blockIdx.x >= cta_first[gi + 1]) gi++;
  return gi;
}

// Krylov scalar state, owned by thread 0 and broadcast through shared memory.
struct BiState {
  double rho[3], rho_old[3], alpha[3], omega[3], tol[3], res[3];
  int active[3], sconv[3], iters[3], conv[3];
  int any, it, first;
};

struct CgState {
  double rz, rz_old, alpha, tol, res, bn;
  int active, it, first;
};

template <typename real, int ND>
__device__ void fwd_group(const FwdCall<real>& A, const SolverOpts& o, Group& g) {
  __shared__ DomStatic D;
  __shared__ BiState bs;
  __shared__ CgState cs;
  __shared__ double s_scale, s_mean;
  copy_to_smem(&D, A.dom);   // static domain description into shared memory
  __syncthreads();
  const int32_t N = D.N;
  const int32_t lo = (int32_t)(((int64_t)N * g.rank) / g.ncta);
  const int32_t hi = (int32_t)(((int64_t)N * (g.rank + 1)) / g.ncta);
  const real* J = reinterpret_cast<const real*>(D.J);
  const real* T = reinterpret_cast<const real*>(D.T);
  const real* AL = reinterpret_cast<const real*>(D.alpha);
  const int NSD = 2 * ND;
  const real dt = (real)A.dt, nu = (real)A.nu, inv_dt = (real)(1.0 / A.dt);
  auto Tm = [&](int j, int k, int32_t i) -> real { return T[(size_t)(j * ND + k) * N + i]; };
  auto for_cells = [&](auto&& f) {
    for (int32_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
      const Cell c = locate<ND>(D, i);
      f(c);
    }
  };
  // boundary-face range of this CTA (outflow update)
  const int32_t flo = (int32_t)(((int64_t)D.nbf * g.rank) / g.ncta);
  const int32_t fhi = (int32_t)(((int64_t)D.nbf * (g.rank + 1)) / g.ncta);
  const int32_t nbf = D.nbf;

  // ------------------------------------------------------------------------
  // F0: advective outflow update (App. A.3, Eq. advOut; reading R10) and
  // inflow/outflow flux balance.
  // ------------------------------------------------------------------------
  if (D.n_out > 0) {
    Acc<real> a[2];
    a[0].zero();
    a[1].zero();
    const real* um = reinterpret_cast<const real*>(D.bf_um);
    for (int32_t f = flo + threadIdx.x; f < fhi; f += blockDim.x) {
      const int32_t P = D.bf_cell[f];
      const int s = D.bf_side[f];
      const int j = s >> 1;
      const real n = (s & 1) ? real(1) : real(-1);
      real ub[ND];
#pragma unroll
      for (int k = 0; k < ND; k++) ub[k] = A.bval[(size_t)k * nbf + f];
      if (D.bf_out[f]) {
        real tu = 0;
#pragma unroll
        for (int k = 0; k < ND; k++) tu += Tm(j, k, P) * um[(size_t)k * nbf + f];
        const real c = real(2) * dt * fabs(tu);
        const real fac = c / (real(1) + c);
#pragma unroll
        for (int k = 0; k < ND; k++) {
          ub[k] = ub[k] - fac * (ub[k] - A.u_in[(size_t)k * N + P]);
          A.bval[(size_t)k * nbf + f] = ub[k];
        }
      }
      real fl = 0;
#pragma unroll
      for (int k = 0; k < ND; k++) fl += Tm(j, k, P) * ub[k];
      fl *= n * J[P];
      if (D.bf_out[f]) a[1].add(fl);
      else a[0].add(-fl);
    }
    publish<real, 2>(g, a);
    if (!group_sync(g)) return;
    double q[2];
    gather<2>(g, q);
    if (threadIdx.x == 0) s_scale = (q[1] != 0.0) ? q[0] / q[1] : 1.0;
    __syncthreads();
    const real sc = (real)s_scale;
    for (int32_t f = flo + threadIdx.x; f < fhi; f += blockDim.x)
      if (D.bf_out[f]) {
#pragma unroll
        for (int k = 0; k < ND; k++) A.bval[(size_t)k * nbf + f] *= sc;
      }
  }
  // record the boundary values used by this step
  for (int32_t f = flo + threadIdx.x; f < fhi; f += blockDim.x)
#pragma unroll
    for (int k = 0; k < ND; k++) A.bval_rec[(size_t)k * nbf + f] = A.bval[(size_t)k * nbf + f];

  // ------------------------------------------------------------------------
  // F1: contravariant flux U^j = J T_j . u^n (App. A.2) and the tape copy of u^n
  // ------------------------------------------------------------------------
  for_cells([&](const Cell& c) {
    const int32_t P = c.i;
    real u[ND];
#pragma unroll
    for (int k = 0; k < ND; k++) {
      u[k] = A.u_in[(size_t)k * N + P];
      A.un[(size_t)k * N + P] = u[k];
    }
#pragma unroll
    for (int j = 0; j < ND; j++) {
      real s = 0;
#pragma unroll
      for (int k = 0; k < ND; k++) s += Tm(j, k, P) * u[k];
      A.U[(size_t)j * N + P] = J[P] * s;
    }
  });
  if (!group_sync(g)) return;

  // ------------------------------------------------------------------------
  // F2: assemble C and the right-hand sides (Eqs. advMatDiscrete,
  // difMatDiscrete, velRHSdiscrete; per-unit-volume rows, R1), predictor rhs
  // b = rhs0 - grad p^n (R4), BiCGStab start r = b - C u^n.
  // ------------------------------------------------------------------------
  {
    Acc<real> a[2 * ND];
#pragma unroll
    for (int k = 0; k < 2 * ND; k++) a[k].zero();
    for_cells([&](const Cell& c) {
      const int32_t P = c.i;
      const real invJ = real(1) / J[P];
      real diag = inv_dt;
      real rhs[ND];
      real off[2 * ND];
#pragma unroll
      for (int k = 0; k < ND; k++)
        rhs[k] = A.u_in[(size_t)k * N + P] * inv_dt + (A.S ? A.S[(size_t)k * N + P] : real(0));
#pragma unroll
      for (int s = 0; s < NSD; s++) {
        const int j = s >> 1;
        const real n = (s & 1) ? real(1) : real(-1);
        const int32_t F = c.nb[s];
        const real aP = AL[(size_t)j * N + P];
        if (F >= 0) {
          const real Uf = real(0.5) * (A.U[(size_t)j * N + P] + A.U[(size_t)j * N + F]);
          const real Df = nu * real(0.5) * (aP + AL[(size_t)j * N + F]);
          off[s] = (real(0.5) * n * Uf - Df) * invJ;
          diag += (real(0.5) * n * Uf + Df) * invJ;
        } else {
          const int32_t f = -1 - F;
          real ub[ND], tu = 0;
#pragma unroll
          for (int k = 0; k < ND; k++) {
            ub[k] = A.bval[(size_t)k * nbf + f];
            tu += Tm(j, k, P) * ub[k];
          }
          const real Ub = J[P] * tu;
          diag += real(2) * aP * nu * invJ;
          const real w = (real(2) * aP * nu - n * Ub) * invJ;
#pragma unroll
          for (int k = 0; k < ND; k++) rhs[k] += ub[k] * w;
          off[s] = real(0);
        }
        A.Coff[(size_t)s * N + P] = off[s];
      }
      A.Cdiag[P] = diag;
      // pressure gradient of p^n (Eq. velCorrDiscrete with R5)
      real gp[ND];
#pragma unroll
      for (int k = 0; k < ND; k++) gp[k] = 0;
      if (o.pred_grad_p) {
        const real pP = A.p_in[P];
#pragma unroll
        for (int j = 0; j < ND; j++) {
          const real pp = c.nb[2 * j + 1] >= 0 ? A.p_in[c.nb[2 * j + 1]] : pP;
          const real pm = c.nb[2 * j] >= 0 ? A.p_in[c.nb[2 * j]] : pP;
          const real dp = real(0.5) * (pp - pm);
#pragma unroll
          for (int k = 0; k < ND; k++) gp[k] += Tm(j, k, P) * dp;
        }
      }
#pragma unroll
      for (int k = 0; k < ND; k++) {
        A.rhs0[(size_t)k * N + P] = rhs[k];
        const real b = rhs[k] - gp[k];
        const real* x = A.u_in + (size_t)k * N;
        real cx = diag * x[P];
#pragma unroll
        for (int s = 0; s < NSD; s++)
          if (c.nb[s] >= 0) cx += off[s] * x[c.nb[s]];
        const real r = b - cx;
        A.r[(size_t)k * N + P] = r;
        A.rhat[(size_t)k * N + P] = r;
        A.ustar[(size_t)k * N + P] = x[P];
        a[k].add_prod(b, b);
        a[ND + k].add_prod(r, r);
      }
    });
    publish<real, 2 * ND>(g, a);
    if (!group_sync(g)) return;
    double q[2 * ND];
    gather<2 * ND>(g, q);
    if (threadIdx.x == 0) {
      bs.any = 0;
      bs.it = 0;
      for (int k = 0; k < ND; k++) {
        const double bn = sqrt(q[k]);
        bs.tol[k] = fmax(o.adv_rtol * bn, o.atol);
        bs.res[k] = sqrt(q[ND + k]);
        bs.rho[k] = q[ND + k];
        bs.rho_old[k] = 1.0;
        bs.alpha[k] = 1.0;
        bs.omega[k] = 1.0;
        bs.iters[k] = 0;
        bs.sconv[k] = 0;
        bs.conv[k] = !(bs.res[k] > bs.tol[k]);
        bs.active[k] = !bs.conv[k];
        if (bs.res[k] != bs.res[k]) { bs.active[k] = 0; atomicOr(g.status, PISO_ERR_NAN); }
        bs.any |= bs.active[k];
      }
      bs.first = 1;
    }
    __syncthreads();
  }

  // ------------------------------------------------------------------------
  // predictor solve: BiCGStab (van der Vorst) on C u* = b, the d components
  // share C and run with their own scalars; converged components freeze.
  // ------------------------------------------------------------------------
  int cur = 0;
  while (bs.any && bs.it < o.adv_maxit) {
    // BA: p = r + beta (p - omega v) (on the fly at the stencil), v = C p
    {
      Acc<real> a[ND];
#pragma unroll
      for (int k = 0; k < ND; k++) a[k].zero();
      real beta[ND], om[ND];
      int act[ND];
#pragma unroll
      for (int k = 0; k < ND; k++) {
        act[k] = bs.active[k];
        beta[k] = bs.first ? real(0) : (real)((bs.rho[k] / bs.rho_old[k]) * (bs.alpha[k] / bs.omega[k]));
        om[k] = (real)bs.omega[k];
      }
      const int first = bs.first;
      const real* pold = A.pv[cur ^ 1];
      const real* vold = A.vv[cur ^ 1];
      real* pnew = A.pv[cur];
      real* vnew = A.vv[cur];
      for_cells([&](const Cell& c) {
        const int32_t P = c.i;
        const real diag = A.Cdiag[P];
        real off[2 * ND];
#pragma unroll
        for (int s = 0; s < NSD; s++) off[s] = A.Coff[(size_t)s * N + P];
#pragma unroll
        for (int k = 0; k < ND; k++) {
          if (!act[k]) continue;
          const size_t o_ = (size_t)k * N;
          auto pn = [&](int32_t Q) -> real {
            const real rq = A.r[o_ + Q];
            return first ? rq : rq + beta[k] * (pold[o_ + Q] - om[k] * vold[o_ + Q]);
          };
          const real pP = pn(P);
          real v = diag * pP;
#pragma unroll
          for (int s = 0; s < NSD; s++)
            if (c.nb[s] >= 0) v += off[s] * pn(c.nb[s]);
          pnew[o_ + P] = pP;
          vnew[o_ + P] = v;
          a[k].add_prod(A.rhat[o_ + P], v);
        }
      });
      publish<real, ND>(g, a);
      if (!group_sync(g)) return;
      double q[ND];
      gather<ND>(g, q);
      if (threadIdx.x == 0) {
        bs.it++;
        for (int k = 0; k < ND; k++) {
          if (!bs.active[k]) continue;
          bs.iters[k]++;
          if (q[k] == 0.0 || q[k] != q[k]) {
            bs.active[k] = 0;
            atomicOr(g.status, q[k] == 0.0 ? PISO_ERR_BREAKDOWN : PISO_ERR_NAN);
            continue;
          }
          bs.alpha[k] = bs.rho[k] / q[k];
        }
      }
      __syncthreads();
    }
    // BB: s = r - alpha v (on the fly at the stencil), t = C s
    {
      Acc<real> a[3 * ND];
#pragma unroll
      for (int k = 0; k < 3 * ND; k++) a[k].zero();
      real al[ND];
      int act[ND];
#pragma unroll
      for (int k = 0; k < ND; k++) {
        act[k] = bs.active[k];
        al[k] = (real)bs.alpha[k];
      }
      const real* vnew = A.vv[cur];
      for_cells([&](const Cell& c) {
        const int32_t P = c.i;
        const real diag = A.Cdiag[P];
        real off[2 * ND];
#pragma unroll
        for (int s = 0; s < NSD; s++) off[s] = A.Coff[(size_t)s * N + P];
#pragma unroll
        for (int k = 0; k < ND; k++) {
          if (!act[k]) continue;
          const size_t o_ = (size_t)k * N;
          auto sv = [&](int32_t Q) -> real { return A.r[o_ + Q] - al[k] * vnew[o_ + Q]; };
          const real sP = sv(P);
          real tt = diag * sP;
#pragma unroll
          for (int s = 0; s < NSD; s++)
            if (c.nb[s] >= 0) tt += off[s] * sv(c.nb[s]);
          A.t[o_ + P] = tt;
          a[k].add_prod(tt, sP);
          a[ND + k].add_prod(tt, tt);
          a[2 * ND + k].add_prod(sP, sP);
        }
      });
      publish<real, 3 * ND>(g, a);
      if (!group_sync(g)) return;
      double q[3 * ND];
      gather<3 * ND>(g, q);
      if (threadIdx.x == 0) {
        for (int k = 0; k < ND; k++) {
          if (!bs.active[k]) continue;
          const double sn = sqrt(q[2 * ND + k]);
          if (!(sn > bs.tol[k])) {
            bs.sconv[k] = 1;
            bs.res[k] = sn;
          } else if (q[ND + k] == 0.0 || q[ND + k] != q[ND + k]) {
            bs.active[k] = 0;
            atomicOr(g.status, q[ND + k] == 0.0 ? PISO_ERR_BREAKDOWN : PISO_ERR_NAN);
          } else {
            bs.omega[k] = q[k] / q[ND + k];
          }
        }
      }
      __syncthreads();
    }
    // BC: x += alpha p + omega s, r = s - omega t
    {
      Acc<real> a[2 * ND];
#pragma unroll
      for (int k = 0; k < 2 * ND; k++) a[k].zero();
      real al[ND], om[ND];
      int act[ND], sc[ND];
#pragma unroll
      for (int k = 0; k < ND; k++) {
        act[k] = bs.active[k];
        sc[k] = bs.sconv[k];
        al[k] = (real)bs.alpha[k];
        om[k] = (real)bs.omega[k];
      }
      const real* pnew = A.pv[cur];
      const real* vnew = A.vv[cur];
      for (int32_t P = lo + threadIdx.x; P < hi; P += blockDim.x) {
#pragma unroll
        for (int k = 0; k < ND; k++) {
          if (!act[k]) continue;
          const size_t o_ = (size_t)k * N;
          const real sP = A.r[o_ + P] - al[k] * vnew[o_ + P];
          if (sc[k]) {
            A.ustar[o_ + P] += al[k] * pnew[o_ + P];
            continue;
          }
          A.ustar[o_ + P] += al[k] * pnew[o_ + P] + om[k] * sP;
          const real r = sP - om[k] * A.t[o_ + P];
          A.r[o_ + P] = r;
          a[k].add_prod(A.rhat[o_ + P], r);
          a[ND + k].add_prod(r, r);
        }
      }
      publish<real, 2 * ND>(g, a);
      if (!group_sync(g)) return;
      double q[2 * ND];
      gather<2 * ND>(g, q);
      if (threadIdx.x == 0) {
        bs.any = 0;
        for (int k = 0; k < ND; k++) {
          if (!bs.active[k]) continue;
          if (bs.sconv[k]) {
            bs.active[k] = 0;
            bs.conv[k] = 1;
            continue;
          }
          bs.res[k] = sqrt(q[ND + k]);
          if (bs.res[k] != bs.res[k]) {
            bs.active[k] = 0;
            atomicOr(g.status, PISO_ERR_NAN);
          } else if (!(bs.res[k] > bs.tol[k])) {
            bs.active[k] = 0;
            bs.conv[k] = 1;
          } else if (q[k] == 0.0) {
            bs.active[k] = 0;
            atomicOr(g.status, PISO_ERR_BREAKDOWN);
          } else {
            bs.rho_old[k] = bs.rho[k];
            bs.rho[k] = q[k];
          }
          bs.any |= bs.active[k];
        }
        bs.first = 0;
      }
      __syncthreads();
    }
    cur ^= 1;
  }
  if (threadIdx.x == 0 && g.rank == 0) {
    int nc = 0;
    for (int k = 0; k < ND; k++) {
      A.istats[k] = bs.iters[k];
      A.dstats[k] = bs.res[k];
      if (!bs.conv[k]) nc = 1;
    }
    if (nc) atomicOr(g.status, PISO_ERR_NOCONV_ADV);
  }

  // ------------------------------------------------------------------------
  // correctors (App. A.1 Eqs. pressureRHS, pressure, correction; App. A.2
  // Eqs. pMatDiscrete, pressureRHSdiscrete, pressureRHSdivDiscrete,
  // velCorrDiscrete)
  // ------------------------------------------------------------------------
  for (int kc = 0; kc < o.n_corr; kc++) {
    const real* uk = (kc == 0) ? A.ustar : A.uc[kc - 1];
    const real* xprev = (kc == 0) ? A.p_in : A.xk[kc - 1];
    real* h = A.h[kc];
    // C1: (kc == 0) pressure matrix from A = diag C; h = A^-1 (rhs0 - H u); Fh = J T . h.
    //     (kc > 0) also finish the previous corrector's mean-free pressure.
    for_cells([&](const Cell& c) {
      const int32_t P = c.i;
      const real aP = A.Cdiag[P];
      if (kc == 0) {
        real pd = 0;
#pragma unroll
        for (int s = 0; s < NSD; s++) {
          const int j = s >> 1;
          const int32_t F = c.nb[s];
          real pf = 0;
          if (F >= 0) pf = real(0.5) * (AL[(size_t)j * N + P] / aP + AL[(size_t)j * N + F] / A.Cdiag[F]);
          pd -= pf;
          if (s & 1) A.Poff[(size_t)j * N + P] = pf;
        }
        A.Pdiag[P] = pd;
      } else {
        A.xk[kc - 1][P] = A.cx[P] - (real)s_mean;
      }
      real hv[ND];
#pragma unroll
      for (int k = 0; k < ND; k++) {
        const real* x = uk + (size_t)k * N;
        real hu = 0;
#pragma unroll
        for (int s = 0; s < NSD; s++)
          if (c.nb[s] >= 0) hu += A.Coff[(size_t)s * N + P] * x[c.nb[s]];
        hv[k] = (A.rhs0[(size_t)k * N + P] - hu) / aP;
        h[(size_t)k * N + P] = hv[k];
      }
#pragma unroll
      for (int j = 0; j < ND; j++) {
        real s = 0;
#pragma unroll
        for (int k = 0; k < ND; k++) s += Tm(j, k, P) * hv[k];
        A.Fh[(size_t)j * N + P] = J[P] * s;
      }
    });
    if (!group_sync(g)) return;
    // C2: b = sum_f N_f mean(J T_j . h) + boundary flux (R6)
    {
      Acc<real> a[1];
      a[0].zero();
      for_cells([&](const Cell& c) {
        const int32_t P = c.i;
        real b = 0;
#pragma unroll
        for (int s = 0; s < NSD; s++) {
          const int j = s >> 1;
          const real n = (s & 1) ? real(1) : real(-1);
          const int32_t F = c.nb[s];
          if (F >= 0) {
            b += n * real(0.5) * (A.Fh[(size_t)j * N + P] + A.Fh[(size_t)j * N + F]);
          } else {
            const int32_t f = -1 - F;
            real tu = 0;
#pragma unroll
            for (int k = 0; k < ND; k++) tu += Tm(j, k, P) * A.bval[(size_t)k * nbf + f];
            b += n * J[P] * tu;
          }
        }
        A.b[P] = b;
        a[0].add(b);
      });
      publish<real, 1>(g, a);
      if (!group_sync(g)) return;
      double q[1];
      gather<1>(g, q);
      if (threadIdx.x == 0) s_mean = q[0] / (double)N;
      __syncthreads();
    }
    // C3: PCG start on -P x = -(b - mean b) (R7), x0 = previous pressure
    {
      Acc<real> a[3];
#pragma unroll
      for (int k = 0; k < 3; k++) a[k].zero();
      const real mb = (real)s_mean;
      for_cells([&](const Cell& c) {
        const int32_t P = c.i;
        const real bp = -(A.b[P] - mb);
        const real pd = A.Pdiag[P];
        real px = pd * xprev[P];
#pragma unroll
        for (int s = 0; s < NSD; s++) {
          const int j = s >> 1;
          const int32_t F = c.nb[s];
          if (F >= 0) {
            const real pf = (s & 1) ? A.Poff[(size_t)j * N + P] : A.Poff[(size_t)j * N + F];
            px += pf * xprev[F];
          }
        }
        const real r = bp + px;          // b' - (-P) x0
        const real z = r / (-pd);
        A.cx[P] = xprev[P];
        A.cr[P] = r;
        A.cz[P] = z;
        a[0].add_prod(bp, bp);
        a[1].add_prod(r, r);
        a[2].add_prod(r, z);
      });
      publish<real, 3>(g, a);
      if (!group_sync(g)) return;
      double q[3];
      gather<3>(g, q);
      if (threadIdx.x == 0) {
        cs.bn = sqrt(q[0]);
        cs.tol = fmax(o.p_rtol * cs.bn, o.atol);
        cs.res = sqrt(q[1]);
        cs.rz = q[2];
        cs.it = 0;
        cs.first = 1;
        cs.active = cs.res > cs.tol;
        if (cs.res != cs.res) { cs.active = 0; atomicOr(g.status, PISO_ERR_NAN); }
      }
      __syncthreads();
    }
    // Jacobi-PCG iterations (two barriers each; d is formed on the fly)
    int cc = 0;
    while (cs.active && cs.it < o.p_maxit) {
      {
        Acc<real> a[1];
        a[0].zero();
        const real beta = cs.first ? real(0) : (real)(cs.rz / cs.rz_old);
        const int first = cs.first;
        const real* dold = A.cd[cc ^ 1];
        real* dnew = A.cd[cc];
        for_cells([&](const Cell& c) {
          const int32_t P = c.i;
          auto dn = [&](int32_t Q) -> real { return first ? A.cz[Q] : A.cz[Q] + beta * dold[Q]; };
          const real dP = dn(P);
          const real pd = A.Pdiag[P];
          real q = -pd * dP;
#pragma unroll
          for (int s = 0; s < NSD; s++) {
            const int j = s >> 1;
            const int32_t F = c.nb[s];
            if (F >= 0) {
              const real pf = (s & 1) ? A.Poff[(size_t)j * N + P] : A.Poff[(size_t)j * N + F];
              q -= pf * dn(F);
            }
          }
          dnew[P] = dP;
          A.cq[P] = q;
          a[0].add_prod(dP, q);
        });
        publish<real, 1>(g, a);
        if (!group_sync(g)) return;
        double q[1];
        gather<1>(g, q);
        if (threadIdx.x == 0) {
          cs.it++;
          if (q[0] == 0.0 || q[0] != q[0]) {
            cs.active = 0;
            atomicOr(g.status, q[0] == 0.0 ? PISO_ERR_BREAKDOWN : PISO_ERR_NAN);
          } else {
            cs.alpha = cs.rz / q[0];
          }
        }
        __syncthreads();
      }
      if (!cs.active) break;
      {
        Acc<real> a[2];
        a[0].zero();
        a[1].zero();
        const real al = (real)cs.alpha;
        const real* dnew = A.cd[cc];
        for (int32_t P = lo + threadIdx.x; P < hi; P += blockDim.x) {
          A.cx[P] += al * dnew[P];
          const real r = A.cr[P] - al * A.cq[P];
          const real z = r / (-A.Pdiag[P]);
          A.cr[P] = r;
          A.cz[P] = z;
          a[0].add_prod(r, r);
          a[1].add_prod(r, z);
        }
        publish<real, 2>(g, a);
        if (!group_sync(g)) return;
        double q[2];
        gather<2>(g, q);
        if (threadIdx.x == 0) {
          cs.res = sqrt(q[0]);
          if (cs.res != cs.res) {
            cs.active = 0;
            atomicOr(g.status, PISO_ERR_NAN);
          } else if (!(cs.res > cs.tol)) {
            cs.active = 0;
          } else {
            cs.rz_old = cs.rz;
            cs.rz = q[1];
            cs.first = 0;
          }
        }
        __syncthreads();
      }
      cc ^= 1;
    }
    if (threadIdx.x == 0 && g.rank == 0) {
      A.istats[4 + kc] = cs.it;
      A.dstats[4 + kc] = cs.res;
      if (cs.res > cs.tol) atomicOr(g.status, PISO_ERR_NOCONV_P);
    }
    // C4: u = h - A^-1 grad x (Eq. velCorrDiscrete, R5); mean of x for R7
    {
      Acc<real> a[1];
      a[0].zero();
      real* uo = (kc == o.n_corr - 1) ? A.u_out : A.uc[kc];
      for_cells([&](const Cell& c) {
        const int32_t P = c.i;
        const real xP = A.cx[P];
        real gp[ND];
#pragma unroll
        for (int k = 0; k < ND; k++) gp[k] = 0;
#pragma unroll
        for (int j = 0; j < ND; j++) {
          const real xp = c.nb[2 * j + 1] >= 0 ? A.cx[c.nb[2 * j + 1]] : xP;
          const real xm = c.nb[2 * j] >= 0 ? A.cx[c.nb[2 * j]] : xP;
          const real d = real(0.5) * (xp - xm);
#pragma unroll
          for (int k = 0; k < ND; k++) gp[k] += Tm(j, k, P) * d;
        }
        const real aP = A.Cdiag[P];
#pragma unroll
        for (int k = 0; k < ND; k++) uo[(size_t)k * N + P] = h[(size_t)k * N + P] - gp[k] / aP;
        a[0].add(xP);
      });
      publish<real, 1>(g, a);
      if (!group_sync(g)) return;
      double q[1];
      gather<1>(g, q);
      if (threadIdx.x == 0) s_mean = q[0] / (double)N;
      __syncthreads();
    }
  }
  // final pressure (mean-free) and the tape record of the last corrector
  {
    const real m = (real)s_mean;
    const int kl = o.n_corr - 1;
    for (int32_t P = lo + threadIdx.x; P < hi; P += blockDim.x) {
      const real x = A.cx[P] - m;
      A.xk[kl][P] = x;
      A.p_out[P] = x;
    }
  }
}

template <typename real, int ND>
__global__ void __launch_bounds__(512, 1) fwd_kernel(const __grid_constant__ FwdLaunch<real> L) {
  __shared__ FwdCall<real> A;
  const int gi = find_group(L.ngroups, L.cta_first);
  copy_to_smem(&A, L.calls ? L.calls + gi : &L.call0);
  __syncthreads();
  Group g;
  g.bar = A.bar;
  g.partials = A.partials;
  g.status = A.status;
  g.ncta = A.ncta;
  g.rank = blockIdx.x - A.cta0;
  g.epoch = 0;
  g.timeout_ns = L.o.timeout_ns;
  fwd_group<real, ND>(A, L.o, g);
}

}  // namespace piso
