// Forward PISO step as one persistent cooperative launch (arXiv:2505.16992,
// Sec. 2.1 and App. A.1-A.3): outflow update, assembly of C = A + H and the
// predictor right-hand side, BiCGStab for the d velocity components sharing
// C, assembly of the pressure matrix P, and n correctors (h, div h,
// Jacobi-CG on -P, velocity correction).  Every phase walks this CTA's cell
// range; phases are separated by the group barrier.
#pragma once
#include "piso_krylov.cuh"
#include "piso_nonortho.cuh"

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
  real* bval_in_rec;         // [d][nbf] boundary values before the outflow update
  double* hdr;               // tape header: dt, nu
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
  real* Pinv;                // [N]    1 / diag(-P)
  real* invA;                // [N]    1 / A
  real* Aw;                  // [d][N] alpha_jj / A
  real* Fh;                  // [d][N] J T . h
  real* b;                   // [N]
  real* cx;                  // [N]
  real* crb[2];              // [N]
  real* cwb[2];              // [N]
  real* csb[2];              // [N]
  real* cp;                  // [N]
  double* x64;               // [N]    refined pressure (FP32 mode)
  real* rin;                 // [N]    refinement residual
  real* ce;                  // [N]    refinement correction
  real* lfa;                 // [N]    y-line preconditioner factors (when p_line)
  real* lfm;
  real* lfc;
  int32_t p_line;            // 1: the pressure CG uses the y-line preconditioner
  IluTab ilu;                // ILU(0) tables of the launch layout (when adv_ilu)
  real* ilud;                // [N]    ILU(0) reciprocal pivots
  int32_t adv_ilu;           // BiCGStab preconditioner: 0 none, 1 ILU(0), 2 ILU(0) after a failed plain solve
                             // (read by the extended instantiation of the kernel only)
  int32_t n_nonortho;        // non-orthogonal mesh: solves per predictor / pressure solve (0: orthogonal)
  real* bx;                  // [N]    pressure right-hand side with the cross terms (non-orthogonal)
  real* pn;                  // [N]    tape: p^n (non-orthogonal meshes; null otherwise)
  real* xit[4];              // [3][N] tape: per corrector the pressure iterates 1..n-1 of its non-orthogonal loop
  real* usit;                // [3][d][N] tape: the predictor iterates 1..n-1
  // group control
  uint32_t* bar;
  double* partials;
  int32_t* status;
  int32_t* istats;           // [16]
  double* dstats;            // [16]
  int32_t cta0, ncta;
};

// Launch arguments.  One domain: its call travels by value in call0.  A batch:
// calls[] and cta_first[] live in device memory (CTA c belongs to group g when
// cta_first[g] <= c < cta_first[g+1]).
template <typename CallT>
struct Launch {
  int32_t ngroups;
  SolverOpts o;
  const int32_t* cta_first;
  const CallT* calls;
  CallT call0;
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

template <typename real, int ND, int MODE>
__device__ void fwd_group(const FwdCall<real>& A, const SolverOpts& o, Group& g) {
  __shared__ DomStatic D;
  __shared__ BiState bs;
  __shared__ CgState cs;
  __shared__ RefState rs;
  __shared__ double s_scale, s_mean;
  __shared__ float s_scale_f, s_mean_f, s_cf[3];
  __shared__ double s_cd[3];
  copy_to_smem(&D, A.dom);
  if (threadIdx.x == 0) {           // step constants in both precisions (no per-thread FP64 work)
    s_cd[0] = A.dt;
    s_cd[1] = A.nu;
    s_cd[2] = 1.0 / A.dt;
    for (int q = 0; q < 3; q++) s_cf[q] = (float)s_cd[q];
  }
  __syncthreads();
  const int32_t N = D.N;
  const int32_t lo = (int32_t)(((int64_t)N * g.rank) / g.ncta);
  const int32_t hi = (int32_t)(((int64_t)N * (g.rank + 1)) / g.ncta);
  const bool lines = A.p_line && o.line_cap > 0;
  LinePre<real> LP{};
  if (lines) LP = line_setup<real, ND>(D, g, o, A.lfa, A.lfm, A.lfc);
  // neighbour frames only in the extended instantiation (a compile-time null
  // elsewhere, so the plain Krylov rows carry no frame test)
  const int16_t* frames = nullptr;
  if constexpr (MODE == 2) frames = D.nbfr;
  const Ctx<real, ND> X{D, g, lo, hi, N, build_nbt<ND>(D, lo, hi, o.nbt_cap), lines ? &LP : nullptr, frames};
  const real* J = reinterpret_cast<const real*>(D.J);
  const real* T = reinterpret_cast<const real*>(D.T);
  const real* AL = reinterpret_cast<const real*>(D.alpha);
  const int NSD = 2 * ND;
  const real dt = pick<real>(s_cd[0], s_cf[0]), nu = pick<real>(s_cd[1], s_cf[1]);
  const real inv_dt = pick<real>(s_cd[2], s_cf[2]);
  auto Tm = [&](int j, int k, int32_t i) -> real { return T[(size_t)(j * ND + k) * N + i]; };
  const int32_t nbf = D.nbf;
  const int32_t flo = (int32_t)(((int64_t)nbf * g.rank) / g.ncta);
  const int32_t fhi = (int32_t)(((int64_t)nbf * (g.rank + 1)) / g.ncta);

  // F0: advective outflow update (App. A.3, Eq. advOut, reading R10) and the
  // inflow/outflow flux balance.
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
      for (int k = 0; k < ND; k++) {
        ub[k] = A.bval[(size_t)k * nbf + f];
        A.bval_in_rec[(size_t)k * nbf + f] = ub[k];
      }
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
    if (!reduce_sync<real, 2>(g, a, [&](const double* q) {
          s_scale = (q[1] != 0.0) ? q[0] / q[1] : 1.0;
          s_scale_f = (float)s_scale;
        }))
      return;
    const real sc = pick<real>(s_scale, s_scale_f);
    for (int32_t f = flo + threadIdx.x; f < fhi; f += blockDim.x)
      if (D.bf_out[f]) {
#pragma unroll
        for (int k = 0; k < ND; k++) A.bval[(size_t)k * nbf + f] *= sc;
      }
  }
  for (int32_t f = flo + threadIdx.x; f < fhi; f += blockDim.x)
#pragma unroll
    for (int k = 0; k < ND; k++) {
      const real v = A.bval[(size_t)k * nbf + f];
      A.bval_rec[(size_t)k * nbf + f] = v;
      if (D.n_out == 0) A.bval_in_rec[(size_t)k * nbf + f] = v;
    }
  if (threadIdx.x == 0 && g.rank == 0) {
    A.hdr[0] = A.dt;
    A.hdr[1] = A.nu;
    A.hdr[2] = (MODE == 2) ? (double)A.n_nonortho : 0.0;
  }

  // F1: contravariant flux U^j = J T_j . u^n (App. A.2) and the tape copy of u^n
  X.own([&](int32_t P) {
    real u[ND];
#pragma unroll
    for (int k = 0; k < ND; k++) {
      u[k] = A.u_in[(size_t)k * N + P];
      A.un[(size_t)k * N + P] = u[k];
    }
    if constexpr (MODE == 2) {
      if (A.n_nonortho && A.pn) A.pn[P] = A.p_in[P];   // the first corrector's starting pressure
    }
#pragma unroll
    for (int j = 0; j < ND; j++) {
      real s = 0;
#pragma unroll
      for (int k = 0; k < ND; k++) s += Tm(j, k, P) * u[k];
      A.U[(size_t)j * N + P] = J[P] * s;
    }
  });
  if (!plain_sync(g)) return;

  // F2: assemble C and the right-hand sides (Eqs. advMatDiscrete,
  // difMatDiscrete, velRHSdiscrete; per-unit-volume rows, R1), predictor
  // rhs b = rhs0 (- grad p^n when enabled, R4), BiCGStab start r = b - C u^n.
  {
    Acc<real> a[2 * ND];
#pragma unroll
    for (int k = 0; k < 2 * ND; k++) a[k].zero();
    X.cells([&](const Cell& c) {
      const int32_t P = c.i;
      const real invJ = real(1) / J[P];
      real diag = inv_dt;
      real rhs[ND];
      real off[2 * ND];
#pragma unroll
      for (int k = 0; k < ND; k++)
        rhs[k] = A.u_in[(size_t)k * N + P] * inv_dt + (A.S ? A.S[(size_t)k * N + P] : real(0));
      // non-orthogonal meshes: the direct-neighbour cross entries of Eq.
      // difNonOrthoMatDiscrete (C gets -(nu/J_P) W_k (q_{k+} - q_{k-}) / 2, a
      // Dirichlet ghost 2 u_b - q_P putting its -q_P part on the diagonal and
      // its 2 u_b part on rhs0, beside the tangential fluxes through P's
      // Dirichlet faces)
      real Wx[ND], bx[ND];
#pragma unroll
      for (int k = 0; k < ND; k++) Wx[k] = bx[k] = 0;
      bool nonortho = false;
      if constexpr (MODE == 2) {
        nonortho = A.n_nonortho > 0;
        if (nonortho) cross_w<real, ND>(c, reinterpret_cast<const real*>(D.Gx), N, Wx, D.nbfr);
      }
#pragma unroll
      for (int s = 0; s < NSD; s++) {
        const int j = s >> 1;
        const real n = (s & 1) ? real(1) : real(-1);
        const int32_t F = c.nb[s];
        const real aP = AL[(size_t)j * N + P];
        if (F >= 0) {
          int jF = j;
          real eF = real(1);
          if constexpr (MODE == 2) {
            // a joint with exchanged or reversed axes: the neighbour's flux and
            // alpha are its own axis's, in its orientation
            if (D.nbfr) {
              const int code = D.nbfr[(size_t)s * N + P];
              jF = fr_ax(code, j);
              if (fr_neg(code, j)) eF = real(-1);
            }
          }
          const real Uf = real(0.5) * (A.U[(size_t)j * N + P] + eF * A.U[(size_t)jF * N + F]);
          const real Df = nu * real(0.5) * (aP + AL[(size_t)jF * N + F]);
          off[s] = (real(0.5) * n * Uf - Df) * invJ;
          diag += (real(0.5) * n * Uf + Df) * invJ;
          if constexpr (MODE == 2) {
            if (nonortho) off[s] -= n * real(0.5) * Wx[j] * nu * invJ;
          }
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
          if constexpr (MODE == 2) {
            if (nonortho) {
              diag += n * real(0.5) * Wx[j] * nu * invJ;
#pragma unroll
              for (int k = 0; k < ND; k++) bx[k] += n * Wx[j] * ub[k];
              cross_bface<real, ND>(D, c, s, A.bval, nbf, reinterpret_cast<const real*>(D.Gx), bx);
            }
          }
        }
        A.Coff[(size_t)s * N + P] = off[s];
      }
      if constexpr (MODE == 2) {
        if (nonortho)
#pragma unroll
          for (int k = 0; k < ND; k++) rhs[k] += nu * invJ * bx[k];
      }
      A.Cdiag[P] = diag;
      const real ia = real(1) / diag;
      A.invA[P] = ia;
#pragma unroll
      for (int j = 0; j < ND; j++) A.Aw[(size_t)j * N + P] = AL[(size_t)j * N + P] * ia;
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
      real xv[ND];
#pragma unroll
      for (int k = 0; k < ND; k++) xv[k] = 0;
      if constexpr (MODE == 2) {
        if (A.n_nonortho)
          cross_visc<real, ND>(D, c, A.u_in, A.bval, nbf, reinterpret_cast<const real*>(D.Gx), J, nu, xv);
      }
#pragma unroll
      for (int k = 0; k < ND; k++) {
        A.rhs0[(size_t)k * N + P] = rhs[k];
        const real b = rhs[k] - gp[k] + xv[k];
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
    if (!reduce_sync<real, 2 * ND>(g, a, [&](const double* q) {
          bicg_start<ND>(bs, q, o.adv_rtol, o.atol, g.status);
        }))
      return;
  }

  // predictor solve (App. A.5: BiCGStab, ILU(0)-preconditioned throughout or
  // only after the plain solve failed)
  int ilu_used = 0;
  int adv_prev[3] = {0, 0, 0};   // thread 0: iterations of earlier non-orthogonal predictor solves
  if constexpr (MODE >= 1) {
    // the level tables exist only when the ILU(0) preconditioner is on (the extended
    // instantiation also runs non-orthogonal meshes without it)
    const IluPre<real> IP = A.adv_ilu ? ilu_setup<real>(A.ilu, A.ilud, g.rank) : IluPre<real>{};
    const IluSmem<real, ND> IS = ilu_smem<real, ND>(X, o);
    bool factored = false;
    auto solve = [&]() -> bool {
      if (A.adv_ilu == 1) {
        if (!factored) ilu_factor<real, ND>(X, IP, A.Cdiag, A.Coff, IS);
        factored = true;
        ilu_used = 1;
        return bicgstab_ilu<real, ND, false>(X, IP, bs, o.adv_maxit, A.Cdiag, A.Coff, A.ustar, A.r, A.rhat, A.pv[0],
                                             A.vv[0], A.pv[1], A.vv[1], A.t, IS);
      }
      if (!bicgstab<real, ND, false>(X, bs, o.adv_maxit, A.Cdiag, A.Coff, A.ustar, A.r, A.rhat, A.pv, A.vv, A.t))
        return false;
      // bs is the same in every CTA (each runs the same updates on the same
      // reduced values), so all CTAs take the same branch
      if (A.adv_ilu == 2 && !bicg_all_conv<ND>(bs)) {
        bicg_restart<real, ND>(X, bs, A.ustar, A.u_in, A.r, A.rhat, o.adv_rtol, o.atol, g.status);
        if (!factored) ilu_factor<real, ND>(X, IP, A.Cdiag, A.Coff, IS);
        factored = true;
        ilu_used = 2;
        return bicgstab_ilu<real, ND, false>(X, IP, bs, o.adv_maxit, A.Cdiag, A.Coff, A.ustar, A.r, A.rhat, A.pv[0],
                                             A.vv[0], A.pv[1], A.vv[1], A.t, IS);
      }
      return true;
    };
    if (!solve()) return;
    // non-orthogonal corrector steps: the cross terms of the latest u*, then
    // the predictor solve again from it
    if constexpr (MODE == 2)
    for (int m = 1; m < A.n_nonortho; m++) {
      if (threadIdx.x == 0)
        for (int k = 0; k < ND; k++) adv_prev[k] += bs.iters[k] + bs.iters_prev[k];
      Acc<real> a[2 * ND];
#pragma unroll
      for (int k = 0; k < 2 * ND; k++) a[k].zero();
      X.cells([&](const Cell& c) {
        const int32_t P = c.i;
        real xv[ND];
        cross_visc<real, ND>(D, c, A.ustar, A.bval, nbf, reinterpret_cast<const real*>(D.Gx), J, nu, xv);
        if (A.usit)   // tape: the predictor iterate u*_m for the adjoint
#pragma unroll
          for (int k = 0; k < ND; k++)
            A.usit[((size_t)(m - 1) * ND + k) * N + P] = A.ustar[(size_t)k * N + P];
#pragma unroll
        for (int k = 0; k < ND; k++) {
          const real b = A.rhs0[(size_t)k * N + P] + xv[k];
          const real* x = A.ustar + (size_t)k * N;
          real cx = A.Cdiag[P] * x[P];
#pragma unroll
          for (int s = 0; s < NSD; s++)
            if (c.nb[s] >= 0) cx += A.Coff[(size_t)s * N + P] * x[c.nb[s]];
          const real r = b - cx;
          A.r[(size_t)k * N + P] = r;
          A.rhat[(size_t)k * N + P] = r;
          a[k].add_prod(b, b);
          a[ND + k].add_prod(r, r);
        }
      });
      if (!reduce_sync<real, 2 * ND>(g, a, [&](const double* q) { bicg_start<ND>(bs, q, o.adv_rtol, o.atol, g.status); }))
        return;
      if (!solve()) return;
    }
  } else {
    if (!bicgstab<real, ND, false>(X, bs, o.adv_maxit, A.Cdiag, A.Coff, A.ustar, A.r, A.rhat, A.pv, A.vv, A.t))
      return;
  }
  if (threadIdx.x == 0 && g.rank == 0) {
    int nc = 0;
    for (int k = 0; k < ND; k++) {
      A.istats[k] = adv_prev[k] + bs.iters[k] + bs.iters_prev[k];
      A.dstats[k] = sqrt(bs.res2[k]);
      if (!bs.conv[k]) nc = 1;
    }
    A.istats[3] = ilu_used;
    if (nc) atomicOr(g.status, PISO_ERR_NOCONV_ADV);
    if (bs.err) atomicOr(g.status, bs.err);
  }

  // correctors (App. A.1 Eqs. pressureRHS, pressure, correction; App. A.2
  // Eqs. pMatDiscrete, pressureRHSdiscrete, pressureRHSdivDiscrete,
  // velCorrDiscrete)
  for (int kc = 0; kc < o.n_corr; kc++) {
    const real* uk = (kc == 0) ? A.ustar : A.uc[kc - 1];
    const real* xprev = (kc == 0) ? A.p_in : A.xk[kc - 1];
    real* h = A.h[kc];
    // C1: (kc == 0) pressure matrix from A = diag C; h = A^-1 (rhs0 - H u),
    // Fh = J T . h; (kc > 0) also the previous corrector's mean-free pressure.
    X.cells([&](const Cell& c) {
      const int32_t P = c.i;
      const real ia = A.invA[P];
      if (kc == 0) {
        real pd = 0;
#pragma unroll
        for (int s = 0; s < NSD; s++) {
          const int j = s >> 1;
          const int32_t F = c.nb[s];
          real pf = 0;
          int jF = j;
          if constexpr (MODE == 2) {
            if (D.nbfr && F >= 0) jF = fr_ax(D.nbfr[(size_t)s * N + P], j);
          }
          if (F >= 0) pf = real(0.5) * (A.Aw[(size_t)j * N + P] + A.Aw[(size_t)jF * N + F]);
          pd -= pf;
          if constexpr (MODE == 2) {
            if (D.nbfr) A.Poff[(size_t)s * N + P] = pf;        // every face kept by its cell
            else if (s & 1) A.Poff[(size_t)j * N + P] = pf;
          } else {
            if (s & 1) A.Poff[(size_t)j * N + P] = pf;
          }
        }
        A.Pdiag[P] = pd;
        A.Pinv[P] = real(1) / (-pd);
      } else {
        A.xk[kc - 1][P] = A.cx[P] - pick<real>(s_mean, s_mean_f);
      }
      real hv[ND], xv[ND];
#pragma unroll
      for (int k = 0; k < ND; k++) xv[k] = 0;
      if constexpr (MODE == 2) {
        if (A.n_nonortho)
          cross_visc<real, ND>(D, c, uk, A.bval, nbf, reinterpret_cast<const real*>(D.Gx), J, nu, xv);
      }
#pragma unroll
      for (int k = 0; k < ND; k++) {
        const real* x = uk + (size_t)k * N;
        real hu = 0;
#pragma unroll
        for (int s = 0; s < NSD; s++)
          if (c.nb[s] >= 0) hu += A.Coff[(size_t)s * N + P] * x[c.nb[s]];
        hv[k] = (A.rhs0[(size_t)k * N + P] + xv[k] - hu) * ia;
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
    if (!plain_sync(g)) return;
    // C2: b = sum_f N_f mean(J T_j . h) + boundary flux (R6); mean of b (R7).
    // Once per step (P is complete after the barrier) the line factors.
    if (kc == 0 && X.lp) line_factor<real, ND>(D, *X.lp, N, A.Pdiag, A.Poff);
    {
      Acc<real> a[1];
      a[0].zero();
      X.cells([&](const Cell& c) {
        const int32_t P = c.i;
        real b = 0;
#pragma unroll
        for (int s = 0; s < NSD; s++) {
          const int j = s >> 1;
          const real n = (s & 1) ? real(1) : real(-1);
          const int32_t F = c.nb[s];
          if (F >= 0) {
            int jF = j;
            real eF = real(1);
            if constexpr (MODE == 2) {
              if (D.nbfr) {
                const int code = D.nbfr[(size_t)s * N + P];
                jF = fr_ax(code, j);
                if (fr_neg(code, j)) eF = real(-1);
              }
            }
            b += n * real(0.5) * (A.Fh[(size_t)j * N + P] + eF * A.Fh[(size_t)jF * N + F]);
          } else {
            const int32_t f = -1 - F;
            real tu = 0;
#pragma unroll
            for (int k = 0; k < ND; k++) tu += Tm(j, k, P) * A.bval[(size_t)k * nbf + f];
            b += n * J[P] * tu;
          }
        }
        A.b[P] = b;
        A.cx[P] = xprev[P];
        a[0].add(b);
      });
      if (!reduce_sync<real, 1>(g, a, [&](const double* q) {
            s_mean = q[0] / (double)N;
            s_mean_f = (float)s_mean;
          }))
        return;
    }
    // pressure solve (App. A.5: CG; Chronopoulos-Gear form), in the FP32 mode
    // refined against an FP64 residual when asked or when the CG stalls
    bool nonortho = false;
    if constexpr (MODE == 2) nonortho = A.n_nonortho > 0;
    if (!nonortho) {
      if (!pressure_solve<real, ND>(X, cs, rs, o, A.Pdiag, A.Pinv, A.Poff, A.b, s_mean, A.cx, A.x64, A.rin, A.ce,
                                    A.crb, A.cwb, A.csb, A.cp, A.istats, A.dstats, kc))
        return;
    } else {
      // non-orthogonal corrector steps: b minus the cross terms of the
      // previous pressure iterate (cx: the previous corrector's, then each
      // solve's), then the pressure solve again from it
      int p_tot = 0;
      for (int m = 0; m < A.n_nonortho; m++) {
        Acc<real> a[1];
        a[0].zero();
        X.cells([&](const Cell& c) {
          const int32_t P = c.i;
          const real bm = A.b[P] - cross_pres<real, ND>(D, c, A.cx, A.invA, reinterpret_cast<const real*>(D.Gx));
          A.bx[P] = bm;
          if (m > 0 && A.xit[kc]) A.xit[kc][(size_t)(m - 1) * N + P] = A.cx[P];   // tape: the iterate x_m
          a[0].add(bm);
        });
        if (!reduce_sync<real, 1>(g, a, [&](const double* q) {
              s_mean = q[0] / (double)N;
              s_mean_f = (float)s_mean;
            }))
          return;
        if (!pressure_solve<real, ND>(X, cs, rs, o, A.Pdiag, A.Pinv, A.Poff, A.bx, s_mean, A.cx, A.x64, A.rin,
                                      A.ce, A.crb, A.cwb, A.csb, A.cp, A.istats, A.dstats, kc))
          return;
        if (threadIdx.x == 0 && g.rank == 0) p_tot += A.istats[4 + kc];
      }
      if (threadIdx.x == 0 && g.rank == 0) A.istats[4 + kc] = p_tot;
    }
    // C4: u = h - A^-1 grad x (Eq. velCorrDiscrete, R5); mean of x (R7)
    {
      Acc<real> a[1];
      a[0].zero();
      real* uo = (kc == o.n_corr - 1) ? A.u_out : A.uc[kc];
      X.cells([&](const Cell& c) {
        const int32_t P = c.i;
        const real xP = A.cx[P];
        real gp[ND];
#pragma unroll
        for (int k = 0; k < ND; k++) gp[k] = 0;
#pragma unroll
        for (int j = 0; j < ND; j++) {
          const real xp = c.nb[2 * j + 1] >= 0 ? A.cx[c.nb[2 * j + 1]] : xP;
          const real xm = c.nb[2 * j] >= 0 ? A.cx[c.nb[2 * j]] : xP;
          const real dd = real(0.5) * (xp - xm);
#pragma unroll
          for (int k = 0; k < ND; k++) gp[k] += Tm(j, k, P) * dd;
        }
        const real ia = A.invA[P];
#pragma unroll
        for (int k = 0; k < ND; k++) uo[(size_t)k * N + P] = h[(size_t)k * N + P] - gp[k] * ia;
        a[0].add(xP);
      });
      if (!reduce_sync<real, 1>(g, a, [&](const double* q) {
            s_mean = q[0] / (double)N;
            s_mean_f = (float)s_mean;
          }))
        return;
    }
  }
  // final pressure (mean-free) and the tape record of the last corrector
  {
    const real m = pick<real>(s_mean, s_mean_f);
    const int kl = o.n_corr - 1;
    X.own([&](int32_t P) {
      const real x = A.cx[P] - m;
      A.xk[kl][P] = x;
      A.p_out[P] = x;
    });
  }
}

// MODE 0: the plain step; 1: with the ILU(0)-preconditioned predictor (App.
// A.5); 2: also the non-orthogonal cross terms (App. A.2).  Each mode carries
// only its own code, so a feature's register pressure cannot reach the modes
// without it.
template <typename real, int ND, int MAXT, int MODE>
__global__ void __launch_bounds__(MAXT, 1) fwd_kernel(const __grid_constant__ Launch<FwdCall<real>> L) {
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
  g.withhold = (L.o.withhold_cta == g.rank) ? 1 : 0;
  g.trace = L.o.trace;
  fwd_group<real, ND, MODE>(A, L.o, g);
}

}  // namespace piso
