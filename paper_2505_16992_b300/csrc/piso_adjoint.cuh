// Adjoint of one PISO step as one persistent cooperative launch
// (arXiv:2505.16992, Sec. 2.3 and App. A.4).  The linear solves are
// differentiated by transposed solves (A^T db = dx, dA = -db (x) x on the
// sparsity pattern; App. A.5: the forward solvers with the transposed matrix),
// every other operation by its exact transpose, read off the implemented
// forward operator (reading R9), including the boundary values and the
// advective outflow update.  The gradient paths of Sec. 2.4 (Eq. jnone) are
// selectable: a path left out makes its solve's output a constant of the
// backward pass, so the transposed solve and the terms it feeds are skipped.
// On non-orthogonal meshes (MODE 2, App. A.2 "Non-Orthogonal Grids" with App.
// A.4) the non-orthogonal corrector loops run in reverse: per pressure solve
// the transposed solve, then the transpose of the pressure cross terms in the
// previous iterate and in A (the starting pressure, p^n for the first
// corrector, receives a gradient); per predictor solve the transposed solve,
// then the transpose of the deferred viscous cross terms in the previous
// iterate and the boundary values; the direct-neighbour cross entries of C add
// their viscosity and boundary-value derivatives.
#pragma once
#include "piso_forward.cuh"

namespace piso {

template <typename real>
struct AdjCall {
  const DomStatic* dom;
  // tape (recorded by the forward step)
  const double* hdr;         // [dt, nu]
  const real* Cdiag;
  const real* Coff;
  const real* ustar;
  const real* h[4];
  const real* xk[4];
  const real* uc[4];
  const real* bval;          // [d][nbf] boundary values used by the step
  const real* bval_in;       // [d][nbf] boundary values before its outflow update
  const real* un;            // [d][N]   u^n
  // seeds and results
  const real* du_out;        // [d][N]
  const real* dp_out;        // [N] or nullptr
  real* du_in;               // [d][N]
  real* dp_in;               // [N] or nullptr
  real* dS;                  // [d][N] or nullptr
  double* dnu;               // device scalar
  real* gbval;               // [d][nbf] dL/d(boundary values before the outflow update)
  // scratch
  real* Poff;                // [d][N] pressure matrix rebuilt from A
  real* Pdiag;               // [N]
  real* Pinv;                // [N]
  real* gA;                  // [N]       dL/dA, A = diag C
  real* gCoff;               // [2d][N]   dL/d(off-diagonal C)
  real* grhs0;               // [d][N]    dL/d(rhs0)
  real* gw;                  // [d][N]    dL/d(alpha_jj / A)
  real* W;                   // [d][N]    T . (gu / A), later T . z
  real* gg;                  // [d][N]
  real* gu;                  // [d][N]
  real* gx;                  // [N]
  real* z;                   // [d][N]    transposed predictor solve
  real* r;
  real* rhat;
  real* pv[2];
  real* vv[2];
  real* t;
  real* cx;
  real* crb[2];
  real* cwb[2];
  real* csb[2];
  real* cp;
  double* x64;
  real* rin;
  real* ce;
  real* lfa;                 // y-line preconditioner factors (when p_line)
  real* lfm;
  real* lfc;
  int32_t p_line;
  IluTab ilu;                // ILU(0) tables of the launch layout (when adv_ilu)
  real* ilud;                // [N] ILU(0) reciprocal pivots (rebuilt here from the taped C)
  int32_t adv_ilu;           // 0 none, 1 ILU(0), 2 ILU(0) after a failed plain solve
  int32_t n_nonortho;        // non-orthogonal mesh: the domain's n_nonortho (the kernel takes the recorded
                             // step's count from the tape header)
  const real* pn;            // [N] recorded p^n (non-orthogonal meshes)
  const real* xit[4];        // per corrector [3][N]: pressure iterates 1..n-1 of its non-orthogonal loop
  const real* usit;          // [3][d][N]: predictor iterates 1..n-1
  real* gyb;                 // [N]   sum of one corrector's transposed pressure solutions
  real* invA;                // [N]   1 / A (non-orthogonal meshes)
  real* gdk;                 // [d][d][N] sensitivities to the cells' central differences
  uint32_t* bar;
  double* partials;
  int32_t* status;
  int32_t* istats;
  double* dstats;
  int32_t cta0, ncta;
};

template <typename real, int ND, int MODE>
__device__ void adj_group(const AdjCall<real>& A, const SolverOpts& o, Group& g) {
  constexpr bool ILU = MODE >= 1;
  __shared__ DomStatic D;
  __shared__ BiState bs;
  __shared__ CgState cs;
  __shared__ RefState rs;
  __shared__ double s_mean, s_idt;
  __shared__ float s_idt_f;
  __shared__ double s_ymean;          // sum over correctors of mean(y) (the transposed pressure solutions)
  __shared__ double s_ob[4];          // outflow adjoint: scale, dL/dscale, q_in, q_out
  copy_to_smem(&D, A.dom);
  if (threadIdx.x == 0) {
    s_idt = 1.0 / A.hdr[0];
    s_idt_f = (float)s_idt;
    s_ymean = 0.0;
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
  const int32_t nbf = D.nbf;
  auto Tm = [&](int j, int k, int32_t i) -> real { return T[(size_t)(j * ND + k) * N + i]; };
  const real inv_dt = pick<real>(s_idt, s_idt_f);
  const int K = o.n_corr;
  const bool path_adv = (o.grad_paths & 1) != 0;   // Sec. 2.4: gradient through the advection solve
  const bool path_p = (o.grad_paths & 2) != 0;     // Sec. 2.4: gradient through the pressure solves
  int NO = 0;                                       // non-orthogonal corrector steps of the recorded step
  if constexpr (MODE == 2) NO = (int)A.hdr[2];
  const real* Gx = reinterpret_cast<const real*>(D.Gx);
  const real nu_s = pick<real>(A.hdr[1], (float)A.hdr[1]);
  Acc<real> anu[1];                                 // dL/dnu, summed over the phases
  anu[0].zero();

  // (G^T W)_P for the cell-centred central gradient with the R5 boundary rule:
  // G(p)_Q = sum_j T_Q,j . 0.5 (p_{nb(Q,+j)} - p_{nb(Q,-j)}), p_Q standing in
  // for a missing neighbour.  W_j(Q) = T_Q,j . g_Q is precomputed.
  auto gradT = [&](const Cell& c, const real* Wv) -> real {
    real acc = 0;
    if constexpr (MODE == 2) {
      if (D.nbfr) {
        // a neighbour R reads this cell in its own gradient along R's axis of
        // its side facing this cell, with +1/2 (this cell its + neighbour) or
        // -1/2; a missing neighbour stands for this cell itself
#pragma unroll
        for (int s = 0; s < 2 * ND; s++) {
          const int32_t R = c.nb[s];
          if (R >= 0) {
            const int rs = fr_ret(D.nbfr[(size_t)s * N + c.i], s);
            const real w = Wv[(size_t)(rs >> 1) * N + R];
            acc += (rs & 1) ? real(0.5) * w : real(-0.5) * w;
          } else {
            const real w = Wv[(size_t)(s >> 1) * N + c.i];
            acc += (s & 1) ? real(0.5) * w : real(-0.5) * w;
          }
        }
        return acc;
      }
    }
#pragma unroll
    for (int j = 0; j < ND; j++) {
      const real* w = Wv + (size_t)j * N;
      const int32_t Fm = c.nb[2 * j], Fp = c.nb[2 * j + 1];
      const real wP = w[c.i];
      acc += real(0.5) * ((Fm >= 0 ? w[Fm] : real(0)) + (Fp < 0 ? wP : real(0)) - (Fp >= 0 ? w[Fp] : real(0)) -
                          (Fm < 0 ? wP : real(0)));
    }
    return acc;
  };

  for (int k = K - 1; k >= 0; k--) {
    const real* xk = A.xk[k];
    const real* hk = A.h[k];
    const real* uin = (k == 0) ? A.ustar : A.uc[k - 1];
    const real* gsrc = (k == K - 1) ? A.du_out : A.gu;
    // R0: W = T . (gu / A); dL/dA from u = h - A^-1 grad x.  On the first
    // pass also rebuild P from A (Eq. pMatDiscrete) and clear the accumulators.
    X.cells([&](const Cell& c) {
      const int32_t P = c.i;
      const real aP = A.Cdiag[P];
      if (k == K - 1) {
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
          if (F >= 0) pf = real(0.5) * (AL[(size_t)j * N + P] / aP + AL[(size_t)jF * N + F] / A.Cdiag[F]);
          pd -= pf;
          if constexpr (MODE == 2) {
            if (D.nbfr) A.Poff[(size_t)s * N + P] = pf;        // every face kept by its cell
            else if (s & 1) A.Poff[(size_t)j * N + P] = pf;
          } else {
            if (s & 1) A.Poff[(size_t)j * N + P] = pf;
          }
          A.gCoff[(size_t)s * N + P] = 0;
        }
        A.Pdiag[P] = pd;
        A.Pinv[P] = real(1) / (-pd);
        if constexpr (MODE == 2) {
          if (NO) A.invA[P] = real(1) / aP;
        }
#pragma unroll
        for (int s = 0; s < NSD; s++)
          if (c.nb[s] < 0)
#pragma unroll
            for (int i = 0; i < ND; i++) A.gbval[(size_t)i * nbf + (-1 - c.nb[s])] = 0;
#pragma unroll
        for (int i = 0; i < ND; i++) {
          A.grhs0[(size_t)i * N + P] = 0;
          A.gw[(size_t)i * N + P] = 0;
        }
      }
      real gu[ND], gp[ND];
#pragma unroll
      for (int i = 0; i < ND; i++) {
        gu[i] = gsrc[(size_t)i * N + P];
        gp[i] = 0;
      }
      const real xP = xk[P];
#pragma unroll
      for (int j = 0; j < ND; j++) {
        const real xp = c.nb[2 * j + 1] >= 0 ? xk[c.nb[2 * j + 1]] : xP;
        const real xm = c.nb[2 * j] >= 0 ? xk[c.nb[2 * j]] : xP;
        const real dd = real(0.5) * (xp - xm);
        real w = 0;
#pragma unroll
        for (int i = 0; i < ND; i++) {
          gp[i] += Tm(j, i, P) * dd;
          w += Tm(j, i, P) * gu[i];
        }
        A.W[(size_t)j * N + P] = w / aP;
      }
      real ga = 0;
#pragma unroll
      for (int i = 0; i < ND; i++) ga += gu[i] * gp[i];
      ga /= aP * aP;
      A.gA[P] = (k == K - 1) ? ga : A.gA[P] + ga;
    });
    if (!plain_sync(g)) return;
    // R1: gx = -G^T W (+ dL/dp^{n+1} after the last corrector); its mean.
    // Without the pressure path the pressure is a constant: no gx, no solve.
    if (path_p) {
      if (k == K - 1 && X.lp) line_factor<real, ND>(D, *X.lp, N, A.Pdiag, A.Poff);   // P rebuilt in R0
      Acc<real> a[1];
      a[0].zero();
      X.cells([&](const Cell& c) {
        real v = -gradT(c, A.W);
        if (k == K - 1 && A.dp_out) v += A.dp_out[c.i];
        if constexpr (MODE == 2) {
          // dL/d(this corrector's final pressure) through the next corrector's
          // starting pressure (its pressure cross terms)
          if (NO && k < K - 1) v += A.gx[c.i];
        }
        A.gx[c.i] = v;
        A.cx[c.i] = real(0);
        a[0].add(v);
      });
      if (!reduce_sync<real, 1>(g, a, [&](const double* q) { s_mean = q[0] / (double)N; })) return;
    }
    // transposed pressure solve: P y = gx - mean (P is symmetric)
    if (path_p && NO == 0 &&
        !pressure_solve<real, ND>(X, cs, rs, o, A.Pdiag, A.Pinv, A.Poff, A.gx, s_mean, A.cx, A.x64, A.rin, A.ce,
                                  A.crb, A.cwb, A.csb, A.cp, A.istats, A.dstats, k))
      return;
    if constexpr (MODE == 2) {
      // non-orthogonal corrector steps in reverse: x_m = P^+ (b - Y(x_{m-1}; A)),
      // m = NO..1, x_0 the corrector's starting pressure; y_m = P^+ (dL/dx_m) feeds
      // dP (through d(alpha/A)), the divergence (sum of the y_m) and, through
      // -Y^T y_m, dL/dx_{m-1} and dL/dA
      if (path_p && NO) {
        int p_tot = 0;
        for (int m = NO; m >= 1; m--) {
          if (!pressure_solve<real, ND>(X, cs, rs, o, A.Pdiag, A.Pinv, A.Poff, A.gx, s_mean, A.cx, A.x64, A.rin,
                                        A.ce, A.crb, A.cwb, A.csb, A.cp, A.istats, A.dstats, k))
            return;
          if (threadIdx.x == 0 && g.rank == 0) p_tot += A.istats[4 + k];
          const real* xm = (m == NO) ? xk : A.xit[k] + (size_t)(m - 1) * N;
          const real* xm1 = (m == 1) ? (k == 0 ? A.pn : A.xk[k - 1]) : A.xit[k] + (size_t)(m - 2) * N;
          X.cells([&](const Cell& c) {
            const int32_t P = c.i;
            const real yP = A.cx[P];
#pragma unroll
            for (int j = 0; j < ND; j++) {
              real gwj = 0;
#pragma unroll
              for (int e = 0; e < 2; e++) {
                const int32_t F = c.nb[2 * j + e];
                if (F >= 0) gwj += real(0.5) * (yP - A.cx[F]) * (xm[P] - xm[F]);
              }
              A.gw[(size_t)j * N + P] += gwj;
            }
            A.gyb[P] = (m == NO ? real(0) : A.gyb[P]) + yP;
            A.gA[P] += cross_pres_T1<real, ND>(D, c, A.cx, real(-1), xm1, A.invA, Gx, A.gdk);
          });
          if (!plain_sync(g)) return;
          Acc<real> a1[1];
          a1[0].zero();
          X.cells([&](const Cell& c) {
            const real v = cross_diff_T2<real, ND, false>(c, A.gdk, N, nullptr, D.nbfr);
            A.gx[c.i] = v;
            A.cx[c.i] = real(0);
            a1[0].add(v);
          });
          if (!reduce_sync<real, 1>(g, a1, [&](const double* q) { s_mean = q[0] / (double)N; })) return;
        }
        if (threadIdx.x == 0 && g.rank == 0) A.istats[4 + k] = p_tot;
      }
    }
    // R3: dP = -y (x) x on the pattern -> d(alpha/A); h_bar = gu + div^T y;
    //     gg = h_bar / A; dL/dA and dL/drhs0 from h = A^-1 (rhs0 - H u);
    //     boundary values: b has the flux N_b J_P T_j . u_b (R6), so
    //     dL/du_b += N_b J_P T_j (y_P - mean y) (the mean is subtracted at the end)
    Acc<real> ay[1];
    ay[0].zero();
    const real* ysrc = A.cx;      // the transposed pressure solution (the sum of them, MODE 2)
    bool gw_here = true;
    if constexpr (MODE == 2) {
      if (NO) {
        ysrc = A.gyb;
        gw_here = false;          // dP was taken per solve above
      }
    }
    X.cells([&](const Cell& c) {
      const int32_t P = c.i;
      const real yP = path_p ? ysrc[P] : real(0), xP = path_p ? xk[P] : real(0);
      if (path_p) {
        ay[0].add(yP);
#pragma unroll
        for (int s = 0; s < NSD; s++) {
          if (c.nb[s] >= 0) continue;
          const int j = s >> 1;
          const real nJy = ((s & 1) ? real(1) : real(-1)) * J[P] * yP;
          const int32_t f = -1 - c.nb[s];
#pragma unroll
          for (int i = 0; i < ND; i++) A.gbval[(size_t)i * nbf + f] += nJy * Tm(j, i, P);
        }
      }
      const real aP = A.Cdiag[P];
      real Fb[ND];
#pragma unroll
      for (int j = 0; j < ND; j++) Fb[j] = 0;
      if (path_p) {
#pragma unroll
        for (int j = 0; j < ND; j++) {
          real gwj = 0, fb = 0;
#pragma unroll
          for (int e = 0; e < 2; e++) {
            const int s = 2 * j + e;
            const int32_t F = c.nb[s];
            if (F < 0) continue;
            const real n = e ? real(1) : real(-1);
            const real dy = yP - ysrc[F];
            if (gw_here) gwj += real(0.5) * dy * (xP - xk[F]);
            fb += real(0.5) * n * dy;
          }
          if (gw_here) A.gw[(size_t)j * N + P] += gwj;
          Fb[j] = fb * J[P];
        }
      }
      real ga = 0;
#pragma unroll
      for (int i = 0; i < ND; i++) {
        real hb = gsrc[(size_t)i * N + P];
#pragma unroll
        for (int j = 0; j < ND; j++) hb += Tm(j, i, P) * Fb[j];
        const real ggi = hb / aP;
        A.gg[(size_t)i * N + P] = ggi;
        ga += hb * hk[(size_t)i * N + P];
        A.grhs0[(size_t)i * N + P] += ggi;
      }
      A.gA[P] -= ga / aP;
    });
    if (!reduce_sync<real, 1>(g, ay, [&](const double* q) { s_ymean += q[0] / (double)N; })) return;
    // R4: gu_in = -H^T gg; dL/dH = -gg (x) u_in on the pattern
    X.cells([&](const Cell& c) {
      const int32_t P = c.i;
      real ggP[ND];
#pragma unroll
      for (int i = 0; i < ND; i++) ggP[i] = A.gg[(size_t)i * N + P];
#pragma unroll
      for (int s = 0; s < NSD; s++) {
        const int32_t F = c.nb[s];
        if (F < 0) continue;
        real acc = 0;
#pragma unroll
        for (int i = 0; i < ND; i++) acc += ggP[i] * uin[(size_t)i * N + F];
        A.gCoff[(size_t)s * N + P] -= acc;
      }
#pragma unroll
      for (int i = 0; i < ND; i++) {
        real v = 0;
#pragma unroll
        for (int s = 0; s < NSD; s++) {
          const int32_t F = c.nb[s];
          int rs = s ^ 1;      // the neighbour's side facing this cell
          if constexpr (MODE == 2) {
            if (D.nbfr) rs = fr_ret(D.nbfr[(size_t)s * N + P], s);
          }
          if (F >= 0) v += A.Coff[(size_t)rs * N + F] * A.gg[(size_t)i * N + F];
        }
        A.gu[(size_t)i * N + P] = -v;
      }
      if constexpr (MODE == 2) {
        // h carries the deferred viscous cross terms of its input velocity:
        // their transpose (phase 1) and their viscosity derivative
        if (NO) {
          cross_visc_T1<real, ND>(c, A.gg, Gx, J, nu_s, N, A.gdk, D.nbfr);
          real xv[ND];
          cross_visc<real, ND>(D, c, uin, A.bval, nbf, Gx, J, real(1), xv);
#pragma unroll
          for (int i = 0; i < ND; i++) anu[0].add_prod(ggP[i], xv[i]);
        }
      }
    });
    if (!plain_sync(g)) return;
    if constexpr (MODE == 2) {
      if (NO) {
        X.cells([&](const Cell& c) {
#pragma unroll
          for (int i = 0; i < ND; i++)
            A.gu[(size_t)i * N + c.i] +=
                cross_diff_T2<real, ND, true>(c, A.gdk + (size_t)i * ND * N, N, A.gbval + (size_t)i * nbf, D.nbfr);
        });
        if (!plain_sync(g)) return;
      }
    }
  }

  // R5: dL/dA from the pressure matrix (w = alpha / A); start the transposed
  // predictor solve C^T z = gu with z0 = 0.
  {
    Acc<real> a[2 * ND];
#pragma unroll
    for (int k = 0; k < 2 * ND; k++) a[k].zero();
    X.own([&](int32_t P) {
      const real aP = A.Cdiag[P];
      real s = 0;
#pragma unroll
      for (int j = 0; j < ND; j++) s += A.gw[(size_t)j * N + P] * AL[(size_t)j * N + P];
      A.gA[P] -= s / (aP * aP);
#pragma unroll
      if (path_adv) {
#pragma unroll
        for (int i = 0; i < ND; i++) {
          const real b = A.gu[(size_t)i * N + P];
          A.z[(size_t)i * N + P] = 0;
          A.r[(size_t)i * N + P] = b;
          A.rhat[(size_t)i * N + P] = b;
          a[i].add_prod(b, b);
          a[ND + i].add_prod(b, b);
        }
      }
    });
    // without the advection path u* is a constant: z = 0 and no solve
    if (path_adv &&
        !reduce_sync<real, 2 * ND>(g, a, [&](const double* q) { bicg_start<ND>(bs, q, o.adv_rtol, o.atol, g.status); }))
      return;
  }
  // the transposed solve with the preconditioning of the forward one: the
  // factors of C^T are the transposed factors of C (same pivots).  On
  // non-orthogonal meshes the predictor's corrector steps run in reverse:
  // u*_m = C^-1 (rhs0 + X(u*_{m-1})), m = NO..1, u*_0 = u^n; z_m = C^-T dL/du*_m
  // feeds dC, rhs0 and, through X^T z_m, dL/du*_{m-1} and the boundary values.
  int ilu_used = 0;
  int adv_tot[3] = {0, 0, 0};
  if (path_adv) {
    IluPre<real> IP{};
    IluSmem<real, ND> IS{};
    if constexpr (ILU) {
      // the level tables exist only when the ILU(0) preconditioner is on
      if (A.adv_ilu) IP = ilu_setup<real>(A.ilu, A.ilud, g.rank);
      IS = ilu_smem<real, ND>(X, o);
    }
    bool factored = false;
    auto solveT = [&]() -> bool {
      if constexpr (ILU) {
        if (A.adv_ilu == 1) {
          if (!factored) ilu_factor<real, ND>(X, IP, A.Cdiag, A.Coff, IS);
          factored = true;
          ilu_used = 1;
          return bicgstab_ilu<real, ND, true>(X, IP, bs, o.adv_maxit, A.Cdiag, A.Coff, A.z, A.r, A.rhat, A.pv[0],
                                              A.vv[0], A.pv[1], A.vv[1], A.t, IS);
        }
        if (!bicgstab<real, ND, true>(X, bs, o.adv_maxit, A.Cdiag, A.Coff, A.z, A.r, A.rhat, A.pv, A.vv, A.t))
          return false;
        if (A.adv_ilu == 2 && !bicg_all_conv<ND>(bs)) {
          bicg_restart<real, ND>(X, bs, A.z, static_cast<const real*>(nullptr), A.r, A.rhat, o.adv_rtol, o.atol,
                                 g.status);
          if (!factored) ilu_factor<real, ND>(X, IP, A.Cdiag, A.Coff, IS);
          factored = true;
          ilu_used = 2;
          return bicgstab_ilu<real, ND, true>(X, IP, bs, o.adv_maxit, A.Cdiag, A.Coff, A.z, A.r, A.rhat, A.pv[0],
                                              A.vv[0], A.pv[1], A.vv[1], A.t, IS);
        }
        return true;
      } else {
        return bicgstab<real, ND, true>(X, bs, o.adv_maxit, A.Cdiag, A.Coff, A.z, A.r, A.rhat, A.pv, A.vv, A.t);
      }
    };
    for (int m = NO > 0 ? NO : 1; m >= 1; m--) {
      if (!solveT()) return;
      if (threadIdx.x == 0)
        for (int q = 0; q < ND; q++) adv_tot[q] += bs.iters[q] + bs.iters_prev[q];
      if constexpr (MODE == 2) {
        if (NO) {
          const real* usm = (m == NO) ? A.ustar : A.usit + (size_t)(m - 1) * ND * N;
          const real* usm1 = (m == 1) ? A.un : A.usit + (size_t)(m - 2) * ND * N;
          // dC = -z (x) u*_m on the pattern, dL/drhs0 += z, X^T z (phase 1)
          X.cells([&](const Cell& c) {
            const int32_t P = c.i;
            real zP[ND];
            real ga = 0;
#pragma unroll
            for (int i = 0; i < ND; i++) {
              zP[i] = A.z[(size_t)i * N + P];
              ga += zP[i] * usm[(size_t)i * N + P];
              A.grhs0[(size_t)i * N + P] += zP[i];
            }
            A.gA[P] -= ga;
#pragma unroll
            for (int s = 0; s < NSD; s++) {
              const int32_t F = c.nb[s];
              if (F < 0) continue;
              real acc = 0;
#pragma unroll
              for (int i = 0; i < ND; i++) acc += zP[i] * usm[(size_t)i * N + F];
              A.gCoff[(size_t)s * N + P] -= acc;
            }
            cross_visc_T1<real, ND>(c, A.z, Gx, J, nu_s, N, A.gdk, D.nbfr);
            real xv[ND];
            cross_visc<real, ND>(D, c, usm1, A.bval, nbf, Gx, J, real(1), xv);
#pragma unroll
            for (int i = 0; i < ND; i++) anu[0].add_prod(zP[i], xv[i]);
          });
          if (!plain_sync(g)) return;
          // X^T z (phase 2): dL/du*_{m-1}; the next transposed solve starts from it
          Acc<real> a[2 * ND];
#pragma unroll
          for (int q = 0; q < 2 * ND; q++) a[q].zero();
          X.cells([&](const Cell& c) {
            const int32_t P = c.i;
#pragma unroll
            for (int i = 0; i < ND; i++) {
              const real gm = cross_diff_T2<real, ND, true>(c, A.gdk + (size_t)i * ND * N, N, A.gbval + (size_t)i * nbf, D.nbfr);
              if (m > 1) {
                A.z[(size_t)i * N + P] = 0;
                A.r[(size_t)i * N + P] = gm;
                A.rhat[(size_t)i * N + P] = gm;
                a[i].add_prod(gm, gm);
                a[ND + i].add_prod(gm, gm);
              } else {
                A.gu[(size_t)i * N + P] = gm;    // dL/du^n through the predictor's cross terms
              }
            }
          });
          if (m > 1) {
            if (!reduce_sync<real, 2 * ND>(g, a,
                                           [&](const double* q) { bicg_start<ND>(bs, q, o.adv_rtol, o.atol, g.status); }))
              return;
          } else if (!plain_sync(g)) {
            return;
          }
        }
      }
    }
  }
  if (path_adv && threadIdx.x == 0 && g.rank == 0) {
    int nc = 0;
    for (int k = 0; k < ND; k++) {
      A.istats[k] = adv_tot[k];
      A.dstats[k] = sqrt(bs.res2[k]);
      if (!bs.conv[k]) nc = 1;
    }
    A.istats[3] = ilu_used;
    if (nc) atomicOr(g.status, PISO_ERR_NOCONV_ADV);
    if (bs.err) atomicOr(g.status, bs.err);
  }
  // R6: dC = -z (x) u* on the pattern; dL/drhs0 += z; outputs dS and the
  //     1/dt part of du_in; W = T . z for the predictor pressure gradient
  bool z_here = path_adv;     // MODE 2 took the z terms per predictor solve above
  if constexpr (MODE == 2) {
    if (NO) z_here = false;
  }
  X.cells([&](const Cell& c) {
    const int32_t P = c.i;
    real zP[ND];
#pragma unroll
    for (int i = 0; i < ND; i++) zP[i] = 0;
    if (z_here) {
      real ga = 0;
#pragma unroll
      for (int i = 0; i < ND; i++) {
        zP[i] = A.z[(size_t)i * N + P];
        ga += zP[i] * A.ustar[(size_t)i * N + P];
      }
      A.gA[P] -= ga;
#pragma unroll
      for (int s = 0; s < NSD; s++) {
        const int32_t F = c.nb[s];
        if (F < 0) continue;
        real acc = 0;
#pragma unroll
        for (int i = 0; i < ND; i++) acc += zP[i] * A.ustar[(size_t)i * N + F];
        A.gCoff[(size_t)s * N + P] -= acc;
      }
    }
    real gr[ND];
#pragma unroll
    for (int i = 0; i < ND; i++) {
      gr[i] = A.grhs0[(size_t)i * N + P] + zP[i];
      A.du_in[(size_t)i * N + P] = gr[i] * inv_dt;
      if (A.dS) A.dS[(size_t)i * N + P] = gr[i];
    }
    if constexpr (MODE == 2) {
      if (NO) {
        // dL/du^n through the predictor's cross terms; rhs0 holds the
        // constant part of the direct-neighbour cross entries (linear in nu
        // and in the boundary values)
        if (path_adv)
#pragma unroll
          for (int i = 0; i < ND; i++) A.du_in[(size_t)i * N + P] += A.gu[(size_t)i * N + P];
        real W[ND], x0[ND];
        cross_w<real, ND>(c, Gx, N, W, D.nbfr);
        cross_const<real, ND>(D, c, W, A.bval, nbf, Gx, J, x0);
#pragma unroll
        for (int i = 0; i < ND; i++) anu[0].add_prod(gr[i], x0[i]);
        cross_const_T<real, ND>(D, c, W, A.grhs0, Gx, J, nu_s, nbf, A.gbval);
      }
    }
    if (o.pred_grad_p) {
#pragma unroll
      for (int j = 0; j < ND; j++) {
        real w = 0;
#pragma unroll
        for (int i = 0; i < ND; i++) w += Tm(j, i, P) * zP[i];
        A.W[(size_t)j * N + P] = w;
      }
    }
    // nu from the Dirichlet terms of the right-hand side (Eq. velRHSdiscrete),
    // and the boundary values there: rhs0_i += u_b,i (2 alpha nu / J - N_f T_j . u_b)
    const real invJ = real(1) / J[P];
#pragma unroll
    for (int s = 0; s < NSD; s++) {
      const int32_t F = c.nb[s];
      if (F >= 0) continue;
      const int32_t f = -1 - F;
      const int j = s >> 1;
      const real n = (s & 1) ? real(1) : real(-1);
      const real two_a = real(2) * AL[(size_t)j * N + P] * invJ;
      real acc = 0, tu = 0;
      real ub[ND];
#pragma unroll
      for (int i = 0; i < ND; i++) {
        ub[i] = A.bval[(size_t)i * nbf + f];
        acc += gr[i] * ub[i];
        tu += Tm(j, i, P) * ub[i];
      }
      anu[0].add(acc * two_a);
      const real a = two_a * nu_s - n * tu;
#pragma unroll
      for (int i = 0; i < ND; i++) A.gbval[(size_t)i * nbf + f] += gr[i] * a - n * Tm(j, i, P) * acc;
    }
  });
  if (!plain_sync(g)) return;
  // R7: dp_in = -G^T (T . z) (reading R4 option); assembly adjoint: the face
  //     fluxes U_f = (U_P + U_F)/2, U = J T . u^n, and the nu terms of C
  X.cells([&](const Cell& c) {
    const int32_t P = c.i;
    const real invJ = real(1) / J[P];
    const real gAP = A.gA[P];
    if constexpr (MODE == 2) {
      if (NO) {
        // dL/dp^n through the first corrector's pressure cross terms; nu
        // through the direct-neighbour cross entries of C (C = ... - nu M1)
        if (A.dp_in) A.dp_in[P] = path_p ? A.gx[P] : real(0);
        real W[ND];
        cross_w<real, ND>(c, Gx, N, W, D.nbfr);
        real m = 0;
#pragma unroll
        for (int s = 0; s < NSD; s++) {
          const real n = (s & 1) ? real(1) : real(-1);
          const real h = n * real(0.5) * W[s >> 1] * invJ;
          if (c.nb[s] >= 0) m += A.gCoff[(size_t)s * N + P] * h;
          else m -= gAP * h;
        }
        anu[0].add(-m);
      } else if (A.dp_in) {
        A.dp_in[P] = o.pred_grad_p ? -gradT(c, A.W) : real(0);
      }
    } else if (A.dp_in) {
      A.dp_in[P] = o.pred_grad_p ? -gradT(c, A.W) : real(0);
    }
    real Ub[ND];
#pragma unroll
    for (int j = 0; j < ND; j++) Ub[j] = 0;
#pragma unroll
    for (int s = 0; s < NSD; s++) {
      const int j = s >> 1;
      const real n = (s & 1) ? real(1) : real(-1);
      const int32_t F = c.nb[s];
      const real aP = AL[(size_t)j * N + P];
      if (F >= 0) {
        const real gcP = A.gCoff[(size_t)s * N + P];
        int rs = s ^ 1;        // the neighbour's side facing this cell
        if constexpr (MODE == 2) {
          if (D.nbfr) rs = fr_ret(D.nbfr[(size_t)s * N + P], s);
        }
        const real gcF = A.gCoff[(size_t)rs * N + F];
        const real own = real(0.5) * n * (gcP + gAP) * invJ;
        const real nbr = -real(0.5) * n * (gcF + A.gA[F]) / J[F];
        Ub[j] += real(0.5) * (own + nbr);
        int jF = j;
        if constexpr (MODE == 2) {
          if (D.nbfr) jF = fr_ax(D.nbfr[(size_t)s * N + P], j);
        }
        const real Df = real(0.5) * (aP + AL[(size_t)jF * N + F]);
        anu[0].add((gAP - gcP) * Df * invJ);
      } else {
        anu[0].add(gAP * real(2) * aP * invJ);
      }
    }
#pragma unroll
    for (int i = 0; i < ND; i++) {
      real v = 0;
#pragma unroll
      for (int j = 0; j < ND; j++) v += Tm(j, i, P) * Ub[j];
      A.du_in[(size_t)i * N + P] += J[P] * v;
    }
  });
  if (!reduce_sync<real, 1>(g, anu, [&](const double* q) {
        if (g.rank == 0) *A.dnu = q[0];
      }))
    return;
  if (nbf == 0) return;
  // Boundary values: finish dL/du_b (the divergence term used y, not y - mean y)
  // and, with advective outflow faces, differentiate the outflow update
  // (App. A.3, Eq. advOut, R10): b1 = (1 - f) b + f u_P on outflow faces,
  // q_out = sum N J T_j . b1 over them, q_in = -sum N J T_j . b over the other
  // Dirichlet faces, u_b = (q_in / q_out) b1 on outflow faces.
  const real ym = pick<real>(s_ymean, (float)s_ymean);
  const real* um = reinterpret_cast<const real*>(D.bf_um);
  const real dt_s = pick<real>(A.hdr[0], (float)A.hdr[0]);
  auto face_fac = [&](int32_t P, int j, int32_t f) -> real {
    real tu = 0;
#pragma unroll
    for (int i = 0; i < ND; i++) tu += Tm(j, i, P) * um[(size_t)i * nbf + f];
    const real cc = real(2) * dt_s * fabs(tu);
    return cc / (real(1) + cc);
  };
  if (D.n_out > 0) {
    Acc<real> ao[3];   // dL/dscale, q_in, q_out
    ao[0].zero();
    ao[1].zero();
    ao[2].zero();
    X.cells([&](const Cell& c) {
      const int32_t P = c.i;
#pragma unroll
      for (int s = 0; s < NSD; s++) {
        if (c.nb[s] >= 0) continue;
        const int j = s >> 1;
        const real nJ = ((s & 1) ? real(1) : real(-1)) * J[P];
        const int32_t f = -1 - c.nb[s];
        real flux_in = 0, flux_b1 = 0, gdot = 0;
#pragma unroll
        for (int i = 0; i < ND; i++) {
          real* gb = A.gbval + (size_t)i * nbf + f;
          *gb -= ym * nJ * Tm(j, i, P);
          const real b = A.bval_in[(size_t)i * nbf + f];
          flux_in += nJ * Tm(j, i, P) * b;
          if (D.bf_out[f]) {
            const real fac = face_fac(P, j, f);
            const real b1 = b - fac * (b - A.un[(size_t)i * N + P]);
            flux_b1 += nJ * Tm(j, i, P) * b1;
            gdot += *gb * b1;
          }
        }
        if (D.bf_out[f]) {
          ao[0].add(gdot);
          ao[2].add(flux_b1);
        } else {
          ao[1].add(-flux_in);
        }
      }
    });
    if (!reduce_sync<real, 3>(g, ao, [&](const double* q) {
          const bool scaled = q[2] != 0.0;
          s_ob[0] = scaled ? q[1] / q[2] : 1.0;
          s_ob[1] = scaled ? q[0] : 0.0;   // no rescaling when q_out = 0
          s_ob[2] = q[1];
          s_ob[3] = scaled ? q[2] : 1.0;
        }))
      return;
    const real sc = pick<real>(s_ob[0], (float)s_ob[0]);
    const real c_out = pick<real>(-s_ob[1] * s_ob[2] / (s_ob[3] * s_ob[3]), (float)(-s_ob[1] * s_ob[2] / (s_ob[3] * s_ob[3])));
    const real c_in = pick<real>(-s_ob[1] / s_ob[3], (float)(-s_ob[1] / s_ob[3]));
    X.cells([&](const Cell& c) {
      const int32_t P = c.i;
#pragma unroll
      for (int s = 0; s < NSD; s++) {
        if (c.nb[s] >= 0) continue;
        const int j = s >> 1;
        const real nJ = ((s & 1) ? real(1) : real(-1)) * J[P];
        const int32_t f = -1 - c.nb[s];
        if (D.bf_out[f]) {
          const real fac = face_fac(P, j, f);
#pragma unroll
          for (int i = 0; i < ND; i++) {
            real* gb = A.gbval + (size_t)i * nbf + f;
            const real gb1 = sc * *gb + c_out * nJ * Tm(j, i, P);
            *gb = (real(1) - fac) * gb1;
            A.du_in[(size_t)i * N + P] += fac * gb1;
          }
        } else {
#pragma unroll
          for (int i = 0; i < ND; i++) A.gbval[(size_t)i * nbf + f] += c_in * nJ * Tm(j, i, P);
        }
      }
    });
  } else {
    X.cells([&](const Cell& c) {
      const int32_t P = c.i;
#pragma unroll
      for (int s = 0; s < NSD; s++) {
        if (c.nb[s] >= 0) continue;
        const int j = s >> 1;
        const real nJ = ((s & 1) ? real(1) : real(-1)) * J[P];
        const int32_t f = -1 - c.nb[s];
#pragma unroll
        for (int i = 0; i < ND; i++) A.gbval[(size_t)i * nbf + f] -= ym * nJ * Tm(j, i, P);
      }
    });
  }
}

// MODE 0: the plain step's adjoint; 1: with the ILU(0)-preconditioned
// transposed predictor solve; 2: also the non-orthogonal terms.
template <typename real, int ND, int MAXT, int MODE>
__global__ void __launch_bounds__(MAXT, 1) adj_kernel(const __grid_constant__ Launch<AdjCall<real>> L) {
  __shared__ AdjCall<real> A;
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
  adj_group<real, ND, MODE>(A, L.o, g);
}

}  // namespace piso
