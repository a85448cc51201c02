// Krylov solvers used by the forward and adjoint PISO kernels (arXiv:2505.16992,
// App. A.5: BiCGStab for advection-diffusion, CG for the pressure; Sec. 2.3:
// the adjoint re-uses them with the transposed matrix).  They run inside the
// persistent kernel: every iteration phase walks the CTA's cells and ends in a
// deterministic group reduction.
#pragma once
#include "piso_device.cuh"

namespace piso {

struct SolverOpts {
  int32_t n_corr, pred_grad_p, adv_maxit, p_maxit;
  double adv_rtol, p_rtol, atol;
  uint64_t timeout_ns;
  int32_t nbt_cap;           // cells per CTA the shared neighbour table can hold
  int32_t line_cap;          // reals per staging array of the y-line preconditioner (0: not available)
  int32_t withhold_cta;      // fault injection: group rank that skips its first barrier arrival (-1 off)
  double p_refine_rtol;      // FP32 mode: outer FP64 residual tolerance of the pressure solve (0 = off)
  double p_inner_rtol;       // FP32 mode: inner CG tolerance per refinement round
  int32_t grad_paths;        // adjoint: bit 1 keeps the advection-solve paths, bit 2 the pressure-solve paths
  int32_t ilu_soff;          // byte offset of the ILU(0) sweep area in dynamic shared memory, -1: none
  uint64_t* trace;           // phase-timing ring of PISO_TRACE builds ([PISO_TRACE_LEN][4]), else nullptr
  // plan of the fused y-line CG iteration (cg_pressure_fused), or lf_off == nullptr
  const int32_t* lf_off;     // [ncta + 1] CTA r's local lines are lf_lines[lf_off[r] .. lf_off[r + 1])
  const int32_t* lf_nown;    // [ncta] the first lf_nown[r] of them are its own lines
  const int32_t* lf_lines;   // line ids
  const int16_t* lf_nbs;     // [ncta][2 ND][lf_own_cap] neighbour slots of the own cells
  int32_t lf_own_cap;        // own cells per CTA the plan reserves (own lines x longest line)
  int32_t lf_slot_cap;       // staged cells per CTA (pitch x longest line)
  int32_t lf_bytes;          // bytes of the fused arrays in dynamic shared memory
};

// Fill the CTA's neighbour table (dynamic shared memory) when its cell range
// fits; returns the table or nullptr.
template <int ND>
__device__ __forceinline__ const int32_t* build_nbt(const DomStatic& D, int32_t lo, int32_t hi, int32_t cap) {
  extern __shared__ int32_t s_nbt[];
  const int32_t n = hi - lo;
  if (n > cap) return nullptr;
  for (int32_t l = threadIdx.x; l < n; l += blockDim.x) {
    const Cell c = locate<ND>(D, lo + l);
#pragma unroll
    for (int s = 0; s < 2 * ND; s++) s_nbt[s * n + l] = c.nb[s];
  }
  __syncthreads();
  return s_nbt;
}

// Execution context of one CTA inside its group.  Which cells a thread visits:
//  - with a neighbour table (the CTA's range fits in shared memory): the CTA's
//    contiguous range [lo, hi), thread t taking lo + t, lo + t + T, ...;
//  - without one (large domains): the group's cells interleaved in passes of
//    ncta * T, so CTA r takes [(j ncta + r) T, (j ncta + r + 1) T) on pass j.
//    All CTAs then sweep the same window of the domain at the same time, and
//    the +-y and +-z neighbours a pass reads (one row / one plane away) were
//    read by another CTA of the same or the previous pass: they are L2 hits,
//    whereas contiguous ranges larger than a plane read every z neighbour
//    stream a second time from DRAM.
// Each thread's cell set and visiting order are fixed, so reductions stay
// deterministic, and every loop of a phase (cells, cells_pf, own) uses the
// same partition.
template <typename real, int ND>
struct Ctx {
  const DomStatic& D;   // shared-memory copy
  Group& g;
  int32_t lo, hi, N;
  const int32_t* nbt;   // [2*ND][hi-lo] neighbour table in shared memory, or nullptr
  const LinePre<real>* lp;   // y-line preconditioner of the pressure CG, or nullptr (Jacobi)
  const int16_t* fr;    // neighbour frames [2*ND][N] when some joint exchanges or reverses axes, else nullptr
  // first cell, stride and end of this thread's walk
  __device__ __forceinline__ int32_t first() const {
    return nbt ? lo + (int32_t)threadIdx.x : g.rank * (int32_t)blockDim.x + (int32_t)threadIdx.x;
  }
  __device__ __forceinline__ int32_t stride() const {
    return nbt ? (int32_t)blockDim.x : g.ncta * (int32_t)blockDim.x;
  }
  __device__ __forceinline__ int32_t end() const { return nbt ? hi : N; }
  __device__ __forceinline__ Cell cell(int32_t i) const {
    Cell c;
    if (nbt) {
      const int32_t n = hi - lo, l = i - lo;
      c.i = i;
#pragma unroll
      for (int s = 0; s < 2 * ND; s++) c.nb[s] = nbt[s * n + l];
    } else {
      c = locate<ND>(D, i);
    }
    return c;
  }
  // cells with an L2 prefetch of the cell this thread visits next: when a
  // thread visits more than one cell, the next cell's streams are requested a
  // full visit ahead (memory-level parallelism for the bandwidth-bound sizes)
  template <typename F, typename PF>
  __device__ __forceinline__ void cells_pf(F&& f, PF&& pf) const {
    const int32_t e = end(), st = stride();
    for (int32_t i = first(); i < e; i += st) {
      if (i + st < e) pf(i + st);
      f(cell(i));
    }
  }
  template <typename F>
  __device__ __forceinline__ void cells(F&& f) const {
    const int32_t e = end(), st = stride();
    for (int32_t i = first(); i < e; i += st) f(cell(i));
  }
  template <typename F>
  __device__ __forceinline__ void own(F&& f) const {
    const int32_t e = end(), st = stride();
    for (int32_t i = first(); i < e; i += st) f(i);
  }
};

__device__ __forceinline__ void prefetch_l2(const void* p) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

// Four consecutive cells of one [comp][N] array as one aligned vector access
// (16 bytes in FP32, two 16-byte halves in FP64).
template <typename real>
struct V4 {
  real v[4];
};
__device__ __forceinline__ V4<float> ld4(const float* __restrict__ p) {
  const float4 t = *reinterpret_cast<const float4*>(p);
  return V4<float>{{t.x, t.y, t.z, t.w}};
}
__device__ __forceinline__ V4<double> ld4(const double* __restrict__ p) {
  const double2 a = reinterpret_cast<const double2*>(p)[0], b = reinterpret_cast<const double2*>(p)[1];
  return V4<double>{{a.x, a.y, b.x, b.y}};
}
__device__ __forceinline__ void st4(float* __restrict__ p, const V4<float>& t) {
  *reinterpret_cast<float4*>(p) = make_float4(t.v[0], t.v[1], t.v[2], t.v[3]);
}
__device__ __forceinline__ void st4(double* __restrict__ p, const V4<double>& t) {
  reinterpret_cast<double2*>(p)[0] = make_double2(t.v[0], t.v[1]);
  reinterpret_cast<double2*>(p)[1] = make_double2(t.v[2], t.v[3]);
}
__device__ __forceinline__ bool aligned16(const void* p) { return ((uintptr_t)p & 15) == 0; }

// Row coefficients of C (TR = false) or C^T (TR = true) for cell c:
// (M y)_P = diag * y_P + sum_s cf[s] * y_{nb(P,s)} over inner faces.  The
// entry of C^T on the face to F = nb(P,s) is F's own coefficient on the
// opposite side (gather form, no atomics).
template <typename real, int ND, bool TR>
__device__ __forceinline__ void c_row(const Cell& c, int32_t N, const real* Cdiag, const real* Coff, real& diag,
                                      real (&cf)[2 * ND], const int16_t* fr = nullptr) {
  diag = Cdiag[c.i];
#pragma unroll
  for (int s = 0; s < 2 * ND; s++) {
    const int32_t Q = c.nb[s];
    if (Q >= 0) {
      if (TR) {   // the neighbour's coefficient on its side facing this cell
        const int rs = fr ? fr_ret(fr[(size_t)s * N + c.i], s) : (s ^ 1);
        cf[s] = Coff[(size_t)rs * N + Q];
      } else {
        cf[s] = Coff[(size_t)s * N + c.i];
      }
    } else {
      cf[s] = real(0);
    }
  }
}

// Face coefficients of the pressure matrix P for cell c (symmetric: the - face
// of P is the + face of its - neighbour).  Domains with joints that exchange
// or reverse axes (own != nullptr... fr set) keep every cell's 2d face
// coefficients itself ([2d][N]), since a neighbour's face towards the cell
// need not be its + face there.
template <typename real, int ND>
__device__ __forceinline__ void p_row(const Cell& c, int32_t N, const real* Poff, real (&pf)[2 * ND],
                                      const int16_t* fr = nullptr) {
#pragma unroll
  for (int s = 0; s < 2 * ND; s++) {
    const int j = s >> 1;
    const int32_t Q = c.nb[s];
    if (fr) pf[s] = Q >= 0 ? Poff[(size_t)s * N + c.i] : real(0);
    else pf[s] = Q >= 0 ? ((s & 1) ? Poff[(size_t)j * N + c.i] : Poff[(size_t)j * N + Q]) : real(0);
  }
}

// Krylov scalar state, owned by thread 0 and broadcast through shared memory.
// Thread 0 also stores the coefficients the cell loops need in both storage
// precisions (the *_f copies), so no other thread converts or divides in FP64.
struct BiState {
  double rho[3], rho_old[3], alpha[3], omega[3], tol2[3], res2[3];
  double beta_d[3];
  double q0[6];              // ||b||^2 and ||r0||^2 per component (a restart reuses them)
  float beta_f[3], alpha_f[3], omega_f[3];
  int active[3], sconv[3], iters[3], conv[3];
  int iters_prev[3];         // iterations of an earlier, failed attempt (ILU(0) fallback)
  int any, it, first;
  int err;                   // breakdown / NaN bits of the solve, passed to the step status by the caller
};

// Residual replacement period of the pressure CG (0 = off, the default).
// Replacing the recursive residual by b - A x caps the attainable relative
// residual at the accuracy of evaluating b - A x (about eps * ||P|| ||x|| /
// ||b||); measured on the BFS grid in FP64 that floor is ~7e-10, above the
// 1e-12 parity tolerance, so the default keeps the recursive residual.
#ifndef PISO_CG_REPLACE
#define PISO_CG_REPLACE 0
#endif
constexpr int CG_REPLACE = PISO_CG_REPLACE;

struct CgState {
  double gam, delta, alpha, beta, tol2, res2;
  double inv_gam;   // 1 / gamma of the last iteration
  double kappa;     // 1 / (gamma alpha) of the last iteration
  double best;      // smallest ||r||^2 that was a 2x (norm) improvement, and its iteration
  // FP32 mode: the loop's scalar state as float pairs (gamma, 1 / alpha, best,
  // tolerance and residual ||r||^2); res2 is converted back when the loop ends
  f2 fgam, finv_alpha, fbest, ftol2, fres2;
  float alpha_f, beta_f;
  int active, it, first, conv, best_it, stalled;
};

// Thread 0, end of one CG iteration (FP64 mode): convergence, stall and
// breakdown tests on ||r||^2, then cg_coeffs from gamma = (r, u), delta = (w, u).
__device__ __forceinline__ void cg_iter_update(CgState& cs, double gam, double delta, double res2, int stall_window,
                                               int32_t* status);

// Thread 0, end of one CG iteration (FP32 mode), all in float-pair arithmetic
// on the FP32 pipe.  Only ratio-form quantities are kept (gamma / gamma_old,
// gamma / alpha_old, den / gamma), which stay inside the float exponent range
// even when ||r||^2 itself is far below 1e-20 (small adjoint right-hand sides).
__device__ __forceinline__ void cg_iter_update_f2(CgState& cs, f2 gam, f2 delta, f2 res2, int stall_window,
                                                  int32_t* status) {
  cs.it++;
  cs.first = 0;
  cs.fres2 = res2;
  if (res2.hi != res2.hi) {
    cs.active = 0;
    atomicOr(status, PISO_ERR_NAN);
    return;
  }
  if (!f2_gt(res2, cs.ftol2)) {
    cs.active = 0;
    cs.conv = 1;
    return;
  }
  const bool improved = f2_gt(f2{0.25f * cs.fbest.hi, 0.25f * cs.fbest.lo}, res2);
  if (stall_window > 0 && !improved && cs.it - cs.best_it >= stall_window) {
    cs.active = 0;
    cs.stalled = 1;
    return;
  }
  if (improved) {
    cs.fbest = res2;
    cs.best_it = cs.it;
  }
  const f2 beta = f2_div(gam, cs.fgam);
  const f2 den = f2_add(delta, f2_neg(f2_mul(beta, f2_mul(gam, cs.finv_alpha))));
  if (den.hi == 0.f || gam.hi == 0.f || den.hi != den.hi) {
    cs.active = 0;
    atomicOr(status, den.hi != den.hi ? PISO_ERR_NAN : PISO_ERR_BREAKDOWN);
    return;
  }
  const f2 alpha = f2_div(gam, den);
  cs.finv_alpha = f2_div(den, gam);
  cs.fgam = gam;
  cs.alpha_f = alpha.hi;
  cs.beta_f = beta.hi;
}

// FP32 pressure CG: a solve whose best residual norm has not halved for this
// many iterations is stalled (finite-precision plateau near the attainable
// accuracy of FP32 vectors) and is finished by FP64-residual refinement rounds.
constexpr int CG_STALL_WINDOW = 200;

// Thread 0: Chronopoulos–Gear coefficients from gamma = (r, u), delta = (w, u):
// beta = gamma / gamma_old and alpha = gamma / (delta - beta gamma / alpha_old).
// The denominator is formed as delta - gamma^2 kappa with kappa = 1 / (gamma_old
// alpha_old) carried over from the previous iteration, so a single division
// (gamma / den) lies on the critical path of the update that every thread of
// the CTA waits for; 1 / gamma for the next kappa is independent of it.  (A
// dependent FP64 division costs ~600 cycles on this GPU, an FP64 FMA ~64.)
// first: the start of the recurrence (beta = 0, alpha = gamma / delta).
// Returns false on breakdown (den or gamma zero) or NaN, with the status set.
__device__ __forceinline__ bool cg_coeffs(CgState& cs, double gam, double delta, bool first, int32_t* status) {
  const double beta = first ? 0.0 : gam * cs.inv_gam;
  const double den = first ? delta : fma(-gam * gam, cs.kappa, delta);
  if (den == 0.0 || gam == 0.0 || den != den) {
    cs.active = 0;
    atomicOr(status, den != den ? PISO_ERR_NAN : PISO_ERR_BREAKDOWN);
    return false;
  }
  const double alpha = gam / den;
  const double ig = 1.0 / gam;
  cs.kappa = den * ig * ig;
  cs.inv_gam = ig;
  cs.gam = gam;
  cs.delta = delta;
  cs.alpha = alpha;
  cs.beta = beta;
  cs.alpha_f = (float)alpha;
  cs.beta_f = (float)beta;
  return true;
}

// A scalar in the storage precision: the float copy for FP32, the double for FP64.
template <typename real>
__device__ __forceinline__ real pick(double d, float f) {
  if constexpr (sizeof(real) == 4) return f;
  else return d;
}

// Thread 0: BiCGStab beta for the next BA phase, both precisions.
__device__ __forceinline__ void bicg_set_beta(BiState& bs, int k) {
  const double b = bs.first ? 0.0 : (bs.rho[k] / bs.rho_old[k]) * (bs.alpha[k] / bs.omega[k]);
  bs.beta_d[k] = b;
  bs.beta_f[k] = (float)b;
  bs.omega_f[k] = (float)bs.omega[k];
}

// Outer state of the iteratively refined pressure solve.
struct RefState {
  double bn2, res2, tol2, rmean;
  int rounds, conv, inner_it;
};

// Thread 0: BiCGStab start from the reduced ||b||^2 and ||r0||^2 per component.
template <int ND>
__device__ __forceinline__ void bicg_start(BiState& bs, const double* q, double rtol, double atol, int32_t* status) {
  bs.any = 0;
  bs.it = 0;
  bs.first = 1;
  bs.err = 0;
  for (int k = 0; k < 2 * ND; k++) bs.q0[k] = q[k];
  for (int k = 0; k < ND; k++) {
    bs.tol2[k] = fmax(rtol * rtol * q[k], atol * atol);
    bs.res2[k] = q[ND + k];
    bs.rho[k] = q[ND + k];
    bs.rho_old[k] = bs.alpha[k] = bs.omega[k] = 1.0;
    bs.iters[k] = 0;
    bs.iters_prev[k] = 0;
    bs.sconv[k] = 0;
    bs.conv[k] = !(bs.res2[k] > bs.tol2[k]);
    bs.active[k] = !bs.conv[k];
    if (bs.res2[k] != bs.res2[k]) {
      bs.active[k] = 0;
      bs.conv[k] = 0;
      atomicOr(status, PISO_ERR_NAN);
    }
    bs.any |= bs.active[k];
    bicg_set_beta(bs, k);
  }
}

// Thread 0, after the reduction of (rhat, v): alpha per component.
template <int ND>
__device__ __forceinline__ void bicg_update_alpha(BiState& bs, const double* q) {
  bs.it++;
  for (int k = 0; k < ND; k++) {
    if (!bs.active[k]) continue;
    bs.iters[k]++;
    if (q[k] == 0.0 || q[k] != q[k]) {
      bs.active[k] = 0;
      bs.err |= q[k] == 0.0 ? PISO_ERR_BREAKDOWN : PISO_ERR_NAN;
      continue;
    }
    bs.alpha[k] = bs.rho[k] / q[k];
    bs.alpha_f[k] = (float)bs.alpha[k];
  }
}

// Thread 0, after the reduction of (t, s), (t, t), (s, s): the s-convergence
// test, then omega.
template <int ND>
__device__ __forceinline__ void bicg_update_omega(BiState& bs, const double* q) {
  for (int k = 0; k < ND; k++) {
    if (!bs.active[k]) continue;
    if (!(q[2 * ND + k] > bs.tol2[k])) {
      bs.sconv[k] = 1;
      bs.res2[k] = q[2 * ND + k];
    } else if (q[ND + k] == 0.0 || q[ND + k] != q[ND + k]) {
      bs.active[k] = 0;
      bs.err |= q[ND + k] == 0.0 ? PISO_ERR_BREAKDOWN : PISO_ERR_NAN;
    } else {
      bs.omega[k] = q[k] / q[ND + k];
      bs.omega_f[k] = (float)bs.omega[k];
    }
  }
}

// Thread 0, after the reduction of (rhat, r), (r, r): convergence, rho and the
// next beta.
template <int ND>
__device__ __forceinline__ void bicg_update_rho(BiState& bs, const double* q) {
  bs.any = 0;
  for (int k = 0; k < ND; k++) {
    if (!bs.active[k]) continue;
    if (bs.sconv[k]) {
      bs.active[k] = 0;
      bs.conv[k] = 1;
      continue;
    }
    bs.res2[k] = q[ND + k];
    if (bs.res2[k] != bs.res2[k]) {
      bs.active[k] = 0;
      bs.err |= PISO_ERR_NAN;
    } else if (!(bs.res2[k] > bs.tol2[k])) {
      bs.active[k] = 0;
      bs.conv[k] = 1;
    } else if (q[k] == 0.0) {
      bs.active[k] = 0;
      bs.err |= PISO_ERR_BREAKDOWN;
    } else {
      bs.rho_old[k] = bs.rho[k];
      bs.rho[k] = q[k];
    }
    bs.any |= bs.active[k];
  }
  bs.first = 0;
  for (int k = 0; k < ND; k++)
    if (bs.active[k]) bicg_set_beta(bs, k);
}

// Thread 0: every component converged?
template <int ND>
__device__ __forceinline__ bool bicg_all_conv(const BiState& bs) {
  for (int k = 0; k < ND; k++)
    if (!bs.conv[k]) return false;
  return true;
}

// The three cell sweeps of a BiCGStab iteration.  Each array is touched
// through one pointer only (ping-pong buffers), so the pointers are
// __restrict__: after inlining the compiler knows a cell's stores cannot alias
// the next cell's loads, and the 2x unrolled loops keep two cells' loads in
// flight.
// BA: p = r + beta (p - omega v), v = M p (p formed on the fly at the stencil), (rhat, v)
template <typename real, int ND, bool TR>
__device__ __forceinline__ void bicg_sweep_a(const Ctx<real, ND>& X, int first, const int (&act)[ND],
                                             const real (&beta)[ND], const real (&om)[ND],
                                             const real* __restrict__ Cdiag, const real* __restrict__ Coff,
                                             const real* __restrict__ r, const real* __restrict__ pold,
                                             const real* __restrict__ vold, const real* __restrict__ rhat,
                                             real* __restrict__ pnew, real* __restrict__ vnew, Acc<real> (&a)[ND]) {
  const int32_t N = X.N, e = X.end(), st = X.stride();
#pragma unroll 2
  for (int32_t i = X.first(); i < e; i += st) {
    const int32_t nx_ = i + st;
    if (nx_ < e) {
      prefetch_l2(Cdiag + nx_);
#pragma unroll
      for (int s = 0; s < 2 * ND; s++) prefetch_l2(Coff + (size_t)s * N + nx_);
#pragma unroll
      for (int k = 0; k < ND; k++) {
        prefetch_l2(r + (size_t)k * N + nx_);
        prefetch_l2(pold + (size_t)k * N + nx_);
        prefetch_l2(vold + (size_t)k * N + nx_);
        prefetch_l2(rhat + (size_t)k * N + nx_);
      }
    }
    const Cell c = X.cell(i);
    real diag, cf[2 * ND];
    c_row<real, ND, TR>(c, N, Cdiag, Coff, diag, cf, X.fr);
    real pP[ND], v[ND], rh[ND];
#pragma unroll
    for (int k = 0; k < ND; k++) {
      pP[k] = v[k] = rh[k] = real(0);
      if (!act[k]) continue;
      const size_t o_ = (size_t)k * N;
      auto pn = [&](int32_t Q) -> real {
        const real rq = r[o_ + Q];
        return first ? rq : rq + beta[k] * (pold[o_ + Q] - om[k] * vold[o_ + Q]);
      };
      pP[k] = pn(c.i);
      real vv_ = diag * pP[k];
#pragma unroll
      for (int s = 0; s < 2 * ND; s++)
        if (c.nb[s] >= 0) vv_ += cf[s] * pn(c.nb[s]);
      v[k] = vv_;
      rh[k] = rhat[o_ + c.i];
    }
#pragma unroll
    for (int k = 0; k < ND; k++) {
      if (!act[k]) continue;
      const size_t o_ = (size_t)k * N;
      pnew[o_ + c.i] = pP[k];
      vnew[o_ + c.i] = v[k];
      a[k].add_prod(rh[k], v[k]);
    }
  }
}

// BB: s = r - alpha v, t = M s (s formed on the fly), (t, s), (t, t), (s, s)
template <typename real, int ND, bool TR>
__device__ __forceinline__ void bicg_sweep_b(const Ctx<real, ND>& X, const int (&act)[ND], const real (&al)[ND],
                                             const real* __restrict__ Cdiag, const real* __restrict__ Coff,
                                             const real* __restrict__ r, const real* __restrict__ vnew,
                                             real* __restrict__ t, Acc<real> (&a)[3 * ND]) {
  const int32_t N = X.N, e = X.end(), st = X.stride();
#pragma unroll 2
  for (int32_t i = X.first(); i < e; i += st) {
    const int32_t nx_ = i + st;
    if (nx_ < e) {
      prefetch_l2(Cdiag + nx_);
#pragma unroll
      for (int s = 0; s < 2 * ND; s++) prefetch_l2(Coff + (size_t)s * N + nx_);
#pragma unroll
      for (int k = 0; k < ND; k++) {
        prefetch_l2(r + (size_t)k * N + nx_);
        prefetch_l2(vnew + (size_t)k * N + nx_);
      }
    }
    const Cell c = X.cell(i);
    real diag, cf[2 * ND];
    c_row<real, ND, TR>(c, N, Cdiag, Coff, diag, cf, X.fr);
    real sP[ND], tt[ND];
#pragma unroll
    for (int k = 0; k < ND; k++) {
      sP[k] = tt[k] = real(0);
      if (!act[k]) continue;
      const size_t o_ = (size_t)k * N;
      auto sv = [&](int32_t Q) -> real { return r[o_ + Q] - al[k] * vnew[o_ + Q]; };
      sP[k] = sv(c.i);
      real t_ = diag * sP[k];
#pragma unroll
      for (int s = 0; s < 2 * ND; s++)
        if (c.nb[s] >= 0) t_ += cf[s] * sv(c.nb[s]);
      tt[k] = t_;
    }
#pragma unroll
    for (int k = 0; k < ND; k++) {
      if (!act[k]) continue;
      t[(size_t)k * N + c.i] = tt[k];
      a[k].add_prod(tt[k], sP[k]);
      a[ND + k].add_prod(tt[k], tt[k]);
      a[2 * ND + k].add_prod(sP[k], sP[k]);
    }
  }
}

// BC: x += alpha p + omega s, r = s - omega t (own cell only), (rhat, r), (r, r)
template <typename real, int ND>
__device__ __forceinline__ void bicg_sweep_c(const Ctx<real, ND>& X, const int (&act)[ND], const int (&sc)[ND],
                                             const real (&al)[ND], const real (&om)[ND],
                                             const real* __restrict__ pnew, const real* __restrict__ vnew,
                                             const real* __restrict__ t, const real* __restrict__ rhat,
                                             real* __restrict__ x, real* __restrict__ r, Acc<real> (&a)[2 * ND]) {
  const int32_t N = X.N, e = X.end(), st = X.stride();
#pragma unroll 2
  for (int32_t P = X.first(); P < e; P += st) {
    real xn[ND], rr[ND], rh[ND];
#pragma unroll
    for (int k = 0; k < ND; k++) {
      xn[k] = rr[k] = rh[k] = real(0);
      if (!act[k]) continue;
      const size_t o_ = (size_t)k * N;
      const real sP = r[o_ + P] - al[k] * vnew[o_ + P];
      if (sc[k]) {
        xn[k] = x[o_ + P] + al[k] * pnew[o_ + P];
        continue;
      }
      xn[k] = x[o_ + P] + (al[k] * pnew[o_ + P] + om[k] * sP);
      rr[k] = sP - om[k] * t[o_ + P];
      rh[k] = rhat[o_ + P];
    }
#pragma unroll
    for (int k = 0; k < ND; k++) {
      if (!act[k]) continue;
      const size_t o_ = (size_t)k * N;
      x[o_ + P] = xn[k];
      if (sc[k]) continue;
      r[o_ + P] = rr[k];
      a[k].add_prod(rh[k], rr[k]);
      a[ND + k].add_prod(rr[k], rr[k]);
    }
  }
}

// Neighbours of a quad of four cells (cells 4m .. 4m+3 of a DomStatic::vec4
// domain walked in interleaved passes): the cell left of the quad, the cell
// right of it, and per y/z side the first cell of the neighbour quad (or a
// negative boundary-face code: all four cells have a boundary face there).
template <int ND>
struct Quad {
  int32_t i0, nL, nR;
  int32_t nb[2 * ND];
};
template <int ND>
__device__ __forceinline__ Quad<ND> quad_at(const DomStatic& D, int32_t i0) {
  const Cell c = locate<ND>(D, i0);
  const BlockInfo& B = D.blk[c.b];
  Quad<ND> q;
  q.i0 = i0;
  q.nL = c.nb[0];
  q.nR = (c.x + 4 < B.nx) ? i0 + 4 : side_nbr(D, B, i0 + 3, c.x + 3, c.y, c.z, 1);
#pragma unroll
  for (int s = 0; s < 2 * ND; s++) q.nb[s] = c.nb[s];
  return q;
}

// Row coefficients of C (TR = false) or C^T (TR = true) for the four cells of
// a quad, as c_row gives them cell by cell: cf[s].v[k] for side s of cell k
// (zero across a boundary face), diag.v[k].
template <typename real, int ND, bool TR>
__device__ __forceinline__ void c_row4(const Quad<ND>& q, int32_t N, const real* __restrict__ Cdiag,
                                       const real* __restrict__ Coff, V4<real>& diag, V4<real> (&cf)[2 * ND]) {
  const int32_t i0 = q.i0;
  diag = ld4(Cdiag + i0);
  if (!TR) {
#pragma unroll
    for (int s = 0; s < 2 * ND; s++) cf[s] = ld4(Coff + (size_t)s * N + i0);
    if (q.nL < 0) cf[0].v[0] = real(0);
    if (q.nR < 0) cf[1].v[3] = real(0);
#pragma unroll
    for (int s = 2; s < 2 * ND; s++)
      if (q.nb[s] < 0) cf[s] = V4<real>{{real(0), real(0), real(0), real(0)}};
  } else {
    // the neighbour's coefficient on its side facing the cell: -x side of
    // cell k is the +x coefficient of cell k - 1, and so on
    const V4<real> c1 = ld4(Coff + (size_t)1 * N + i0), c0 = ld4(Coff + i0);
    cf[0] = V4<real>{{q.nL >= 0 ? Coff[(size_t)1 * N + q.nL] : real(0), c1.v[0], c1.v[1], c1.v[2]}};
    cf[1] = V4<real>{{c0.v[1], c0.v[2], c0.v[3], q.nR >= 0 ? Coff[q.nR] : real(0)}};
#pragma unroll
    for (int s = 2; s < 2 * ND; s++) {
      const int32_t Q = q.nb[s];
      cf[s] = Q >= 0 ? ld4(Coff + (size_t)(s ^ 1) * N + Q) : V4<real>{{real(0), real(0), real(0), real(0)}};
    }
  }
}

// (M y) on a quad with y formed on the fly by yv(Q) (one cell) and yq(Q0, out)
// (a neighbour quad): diag y_P first, then the sides in order, as the one-cell
// sweeps sum them.
template <typename real, int ND, typename F1, typename F4>
__device__ __forceinline__ void quad_apply(const Quad<ND>& q, const V4<real>& diag, const V4<real> (&cf)[2 * ND],
                                           const real (&yP)[4], F1&& yv, F4&& yq, real (&out)[4]) {
  const real yL = q.nL >= 0 ? yv(q.nL) : real(0), yR = q.nR >= 0 ? yv(q.nR) : real(0);
#pragma unroll
  for (int k = 0; k < 4; k++) {
    real v = diag.v[k] * yP[k];
    v += cf[0].v[k] * (k > 0 ? yP[k - 1] : yL);
    v += cf[1].v[k] * (k < 3 ? yP[k + 1] : yR);
    out[k] = v;
  }
#pragma unroll
  for (int s = 2; s < 2 * ND; s++) {
    if (q.nb[s] < 0) continue;
    real y[4];
    yq(q.nb[s], y);
#pragma unroll
    for (int k = 0; k < 4; k++) out[k] += cf[s].v[k] * y[k];
  }
}

// The BiCGStab sweeps BA, BB, BC with four cells per thread (domains as
// cg_jacobi_sweep4 takes them): every stream one aligned vector access per
// quad, one neighbour lookup per quad; the per-cell arithmetic is that of
// bicg_sweep_a/b/c, only the order of the dot sums changes.
template <typename real, int ND, bool TR>
__device__ __forceinline__ void bicg_sweep_a4(const Ctx<real, ND>& X, int first, const int (&act)[ND],
                                              const real (&beta)[ND], const real (&om)[ND],
                                              const real* __restrict__ Cdiag, const real* __restrict__ Coff,
                                              const real* __restrict__ r, const real* __restrict__ pold,
                                              const real* __restrict__ vold, const real* __restrict__ rhat,
                                              real* __restrict__ pnew, real* __restrict__ vnew, Acc<real> (&a)[ND]) {
  const int32_t N = X.N, nq = N >> 2, st = X.stride();
#pragma unroll 1
  for (int32_t qi = X.first(); qi < nq; qi += st) {
    const Quad<ND> q = quad_at<ND>(X.D, qi << 2);
    const int32_t i0 = q.i0;
    V4<real> diag, cf[2 * ND];
    c_row4<real, ND, TR>(q, N, Cdiag, Coff, diag, cf);
#pragma unroll
    for (int c = 0; c < ND; c++) {
      if (!act[c]) continue;
      const size_t o_ = (size_t)c * N;
      const real be = beta[c], w = om[c];
      auto pn = [&](int32_t Q) -> real {
        const real rq = r[o_ + Q];
        return first ? rq : rq + be * (pold[o_ + Q] - w * vold[o_ + Q]);
      };
      auto pq = [&](int32_t Q0, real (&y)[4]) {
        const V4<real> rq = ld4(r + o_ + Q0);
        V4<real> pq_{}, vq{};
        if (!first) {
          pq_ = ld4(pold + o_ + Q0);
          vq = ld4(vold + o_ + Q0);
        }
#pragma unroll
        for (int k = 0; k < 4; k++) y[k] = first ? rq.v[k] : rq.v[k] + be * (pq_.v[k] - w * vq.v[k]);
      };
      real pP[4], v[4];
      pq(i0, pP);
      quad_apply<real, ND>(q, diag, cf, pP, pn, pq, v);
      st4(pnew + o_ + i0, V4<real>{{pP[0], pP[1], pP[2], pP[3]}});
      st4(vnew + o_ + i0, V4<real>{{v[0], v[1], v[2], v[3]}});
      const V4<real> rh = ld4(rhat + o_ + i0);
#pragma unroll
      for (int k = 0; k < 4; k++) a[c].add_prod(rh.v[k], v[k]);
    }
  }
}

template <typename real, int ND, bool TR>
__device__ __forceinline__ void bicg_sweep_b4(const Ctx<real, ND>& X, const int (&act)[ND], const real (&al)[ND],
                                              const real* __restrict__ Cdiag, const real* __restrict__ Coff,
                                              const real* __restrict__ r, const real* __restrict__ vnew,
                                              real* __restrict__ t, Acc<real> (&a)[3 * ND]) {
  const int32_t N = X.N, nq = N >> 2, st = X.stride();
#pragma unroll 1
  for (int32_t qi = X.first(); qi < nq; qi += st) {
    const Quad<ND> q = quad_at<ND>(X.D, qi << 2);
    const int32_t i0 = q.i0;
    V4<real> diag, cf[2 * ND];
    c_row4<real, ND, TR>(q, N, Cdiag, Coff, diag, cf);
#pragma unroll
    for (int c = 0; c < ND; c++) {
      if (!act[c]) continue;
      const size_t o_ = (size_t)c * N;
      const real alc = al[c];
      auto sv = [&](int32_t Q) -> real { return r[o_ + Q] - alc * vnew[o_ + Q]; };
      auto sq = [&](int32_t Q0, real (&y)[4]) {
        const V4<real> rq = ld4(r + o_ + Q0), vq = ld4(vnew + o_ + Q0);
#pragma unroll
        for (int k = 0; k < 4; k++) y[k] = rq.v[k] - alc * vq.v[k];
      };
      real sP[4], tt[4];
      sq(i0, sP);
      quad_apply<real, ND>(q, diag, cf, sP, sv, sq, tt);
      st4(t + o_ + i0, V4<real>{{tt[0], tt[1], tt[2], tt[3]}});
#pragma unroll
      for (int k = 0; k < 4; k++) {
        a[c].add_prod(tt[k], sP[k]);
        a[ND + c].add_prod(tt[k], tt[k]);
        a[2 * ND + c].add_prod(sP[k], sP[k]);
      }
    }
  }
}

template <typename real, int ND>
__device__ __forceinline__ void bicg_sweep_c4(const Ctx<real, ND>& X, const int (&act)[ND], const int (&sc)[ND],
                                              const real (&al)[ND], const real (&om)[ND],
                                              const real* __restrict__ pnew, const real* __restrict__ vnew,
                                              const real* __restrict__ t, const real* __restrict__ rhat,
                                              real* __restrict__ x, real* __restrict__ r, Acc<real> (&a)[2 * ND]) {
  const int32_t N = X.N, nq = N >> 2, st = X.stride();
#pragma unroll 1
  for (int32_t qi = X.first(); qi < nq; qi += st) {
    const int32_t i0 = qi << 2;
#pragma unroll
    for (int c = 0; c < ND; c++) {
      if (!act[c]) continue;
      const size_t o_ = (size_t)c * N + i0;
      const V4<real> rq = ld4(r + o_), vq = ld4(vnew + o_), pq = ld4(pnew + o_), xq = ld4(x + o_);
      V4<real> xn, rn;
      if (sc[c]) {
#pragma unroll
        for (int k = 0; k < 4; k++) xn.v[k] = xq.v[k] + al[c] * pq.v[k];
        st4(x + o_, xn);
        continue;
      }
      const V4<real> tq = ld4(t + o_), rh = ld4(rhat + o_);
#pragma unroll
      for (int k = 0; k < 4; k++) {
        const real sP = rq.v[k] - al[c] * vq.v[k];
        xn.v[k] = xq.v[k] + (al[c] * pq.v[k] + om[c] * sP);
        rn.v[k] = sP - om[c] * tq.v[k];
      }
      st4(x + o_, xn);
      st4(r + o_, rn);
#pragma unroll
      for (int k = 0; k < 4; k++) {
        a[c].add_prod(rh.v[k], rn.v[k]);
        a[ND + c].add_prod(rn.v[k], rn.v[k]);
      }
    }
  }
}

// BiCGStab (van der Vorst 1992) on M x = b, M = C or C^T, for the ND velocity
// components sharing M, each with its own scalars; converged components
// freeze.  On entry x = x0, r = b - M x0, rhat = r and bs came from bicg_start.
// Three reductions per iteration; p and s are formed on the fly at the stencil.
template <typename real, int ND, bool TR>
__device__ bool bicgstab(const Ctx<real, ND>& X, BiState& bs, int maxit, const real* Cdiag, const real* Coff,
                         real* x, real* r, const real* rhat, real* const (&pv)[2], real* const (&vv)[2], real* t) {
  // four cells per thread where the layout allows it (as cg_jacobi_sweep4)
  const bool v4 = X.D.vec4 && !X.nbt && !X.fr && aligned16(Cdiag) && aligned16(Coff) && aligned16(x) &&
                  aligned16(r) && aligned16(rhat) && aligned16(pv[0]) && aligned16(pv[1]) && aligned16(vv[0]) &&
                  aligned16(vv[1]) && aligned16(t);
  int cur = 0;
  while (bs.any && bs.it < maxit) {
    // BA: p = r + beta (p - omega v), v = M p
    {
      Acc<real> a[ND];
      real beta[ND], om[ND];
      int act[ND];
#pragma unroll
      for (int k = 0; k < ND; k++) {
        a[k].zero();
        act[k] = bs.active[k];
        beta[k] = pick<real>(bs.beta_d[k], bs.beta_f[k]);
        om[k] = pick<real>(bs.omega[k], bs.omega_f[k]);
      }
      const int first = bs.first;
      const real* pold = pv[cur ^ 1];
      const real* vold = vv[cur ^ 1];
      real* pnew = pv[cur];
      real* vnew = vv[cur];
      if (v4)
        bicg_sweep_a4<real, ND, TR>(X, first, act, beta, om, Cdiag, Coff, r, pold, vold, rhat, pnew, vnew, a);
      else
        bicg_sweep_a<real, ND, TR>(X, first, act, beta, om, Cdiag, Coff, r, pold, vold, rhat, pnew, vnew, a);
      const bool ok = reduce_sync<real, ND>(X.g, a, [&](const double* q) { bicg_update_alpha<ND>(bs, q); });
      if (!ok) return false;
    }
    // BB: s = r - alpha v, t = M s
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
      if (v4)
        bicg_sweep_b4<real, ND, TR>(X, act, al, Cdiag, Coff, r, vv[cur], t, a);
      else
        bicg_sweep_b<real, ND, TR>(X, act, al, Cdiag, Coff, r, vv[cur], t, a);
      const bool ok = reduce_sync<real, 3 * ND>(X.g, a, [&](const double* q) { bicg_update_omega<ND>(bs, q); });
      if (!ok) return false;
    }
    // BC: x += alpha p + omega s, r = s - omega t
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
      if (v4)
        bicg_sweep_c4<real, ND>(X, act, sc, al, om, pv[cur], vv[cur], t, rhat, x, r, a);
      else
        bicg_sweep_c<real, ND>(X, act, sc, al, om, pv[cur], vv[cur], t, rhat, x, r, a);
      const bool ok = reduce_sync<real, 2 * ND>(X.g, a, [&](const double* q) { bicg_update_rho<ND>(bs, q); });
      if (!ok) return false;
    }
    cur ^= 1;
  }
  return true;
}

}  // namespace piso
#include "piso_lines.cuh"
#include "piso_ilu.cuh"
namespace piso {

// One iteration's cell sweep of the Jacobi CG below (all of the CTA's cells):
// p = u + beta p, x += alpha p, s = w + beta s, r1 = r - alpha s, w1 = A' u1
// with u1 = D^-1 r1 formed on the fly at the neighbours, and the three dot
// products.  The arrays are distinct (ping-pong buffers; p and x are touched
// only at the own cell), so the pointer arguments are __restrict__: after
// inlining the compiler still knows a cell's stores cannot alias the next
// cell's loads, and the 2x unrolled loop keeps two cells' loads in flight.
template <typename real, int ND>
__device__ __forceinline__ void cg_jacobi_sweep(const Ctx<real, ND>& X, int first, real al, real be,
                                                const real* __restrict__ r_i, const real* __restrict__ w_i,
                                                const real* __restrict__ s_o, const real* __restrict__ Pinv,
                                                const real* __restrict__ Poff, real* __restrict__ pdir,
                                                real* __restrict__ x, real* __restrict__ s_n, real* __restrict__ r_n,
                                                real* __restrict__ w_n, Acc<real> (&a)[3]) {
  const int32_t N = X.N, e = X.end(), st = X.stride();
#pragma unroll 4
  for (int32_t i = X.first(); i < e; i += st) {
    const int32_t nx_ = i + st;
    if (nx_ < e) {
      prefetch_l2(r_i + nx_);
      prefetch_l2(w_i + nx_);
      prefetch_l2(s_o + nx_);
      prefetch_l2(Pinv + nx_);
      prefetch_l2(pdir + nx_);
      prefetch_l2(x + nx_);
#pragma unroll
      for (int j = 0; j < ND; j++) prefetch_l2(Poff + (size_t)j * N + nx_);
    }
    const Cell c = X.cell(i);
    real pf[2 * ND];
    p_row<real, ND>(c, N, Poff, pf, X.fr);
    auto sQ = [&](int32_t Q) -> real { return first ? w_i[Q] : w_i[Q] + be * s_o[Q]; };
    auto u1 = [&](int32_t Q) -> real { return (r_i[Q] - al * sQ(Q)) * Pinv[Q]; };
    const int32_t P = c.i;
    const real iP = Pinv[P];
    const real rP = r_i[P];
    const real pOld = first ? real(0) : pdir[P];
    const real xP = x[P];
    const real sP = sQ(P);
    real uq[2 * ND];
#pragma unroll
    for (int s = 0; s < 2 * ND; s++) uq[s] = c.nb[s] >= 0 ? u1(c.nb[s]) : real(0);
    const real uP = rP * iP;
    const real p = first ? uP : uP + be * pOld;
    const real r1 = rP - al * sP;
    const real u1P = r1 * iP;
    real w1 = 0;
#pragma unroll
    for (int s = 0; s < 2 * ND; s++)
      if (c.nb[s] >= 0) w1 += pf[s] * (u1P - uq[s]);
    pdir[P] = p;
    x[P] = xP + al * p;
    s_n[P] = sP;
    r_n[P] = r1;
    w_n[P] = w1;
    a[0].add_prod(r1, u1P);
    a[1].add_prod(w1, u1P);
    a[2].add_prod(r1, r1);
  }
}


// The sweep of cg_jacobi_sweep with four consecutive cells per thread (domains
// walked in interleaved passes whose blocks all have nx a multiple of 4 and
// plain joints, DomStatic::vec4).  The four cells share block, row, and their
// y and z neighbours are four consecutive cells too (or all boundary faces), so
// every stream is read and written as one aligned vector per array: the own
// cells' 9 streams, the 4 streams of each y/z neighbour quad and the -y/-z face
// coefficients of P; inside the quad the x neighbours' values are the quad's
// own, and only the cells left and right of it are read singly.  Each cell's
// arithmetic is that of cg_jacobi_sweep, term for term (same values, same
// summation order of A'u), so only the order of the three dot sums differs.
// Four times the bytes per load instruction and one neighbour lookup per four
// cells: the sweep is bound by the memory system, not by the loads a warp can
// keep in flight or by instruction issue.
template <typename real, int ND>
__device__ __forceinline__ void cg_jacobi_sweep4(const Ctx<real, ND>& X, int first, real al, real be,
                                                 const real* __restrict__ r_i, const real* __restrict__ w_i,
                                                 const real* __restrict__ s_o, const real* __restrict__ Pinv,
                                                 const real* __restrict__ Poff, real* __restrict__ pdir,
                                                 real* __restrict__ x, real* __restrict__ s_n,
                                                 real* __restrict__ r_n, real* __restrict__ w_n, Acc<real> (&a)[3]) {
  const int32_t N = X.N, nq = N >> 2, st = X.stride();
  // u1 = D^-1 (r - al s) at one cell (s = w + be s_old), as cg_jacobi_sweep forms it
  auto u1s = [&](int32_t Q) -> real {
    const real sQ = first ? w_i[Q] : w_i[Q] + be * s_o[Q];
    return (r_i[Q] - al * sQ) * Pinv[Q];
  };
  auto u1q = [&](int32_t Q0, real (&u)[4]) {
    const V4<real> rq = ld4(r_i + Q0), wq = ld4(w_i + Q0), iq = ld4(Pinv + Q0);
    V4<real> sq{};
    if (!first) sq = ld4(s_o + Q0);
#pragma unroll
    for (int k = 0; k < 4; k++) u[k] = (rq.v[k] - al * (first ? wq.v[k] : wq.v[k] + be * sq.v[k])) * iq.v[k];
  };
#pragma unroll 1
  for (int32_t q = X.first(); q < nq; q += st) {
    const int32_t i0 = q << 2;
    const int32_t nxt = (q + st) << 2;
    if (q + st < nq) {
      prefetch_l2(r_i + nxt);
      prefetch_l2(w_i + nxt);
      prefetch_l2(Pinv + nxt);
      prefetch_l2(x + nxt);
      if (!first) {
        prefetch_l2(s_o + nxt);
        prefetch_l2(pdir + nxt);
      }
#pragma unroll
      for (int j = 0; j < ND; j++) prefetch_l2(Poff + (size_t)j * N + nxt);
    }
    const Cell c = locate<ND>(X.D, i0);
    const BlockInfo& B = X.D.blk[c.b];
    const int32_t nR = (c.x + 4 < B.nx) ? i0 + 4 : side_nbr(X.D, B, i0 + 3, c.x + 3, c.y, c.z, 1);
    const int32_t nL = c.nb[0];
    // own cells, in an order that lets each value die early: s, r and their
    // dot products; then p and x (touched only here); then the stencil
    real u1P[4], w1[4];
    {
      const V4<real> rP = ld4(r_i + i0), wP = ld4(w_i + i0), iP = ld4(Pinv + i0);
      V4<real> sO{};
      if (!first) sO = ld4(s_o + i0);
      V4<real> sn, rn;
#pragma unroll
      for (int k = 0; k < 4; k++) {
        sn.v[k] = first ? wP.v[k] : wP.v[k] + be * sO.v[k];
        rn.v[k] = rP.v[k] - al * sn.v[k];
        u1P[k] = rn.v[k] * iP.v[k];
      }
      st4(s_n + i0, sn);
      st4(r_n + i0, rn);
#pragma unroll
      for (int k = 0; k < 4; k++) {
        a[0].add_prod(rn.v[k], u1P[k]);
        a[2].add_prod(rn.v[k], rn.v[k]);
      }
      const V4<real> xP = ld4(x + i0);
      V4<real> pO{};
      if (!first) pO = ld4(pdir + i0);
      V4<real> pn, xn;
#pragma unroll
      for (int k = 0; k < 4; k++) {
        const real uP = rP.v[k] * iP.v[k];
        pn.v[k] = first ? uP : uP + be * pO.v[k];
        xn.v[k] = xP.v[k] + al * pn.v[k];
      }
      st4(pdir + i0, pn);
      st4(x + i0, xn);
    }
    // x faces (sides 0, 1): inside the quad from registers, the cells left and
    // right of it read singly
    {
      const V4<real> px = ld4(Poff + i0);
      const real uL = nL >= 0 ? u1s(nL) : real(0), cL = nL >= 0 ? Poff[nL] : real(0);
      const real uR = nR >= 0 ? u1s(nR) : real(0);
#pragma unroll
      for (int k = 0; k < 4; k++) {
        real w = 0;
        if (k > 0) w += px.v[k - 1] * (u1P[k] - u1P[k - 1]);
        else if (nL >= 0) w += cL * (u1P[0] - uL);
        if (k < 3) w += px.v[k] * (u1P[k] - u1P[k + 1]);
        else if (nR >= 0) w += px.v[3] * (u1P[3] - uR);
        w1[k] = w;
      }
    }
    // y and z faces (sides 2 .. 2 ND - 1): a neighbour quad, or boundary faces
#pragma unroll
    for (int j = 1; j < ND; j++) {
      const int32_t Qm = c.nb[2 * j], Qp = c.nb[2 * j + 1];
      if (Qm >= 0) {
        real u[4];
        u1q(Qm, u);
        const V4<real> cm = ld4(Poff + (size_t)j * N + Qm);
#pragma unroll
        for (int k = 0; k < 4; k++) w1[k] += cm.v[k] * (u1P[k] - u[k]);
      }
      if (Qp >= 0) {
        real u[4];
        u1q(Qp, u);
        const V4<real> cp = ld4(Poff + (size_t)j * N + i0);
#pragma unroll
        for (int k = 0; k < 4; k++) w1[k] += cp.v[k] * (u1P[k] - u[k]);
      }
    }
    V4<real> wn;
#pragma unroll
    for (int k = 0; k < 4; k++) {
      wn.v[k] = w1[k];
      a[1].add_prod(w1[k], u1P[k]);
    }
    st4(w_n + i0, wn);
  }
}

// Jacobi-preconditioned CG in the single-reduction form of Chronopoulos and
// Gear (1989) for  (-P) x = -(b - bmean)  (R7: the pressure system is singular
// and b is projected to zero mean).  D = -diag(P) is the preconditioner.  On
// entry x holds x0; on return x holds the solution (not mean-corrected).
// rb, wb, sb are ping-pong buffers for r, w = A u and s = A p; pdir holds p.
template <typename real, int ND>
__device__ bool cg_pressure(const Ctx<real, ND>& X, CgState& cs, double rtol, double atol, int maxit,
                            const real* Pdiag, const real* Pinv, const real* Poff, const real* b, double bmean,
                            real* x, real* const (&rb)[2], real* const (&wb)[2], real* const (&sb)[2],
                            real* pdir, int stall_window = 0) {
  if (X.lp) {   // y-line preconditioner (piso_lines.cuh)
    if (X.lp->fl)
      return cg_pressure_fused<real, ND>(X, cs, rtol, atol, maxit, Poff, b, bmean, x, rb, wb, sb, stall_window);
    return cg_pressure_line<real, ND>(X, cs, rtol, atol, maxit, Poff, b, bmean, x, rb[0], rb[1], wb[0], sb[0], pdir,
                                      stall_window);
  }
  const int32_t N = X.N;
  // I1: r0 = b' - A' x0 with b' = -(b - mean), A' = -P
  __shared__ double s_mb;
  __shared__ float s_mbf;
  {
    Acc<real> a[2];
    a[0].zero();
    a[1].zero();
    if (threadIdx.x == 0) {
      s_mb = bmean;
      s_mbf = (float)bmean;
    }
    __syncthreads();
    const real mb = pick<real>(s_mb, s_mbf);
    X.cells([&](const Cell& c) {
      real pf[2 * ND];
      p_row<real, ND>(c, N, Poff, pf, X.fr);
      const real bp = -(b[c.i] - mb);
      const real xP = x[c.i];
      real px = 0;   // (P x)_P = sum_f P_F (x_F - x_P): exact zero on constants in any precision
#pragma unroll
      for (int s = 0; s < 2 * ND; s++)
        if (c.nb[s] >= 0) px += pf[s] * (x[c.nb[s]] - xP);
      const real r = bp + px;
      rb[0][c.i] = r;
      a[0].add_prod(bp, bp);
      a[1].add_prod(r, r);
    });
    const bool ok = reduce_sync<real, 2>(X.g, a, [&](const double* q) {
      cs.tol2 = fmax(rtol * rtol * q[0], atol * atol);
      cs.res2 = q[1];
      cs.best = q[1];
      if (sizeof(real) == 4) {
        cs.ftol2 = f2_from_double(cs.tol2);
        cs.fbest = f2_from_double(q[1]);
        cs.fres2 = cs.fbest;
      }
      cs.best_it = 0;
      cs.stalled = 0;
      cs.it = 0;
      cs.first = 1;
      cs.conv = !(cs.res2 > cs.tol2);
      cs.active = !cs.conv;
      if (cs.res2 != cs.res2) {
        cs.active = 0;
        cs.conv = 0;
        atomicOr(X.g.status, PISO_ERR_NAN);
      }
    });
    if (!ok) return false;
  }
  if (!cs.active) return true;
  // I2: w0 = A' u0, u0 = D^-1 r0
  {
    Acc<real> a[2];
    a[0].zero();
    a[1].zero();
    const real* r0 = rb[0];
    X.cells([&](const Cell& c) {
      real pf[2 * ND];
      p_row<real, ND>(c, N, Poff, pf, X.fr);
      const real rP = r0[c.i];
      const real uP = rP * Pinv[c.i];
      real w = 0;    // (A' u)_P = sum_f P_F (u_P - u_F)
#pragma unroll
      for (int s = 0; s < 2 * ND; s++) {
        const int32_t Q = c.nb[s];
        if (Q >= 0) w += pf[s] * (uP - r0[Q] * Pinv[Q]);
      }
      wb[0][c.i] = w;
      a[0].add_prod(rP, uP);
      a[1].add_prod(w, uP);
    });
    const bool ok = reduce_sync<real, 2>(X.g, a, [&](const double* q) {
      if (cg_coeffs(cs, q[0], q[1], true, X.g.status) && sizeof(real) == 4) {
        cs.fgam = f2_from_double(q[0]);
        cs.finv_alpha = f2_div(f2_from_double(q[1]), cs.fgam);
      }
    });
    if (!ok) return false;
  }
  // four cells per thread where the layout allows it (cg_jacobi_sweep4)
  const bool v4 = X.D.vec4 && !X.nbt && !X.fr && aligned16(rb[0]) && aligned16(rb[1]) && aligned16(wb[0]) &&
                  aligned16(wb[1]) && aligned16(sb[0]) && aligned16(sb[1]) && aligned16(Pinv) && aligned16(Poff) &&
                  aligned16(pdir) && aligned16(x);
  int cur = 0;
  while (cs.active && cs.it < maxit) {
    Acc<real> a[3];
    a[0].zero();
    a[1].zero();
    a[2].zero();
    const real al = pick<real>(cs.alpha, cs.alpha_f), be = pick<real>(cs.beta, cs.beta_f);
    const int first = cs.first;
    const real* r_i = rb[cur];
    const real* w_i = wb[cur];
    const real* s_o = sb[cur ^ 1];
    real* s_n = sb[cur];
    real* r_n = rb[cur ^ 1];
    real* w_n = wb[cur ^ 1];
    if (v4)
      cg_jacobi_sweep4<real, ND>(X, first, al, be, r_i, w_i, s_o, Pinv, Poff, pdir, x, s_n, r_n, w_n, a);
    else
      cg_jacobi_sweep<real, ND>(X, first, al, be, r_i, w_i, s_o, Pinv, Poff, pdir, x, s_n, r_n, w_n, a);
    bool ok;
    if constexpr (sizeof(real) == 4)
      ok = reduce_sync<real, 3, true>(X.g, a, [&](const double* q) {
        cg_iter_update_f2(cs, f2_unpack(q[0]), f2_unpack(q[1]), f2_unpack(q[2]), stall_window, X.g.status);
      });
    else
      ok = reduce_sync<real, 3>(
          X.g, a, [&](const double* q) { cg_iter_update(cs, q[0], q[1], q[2], stall_window, X.g.status); });
    if (!ok) return false;
    cur ^= 1;
    // residual replacement (Cools & Vanroose): every CG_REPLACE iterations the
    // recursively updated r, w = A u and s = A p are recomputed from x and p,
    // which keeps the single-reduction recurrences from drifting in FP32
    if (CG_REPLACE > 0 && cs.active && cs.it % CG_REPLACE == 0) {
      const real mb = pick<real>(s_mb, s_mbf);
      real* r_t = rb[cur];
      X.cells([&](const Cell& c) {
        real pf[2 * ND];
        p_row<real, ND>(c, N, Poff, pf, X.fr);
        const real xP = x[c.i];
        real px = 0;
#pragma unroll
        for (int s = 0; s < 2 * ND; s++)
          if (c.nb[s] >= 0) px += pf[s] * (x[c.nb[s]] - xP);
        r_t[c.i] = -(b[c.i] - mb) + px;
      });
      if (!plain_sync(X.g)) return false;
      Acc<real> a2[3];
      a2[0].zero();
      a2[1].zero();
      a2[2].zero();
      real* w_t = wb[cur];
      real* s_t = sb[cur ^ 1];
      X.cells([&](const Cell& c) {
        real pf[2 * ND];
        p_row<real, ND>(c, N, Poff, pf, X.fr);
        const int32_t P = c.i;
        const real uP = r_t[P] * Pinv[P];
        const real pP = pdir[P];
        real w = 0, sv = 0;
#pragma unroll
        for (int s = 0; s < 2 * ND; s++) {
          const int32_t Q = c.nb[s];
          if (Q >= 0) {
            w += pf[s] * (uP - r_t[Q] * Pinv[Q]);
            sv += pf[s] * (pP - pdir[Q]);
          }
        }
        w_t[P] = w;
        s_t[P] = sv;
        a2[0].add_prod(r_t[P], uP);
        a2[1].add_prod(w, uP);
        a2[2].add_prod(r_t[P], r_t[P]);
      });
      const bool ok2 = reduce_sync<real, 3>(X.g, a2, [&](const double* q) {
        cs.res2 = q[2];
        if (sizeof(real) == 4) cs.fres2 = f2_from_double(q[2]);
        if (!(cs.res2 > cs.tol2)) {
          cs.active = 0;
          cs.conv = 1;
          return;
        }
        if (cg_coeffs(cs, q[0], q[1], false, X.g.status) && sizeof(real) == 4) {
          cs.fgam = f2_from_double(q[0]);
          cs.finv_alpha = f2_from_double(1.0 / cs.alpha);
        }
      });
      if (!ok2) return false;
    }
  }
  if (sizeof(real) == 4 && threadIdx.x == 0) cs.res2 = f2_to_double(cs.fres2);
  return true;
}

// Iteratively refined pressure solve for the FP32 mode: the solution x64 and
// the outer residual r = b' - A' x64 (b' = -(b - mean), A' = -P) live in FP64;
// each round solves A' e = r in FP32 with cg_pressure to inner_rtol and adds e
// to x64 in FP64, until ||r|| <= max(outer_rtol ||b'||, atol).  Every residual
// phase also writes x = (float) x64, so x holds the refined solution after the
// final (converged) residual phase and its barrier.  e, rin: FP32 scratch.
template <typename real, int ND>
__device__ bool cg_pressure_refined(const Ctx<real, ND>& X, CgState& cs, RefState& rs, double outer_rtol,
                                    double inner_rtol, double atol, int maxit, int max_rounds, const real* Pdiag,
                                    const real* Pinv, const real* Poff, const real* b, double bmean, real* x,
                                    double* x64, real* rin, real* e, real* const (&rb)[2], real* const (&wb)[2],
                                    real* const (&sb)[2], real* pdir) {
  const int32_t N = X.N;
  for (int round = 0;; round++) {
    // residual in FP64, measured and corrected in the zero-mean subspace (R7:
    // the rounded P has row sums of order the FP32 unit roundoff, so the
    // constant mode of r is not reducible and carries no pressure gradient)
    {
      Acc<double> a[3];
      a[0].zero();
      a[1].zero();
      a[2].zero();
      X.cells([&](const Cell& c) {
        real pf[2 * ND];
        p_row<real, ND>(c, N, Poff, pf, X.fr);
        auto xs = [&](int32_t Q) -> double { return round == 0 ? (double)x[Q] : x64[Q]; };
        const int32_t P = c.i;
        const double bp = -((double)b[P] - bmean);
        const double xP = xs(P);
        double px = 0;
#pragma unroll
        for (int s = 0; s < 2 * ND; s++)
          if (c.nb[s] >= 0) px += (double)pf[s] * (xs(c.nb[s]) - xP);
        const double r = bp + px;
        if (round == 0) x64[P] = xP;
        else x[P] = (real)xP;
        rin[P] = (real)(-r);
        e[P] = real(0);
        a[0].add(r);
        a[1].add_prod(r, r);
        a[2].add_prod(bp, bp);
      });
      const bool ok = reduce_sync<double, 3>(X.g, a, [&](const double* q) {
        if (round == 0) {
          rs.bn2 = q[2];
          rs.tol2 = fmax(outer_rtol * outer_rtol * q[2], atol * atol);
          rs.inner_it = 0;
        }
        const double mean = q[0] / (double)N;
        rs.rmean = mean;
        rs.res2 = fmax(q[1] - (double)N * mean * mean, 0.0);
        rs.rounds = round;
        rs.conv = !(rs.res2 > rs.tol2);
        if (rs.res2 != rs.res2) {
          rs.conv = 0;
          atomicOr(X.g.status, PISO_ERR_NAN);
        }
      });
      if (!ok) return false;
    }
    if (rs.conv || rs.res2 != rs.res2 || round >= max_rounds || rs.inner_it >= maxit) return true;
    // inner FP32 solve of A' e = r (a stalled inner solve just ends the round)
    if (!cg_pressure<real, ND>(X, cs, inner_rtol, 0.0, maxit - rs.inner_it, Pdiag, Pinv, Poff, rin, -rs.rmean, e,
                               rb, wb, sb, pdir, CG_STALL_WINDOW))
      return false;
    if (threadIdx.x == 0) rs.inner_it += cs.it;
    // x64 += e
    X.own([&](int32_t P) { x64[P] += (double)e[P]; });
    if (!plain_sync(X.g)) return false;
  }
}

__device__ __forceinline__ void cg_iter_update(CgState& cs, double gam, double delta, double res2, int stall_window,
                                               int32_t* status) {
  cs.it++;
  cs.res2 = res2;
  cs.first = 0;
  if (res2 != res2) {
    cs.active = 0;
    atomicOr(status, PISO_ERR_NAN);
  } else if (!(res2 > cs.tol2)) {
    cs.active = 0;
    cs.conv = 1;
  } else if (stall_window > 0 && !(res2 < 0.25 * cs.best) && cs.it - cs.best_it >= stall_window) {
    cs.active = 0;
    cs.stalled = 1;
  } else {
    if (res2 < 0.25 * cs.best) {
      cs.best = res2;
      cs.best_it = cs.it;
    }
    cg_coeffs(cs, gam, delta, false, status);
  }
}

// One corrector's pressure solve P x = b - mean (forward or adjoint), x holding
// the initial guess: a CG to rtol, or in the FP32 mode with p_refine_rtol > 0 an
// FP64-refined solve; an FP32 CG that stalls is finished by refinement rounds
// to the same tolerance from where it stopped.  Thread 0 of group rank 0
// records iterations, refinement rounds, residual and right-hand-side norms in
// stats slot k and flags non-convergence.  Returns false if the group aborted.
template <typename real, int ND>
__device__ bool pressure_solve(const Ctx<real, ND>& X, CgState& cs, RefState& rs, const SolverOpts& o,
                               const real* Pdiag, const real* Pinv, const real* Poff, const real* b, double bmean,
                               real* x, double* x64, real* rin, real* ce, real* const (&rb)[2],
                               real* const (&wb)[2], real* const (&sb)[2], real* pdir, int32_t* istats,
                               double* dstats, int k) {
  constexpr bool F32 = sizeof(real) == 4;
  const Group& g = X.g;
  if (F32 && o.p_refine_rtol > 0) {
    if (!cg_pressure_refined<real, ND>(X, cs, rs, o.p_refine_rtol, o.p_inner_rtol, o.atol, o.p_maxit, 20, Pdiag,
                                       Pinv, Poff, b, bmean, x, x64, rin, ce, rb, wb, sb, pdir))
      return false;
    if (threadIdx.x == 0 && g.rank == 0) {
      istats[4 + k] = rs.inner_it;
      istats[8 + k] = rs.rounds;
      dstats[4 + k] = sqrt(rs.res2);
      dstats[8 + k] = sqrt(rs.bn2);
      if (!rs.conv) atomicOr(g.status, PISO_ERR_NOCONV_P);
    }
    return true;
  }
  if (!cg_pressure<real, ND>(X, cs, o.p_rtol, o.atol, o.p_maxit, Pdiag, Pinv, Poff, b, bmean, x, rb, wb, sb, pdir,
                             F32 ? CG_STALL_WINDOW : 0))
    return false;
  if (F32 && cs.stalled) {
    const int plain_it = cs.it;
    if (!cg_pressure_refined<real, ND>(X, cs, rs, o.p_rtol, o.p_inner_rtol, o.atol, o.p_maxit - plain_it, 20, Pdiag,
                                       Pinv, Poff, b, bmean, x, x64, rin, ce, rb, wb, sb, pdir))
      return false;
    // the refined result lives in x64; x holds it rounded (written by the last
    // residual pass of the refinement)
    if (threadIdx.x == 0 && g.rank == 0) {
      istats[4 + k] = plain_it + rs.inner_it;
      istats[8 + k] = 1 + rs.rounds;
      dstats[4 + k] = sqrt(rs.res2);
      dstats[8 + k] = sqrt(rs.bn2);
      if (!rs.conv) atomicOr(g.status, PISO_ERR_NOCONV_P);
    }
    return true;
  }
  if (threadIdx.x == 0 && g.rank == 0) {
    istats[4 + k] = cs.it;
    dstats[4 + k] = sqrt(cs.res2);
    dstats[8 + k] = sqrt(cs.tol2) / fmax(o.p_rtol, 1e-300);
    if (!cs.conv) atomicOr(g.status, PISO_ERR_NOCONV_P);
  }
  return true;
}

}  // namespace piso
