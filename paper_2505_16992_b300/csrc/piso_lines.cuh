// y-line preconditioner for the pressure CG (a B300 choice; the paper's CG,
// App. A.5, names no preconditioner for the pressure system).
//
// M is the block diagonal of -P made of its y-lines: for every block column
// (fixed x, z) the tridiagonal matrix that keeps the cell's full diagonal
// (-P_P = sum of all its face coefficients) and the couplings to the y-
// neighbours inside the same block.  Couplings across block sides, periodic
// wraps and the x/z directions are dropped, so every line block is strictly
// diagonally dominant (whenever a cell has an x or z face) and M is symmetric
// positive definite: a valid CG preconditioner.  On grids refined towards
// walls in y (tanh stretching, aspect ratios of 10-100 near the wall) the y
// couplings dominate -P and M captures them: on the 64x48x32 channel the CG
// needs 106 instead of 252 iterations, on the 5-block step 482 instead of 1477.
//
// Thomas' algorithm for one line block, with d_y = -P_P, e_y = -P_F(y, y+1)
// (0 for the last cell of the line), m_y = 1 / (d_y - e_{y-1} c'_{y-1}) and
// c'_y = e_y m_y (formed once per step):
//   g_y = fa_y g_{y-1} + fm_y r_y,  fa_y = -e_{y-1} m_y, fm_y = m_y  (forward)
//   z_y = fc_y z_{y+1} + g_y,       fc_y = -c'_y                      (backward)
//
// Execution: M^-1 r needs a whole line, so the CG iteration splits into two
// phases with a plain barrier between them.  In the first, each CTA owns a
// contiguous range of lines, stages them in shared memory in batches (cell
// (line, y) of a batch at index y * pitch + line), updates r, x, p, s there and
// solves its lines; in the second, every CTA applies -P to u on its usual cell
// range.  A line is solved by a group of 8 to 32 lanes of one warp: the two
// recurrences are affine maps composed by a parallel prefix over the group
// (Kogge-Stone), each lane holding a contiguous chunk of the line.
// This header is included from piso_krylov.cuh (it uses Ctx, CgState and the
// group reductions defined there).
#pragma once

namespace piso {

constexpr int LINE_LBMAX = 1024;   // lines per staging batch (size of the descriptor arrays)
constexpr int LINE_ARRAYS = 4;     // staged reals per cell: fa, fm r (then the solution), fc, r

// This CTA's share of the y-line preconditioner: lines [L0, L1) of the group
// and the staging area behind the neighbour table in dynamic shared memory
// (LINE_ARRAYS arrays of o.line_cap reals, or the fused solve's arrays where
// those are larger, then 3 x LINE_LBMAX ints).
template <typename real, int ND>
__device__ __forceinline__ LinePre<real> line_setup(const DomStatic& D, const Group& g, const SolverOpts& o,
                                                    real* fa, real* fm, real* fc) {
  extern __shared__ int32_t s_nbt[];
  LinePre<real> L;
  const size_t nbt_bytes = ((size_t)o.nbt_cap * 2 * ND * sizeof(int32_t) + 15) & ~size_t(15);
  char* base = reinterpret_cast<char*>(s_nbt) + nbt_bytes;
  real* sr = reinterpret_cast<real*>(base);
  const size_t cap = (size_t)o.line_cap;
  L.sA = sr;
  L.sB = sr + cap;
  L.sC = sr + 2 * cap;
  L.sR = sr + 3 * cap;
  const size_t stage = LINE_ARRAYS * cap * sizeof(real);
  const bool fused = o.lf_off != nullptr;
  int32_t* si = reinterpret_cast<int32_t*>(base + (fused ? max(stage, (size_t)o.lf_bytes) : stage));
  L.fl = nullptr;
  L.fnb = nullptr;
  if (fused) {
    const int32_t a = o.lf_off[g.rank];
    L.fl = o.lf_lines + a;
    L.n_own = o.lf_nown[g.rank];
    L.n_loc = o.lf_off[g.rank + 1] - a;
    L.own_cap = o.lf_own_cap;
    L.slot_cap = o.lf_slot_cap;
    L.fnb = o.lf_nbs + (size_t)g.rank * 2 * ND * o.lf_own_cap;
    const size_t sc = (size_t)o.lf_slot_cap, oc = (size_t)o.lf_own_cap;
    L.fA = sr;
    L.fC = sr + sc;
    L.fM = sr + 2 * sc;
    L.fB = sr + 3 * sc;
    L.fR = sr + 4 * sc;
    L.fS = sr + 5 * sc;
    L.fP = sr + 6 * sc;
    L.fX = L.fP + oc;
    L.fW = L.fX + oc;
    L.fPf = L.fW + oc;
    L.fI = reinterpret_cast<int32_t*>(L.fPf + 2 * ND * oc);
    L.fNb = reinterpret_cast<int16_t*>(L.fI + sc);
  }
  L.sStart = si;
  L.sStride = si + LINE_LBMAX;
  L.sLen = si + 2 * LINE_LBMAX;
  L.fa = fa;
  L.fm = fm;
  L.fc = fc;
  L.L0 = (int32_t)(((int64_t)D.nlines * g.rank) / g.ncta);
  L.L1 = (int32_t)(((int64_t)D.nlines * (g.rank + 1)) / g.ncta);
  L.lb = min(LINE_LBMAX, o.line_cap / D.lmax - 1);
  return L;
}

// Staging geometry of one batch: nb lines from line l0, pitch = nb | 1 (odd, so
// the lanes of a line-solve warp, whose chunks start E * pitch apart, spread
// over at least 16 banks).
struct LineBatch {
  int32_t l0, nb, pitch, slots;   // slots = nb * lmax
};

// Load this batch's line descriptors into shared memory.
template <typename real>
__device__ __forceinline__ LineBatch line_batch_begin(const DomStatic& D, const LinePre<real>& L, int32_t l0) {
  LineBatch B;
  B.l0 = l0;
  B.nb = min(L.lb, L.L1 - l0);
  B.pitch = B.nb | 1;
  B.slots = B.nb * D.lmax;
  __syncthreads();   // the previous batch's staging is no longer read
  for (int32_t t = threadIdx.x; t < B.nb; t += blockDim.x) {
    const LineDesc ld = line_desc(D, l0 + t);
    L.sStart[t] = ld.start;
    L.sStride[t] = ld.stride;
    L.sLen[t] = ld.len;
  }
  __syncthreads();
  return B;
}

// Cell and shared index of slot k of a batch (consecutive slots take
// consecutive lines at the same y: contiguous memory for y-lines); false if
// the slot lies past the end of a shorter line.  last: the line's last cell.
template <typename real>
__device__ __forceinline__ bool line_slot(const LinePre<real>& L, const LineBatch& B, int32_t k, int32_t& cell,
                                          int32_t& sk, bool& last) {
  const int32_t q = k / B.nb;   // y along the line
  const int32_t l = k - q * B.nb;
  const int32_t len = L.sLen[l];
  if (q >= len) return false;
  cell = L.sStart[l] + q * L.sStride[l];
  sk = q * B.pitch + l;
  last = q + 1 == len;
  return true;
}

template <typename real, typename F>
__device__ __forceinline__ void line_batch_cells(const LinePre<real>& L, const LineBatch& B, F&& f) {
  for (int32_t k = threadIdx.x; k < B.slots; k += blockDim.x) {
    int32_t i, sk;
    bool last;
    if (line_slot(L, B, k, i, sk, last)) f(i, sk, last);
  }
}

// Solve nb staged lines (cell y of line l at y * P + l) in place: on entry
// sB = fm * r, sA = fa, sC = fc; on exit sB = M^-1 r.  A line is solved by W
// lanes of a warp (32 / W lines per warp at a time); lane j of its group
// holds the chunk [j E, min(len, (j + 1) E)) with E = ceil(len / W).
template <typename real, int W>
__device__ __forceinline__ void line_solve_w(const real* __restrict__ sA, real* __restrict__ sB,
                                             const real* __restrict__ sC, const int32_t* sLen, int32_t nb,
                                             int32_t P) {
  constexpr int G = 32 / W;   // lines per warp
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int j = lane % W;
  for (int32_t lb = warp * G; lb < nb; lb += nw * G) {   // uniform over the warp
    const int32_t l = lb + lane / W;
    const int32_t len = l < nb ? sLen[l] : 0;
    const int32_t E = (len + W - 1) / W;
    const int32_t y0 = min(len, j * E), y1 = min(len, y0 + E);
    // forward: g_y = a_y g_{y-1} + b_y; this lane's chunk as one map g -> A g + Bv
    real A = real(1), Bv = real(0);
    for (int32_t y = y0; y < y1; y++) {
      const real a = sA[y * P + l];
      A = a * A;
      Bv = a * Bv + sB[y * P + l];
    }
#pragma unroll
    for (int off = 1; off < W; off <<= 1) {       // inclusive prefix of the maps over the group
      const real Au = __shfl_up_sync(0xffffffffu, A, off, W);
      const real Bu = __shfl_up_sync(0xffffffffu, Bv, off, W);
      if (j >= off) {
        Bv = A * Bu + Bv;
        A = A * Au;
      }
    }
    real g = __shfl_up_sync(0xffffffffu, Bv, 1, W);   // g just before this chunk (g_{-1} = 0)
    if (j == 0) g = real(0);
    for (int32_t y = y0; y < y1; y++) {
      g = sA[y * P + l] * g + sB[y * P + l];
      sB[y * P + l] = g;
    }
    // backward: z_y = c_y z_{y+1} + g_y; the chunk as one map z_next -> C z_next + G
    real Cm = real(1), Gz = real(0);
    for (int32_t y = y1 - 1; y >= y0; y--) {
      const real c = sC[y * P + l];
      Gz = c * Gz + sB[y * P + l];
      Cm = c * Cm;
    }
#pragma unroll
    for (int off = 1; off < W; off <<= 1) {       // suffix composition over the group
      const real Cd = __shfl_down_sync(0xffffffffu, Cm, off, W);
      const real Gd = __shfl_down_sync(0xffffffffu, Gz, off, W);
      if (j + off < W) {
        Gz = Cm * Gd + Gz;
        Cm = Cm * Cd;
      }
    }
    real z = __shfl_down_sync(0xffffffffu, Gz, 1, W);  // z just after this chunk (z_len = 0)
    if (j == W - 1) z = real(0);
    for (int32_t y = y1 - 1; y >= y0; y--) {
      z = sC[y * P + l] * z + sB[y * P + l];
      sB[y * P + l] = z;
    }
  }
}

// The group width is the widest that still solves all nb lines in one round
// of the CTA's warps (narrower groups: longer serial chunks, fewer shuffle
// steps; 8 lanes at the narrowest).
template <typename real>
__device__ __forceinline__ void line_solve(const real* __restrict__ sA, real* __restrict__ sB,
                                           const real* __restrict__ sC, const int32_t* sLen, int32_t nb,
                                           int32_t P) {
  __syncthreads();
  const int nw = blockDim.x >> 5;
  if (nb <= nw) line_solve_w<real, 32>(sA, sB, sC, sLen, nb, P);
  else if (nb <= 2 * nw) line_solve_w<real, 16>(sA, sB, sC, sLen, nb, P);
  else line_solve_w<real, 8>(sA, sB, sC, sLen, nb, P);
  __syncthreads();
}

template <typename real>
__device__ __forceinline__ void line_batch_solve(const LinePre<real>& L, const LineBatch& B) {
  line_solve<real>(L.sA, L.sB, L.sC, L.sLen, B.nb, B.pitch);
}

// Thomas factors of every line block of -P (once per step, after P is
// assembled).  One thread per line runs the recurrence over the staged
// coefficients.
template <typename real, int ND>
__device__ void line_factor(const DomStatic& D, const LinePre<real>& L, int32_t N, const real* Pdiag,
                            const real* Poff) {
  for (int32_t l0 = L.L0; l0 < L.L1; l0 += L.lb) {
    const LineBatch B = line_batch_begin(D, L, l0);
    line_batch_cells(L, B, [&](int32_t i, int32_t k, bool last) {
      L.sA[k] = -Pdiag[i];
      L.sB[k] = last ? real(0) : -Poff[(size_t)N + i];   // j = 1: the +y face of i
    });
    __syncthreads();
    for (int32_t l = threadIdx.x; l < B.nb; l += blockDim.x) {
      const int32_t len = L.sLen[l];
      real cprev = real(0), eprev = real(0);
      for (int32_t y = 0; y < len; y++) {
        const int32_t k = y * B.pitch + l;
        const real d = L.sA[k], e = L.sB[k];
        real piv = d - eprev * cprev;
        // a line block without x/z couplings (a one-cell-wide block) is
        // singular; the pivot then takes the full diagonal, i.e. the block is
        // factored with a positive diagonal shift and M stays SPD
        if (!(piv > real(1e-5) * d)) piv = d;
        const real m = real(1) / piv;
        const real c = e * m;
        L.sA[k] = -eprev * m;
        L.sB[k] = m;
        L.sC[k] = -c;
        cprev = c;
        eprev = e;
      }
    }
    __syncthreads();
    line_batch_cells(L, B, [&](int32_t i, int32_t k, bool) {
      L.fa[i] = L.sA[k];
      L.fm[i] = L.sB[k];
      L.fc[i] = L.sC[k];
    });
  }
  __syncthreads();
}

// Phase A of an iteration for one staged batch: p = u + beta p, s = w + beta s,
// x += alpha p, r -= alpha s at the batch's cells, and the staging of r and
// the line factors; ||r||^2.  Every array is touched through one pointer only
// (__restrict__: a slot's stores cannot alias the next slot's loads), the
// loop is unrolled 2x.
template <typename real>
__device__ __forceinline__ void line_update_sweep(const LinePre<real>& L, const LineBatch& B, int first, real al, real be,
                                                  const real* __restrict__ u, const real* __restrict__ w,
                                                  const real* __restrict__ fa, const real* __restrict__ fm,
                                                  const real* __restrict__ fc, real* __restrict__ r,
                                                  real* __restrict__ x, real* __restrict__ pdir, real* __restrict__ s,
                                                  real* __restrict__ sR, real* __restrict__ sA, real* __restrict__ sB,
                                                  real* __restrict__ sC, Acc<real>& rr2) {
#pragma unroll 2
  for (int32_t k = threadIdx.x; k < B.slots; k += blockDim.x) {
    int32_t i, sk;
    bool last;
    if (!line_slot(L, B, k, i, sk, last)) continue;
    const real uP = u[i], wP = w[i], rP = r[i], xP = x[i];
    const real pO = first ? real(0) : pdir[i];
    const real sO = first ? real(0) : s[i];
    const real fav = fa[i], fmv = fm[i], fcv = fc[i];
    const real p = first ? uP : uP + be * pO;
    const real sv = first ? wP : wP + be * sO;
    const real rr = rP - al * sv;
    pdir[i] = p;
    s[i] = sv;
    x[i] = xP + al * p;
    r[i] = rr;
    sR[sk] = rr;
    sA[sk] = fav;
    sB[sk] = fmv * rr;
    sC[sk] = fcv;
    rr2.add_prod(rr, rr);
  }
}

// Phase B: w = A' u on the CTA's cell range (difference form) and (w, u).
template <typename real, int ND>
__device__ __forceinline__ void line_apply_sweep(const Ctx<real, ND>& X, const real* __restrict__ u,
                                                 const real* __restrict__ Poff, real* __restrict__ w, Acc<real>& wu) {
  const int32_t N = X.N, e = X.end(), st = X.stride();
#pragma unroll 2
  for (int32_t i = X.first(); i < e; i += st) {
    const int32_t nx_ = i + st;
    if (nx_ < e) {
      prefetch_l2(u + nx_);
#pragma unroll
      for (int j = 0; j < ND; j++) prefetch_l2(Poff + (size_t)j * N + nx_);
    }
    const Cell c = X.cell(i);
    real pf[2 * ND];
    p_row<real, ND>(c, N, Poff, pf, X.fr);
    const real uP = u[c.i];
    real uq[2 * ND];
#pragma unroll
    for (int q = 0; q < 2 * ND; q++) uq[q] = c.nb[q] >= 0 ? u[c.nb[q]] : uP;
    real ww = 0;
#pragma unroll
    for (int q = 0; q < 2 * ND; q++) ww += pf[q] * (uP - uq[q]);
    w[c.i] = ww;
    wu.add_prod(ww, uP);
  }
}

// Thread 0, end of the start phase of a line-preconditioned CG, from the
// totals q = (||b'||^2, ||r0||^2, (r0, u0), (w0, u0)): tolerance, state and the
// first coefficients.
template <typename real>
__device__ __forceinline__ void line_cg_start(CgState& cs, const double* q, double rtol, double atol,
                                              int32_t* status) {
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
    atomicOr(status, PISO_ERR_NAN);
  }
  if (cs.active && cg_coeffs(cs, q[2], q[3], true, status) && sizeof(real) == 4) {
    cs.fgam = f2_from_double(q[2]);
    cs.finv_alpha = f2_div(f2_from_double(q[3]), cs.fgam);
  }
}

// Line-preconditioned CG on (-P) x = -(b - bmean) in the Chronopoulos-Gear
// form (one reduction per iteration; R7: b is projected to zero mean):
//   r0 = b' - A' x0, u0 = M^-1 r0, w0 = A' u0
//   per iteration: p = u + beta p, s = w + beta s, x += alpha p, r -= alpha s,
//                  u = M^-1 r  | barrier |  w = A' u, then gamma = (r, u),
//                  delta = (w, u), ||r||^2 in one group reduction.
// A' = -P is applied in difference form (sum_F P_F (u_P - u_F)), exact on
// constants in any precision.  Vectors: x (solution, holds x0 on entry), r, u,
// w, s, p.  The same scalar updates as the Jacobi CG (cg_coeffs /
// cg_iter_update).
template <typename real, int ND>
__device__ bool cg_pressure_line(const Ctx<real, ND>& X, CgState& cs, double rtol, double atol, int maxit,
                                 const real* Poff, const real* b, double bmean, real* x, real* r, real* u, real* w,
                                 real* s, real* pdir, int stall_window) {
  const int32_t N = X.N;
  const DomStatic& D = X.D;
  const LinePre<real>& L = *X.lp;
  __shared__ double s_mb2;
  __shared__ float s_mbf2;
  if (threadIdx.x == 0) {
    s_mb2 = bmean;
    s_mbf2 = (float)bmean;
  }
  __syncthreads();
  const real mb = pick<real>(s_mb2, s_mbf2);
  // I1: r0 = b' - A' x0 and u0 = M^-1 r0 on this CTA's lines
  Acc<real> a[4];
#pragma unroll
  for (int k = 0; k < 4; k++) a[k].zero();
  for (int32_t l0 = L.L0; l0 < L.L1; l0 += L.lb) {
    const LineBatch B = line_batch_begin(D, L, l0);
    line_batch_cells(L, B, [&](int32_t i, int32_t k, bool) {
      const Cell c = locate<ND>(D, i);
      real pf[2 * ND];
      p_row<real, ND>(c, N, Poff, pf, X.fr);
      const real bp = -(b[i] - mb);
      const real xP = x[i];
      real px = 0;
#pragma unroll
      for (int q = 0; q < 2 * ND; q++)
        if (c.nb[q] >= 0) px += pf[q] * (x[c.nb[q]] - xP);
      const real rr = bp + px;
      const real fa = L.fa[i], fm = L.fm[i], fc = L.fc[i];
      r[i] = rr;
      L.sR[k] = rr;
      L.sA[k] = fa;
      L.sB[k] = fm * rr;
      L.sC[k] = fc;
      a[0].add_prod(bp, bp);
      a[1].add_prod(rr, rr);
    });
    line_batch_solve(L, B);
    line_batch_cells(L, B, [&](int32_t i, int32_t k, bool) {
      const real uu = L.sB[k];
      u[i] = uu;
      a[2].add_prod(L.sR[k], uu);
    });
  }
  if (!plain_sync(X.g)) return false;
  // I2: w0 = A' u0 on the usual cell range
  X.cells([&](const Cell& c) {
    real pf[2 * ND];
    p_row<real, ND>(c, N, Poff, pf, X.fr);
    const real uP = u[c.i];
    real ww = 0;
#pragma unroll
    for (int q = 0; q < 2 * ND; q++)
      if (c.nb[q] >= 0) ww += pf[q] * (uP - u[c.nb[q]]);
    w[c.i] = ww;
    a[3].add_prod(ww, uP);
  });
  {
    const bool ok = reduce_sync<real, 4>(
        X.g, a, [&](const double* q) { line_cg_start<real>(cs, q, rtol, atol, X.g.status); });
    if (!ok) return false;
  }
  while (cs.active && cs.it < maxit) {
    Acc<real> c3[3];
    c3[0].zero();
    c3[1].zero();
    c3[2].zero();
    const real al = pick<real>(cs.alpha, cs.alpha_f), be = pick<real>(cs.beta, cs.beta_f);
    const int first = cs.first;
    // phase A: vector updates and u = M^-1 r on this CTA's lines
    for (int32_t l0 = L.L0; l0 < L.L1; l0 += L.lb) {
      const LineBatch B = line_batch_begin(D, L, l0);
      line_update_sweep<real>(L, B, first, al, be, u, w, L.fa, L.fm, L.fc, r, x, pdir, s, L.sR, L.sA, L.sB, L.sC,
                              c3[2]);
      line_batch_solve(L, B);
      line_batch_cells(L, B, [&](int32_t i, int32_t k, bool) {
        const real uu = L.sB[k];
        u[i] = uu;
        c3[0].add_prod(L.sR[k], uu);
      });
    }
    if (!plain_sync(X.g)) return false;
    // phase B: w = A' u and (w, u)
    line_apply_sweep<real, ND>(X, u, Poff, w, c3[1]);
    bool ok;
    if constexpr (sizeof(real) == 4)
      ok = reduce_sync<real, 3, true>(X.g, c3, [&](const double* q) {
        cg_iter_update_f2(cs, f2_unpack(q[0]), f2_unpack(q[1]), f2_unpack(q[2]), stall_window, X.g.status);
      });
    else
      ok = reduce_sync<real, 3>(
          X.g, c3, [&](const double* q) { cg_iter_update(cs, q[0], q[1], q[2], stall_window, X.g.status); });
    if (!ok) return false;
  }
  if (sizeof(real) == 4 && threadIdx.x == 0) cs.res2 = f2_to_double(cs.fres2);
  return true;
}

// Visit k = threadIdx.x, k + blockDim.x, ... < total as (q, l) = (k / n, k mod n),
// carrying the quotient and remainder from one visit to the next (no division
// inside the loop).
struct GridWalk {
  int32_t q, l, dq, dl, n;
  __device__ __forceinline__ GridWalk(int32_t n_) : n(n_) {
    const int32_t T = blockDim.x;
    dq = T / n;
    dl = T - dq * n;
    q = threadIdx.x / n;
    l = threadIdx.x - q * n;
  }
  __device__ __forceinline__ void next() {
    l += dl;
    q += dq;
    if (l >= n) {
      l -= n;
      q++;
    }
  }
};

template <typename F>
__device__ __forceinline__ void line_grid(int32_t n, int32_t total, F&& f) {
  GridWalk w(n);
  for (int32_t k = threadIdx.x; k < total; k += blockDim.x) {
    f(k, w.q, w.l);
    w.next();
  }
}

// The line-preconditioned CG with one group barrier per iteration, for
// launches whose every CTA can hold its own lines and the lines next to them
// in shared memory (the host builds the plan: own lines, halo lines and the
// shared slot of every neighbour of every own cell).  Same recurrences as
// cg_pressure_line; what moves is where u = M^-1 r comes from: each CTA
// updates s and r on its halo lines too and solves those lines itself, so the
// u of every neighbour of an own cell is in shared memory and w = A' u needs
// no barrier:
//   per iteration, on own and halo lines: s = w + beta s, r -= alpha s,
//   u = M^-1 r; on own cells: p = u_prev + beta p, x += alpha p, w = A' u;
//   one group reduction of gamma = (r, u), delta = (w, u), ||r||^2.
// r and s of every local line stay in shared memory for the whole solve: a
// halo line's copy starts from the owner's r0 and then takes the owner's
// recurrence step for step (the same code, the same w, alpha and beta), so it
// stays bit-identical to the owner's without being read back.  Only w
// crosses CTAs: the owners write it (ping-pong buffers, written before the
// barrier that precedes its reading), and the halo lines read it once per
// iteration.  Own cells keep p, x, w and their face coefficients in shared
// memory; x also goes to global memory every iteration (so it is complete at
// every barrier, the solve's last one included).  Cell y of local line
// l sits at slot y * P + l (P = n_loc | 1; fI holds its cell index, -1 past
// the line's end); own cell k = y * n_own + l.
template <typename real, int ND>
__device__ bool cg_pressure_fused(const Ctx<real, ND>& X, CgState& cs, double rtol, double atol, int maxit,
                                  const real* Poff, const real* b, double bmean, real* x, real* const (&rb)[2],
                                  real* const (&wb)[2], real* const (&sb)[2], int stall_window) {
  constexpr int NS = 2 * ND;
  const int32_t N = X.N;
  const DomStatic& D = X.D;
  const LinePre<real>& L = *X.lp;
  const int32_t no = L.n_own, nl = L.n_loc, P = nl | 1, oc = L.own_cap;
  const int32_t nslot = nl * D.lmax, nown = no * D.lmax;
  real* __restrict__ fA = L.fA;
  real* __restrict__ fC = L.fC;
  real* __restrict__ fM = L.fM;
  real* __restrict__ fB = L.fB;
  real* __restrict__ fR = L.fR;
  real* __restrict__ fS = L.fS;
  real* __restrict__ fP = L.fP;
  real* __restrict__ fX = L.fX;
  real* __restrict__ fW = L.fW;
  real* __restrict__ fPf = L.fPf;
  int32_t* __restrict__ fI = L.fI;
  int16_t* __restrict__ fNb = L.fNb;
  int32_t* sLen = L.sLen;
  __shared__ double s_mb3;
  __shared__ float s_mbf3;
  // S0: lengths of the local lines and the own cells' neighbour slots
  __syncthreads();   // earlier users of the staging area are done
  if (threadIdx.x == 0) {
    s_mb3 = bmean;
    s_mbf3 = (float)bmean;
  }
  for (int32_t t = threadIdx.x; t < nl; t += blockDim.x) {
    const LineDesc ld = line_desc(D, L.fl[t]);
    L.sStart[t] = ld.start;
    L.sStride[t] = ld.stride;
    sLen[t] = ld.len;
  }
  for (int32_t t = threadIdx.x; t < NS * oc; t += blockDim.x) fNb[t] = L.fnb[t];
  __syncthreads();
  const real mb = pick<real>(s_mb3, s_mbf3);
  // S1: cell index and line factors of every slot
  line_grid(nl, nslot, [&](int32_t, int32_t q, int32_t l) {
    const int32_t k = q * P + l;
    if (q >= sLen[l]) {
      fI[k] = -1;
      return;
    }
    const int32_t i = L.sStart[l] + q * L.sStride[l];
    fI[k] = i;
    fA[k] = L.fa[i];
    fM[k] = L.fm[i];
    fC[k] = L.fc[i];
  });
  __syncthreads();
  // I1: own cells: face coefficients and x0 to shared memory, r0 = b' - A' x0
  Acc<real> a[4];
#pragma unroll
  for (int k = 0; k < 4; k++) a[k].zero();
  line_grid(no, nown, [&](int32_t k, int32_t q, int32_t l) {
    const int32_t i = fI[q * P + l];
    if (i < 0) return;
    const Cell c = locate<ND>(D, i);
    real pf[NS];
    p_row<real, ND>(c, N, Poff, pf);
    const real xP = x[i];
    real px = 0;
#pragma unroll
    for (int s = 0; s < NS; s++) {
      fPf[s * oc + k] = pf[s];
      if (c.nb[s] >= 0) px += pf[s] * (x[c.nb[s]] - xP);
    }
    fX[k] = xP;
    const real bp = -(b[i] - mb);
    const real rr = bp + px;
    rb[0][i] = rr;
    a[0].add_prod(bp, bp);
    a[1].add_prod(rr, rr);
  });
  if (!plain_sync(X.g)) return false;
  // I2: u0 = M^-1 r0 on the local lines, w0 = A' u0 on the own cells
  {
    const real* __restrict__ r0 = rb[0];
    line_grid(nl, nslot, [&](int32_t, int32_t q, int32_t l) {
      const int32_t k = q * P + l, i = fI[k];
      if (i < 0) return;
      const real rr = r0[i];
      fB[k] = fM[k] * rr;
      fR[k] = rr;
    });
  }
  line_solve<real>(fA, fB, fC, sLen, nl, P);
  // w = A' u on the own cells from the solved lines, (r, u) and (w, u)
  auto own_apply = [&](real* __restrict__ w_o, Acc<real>& ru, Acc<real>& wu) {
    line_grid(no, nown, [&](int32_t k, int32_t q, int32_t l) {
      const int32_t sk = q * P + l, i = fI[sk];
      if (i < 0) return;
      const real uP = fB[sk];
      real ww = 0;
#pragma unroll
      for (int s = 0; s < NS; s++) {
        const int32_t nk = fNb[s * oc + k];
        if (nk >= 0) ww += fPf[s * oc + k] * (uP - fB[nk]);
      }
      w_o[i] = ww;
      fW[k] = ww;
      ru.add_prod(fR[sk], uP);
      wu.add_prod(ww, uP);
    });
  };
  own_apply(wb[0], a[2], a[3]);
  {
    const bool ok = reduce_sync<real, 4>(
        X.g, a, [&](const double* q) { line_cg_start<real>(cs, q, rtol, atol, X.g.status); });
    if (!ok) return false;
  }
  int cur = 0;
  while (cs.active && cs.it < maxit) {
    Acc<real> c3[3];
    c3[0].zero();
    c3[1].zero();
    c3[2].zero();
    const real al = pick<real>(cs.alpha, cs.alpha_f), be = pick<real>(cs.beta, cs.beta_f);
    const int first = cs.first;
    const real* __restrict__ w_i = wb[cur];
    real* __restrict__ w_n = wb[cur ^ 1];
    const Group& g = X.g;
    PISO_STAMP(g.epoch, 4);
    // s = w + beta s, r -= alpha s and the line right-hand sides on every local
    // line (r and s from shared memory; w from the own cells' shared copy or,
    // on halo lines, from its owner's global row); p and x on the own cells.
    // Four slots per pass, all their global loads issued before the first use.
    auto stage = [&](int32_t sk, int32_t q, int32_t l, int32_t i, real wO) {
      const real sv = first ? wO : wO + be * fS[sk];
      const real rr = fR[sk] - al * sv;
      if (l < no) {      // the own slot still holds u of the last line solve
        const int32_t ko = q * no + l;
        const real p = first ? fB[sk] : fB[sk] + be * fP[ko];
        const real xn = fX[ko] + al * p;
        fP[ko] = p;
        fX[ko] = xn;
        x[i] = xn;      // complete at every barrier: the caller reads x at the neighbours right after the solve
        c3[2].add_prod(rr, rr);
      }
      fS[sk] = sv;
      fR[sk] = rr;
      fB[sk] = fM[sk] * rr;
    };
    {
      GridWalk gw(nl);
      for (int32_t k = threadIdx.x; k < nslot; k += 4 * (int32_t)blockDim.x) {
        int32_t qq[4], ll[4], ii[4];
        real ww[4];
#pragma unroll
        for (int j = 0; j < 4; j++) {
          qq[j] = gw.q;
          ll[j] = gw.l;
          gw.next();
          ii[j] = k + j * (int32_t)blockDim.x < nslot ? fI[qq[j] * P + ll[j]] : -1;
          ww[j] = 0;
          if (ii[j] >= 0) ww[j] = ll[j] < no ? fW[qq[j] * no + ll[j]] : w_i[ii[j]];
        }
#pragma unroll
        for (int j = 0; j < 4; j++)
          if (ii[j] >= 0) stage(qq[j] * P + ll[j], qq[j], ll[j], ii[j], ww[j]);
      }
    }
    PISO_TRACE_SYNC();
    PISO_STAMP(g.epoch, 5);
    line_solve<real>(fA, fB, fC, sLen, nl, P);
    PISO_STAMP(g.epoch, 6);
    own_apply(w_n, c3[0], c3[1]);
    PISO_TRACE_SYNC();
    PISO_STAMP(g.epoch, 7);
    bool ok;
    if constexpr (sizeof(real) == 4)
      ok = reduce_sync<real, 3, true>(X.g, c3, [&](const double* q) {
        cg_iter_update_f2(cs, f2_unpack(q[0]), f2_unpack(q[1]), f2_unpack(q[2]), stall_window, X.g.status);
      });
    else
      ok = reduce_sync<real, 3>(
          X.g, c3, [&](const double* q) { cg_iter_update(cs, q[0], q[1], q[2], stall_window, X.g.status); });
    if (!ok) return false;
    cur ^= 1;
  }
  if (sizeof(real) == 4 && threadIdx.x == 0) cs.res2 = f2_to_double(cs.fres2);
  return true;
}

}  // namespace piso
