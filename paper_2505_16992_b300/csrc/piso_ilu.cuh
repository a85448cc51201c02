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

// Bytes of the fast path's shared memory for n cells of d components (the
// sweep values, the 2d row coefficients and the pivot in the storage type,
// the 2d neighbour positions as int32); the host reserves this much.
__host__ __device__ constexpr size_t ilu_smem_bytes(int nd, size_t n, size_t elem) {
  return (size_t)(3 * nd + 1) * n * elem + (size_t)(2 * nd) * n * sizeof(int32_t);
}

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
__device__ void ilu_factor_levels(const Ctx<real, ND>& X, const IluPre<real>& P, const real* Cdiag,
                                  const real* Coff) {
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
        c_row<real, ND, true>(c, N, Cdiag, Coff, diag, ct, X.fr);
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
      if (m) c_row<real, ND, TR>(c, N, Cdiag, Coff, diag, cf, X.fr);
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
      c_row<real, ND, TR>(c, N, Cdiag, Coff, diag, cf, X.fr);
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

// ---------------------------------------------------------------------------
// Fast path.  When the CTA owns a contiguous range [lo, hi) of n <= blockDim
// cells (its neighbour table is in shared memory), thread t takes the cell at
// position t of the level order for every sweep of the solve.  The sweep
// values (d x n, by cell position i - lo) and that cell's row of the factors
// (2d coefficients and neighbour positions, the reciprocal pivot; by thread t,
// one array per side) are staged in shared memory once per solve, so a level
// step is a few shared-memory loads and one CTA barrier instead of a chain of
// dependent global loads (level bound, cell, mask, row, values).  Only the
// thread's cell, position, level and mask stay in registers.  This code is
// compiled only into the kernels built for the preconditioned solve, so it
// cannot change the register allocation of the plain ones.
template <typename real, int ND>
struct IluSmem {
  real* zv;       // [ND][n]  sweep values by cell position
  real* rc;       // [2ND][n] row coefficients by thread
  real* rd;       // [n]      reciprocal pivot by thread
  int32_t* rl;    // [2ND][n] neighbour position by thread
  int32_t n;      // 0: no fast path
};

template <typename real, int ND>
struct IluRow {
  int32_t i;      // cell, -1 for a thread without one
  int32_t self;   // its position i - lo
  int32_t lvl;    // its level, -1 for a thread without a cell
  uint32_t m;     // in-block mask (bit s: lower neighbour, bit 8 + s: upper)
};

// The fast path's shared memory, or n = 0 without one.
template <typename real, int ND>
__device__ __forceinline__ IluSmem<real, ND> ilu_smem(const Ctx<real, ND>& X, const SolverOpts& o) {
  extern __shared__ int32_t s_nbt[];
  IluSmem<real, ND> S{};
  if (o.ilu_soff < 0 || X.nbt == nullptr || X.hi - X.lo > (int32_t)blockDim.x) return S;
  const int32_t n = X.hi - X.lo;
  real* b = reinterpret_cast<real*>(reinterpret_cast<char*>(s_nbt) + o.ilu_soff);
  S.zv = b;
  S.rc = b + (size_t)ND * n;
  S.rd = b + (size_t)3 * ND * n;
  S.rl = reinterpret_cast<int32_t*>(b + (size_t)(3 * ND + 1) * n);
  S.n = n;
  return S;
}

// The level l with ls[l] <= t < ls[l + 1] (ls[0] = 0 <= t < ls[nlev]).
template <typename real>
__device__ __forceinline__ int32_t ilu_level_of(const IluPre<real>& P, int32_t t) {
  int32_t a = 0, b = P.nlev;
  while (b - a > 1) {
    const int32_t c = (a + b) >> 1;
    if (P.ls[c] <= t) a = c;
    else b = c;
  }
  return a;
}

template <typename real, int ND>
__device__ __forceinline__ IluRow<real, ND> ilu_row_of(const Ctx<real, ND>& X, const IluPre<real>& P) {
  IluRow<real, ND> R;
  const int32_t t = (int32_t)threadIdx.x;
  R.i = -1;
  R.self = 0;
  R.lvl = -1;
  R.m = 0;
  if (t < X.hi - X.lo) {
    R.i = P.ord[t];
    R.self = R.i - X.lo;
    R.lvl = ilu_level_of(P, t);
    R.m = P.mask[R.i];
  }
  return R;
}

// Stage this thread's row of M (C or C^T) and its pivot (after the pivots
// are formed).
template <typename real, int ND, bool TR>
__device__ __forceinline__ void ilu_stage_rows(const Ctx<real, ND>& X, const IluPre<real>& P, const real* Cdiag,
                                               const real* Coff, const IluRow<real, ND>& R,
                                               const IluSmem<real, ND>& S) {
  const int32_t t = (int32_t)threadIdx.x;
  if (R.i >= 0) {
    const Cell c = X.cell(R.i);
    real diag, cf[2 * ND];
    c_row<real, ND, TR>(c, X.N, Cdiag, Coff, diag, cf, X.fr);
#pragma unroll
    for (int s = 0; s < 2 * ND; s++) {
      const bool in = ((R.m >> s) | (R.m >> (8 + s))) & 1u;
      S.rc[s * S.n + t] = in ? cf[s] : real(0);
      S.rl[s * S.n + t] = in ? c.nb[s] - X.lo : 0;
    }
    S.rd[t] = P.dinv[R.i];
  }
  __syncthreads();
}

// Pivots, fast path.  Same arithmetic, in the same order, as
// ilu_factor_levels: d_i = c_ii - sum (c_ik c_ki) / d_k.
template <typename real, int ND>
__device__ void ilu_factor_fast(const Ctx<real, ND>& X, const IluPre<real>& P, const real* Cdiag, const real* Coff,
                                const IluSmem<real, ND>& S) {
  const IluRow<real, ND> R = ilu_row_of<real, ND>(X, P);
  const int32_t t = (int32_t)threadIdx.x, n = S.n;
  const uint32_t m = R.m & 0xffu;
  __syncthreads();   // the staging area may still be read by an earlier solve
  if (R.i >= 0) {
    const Cell c = X.cell(R.i);
    real diag, cf[2 * ND], ct[2 * ND];
    c_row<real, ND, false>(c, X.N, Cdiag, Coff, diag, cf);
    c_row<real, ND, true>(c, X.N, Cdiag, Coff, diag, ct, X.fr);
#pragma unroll
    for (int s = 0; s < 2 * ND; s++) {
      S.rc[s * n + t] = ((m >> s) & 1u) ? cf[s] * ct[s] : real(0);
      S.rl[s * n + t] = ((m >> s) & 1u) ? c.nb[s] - X.lo : 0;
    }
    S.rd[t] = diag;
  }
  __syncthreads();
  for (int l = 0; l < P.nlev; l++) {
    if (R.lvl == l) {
      const real diag = S.rd[t];
      real d = diag;
#pragma unroll
      for (int s = 0; s < 2 * ND; s++)
        if ((m >> s) & 1u) d -= S.rc[s * n + t] * S.zv[S.rl[s * n + t]];
      if (!(d > real(1e-5) * diag)) d = diag;
      S.zv[R.self] = real(1) / d;
    }
    __syncthreads();
  }
  if (R.i >= 0) P.dinv[R.i] = S.zv[R.self];
  __syncthreads();
}

// z = M^-1 w, fast path: the source values are staged first (one load round
// trip for all cells), then the sweeps of ilu_apply run on shared memory and
// the CTA's values are stored to z.  Rows staged by ilu_stage_rows.
template <typename real, int ND, typename SRC>
__device__ __forceinline__ void ilu_apply_fast(const Ctx<real, ND>& X, const IluPre<real>& P,
                                               const IluRow<real, ND>& R, const IluSmem<real, ND>& S,
                                               const int (&act)[ND], SRC&& src, real* z) {
  const int32_t N = X.N, n = S.n, t = (int32_t)threadIdx.x;
  __syncthreads();
  if (R.i >= 0) {
#pragma unroll
    for (int k = 0; k < ND; k++)
      if (act[k]) S.zv[k * n + R.self] = src(k, R.i);
  }
  __syncthreads();
  for (int l = 0; l < P.nlev; l++) {
    if (R.lvl == l) {
      const real di = S.rd[t];
#pragma unroll
      for (int k = 0; k < ND; k++) {
        if (!act[k]) continue;
        real w = S.zv[k * n + R.self];
#pragma unroll
        for (int s = 0; s < 2 * ND; s++)
          if ((R.m >> s) & 1u) w -= S.rc[s * n + t] * S.zv[k * n + S.rl[s * n + t]];
        S.zv[k * n + R.self] = w * di;
      }
    }
    __syncthreads();
  }
  for (int l = P.nlev - 1; l >= 0; l--) {
    if (R.lvl == l && (R.m >> 8)) {
      const real di = S.rd[t];
#pragma unroll
      for (int k = 0; k < ND; k++) {
        if (!act[k]) continue;
        real acc = 0;
#pragma unroll
        for (int s = 0; s < 2 * ND; s++)
          if ((R.m >> (8 + s)) & 1u) acc += S.rc[s * n + t] * S.zv[k * n + S.rl[s * n + t]];
        S.zv[k * n + R.self] -= di * acc;
      }
    }
    __syncthreads();
  }
  if (R.i >= 0) {
#pragma unroll
    for (int k = 0; k < ND; k++)
      if (act[k]) z[(size_t)k * N + R.i] = S.zv[k * n + R.self];
  }
}

// Pivots of this CTA's block: the shared-memory sweep when S is set up.
template <typename real, int ND>
__device__ void ilu_factor(const Ctx<real, ND>& X, const IluPre<real>& P, const real* Cdiag, const real* Coff,
                           const IluSmem<real, ND>& S) {
  if (S.n) ilu_factor_fast<real, ND>(X, P, Cdiag, Coff, S);
  else ilu_factor_levels<real, ND>(X, P, Cdiag, Coff);
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
                             real* v, real* y, real* z, real* t, const IluSmem<real, ND>& S) {
  const int32_t N = X.N;
  IluRow<real, ND> R{};
  if (S.n) {
    R = ilu_row_of<real, ND>(X, P);
    ilu_stage_rows<real, ND, TR>(X, P, Cdiag, Coff, R, S);
  }
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
      auto src = [&](int k, int32_t i) -> real {
        const size_t o_ = (size_t)k * N + i;
        const real pn = first ? r[o_] : r[o_] + beta[k] * (p[o_] - om[k] * v[o_]);
        p[o_] = pn;
        return pn;
      };
      if (S.n) ilu_apply_fast<real, ND>(X, P, R, S, act, src, y);
      else ilu_apply<real, ND, TR>(X, P, Cdiag, Coff, act, src, y);
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
        c_row<real, ND, TR>(c, N, Cdiag, Coff, diag, cf, X.fr);
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
      auto src = [&](int k, int32_t i) -> real {
        const size_t o_ = (size_t)k * N + i;
        return r[o_] - al[k] * v[o_];
      };
      if (S.n) ilu_apply_fast<real, ND>(X, P, R, S, act, src, z);
      else ilu_apply<real, ND, TR>(X, P, Cdiag, Coff, act, src, z);
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
        c_row<real, ND, TR>(c, N, Cdiag, Coff, diag, cf, X.fr);
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
