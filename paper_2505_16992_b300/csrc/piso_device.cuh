// Device-side building blocks of the persistent PISO kernels (sm_103a).
//
// A launch runs one or more *groups*; a group is one simulation domain (the
// multi-block grid of Sec. 2.2 of arXiv:2505.16992) owned by a contiguous set
// of co-resident CTAs.  Each CTA of a group owns a contiguous range of the
// domain's cells and walks the whole PISO step phase by phase; phases are
// separated by a group-wide barrier with a bounded wait, and every Krylov dot
// product is reduced deterministically (fixed tree, fixed order, no float
// atomics), so reruns are bit-identical and every CTA of a group takes the same
// control-flow decisions from the same reduced scalars.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#define PISO_ERR_NOCONV_ADV 1
#define PISO_ERR_NOCONV_P 2
#define PISO_ERR_BREAKDOWN 4
#define PISO_ERR_NAN 8
#define PISO_ERR_TIMEOUT 16

namespace piso {

constexpr int MAXB = 16;     // blocks per domain
constexpr int NSMAX = 12;    // scalars per reduction
constexpr int MAXG = 128;    // groups (domains) per launch
constexpr int MAXW = 32;     // warps per CTA
constexpr int MAXCTA = 1024; // CTAs per group (size of the partials rows)

// ---------------------------------------------------------------------------
// division by a run-time invariant (Granlund & Montgomery 1994, round-up
// multiplier): q = (umulhi(n, m) + n) >> s, valid for n, d < 2^31.
// ---------------------------------------------------------------------------
struct FastDiv {
  uint32_t m, s;
};

__host__ __device__ inline uint32_t fast_div(uint32_t n, FastDiv f) {
#ifdef __CUDA_ARCH__
  uint32_t t = __umulhi(n, f.m);
#else
  uint32_t t = (uint32_t)(((uint64_t)n * f.m) >> 32);
#endif
  return (t + n) >> f.s;
}

inline FastDiv make_fast_div(uint32_t d) {
  uint32_t s = 0;
  while ((1ull << s) < d) s++;
  uint64_t m = (((1ull << 32) * ((1ull << s) - d)) / d) + 1;
  return FastDiv{(uint32_t)m, s};
}

// ---------------------------------------------------------------------------
// static description of one domain (uploaded once at finalize)
// ---------------------------------------------------------------------------
struct BlockInfo {
  int32_t nx, ny, nz, off;   // resolution and first cell (domain index)
  int32_t link[6];           // >= 0: block joined at this side; -1: boundary faces
  int8_t lside[6];           // the joined block's side (the opposite side for a plain joint)
  int8_t lperm[6];           // 1: the side's two tangential axes run along the other side's in exchanged order
  int8_t lflip[6];           // bit i: the side's i-th tangential axis (ascending) runs reversed
  int8_t lplain[6];          // 1: a plain joint (opposite side of the same axis, no exchange, no reversal)
  int32_t bfo[6];            // first boundary face of this side (when link < 0)
  FastDiv dnx, dny;
  int32_t line0;             // first y-line of this block in the domain's line numbering
};

struct DomStatic {
  int32_t ndim, nblocks, N, nbf;
  int32_t n_out;             // number of advective-outflow faces
  int32_t nlines, lmax;      // y-lines (one per block column) and the longest line's length
  int32_t vec4;              // 1: every block's nx is a multiple of 4 and every joint is plain, so four
                             // cells (4m .. 4m+3) always share block, row and the layout of their y/z
                             // neighbours, and [comp][N] arrays hold them in one aligned 4-vector
  BlockInfo blk[MAXB];
  // per-cell metrics, storage precision (void*: float or double)
  const void* J;             // [N]
  const void* T;             // [d*d][N], T[(j*d+k)*N + i] = d xi^j / d x_k
  const void* alpha;         // [d][N]  alpha_jj = J T_j . T_j
  const void* Gx;            // [d(d-1)/2][N] cross metrics alpha_jk, j < k, pairs (0,1) (0,2) (1,2); null
                             // on orthogonal meshes
  const int16_t* nbfr;       // [2d][N] frame of the neighbour across each side (see fr_ax), or null when
                             // every joint is plain (then every frame is the identity)
  // boundary faces
  const int32_t* bf_cell;    // [nbf] adjacent cell
  const int8_t* bf_side;     // [nbf] side of that cell
  const int8_t* bf_out;      // [nbf] 1 if advective outflow
  const void* bf_um;         // [d][nbf] outflow characteristic velocity (0 elsewhere)
};

// ---------------------------------------------------------------------------
// cell location and neighbour lookup (App. A.3: a connection only changes the
// neighbour lookup).  Neighbour >= 0 is a cell of the domain; a negative value
// -1-f names boundary face f.
// ---------------------------------------------------------------------------
struct Cell {
  int32_t i, b, x, y, z;
  int32_t nb[6];
};

// The neighbour of cell (x, y, z) of block B across side s when that side is
// joined to side lside of block O with its tangential axes exchanged (lperm)
// and/or reversed (lflip): the tangential coordinates carried over, the
// normal one at O's side.
__host__ __device__ inline int32_t joint_nbr(const BlockInfo& B, const BlockInfo& O, int32_t x, int32_t y, int32_t z,
                                             int s) {
  const int j = s >> 1, so = B.lside[s], jo = so >> 1;
  const int32_t c[3] = {x, y, z};
  const int32_t nb_[3] = {B.nx, B.ny, B.nz};
  const int32_t no[3] = {O.nx, O.ny, O.nz};
  int32_t oc[3] = {0, 0, 0};
  int ta[2] = {0, 0}, tb[2] = {0, 0}, n = 0, m = 0;
  for (int a = 0; a < 3; a++) {
    if (a != j) ta[n++] = a;
    if (a != jo) tb[m++] = a;
  }
  oc[jo] = (so & 1) ? no[jo] - 1 : 0;
  for (int i = 0; i < 2; i++) {
    int32_t v = c[ta[i]];
    if ((B.lflip[s] >> i) & 1) v = nb_[ta[i]] - 1 - v;
    oc[tb[B.lperm[s] ? 1 - i : i]] = v;
  }
  return O.off + oc[0] + O.nx * (oc[1] + O.ny * oc[2]);
}

__host__ __device__ __forceinline__ int32_t side_nbr(const DomStatic& D, const BlockInfo& B, int32_t i,
                                            int32_t x, int32_t y, int32_t z, int s) {
  switch (s) {
    case 0: if (x > 0) return i - 1; break;
    case 1: if (x < B.nx - 1) return i + 1; break;
    case 2: if (y > 0) return i - B.nx; break;
    case 3: if (y < B.ny - 1) return i + B.nx; break;
    case 4: if (z > 0) return i - B.nx * B.ny; break;
    default: if (z < B.nz - 1) return i + B.nx * B.ny; break;
  }
  const int32_t t = B.link[s];
  if (t >= 0) {
    const BlockInfo& O = D.blk[t];
    if (!B.lplain[s]) return joint_nbr(B, O, x, y, z, s);
    switch (s) {
      case 0: return O.off + (O.nx - 1) + O.nx * (y + O.ny * z);
      case 1: return O.off + O.nx * (y + O.ny * z);
      case 2: return O.off + x + O.nx * ((O.ny - 1) + O.ny * z);
      case 3: return O.off + x + O.nx * (O.ny * z);
      case 4: return O.off + x + O.nx * (y + O.ny * (O.nz - 1));
      default: return O.off + x + O.nx * y;
    }
  }
  int32_t f;
  if (s < 2) f = y + B.ny * z;
  else if (s < 4) f = x + B.nx * z;
  else f = x + B.nx * y;
  return -1 - (B.bfo[s] + f);
}

template <int ND>
__host__ __device__ __forceinline__ Cell locate(const DomStatic& D, int32_t i) {
  Cell c;
  c.i = i;
  int b = 0;
  while (b + 1 < D.nblocks && i >= D.blk[b + 1].off) b++;
  const BlockInfo& B = D.blk[b];
  c.b = b;
  const uint32_t li = (uint32_t)(i - B.off);
  const uint32_t q = fast_div(li, B.dnx);
  c.x = (int32_t)(li - q * (uint32_t)B.nx);
  if (ND == 3) {
    const uint32_t zz = fast_div(q, B.dny);
    c.z = (int32_t)zz;
    c.y = (int32_t)(q - zz * (uint32_t)B.ny);
  } else {
    c.y = (int32_t)q;
    c.z = 0;
  }
#pragma unroll
  for (int s = 0; s < 2 * ND; s++) c.nb[s] = side_nbr(D, B, i, c.x, c.y, c.z, s);
  return c;
}

__device__ __forceinline__ int32_t safe(int32_t nb, int32_t self) { return nb >= 0 ? nb : self; }

// Frame of the neighbour across a side (joints with exchanged or reversed
// axes; App. A.3: a connection only changes the neighbour lookup, but the
// neighbour's per-axis quantities are in its own frame).  A code holds, for
// each axis a of the cell, the neighbour's axis (2 bits at 2a) and whether it
// runs reversed (bit 6 + a); FRAME_ID is the identity.
constexpr int FRAME_ID = 0x24;
__host__ __device__ __forceinline__ int fr_ax(int code, int a) { return (code >> (2 * a)) & 3; }
__host__ __device__ __forceinline__ int fr_neg(int code, int a) { return (code >> (6 + a)) & 1; }
// the neighbour's side that faces the cell, for the cell's side s
__host__ __device__ __forceinline__ int fr_ret(int code, int s) {
  return 2 * fr_ax(code, s >> 1) + (((s & 1) == fr_neg(code, s >> 1)) ? 1 : 0);
}
__device__ __forceinline__ int fr_code(const int16_t* fr, int32_t N, int s, int32_t i) {
  return fr ? (int)fr[(size_t)s * N + i] : FRAME_ID;
}

// Lines of the y-line preconditioner: the cells of one block that share x (and
// z), in order of y.  Line l of block b (l' = l - line0) starts at x = l' mod nx,
// z = l' / nx, y = 0, with stride nx and ny cells; consecutive lines are
// x-neighbours, so a warp that takes one cell of each of 32 consecutive lines
// at the same y reads contiguous memory.
struct LineDesc {
  int32_t start, stride, len;
};

__host__ __device__ __forceinline__ LineDesc line_desc(const DomStatic& D, int32_t l) {
  int b = 0;
  while (b + 1 < D.nblocks && l >= D.blk[b + 1].line0) b++;
  const BlockInfo& B = D.blk[b];
  const uint32_t lp = (uint32_t)(l - B.line0);
  const uint32_t z = fast_div(lp, B.dnx);
  const uint32_t x = lp - z * (uint32_t)B.nx;
  return LineDesc{B.off + (int32_t)x + B.nx * B.ny * (int32_t)z, B.nx, B.ny};
}

// The line holding a located cell (the inverse of line_desc; the cell's y is
// its position along the line).
__host__ __device__ __forceinline__ int32_t line_of(const DomStatic& D, const Cell& c) {
  const BlockInfo& B = D.blk[c.b];
  return B.line0 + c.x + B.nx * c.z;
}

// Per-CTA state of the y-line preconditioner: the Thomas factors of the line
// blocks of -P (device arrays), this CTA's lines [L0, L1), and its shared
// staging area (lb lines per batch).
template <typename real>
struct LinePre {
  real* fa;          // [N] forward multiplier  -e_{y-1} m_y
  real* fm;          // [N] pivot reciprocal     m_y
  real* fc;          // [N] backward multiplier -c'_y
  real* sA;          // shared staging arrays of line_cap reals each
  real* sB;
  real* sC;
  real* sR;
  int32_t* sStart;   // shared line descriptors of the current batch
  int32_t* sStride;
  int32_t* sLen;
  int32_t L0, L1, lb;
  // fused iteration (one group barrier per CG iteration), when this launch has
  // a plan for it, else fl == nullptr: the CTA's local lines (n_own own lines,
  // then the halo lines that hold its cells' other neighbours), the
  // neighbour slots of its own cells ([2 ND][own_cap], -1: boundary face) and
  // the shared arrays of the fused solve (they alias the staging arrays)
  const int32_t* fl;
  const int16_t* fnb;
  int32_t n_own, n_loc, own_cap, slot_cap;
  real *fA, *fC, *fM, *fB, *fR, *fS;   // [slot_cap]: fa, fc, fm, line right-hand side / solution, r, s
  real *fP, *fX, *fW, *fPf;       // [own_cap]: p, x, w of the own cells; [2 ND][own_cap] face coefficients
  int32_t* fI;                    // [slot_cap] cell of each slot, -1 past the end of its line
  int16_t* fNb;                   // [2 ND][own_cap] neighbour slots in shared memory
};

// ---------------------------------------------------------------------------
// accumulators: FP64 mode sums in double; the FP32 mode sums in a float pair
// (TwoSum / FMA-TwoProd, Knuth and Dekker), which carries ~48 significant bits
// on the FP32 pipe (B300's FP64 pipe is a small fraction of its FP32 rate).
// ---------------------------------------------------------------------------
struct f2 {
  float hi, lo;
};

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

__device__ __forceinline__ f2 f2_add(f2 a, f2 b) {
  float s, e;
  two_sum(a.hi, b.hi, s, e);
  e += a.lo + b.lo;
  f2 r;
  two_sum(s, e, r.hi, r.lo);
  return r;
}

// Float-pair (double-word) operations for the FP32 mode's Krylov scalars, so
// thread 0's per-iteration update stays on the FP32 pipe (an FP64 instruction
// issues at ~64 cycles per warp on this GPU).  The product follows Dekker's
// double-length multiplication with an FMA for the exact partial product, the
// quotient one correction step q1 + (a - q1 b) / b with both partial quotients
// taken against the rounded reciprocal of b.hi; relative accuracy ~2^-44.
__device__ __forceinline__ f2 f2_norm(float s, float e) {   // fast two-sum, |s| >= |e|
  f2 r;
  r.hi = s + e;
  r.lo = e - (r.hi - s);
  return r;
}
__device__ __forceinline__ f2 f2_neg(f2 a) { return f2{-a.hi, -a.lo}; }
__device__ __forceinline__ f2 f2_mul(f2 a, f2 b) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  return f2_norm(p, e);
}
__device__ __forceinline__ f2 f2_div(f2 a, f2 b) {
  const float rb = __frcp_rn(b.hi);   // one reciprocal for both partial quotients
  const float q1 = a.hi * rb;
  const f2 r = f2_add(a, f2_neg(f2_mul(f2{q1, 0.f}, b)));
  return f2_norm(q1, r.hi * rb);
}
__device__ __forceinline__ bool f2_gt(f2 a, f2 b) { return a.hi > b.hi || (a.hi == b.hi && a.lo > b.lo); }
__device__ __forceinline__ f2 f2_from_double(double d) {
  f2 r;
  r.hi = (float)d;
  r.lo = (float)(d - (double)r.hi);
  return r;
}
__device__ __forceinline__ double f2_to_double(f2 a) { return (double)a.hi + (double)a.lo; }
// unpack a float pair transported in the bits of a double (Acc<float>::pack)
__device__ __forceinline__ f2 f2_unpack(double w) {
  return f2{__int_as_float(__double2hiint(w)), __int_as_float(__double2loint(w))};
}

template <typename real>
struct Acc;

template <>
struct Acc<double> {
  double v;
  __device__ __forceinline__ void zero() { v = 0.0; }
  __device__ __forceinline__ void add_prod(double a, double b) { v = fma(a, b, v); }
  __device__ __forceinline__ void add(double a) { v += a; }
  __device__ __forceinline__ void shfl_down_add(int off) { v += __shfl_down_sync(0xffffffffu, v, off); }
  __device__ __forceinline__ double to_double() const { return v; }
  __device__ __forceinline__ double pack() const { return v; }
  __device__ __forceinline__ void unpack_add(double w) { v += w; }
};

template <>
struct Acc<float> {
  // Per-thread sums in the form of Ogita, Rump and Oishi's Dot2 (2005): v.hi is
  // the running float sum, v.lo collects the exact rounding errors of the
  // products (FMA) and of the additions (TwoSum) without renormalising, which
  // gives the accuracy of a doubled-precision dot product at ~10 FP32
  // operations per term; the pair is normalised when partial sums are combined.
  f2 v;
  __device__ __forceinline__ void zero() { v.hi = 0.f; v.lo = 0.f; }
  __device__ __forceinline__ void add_prod(float a, float b) {
    const float p = a * b;
    const float pe = fmaf(a, b, -p);
    float s, e;
    two_sum(v.hi, p, s, e);
    v.hi = s;
    v.lo += e + pe;
  }
  __device__ __forceinline__ void add(float a) {
    float s, e;
    two_sum(v.hi, a, s, e);
    v.hi = s;
    v.lo += e;
  }
  __device__ __forceinline__ void shfl_down_add(int off) {
    f2 o{__shfl_down_sync(0xffffffffu, v.hi, off), __shfl_down_sync(0xffffffffu, v.lo, off)};
    v = f2_add(v, o);
  }
  __device__ __forceinline__ double to_double() const { return (double)v.hi + (double)v.lo; }
  // 8-byte transport of the float pair (no FP64 arithmetic on the way)
  __device__ __forceinline__ double pack() const {
    return __hiloint2double(__float_as_int(v.hi), __float_as_int(v.lo));
  }
  __device__ __forceinline__ void unpack_add(double w) {
    f2 o{__int_as_float(__double2hiint(w)), __int_as_float(__double2loint(w))};
    v = f2_add(v, o);
  }
};

// ---------------------------------------------------------------------------
// group barrier (bounded wait) and deterministic group reductions
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t ld_acquire_u32(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

struct Group {
  uint32_t* bar;        // monotone arrival counter, zeroed before the launch
  double* partials;     // [2][NSMAX][ncta]
  int32_t* status;      // error bits of this group
  int32_t ncta, rank;
  uint32_t epoch;
  uint64_t timeout_ns;
  int32_t withhold;     // fault injection: this CTA skips its first arrival (1) or not (0)
  uint64_t* trace;      // phase-timing ring (PISO_TRACE builds), or nullptr
};

// Optional phase-timing trace (build with -DPISO_TRACE): CTA 0 of the launch
// records globaltimer stamps at four points of every phase boundary - work
// done, partials published, barrier passed, totals gathered - into a ring of
// PISO_TRACE_LEN entries of PISO_TRACE_STAMPS stamps at Group::trace (a device
// buffer the host side owns and passes in with the solver options, so every
// translation unit writes the same buffer); stamps 4.. of an entry mark points
// inside the phase's work (PISO_TRACE_SYNC lines the CTA up before such a
// mark).  Off by default; it changes no computation.
#ifdef PISO_TRACE
constexpr int PISO_TRACE_LEN = 8192;
constexpr int PISO_TRACE_STAMPS = 8;
#define PISO_STAMP(slot, k)                                                   \
  do {                                                                        \
    if (g.trace && blockIdx.x == 0 && threadIdx.x == 0) {                     \
      uint64_t t_;                                                            \
      asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t_));                  \
      g.trace[((slot) % PISO_TRACE_LEN) * PISO_TRACE_STAMPS + (k)] = t_;      \
    }                                                                         \
  } while (0)
#define PISO_TRACE_SYNC() __syncthreads()
#else
#define PISO_STAMP(slot, k) \
  do {                      \
  } while (0)
#define PISO_TRACE_SYNC() \
  do {                    \
  } while (0)
#endif

__device__ __forceinline__ void red_release_add(uint32_t* p, uint32_t v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Arrival and bounded wait of one CTA at barrier g.epoch (called by one thread
// after __syncthreads ordered the CTA's writes).  The release increment makes
// those writes visible to every CTA whose acquire load sees the count.
static __device__ __noinline__ int barrier_arrive_wait(const Group& g) {
  const uint32_t target = g.epoch * (uint32_t)g.ncta;
  if (!(g.withhold && g.epoch == 1)) {
#ifdef PISO_FULL_FENCES
    __threadfence();
    atomicAdd(g.bar, 1u);
#else
    red_release_add(g.bar, 1u);
#endif
  }
  int ok = 1;
  if ((int32_t)(ld_acquire_u32(g.bar) - target) < 0) {
    const uint64_t t0 = global_ns();
    while (true) {
      if ((int32_t)(ld_acquire_u32(g.bar) - target) >= 0) break;
      if (*((volatile int32_t*)g.status) & PISO_ERR_TIMEOUT) { ok = 0; break; }
      if (global_ns() - t0 > g.timeout_ns) {
        atomicOr(g.status, PISO_ERR_TIMEOUT);
        ok = 0;
        break;
      }
    }
  }
#ifdef PISO_FULL_FENCES
  __threadfence();
#endif
  return ok;
}

// One phase boundary with a reduction: block-reduce the NS accumulators,
// publish this CTA's partials, wait at the group barrier, sum the group's
// partials in a fixed order (identical in every CTA) and let thread 0 run
// update(totals) on the shared solver state.  Warp k reduces scalar k, so the
// block- and group-level sums of different scalars proceed in parallel and
// each lane issues all its partial loads before adding.  Returns false when
// the barrier wait ran out.
constexpr int GATHER_UNROLL = 8;

// RAW: hand update() the totals in transport form (Acc::pack: the float pair's
// bits in the FP32 mode) instead of converted to double.
template <typename real, int NS, bool RAW = false, typename F>
__device__ __forceinline__ bool reduce_sync(Group& g, Acc<real> (&a)[NS], F&& update) {
  // each warp folds its lanes down to KEEP partials per scalar (fewer shuffle
  // levels in every warp; the rest is summed by one warp per scalar), at most
  // NSMAX values per warp; each instantiation holds its own shared arrays,
  // sized for its NS (static shared memory of the step kernels 70 -> 53 KB)
  constexpr int KEEP = NS * 4 <= NSMAX ? 4 : (NS * 2 <= NSMAX ? 2 : 1);
  __shared__ double s_w[MAXW * NS * KEEP];
  __shared__ double s_tot[NS];
  __shared__ int s_ok;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int k = 0; k < NS; k++) {
#pragma unroll
    for (int off = 16; off >= KEEP; off >>= 1) a[k].shfl_down_add(off);
    if (lane < KEEP) s_w[(k * MAXW + warp) * KEEP + lane] = a[k].pack();
  }
  __syncthreads();
  PISO_STAMP(g.epoch, 0);
  g.epoch++;
  double* P = g.partials + (size_t)(g.epoch & 1) * NSMAX * g.ncta;
  for (int k = warp; k < NS; k += nw) {
    Acc<real> v;
    v.zero();
    for (int t = lane; t < nw * KEEP; t += 32) v.unpack_add(s_w[k * MAXW * KEEP + t]);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v.shfl_down_add(off);
    if (lane == 0) __stcg(P + (size_t)k * g.ncta + g.rank, v.pack());
  }
  __syncthreads();
  PISO_STAMP(g.epoch - 1, 1);
  if (threadIdx.x == 0) s_ok = barrier_arrive_wait(g);
  PISO_STAMP(g.epoch - 1, 2);
  __syncthreads();
  const int ok = s_ok;
  if (ok) {
    for (int k = warp; k < NS; k += nw) {
      const double* src = P + (size_t)k * g.ncta;
      Acc<real> v;
      v.zero();
      for (int base = 0; base < g.ncta; base += 32 * GATHER_UNROLL) {
        double w[GATHER_UNROLL];
#pragma unroll
        for (int u = 0; u < GATHER_UNROLL; u++) {
          const int c = base + lane + 32 * u;
          w[u] = c < g.ncta ? __ldcg(src + c) : 0.0;
        }
#pragma unroll
        for (int u = 0; u < GATHER_UNROLL; u++)
          if (base + lane + 32 * u < g.ncta) v.unpack_add(w[u]);
      }
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) v.shfl_down_add(off);
      if (lane == 0) s_tot[k] = RAW ? v.pack() : v.to_double();
    }
    __syncthreads();
    if (threadIdx.x == 0) update(s_tot);
  }
  PISO_STAMP(g.epoch - 1, 3);
  __syncthreads();
  return ok != 0;
}

// A phase boundary without a reduction.
__device__ __forceinline__ bool plain_sync(Group& g) {
  __shared__ int s_ok2;
  __syncthreads();
  PISO_STAMP(g.epoch, 0);
  PISO_STAMP(g.epoch, 1);
  g.epoch++;
  if (threadIdx.x == 0) s_ok2 = barrier_arrive_wait(g);
  PISO_STAMP(g.epoch - 1, 2);
  PISO_STAMP(g.epoch - 1, 3);
  __syncthreads();
  return s_ok2 != 0;
}

}  // namespace piso
