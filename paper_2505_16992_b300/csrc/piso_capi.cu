// Host side of the PISO library: domain description, metrics and connection
// tables (App. A.2-A.3 and A.5 of arXiv:2505.16992), device workspace, launch
// configuration and the C ABI declared in include/piso.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include <map>
#include <tuple>

#include "../../include/piso.h"
#include "piso_adjoint.cuh"
#include "piso_forward.cuh"
#include "piso_stats.cuh"

using namespace piso;

// The step kernels live in translation units of their own
// (piso_kernels_{fwd,adj}_{f32,f64}.cu, built in parallel); these return the
// address of one instantiation (wide: the 768-thread variant).
namespace piso {
const void* fwd_kernel_addr_f32(int nd, bool wide, int mode);
const void* fwd_kernel_addr_f64(int nd, bool wide, int mode);
const void* adj_kernel_addr_f32(int nd, bool wide, int mode);
const void* adj_kernel_addr_f64(int nd, bool wide, int mode);
}  // namespace piso

namespace {

thread_local std::string g_create_error;

struct SideSpec {
  int kind = 0;            // 0 none, 1 connection, 2 dirichlet, 3 outflow
  int other = -1, other_side = -1;
  int perm = 0, flip = 0;  // connection: tangential axes exchanged / reversed (bit i: this side's axis i)
  std::vector<double> values;   // [face][ndim]
  double um[3] = {0, 0, 0};
};

struct HostBlock {
  int res[3];
  std::vector<double> vertices;
  SideSpec side[6];
};

struct Arena {
  char* base = nullptr;
  size_t size = 0, used = 0;
  void* take(size_t bytes) {
    size_t off = (used + 255) & ~size_t(255);
    used = off + bytes;
    return base ? base + off : nullptr;
  }
};

}  // namespace

struct piso_domain {
  int ndim = 2, prec = 0;
  bool finalized = false;
  std::vector<HostBlock> blocks;
  piso_options opts;
  std::string err;
  // sizes
  int32_t N = 0, nbf = 0, n_out = 0;
  size_t elem = 8;
  // device
  char* dmem = nullptr;
  size_t dmem_bytes = 0;
  DomStatic* d_static = nullptr;
  void* J = nullptr;
  void* T = nullptr;
  void* alpha = nullptr;
  int32_t* bf_cell = nullptr;
  int8_t* bf_side = nullptr;
  int8_t* bf_out = nullptr;
  void* bf_um = nullptr;
  void* bval = nullptr;
  void* gbval = nullptr;       // [d][nbf] dL/d(boundary values) of the last adjoint
  // workspace arrays (element pointers)
  void* ws[64] = {nullptr};
  void* tape_ws = nullptr;     // internal tape (last step)
  bool tape_ws_valid = false;  // tape_ws holds the record of the domain's last forward step (that step was a
                               // piso_step or batch step without a caller tape)
  uint32_t* bar = nullptr;
  double* partials = nullptr;
  int32_t* status = nullptr;
  int32_t* istats = nullptr;
  double* dstats = nullptr;
  double* d_dnu = nullptr;
  // pinned readback
  int32_t* h_status = nullptr;
  int32_t* h_istats = nullptr;
  double* h_dstats = nullptr;
  double* h_dnu = nullptr;
  // launch shape
  int threads = 512, ncta = 1;
  int sms = 148;
  DomStatic h_static;
  double aniso = 1.0;          // max over cells of alpha_yy / alpha_kk (k != y): y-anisotropy of the grid
  int p_line = 0;              // the pressure CG uses the y-line preconditioner
  // ILU(0) tables of the BiCGStab preconditioner for the current launch layout
  void* ilu_buf = nullptr;
  IluTab ilu_tab{};
  bool ilu_ready = false;      // tables match (ncta, threads, ownership) of the launches
  int ilu_key[3] = {-1, -1, -1};
  // plan of the fused y-line CG iteration for the current CTA count
  void* lf_buf = nullptr;
  bool lf_ready = false;
  int lf_ncta = -1;
  int32_t lf_own_cap = 0, lf_slot_cap = 0, lf_bytes = 0;
  const int32_t* lf_off = nullptr;
  const int32_t* lf_nown = nullptr;
  const int32_t* lf_lines = nullptr;
  const int16_t* lf_nbs = nullptr;
  bool has_cross = false;      // some cell has non-zero cross metrics (accepted with n_nonortho >= 1)
  bool twisted = false;        // some joint exchanges or reverses axes (neighbour frames are stored)
  int16_t* nbfr = nullptr;     // [2d][N] neighbour frames on the device (twisted domains)
  void* gx = nullptr;          // [d(d-1)/2][N] cross metrics on the device
  bool pending = false;
  cudaStream_t pending_stream = nullptr;
  int pending_kind = 0;        // 1 forward, 2 adjoint
};

struct piso_batch {
  std::vector<piso_domain*> doms;
  piso_options opts;
  int total_cta = 0;
  std::vector<int32_t> cta_first;
  int32_t* d_cta_first = nullptr;
  size_t call_bytes = 0;       // bytes of one group's call record (the larger of forward and adjoint)
  int mode = 0;                // kernel instantiation: 0 plain, 2 when a member is non-orthogonal
  std::vector<double> weights; // measured work per member (piso_batch_autotune), or empty: the estimate
  void* dev = nullptr;         // piso_batch_dev: device and pinned buffers of the batch launches
  std::string err;
};

namespace {

piso_status fail(piso_domain* d, piso_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (d) d->err = buf;
  else g_create_error = buf;
  return s;
}

#define CUDA_TRY(d, call)                                                              \
  do {                                                                                 \
    cudaError_t e_ = (call);                                                           \
    if (e_ != cudaSuccess)                                                             \
      return fail(d, PISO_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_));      \
  } while (0)

int side_nfaces(const int* r, int s, int nd) {
  int ax = s / 2;
  if (nd == 2) return ax == 0 ? r[1] : r[0];
  if (ax == 0) return r[1] * r[2];
  if (ax == 1) return r[0] * r[2];
  return r[0] * r[1];
}

// d x / d xi at a cell centre from opposite face-centre differences.
void cell_jacobian(const HostBlock& b, int nd, int x, int y, int z, double M[3][3]) {
  const int nx = b.res[0], ny = b.res[1];
  auto V = [&](int i, int j, int k, int c) -> double {
    return b.vertices[((size_t)(k * (ny + 1) + j) * (nx + 1) + i) * nd + c];
  };
  for (int a = 0; a < 3; a++)
    for (int c = 0; c < 3; c++) M[a][c] = (a == c) ? 1.0 : 0.0;
  if (nd == 2) {
    for (int c = 0; c < 2; c++) {
      double fxm = 0.5 * (V(x, y, 0, c) + V(x, y + 1, 0, c));
      double fxp = 0.5 * (V(x + 1, y, 0, c) + V(x + 1, y + 1, 0, c));
      double fym = 0.5 * (V(x, y, 0, c) + V(x + 1, y, 0, c));
      double fyp = 0.5 * (V(x, y + 1, 0, c) + V(x + 1, y + 1, 0, c));
      M[c][0] = fxp - fxm;
      M[c][1] = fyp - fym;
    }
    return;
  }
  for (int c = 0; c < 3; c++) {
    double fxm = 0.25 * (V(x, y, z, c) + V(x, y + 1, z, c) + V(x, y, z + 1, c) + V(x, y + 1, z + 1, c));
    double fxp = 0.25 * (V(x + 1, y, z, c) + V(x + 1, y + 1, z, c) + V(x + 1, y, z + 1, c) +
                         V(x + 1, y + 1, z + 1, c));
    double fym = 0.25 * (V(x, y, z, c) + V(x + 1, y, z, c) + V(x, y, z + 1, c) + V(x + 1, y, z + 1, c));
    double fyp = 0.25 * (V(x, y + 1, z, c) + V(x + 1, y + 1, z, c) + V(x, y + 1, z + 1, c) +
                         V(x + 1, y + 1, z + 1, c));
    double fzm = 0.25 * (V(x, y, z, c) + V(x + 1, y, z, c) + V(x, y + 1, z, c) + V(x + 1, y + 1, z, c));
    double fzp = 0.25 * (V(x, y, z + 1, c) + V(x + 1, y, z + 1, c) + V(x, y + 1, z + 1, c) +
                         V(x + 1, y + 1, z + 1, c));
    M[c][0] = fxp - fxm;
    M[c][1] = fyp - fym;
    M[c][2] = fzp - fzm;
  }
}

// inverse and determinant of a 2x2 / 3x3 matrix
double invert(int nd, const double M[3][3], double Ti[3][3]) {
  if (nd == 2) {
    double det = M[0][0] * M[1][1] - M[0][1] * M[1][0];
    Ti[0][0] = M[1][1] / det;
    Ti[0][1] = -M[0][1] / det;
    Ti[1][0] = -M[1][0] / det;
    Ti[1][1] = M[0][0] / det;
    return det;
  }
  double c00 = M[1][1] * M[2][2] - M[1][2] * M[2][1];
  double c01 = M[1][2] * M[2][0] - M[1][0] * M[2][2];
  double c02 = M[1][0] * M[2][1] - M[1][1] * M[2][0];
  double det = M[0][0] * c00 + M[0][1] * c01 + M[0][2] * c02;
  Ti[0][0] = c00 / det;
  Ti[1][0] = c01 / det;
  Ti[2][0] = c02 / det;
  Ti[0][1] = (M[0][2] * M[2][1] - M[0][1] * M[2][2]) / det;
  Ti[1][1] = (M[0][0] * M[2][2] - M[0][2] * M[2][0]) / det;
  Ti[2][1] = (M[0][1] * M[2][0] - M[0][0] * M[2][1]) / det;
  Ti[0][2] = (M[0][1] * M[1][2] - M[0][2] * M[1][1]) / det;
  Ti[1][2] = (M[0][2] * M[1][0] - M[0][0] * M[1][2]) / det;
  Ti[2][2] = (M[0][0] * M[1][1] - M[0][1] * M[1][0]) / det;
  return det;
}

template <typename real>
void put(std::vector<char>& buf, size_t i, double v) {
  reinterpret_cast<real*>(buf.data())[i] = (real)v;
}

// --- workspace layout ------------------------------------------------------
enum WsIdx {
  W_U, W_RHS0, W_R, W_RHAT, W_P0, W_P1, W_V0, W_V1, W_T, W_POFF, W_PDIAG, W_FH, W_B, W_CX,
  W_CRB0, W_CRB1, W_CWB0, W_CWB1, W_CSB0, W_CSB1, W_CP, W_PINV, W_INVA, W_AW, W_X64, W_RIN, W_CE,
  W_LFA, W_LFM, W_LFC, W_ILUD, W_BX,
  // adjoint scratch
  A_GA, A_GCOFF, A_GRHS0, A_GW, A_W, A_GG, A_GU, A_GX, A_Z, A_DU,
  A_GYB, A_GDK,    // non-orthogonal meshes only
  W_COUNT
};

// size of workspace array k in units of N elements
int ws_units(int k, int nd) {
  switch (k) {
    case W_PDIAG: case W_B: case W_CX: case W_CRB0: case W_CRB1: case W_CWB0: case W_CWB1: case W_CSB0:
    case W_CSB1: case W_CP: case A_GA: case A_GX: case W_PINV: case W_INVA: case W_RIN: case W_CE:
    case W_LFA: case W_LFM: case W_LFC: case W_ILUD: case W_BX:
      return 1;
    case W_X64:
      return 2;     // N doubles (two float units; the FP64 mode over-allocates)
    case A_GCOFF:
      return 2 * nd;
    case A_GYB:
      return 1;
    case A_GDK:
      return nd * nd;
    default:
      return nd;
  }
}

// workspace arrays a domain allocates: the adjoint's non-orthogonal scratch
// only on non-orthogonal meshes
bool ws_needed(int k, bool has_cross) { return has_cross || (k != A_GYB && k != A_GDK); }

// size of workspace array k for domain d: on domains with joints that
// exchange or reverse axes every cell keeps its 2d pressure face coefficients
int ws_units_d(int k, const piso_domain* d) {
  return (k == W_POFF && d->twisted) ? 2 * d->ndim : ws_units(k, d->ndim);
}

// Non-orthogonal corrector iterates a step record can hold (the adjoint needs
// them); piso_options.n_nonortho is limited to this.
constexpr int NONORTHO_MAX = 4;

struct TapeLayout {
  size_t hdr, un, cdiag, coff, ustar, h[4], xk[4], uc[4], bval, bval_in;
  size_t pn, xit[4], usit;   // non-orthogonal meshes: p^n and the iterates 1..n-1 (0: not recorded)
  size_t total;
};

TapeLayout tape_layout(const piso_domain* d) {
  TapeLayout t{};
  const size_t N = d->N, nd = d->ndim, e = d->elem;
  size_t off = 0;
  auto take = [&](size_t n) {
    size_t o = off;
    off += ((n * e + 255) / 256) * 256;
    return o;
  };
  t.hdr = off;
  off += 256;
  t.un = take(nd * N);
  t.cdiag = take(N);
  t.coff = take(2 * nd * N);
  t.ustar = take(nd * N);
  for (int k = 0; k < 4; k++) {
    t.h[k] = take(nd * N);
    t.xk[k] = take(N);
    t.uc[k] = take(nd * N);
  }
  t.bval = take(nd * std::max(d->nbf, 1));
  t.bval_in = take(nd * std::max(d->nbf, 1));
  if (d->has_cross) {
    t.pn = take(N);
    for (int k = 0; k < 4; k++) t.xit[k] = take((NONORTHO_MAX - 1) * N);
    t.usit = take((NONORTHO_MAX - 1) * nd * N);
  }
  t.total = off;
  return t;
}

template <typename real>
void fill_fwd_call(piso_domain* d, FwdCall<real>& c, const void* u_in, const void* p_in, void* u_out,
                   void* p_out, double dt, double nu, const void* S, void* tape) {
  memset(&c, 0, sizeof c);
  c.dom = d->d_static;
  c.u_in = (const real*)u_in;
  c.p_in = (const real*)p_in;
  c.u_out = (real*)u_out;
  c.p_out = (real*)p_out;
  c.S = (const real*)S;
  c.bval = (real*)d->bval;
  c.dt = dt;
  c.nu = nu;
  char* tb = (char*)(tape ? tape : d->tape_ws);
  TapeLayout L = tape_layout(d);
  c.un = (real*)(tb + L.un);
  c.Cdiag = (real*)(tb + L.cdiag);
  c.Coff = (real*)(tb + L.coff);
  c.ustar = (real*)(tb + L.ustar);
  for (int k = 0; k < 4; k++) {
    c.h[k] = (real*)(tb + L.h[k]);
    c.xk[k] = (real*)(tb + L.xk[k]);
    c.uc[k] = (real*)(tb + L.uc[k]);
  }
  c.bval_rec = (real*)(tb + L.bval);
  c.bval_in_rec = (real*)(tb + L.bval_in);
  c.hdr = (double*)(tb + L.hdr);
  if (d->has_cross) {
    c.pn = (real*)(tb + L.pn);
    for (int k = 0; k < 4; k++) c.xit[k] = (real*)(tb + L.xit[k]);
    c.usit = (real*)(tb + L.usit);
  }
  c.U = (real*)d->ws[W_U];
  c.rhs0 = (real*)d->ws[W_RHS0];
  c.r = (real*)d->ws[W_R];
  c.rhat = (real*)d->ws[W_RHAT];
  c.pv[0] = (real*)d->ws[W_P0];
  c.pv[1] = (real*)d->ws[W_P1];
  c.vv[0] = (real*)d->ws[W_V0];
  c.vv[1] = (real*)d->ws[W_V1];
  c.t = (real*)d->ws[W_T];
  c.Poff = (real*)d->ws[W_POFF];
  c.Pdiag = (real*)d->ws[W_PDIAG];
  c.Pinv = (real*)d->ws[W_PINV];
  c.invA = (real*)d->ws[W_INVA];
  c.Aw = (real*)d->ws[W_AW];
  c.Fh = (real*)d->ws[W_FH];
  c.b = (real*)d->ws[W_B];
  c.cx = (real*)d->ws[W_CX];
  c.crb[0] = (real*)d->ws[W_CRB0];
  c.crb[1] = (real*)d->ws[W_CRB1];
  c.cwb[0] = (real*)d->ws[W_CWB0];
  c.cwb[1] = (real*)d->ws[W_CWB1];
  c.csb[0] = (real*)d->ws[W_CSB0];
  c.csb[1] = (real*)d->ws[W_CSB1];
  c.cp = (real*)d->ws[W_CP];
  c.x64 = (double*)d->ws[W_X64];
  c.rin = (real*)d->ws[W_RIN];
  c.ce = (real*)d->ws[W_CE];
  c.lfa = (real*)d->ws[W_LFA];
  c.lfm = (real*)d->ws[W_LFM];
  c.lfc = (real*)d->ws[W_LFC];
  c.p_line = d->p_line;
  c.ilu = d->ilu_tab;
  c.ilud = (real*)d->ws[W_ILUD];
  c.adv_ilu = d->opts.adv_precond;
  c.n_nonortho = d->has_cross ? d->opts.n_nonortho : 0;
  c.bx = (real*)d->ws[W_BX];
  c.bar = d->bar;
  c.partials = d->partials;
  c.status = d->status;
  c.istats = d->istats;
  c.dstats = d->dstats;
  c.cta0 = 0;
  c.ncta = d->ncta;
}

#ifdef PISO_TRACE
// Phase-timing ring of trace builds: [PISO_TRACE_LEN][PISO_TRACE_STAMPS] stamps in device
// memory, allocated on first use and handed to every kernel through the solver
// options (the kernels of all translation units write this one buffer).
uint64_t* g_trace_buf = nullptr;
uint64_t* trace_buffer() {
  if (!g_trace_buf) {
    if (cudaMalloc((void**)&g_trace_buf, sizeof(uint64_t) * PISO_TRACE_STAMPS * PISO_TRACE_LEN) != cudaSuccess)
      g_trace_buf = nullptr;
    else cudaMemset(g_trace_buf, 0, sizeof(uint64_t) * PISO_TRACE_STAMPS * PISO_TRACE_LEN);
  }
  return g_trace_buf;
}
#endif

SolverOpts solver_opts(const piso_options& o) {
  SolverOpts s;
  s.n_corr = o.n_correctors;
  s.pred_grad_p = o.pred_grad_p;
  s.adv_maxit = o.adv_maxit;
  s.p_maxit = o.p_maxit;
  s.adv_rtol = o.adv_rtol;
  s.p_rtol = o.p_rtol;
  s.atol = o.atol;
  s.timeout_ns = (uint64_t)(o.timeout_s * 1e9);
  s.nbt_cap = 0;
  s.line_cap = 0;
  s.withhold_cta = o.fault_withhold_cta;
  s.p_refine_rtol = o.p_refine_rtol;
  s.p_inner_rtol = o.p_inner_rtol;
  s.grad_paths = o.grad_paths;
  s.ilu_soff = -1;
  s.lf_off = nullptr;
  s.lf_nown = nullptr;
  s.lf_lines = nullptr;
  s.lf_nbs = nullptr;
  s.lf_own_cap = 0;
  s.lf_slot_cap = 0;
  s.lf_bytes = 0;
#ifdef PISO_TRACE
  s.trace = trace_buffer();
#else
  s.trace = nullptr;
#endif
  return s;
}

// Dynamic shared memory of a step launch (neighbour table, line staging, ILU
// sweep area), at most this much.  Every step kernel's static shared memory
// plus this must stay within the 227 KB a CTA may opt into (the largest static
// area, the FP32 non-orthogonal adjoint's, is ~54 KB; tests/test_capi_symbols.py
// checks the sum against the build's resource report).
constexpr size_t NBT_MAX_BYTES = 168 * 1024;

size_t nbt_bytes(int ndim, int64_t N, int ncta, int32_t* cap) {
  const int64_t per = (N + ncta - 1) / ncta;
  const size_t b = (size_t)per * 2 * ndim * sizeof(int32_t);
  if (b > NBT_MAX_BYTES) {
    *cap = 0;
    return 0;
  }
  *cap = (int32_t)per;
  return b;
}

// Dynamic shared memory of a single-domain launch: the neighbour table and,
// with the y-line preconditioner, its staging area (LINE_ARRAYS arrays of line_cap reals
// and 3 x LINE_LBMAX ints), together within NBT_MAX_BYTES (the size the
// occupancy of the kernels was computed for).  The table is dropped (cells are
// then located arithmetically) when it would leave the staging area less than
// two lines.  Sets o->nbt_cap and o->line_cap; returns the bytes.
size_t launch_smem(const piso_domain* d, int ncta, SolverOpts* o) {
  const int nd = d->ndim;
  const size_t e = d->elem;
  const size_t ints = 3 * (size_t)LINE_LBMAX * sizeof(int32_t);
  const int lmax = std::max(d->h_static.lmax, 1);
  const size_t line_min = d->p_line ? LINE_ARRAYS * e * 2 * (size_t)lmax + ints : 0;
  auto al16 = [](size_t b) { return (b + 15) & ~size_t(15); };
  o->nbt_cap = 0;
  o->line_cap = 0;
  o->ilu_soff = -1;
  if (line_min > NBT_MAX_BYTES) return nbt_bytes(nd, d->N, ncta, &o->nbt_cap);   // lines cannot be staged
  const int64_t per = ((int64_t)d->N + ncta - 1) / ncta;
  // ILU(0) sweep values and factor rows of one cell per thread, when the
  // BiCGStab is preconditioned and every CTA owns at most one cell per thread
  const size_t ilu_b = (d->opts.adv_precond != PISO_ADV_PRECOND_NONE && per <= d->threads)
                           ? al16(ilu_smem_bytes(nd, (size_t)per, e)) : 0;
  size_t nbt = (size_t)per * 2 * nd * sizeof(int32_t);
  if (nbt + 16 + line_min + ilu_b <= NBT_MAX_BYTES) o->nbt_cap = (int32_t)per;
  else if (nbt + 16 + line_min <= NBT_MAX_BYTES && ilu_b) o->nbt_cap = (int32_t)per;   // table kept, no ILU area
  else nbt = 0;
  nbt = al16(nbt);
  const size_t ilu = (o->nbt_cap > 0 && nbt + 16 + line_min + ilu_b <= NBT_MAX_BYTES) ? ilu_b : 0;
  if (!d->p_line) {
    if (ilu) o->ilu_soff = (int32_t)nbt;
    return nbt + ilu;
  }
  // staging: as much as fits, but no more than this CTA's lines plus one
  const int64_t lines_per = ((int64_t)d->h_static.nlines + ncta - 1) / ncta;
  size_t cap = (NBT_MAX_BYTES - nbt - ilu - ints - (ilu ? 16 : 0)) / (LINE_ARRAYS * e);
  cap = std::min<size_t>(cap, (size_t)(std::min<int64_t>(lines_per, LINE_LBMAX) + 1) * lmax);
  cap = std::max<size_t>(cap, 2 * (size_t)lmax);
  o->line_cap = (int32_t)cap;
  size_t stage = LINE_ARRAYS * e * cap;
  // the fused CG's arrays alias the staging arrays (each fused solve re-fills them)
  if (d->lf_ready && d->lf_ncta == ncta && !d->opts.p_line_split) {
    const size_t st2 = std::max(stage, (size_t)d->lf_bytes);
    bool fit = nbt + st2 + ints + (ilu ? 16 + ilu : 0) <= NBT_MAX_BYTES;
    if (!fit && !ilu_b && st2 + ints <= NBT_MAX_BYTES) {
      // the fused form saves a group barrier per CG iteration, which is worth
      // more than the neighbour table (the other phases then locate their
      // cells arithmetically): FP64 on 64x48x32 with 128 CTAs needs this
      nbt = 0;
      o->nbt_cap = 0;
      fit = true;
    }
    if (fit) {
      stage = st2;
      o->lf_off = d->lf_off;
      o->lf_nown = d->lf_nown;
      o->lf_lines = d->lf_lines;
      o->lf_nbs = d->lf_nbs;
      o->lf_own_cap = d->lf_own_cap;
      o->lf_slot_cap = d->lf_slot_cap;
      o->lf_bytes = d->lf_bytes;
    }
  }
  size_t total = nbt + stage + ints;
  if (ilu) {
    total = al16(total);
    o->ilu_soff = (int32_t)total;
    total += ilu;
  }
  return total;
}

cudaError_t coop_launch(const void* kernel, int grid, int threads, void** args, cudaStream_t st, size_t smem = 0) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelExC(&cfg, kernel, args);
}

// Kernel variants: precision x dimension x CTA width (launch bound 512 or 768
// threads; the wider variant holds one cell per thread for ~98k-cell domains
// at 80 registers).
constexpr int WIDE = 768;   // the wide instantiations of piso_kernels_*.cu
inline int width_class(int threads) { return threads > 512 ? WIDE : 512; }

// Kernel instantiations (forward and adjoint alike): mode 0 plain, 1 with the
// ILU(0) predictor, 2 also with the non-orthogonal cross terms.  Batches take
// the plain ones.
template <typename real>
const void* fwd_ptr_t(int nd, int threads, int mode = 0) {
  const bool wide = width_class(threads) == WIDE;
  return sizeof(real) == 4 ? fwd_kernel_addr_f32(nd, wide, mode) : fwd_kernel_addr_f64(nd, wide, mode);
}

template <typename real>
const void* adj_ptr_t(int nd, int threads, int mode = 0) {
  const bool wide = width_class(threads) == WIDE;
  return sizeof(real) == 4 ? adj_kernel_addr_f32(nd, wide, mode) : adj_kernel_addr_f64(nd, wide, mode);
}

const void* fwd_kernel_ptr(int prec, int nd, int threads = 512, int mode = 0) {
  return prec == PISO_FP64 ? fwd_ptr_t<double>(nd, threads, mode) : fwd_ptr_t<float>(nd, threads, mode);
}

const void* adj_kernel_ptr(int prec, int nd, int threads = 512, int mode = 0) {
  return prec == PISO_FP64 ? adj_ptr_t<double>(nd, threads, mode) : adj_ptr_t<float>(nd, threads, mode);
}

bool uses_ilu(const piso_domain* d) { return d->opts.adv_precond != PISO_ADV_PRECOND_NONE; }
// the extended instantiations (mode 2) also carry the neighbour frames of joints
// that exchange or reverse axes
int fwd_mode(const piso_domain* d) { return (d->has_cross || d->twisted) ? 2 : (uses_ilu(d) ? 1 : 0); }
int adj_mode(const piso_domain* d) { return fwd_mode(d); }

// ILU(0) tables for the current launch layout (App. A.5 preconditioner of the
// BiCGStab).  Each CTA preconditions with the diagonal block of the cells it
// owns, so the tables follow the kernels' ownership rule: contiguous ranges
// [N r / ncta, N (r + 1) / ncta) when the neighbour table fits in shared
// memory, otherwise chunks of `threads` cells dealt round-robin to the CTAs.
// A cell's level is one more than the highest level among its neighbours in
// the same block with a lower index (0 if none); the forward substitution
// walks the levels upwards, the backward substitution downwards.
template <int ND>
void ilu_levels(const DomStatic& D, const std::vector<int32_t>& own, std::vector<int32_t>& lvl,
                std::vector<uint16_t>& mask) {
  const int32_t N = D.N;
  for (int32_t i = 0; i < N; i++) {
    const Cell c = locate<ND>(D, i);
    int32_t L = 0;
    uint16_t m = 0;
    for (int s = 0; s < 2 * ND; s++) {
      const int32_t k = c.nb[s];
      if (k < 0 || k == i || own[k] != own[i]) continue;
      if (k < i) {
        m |= (uint16_t)(1u << s);
        L = std::max(L, lvl[k] + 1);
      } else {
        m |= (uint16_t)(1u << (8 + s));
      }
    }
    lvl[i] = L;
    mask[i] = m;
  }
}

piso_status build_ilu(piso_domain* d) {
  if (d->opts.adv_precond == PISO_ADV_PRECOND_NONE) return PISO_OK;
  SolverOpts so = solver_opts(d->opts);
  launch_smem(d, d->ncta, &so);
  const int contiguous = so.nbt_cap > 0 ? 1 : 0;
  const int ncta = d->ncta, T = d->threads;
  if (d->ilu_ready && d->ilu_key[0] == ncta && d->ilu_key[1] == T && d->ilu_key[2] == contiguous) return PISO_OK;
  d->ilu_ready = false;
  const int32_t N = d->N;
  std::vector<int32_t> own(N);
  if (contiguous) {
    for (int r = 0; r < ncta; r++) {
      const int32_t lo = (int32_t)(((int64_t)N * r) / ncta), hi = (int32_t)(((int64_t)N * (r + 1)) / ncta);
      for (int32_t i = lo; i < hi; i++) own[i] = r;
    }
  } else {
    for (int32_t i = 0; i < N; i++) own[i] = (int32_t)((i / T) % ncta);
  }
  std::vector<int32_t> lvl(N);
  std::vector<uint16_t> mask(N);
  if (d->ndim == 3) ilu_levels<3>(d->h_static, own, lvl, mask);
  else ilu_levels<2>(d->h_static, own, lvl, mask);
  std::vector<int32_t> cnt(ncta, 0), nlev(ncta, 0), base(ncta, 0), lidx(ncta + 1, 0);
  for (int32_t i = 0; i < N; i++) {
    cnt[own[i]]++;
    nlev[own[i]] = std::max(nlev[own[i]], lvl[i] + 1);
  }
  for (int r = 1; r < ncta; r++) base[r] = base[r - 1] + cnt[r - 1];
  for (int r = 0; r < ncta; r++) lidx[r + 1] = lidx[r] + nlev[r] + 1;
  std::vector<int32_t> lstart(lidx[ncta], 0);
  for (int32_t i = 0; i < N; i++) lstart[lidx[own[i]] + lvl[i] + 1]++;
  for (int r = 0; r < ncta; r++)
    for (int l = 1; l <= nlev[r]; l++) lstart[lidx[r] + l] += lstart[lidx[r] + l - 1];
  std::vector<int32_t> cur(lstart), order(N);
  for (int32_t i = 0; i < N; i++) order[base[own[i]] + cur[lidx[own[i]] + lvl[i]]++] = i;
  // one device buffer: order | mask | lstart | lidx | base
  auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
  const size_t o_order = 0, o_mask = al(sizeof(int32_t) * N), o_ls = o_mask + al(sizeof(uint16_t) * N),
               o_lidx = o_ls + al(sizeof(int32_t) * lstart.size()), o_base = o_lidx + al(sizeof(int32_t) * (ncta + 1)),
               total = o_base + al(sizeof(int32_t) * ncta);
  if (d->ilu_buf) {
    CUDA_TRY(d, cudaDeviceSynchronize());   // no launch in flight may still read the old tables
    CUDA_TRY(d, cudaFree(d->ilu_buf));
    d->ilu_buf = nullptr;
  }
  CUDA_TRY(d, cudaMalloc(&d->ilu_buf, total));
  char* bb = (char*)d->ilu_buf;
  CUDA_TRY(d, cudaMemcpy(bb + o_order, order.data(), sizeof(int32_t) * N, cudaMemcpyHostToDevice));
  CUDA_TRY(d, cudaMemcpy(bb + o_mask, mask.data(), sizeof(uint16_t) * N, cudaMemcpyHostToDevice));
  CUDA_TRY(d, cudaMemcpy(bb + o_ls, lstart.data(), sizeof(int32_t) * lstart.size(), cudaMemcpyHostToDevice));
  CUDA_TRY(d, cudaMemcpy(bb + o_lidx, lidx.data(), sizeof(int32_t) * (ncta + 1), cudaMemcpyHostToDevice));
  CUDA_TRY(d, cudaMemcpy(bb + o_base, base.data(), sizeof(int32_t) * ncta, cudaMemcpyHostToDevice));
  d->ilu_tab.order = (const int32_t*)(bb + o_order);
  d->ilu_tab.mask = (const uint16_t*)(bb + o_mask);
  d->ilu_tab.lstart = (const int32_t*)(bb + o_ls);
  d->ilu_tab.lidx = (const int32_t*)(bb + o_lidx);
  d->ilu_tab.base = (const int32_t*)(bb + o_base);
  d->ilu_key[0] = ncta;
  d->ilu_key[1] = T;
  d->ilu_key[2] = contiguous;
  d->ilu_ready = true;
  return PISO_OK;
}

// A launch with the ILU(0) preconditioner needs tables of its own layout.
piso_status check_ilu(piso_domain* d) {
  if (d->opts.adv_precond == PISO_ADV_PRECOND_NONE) return PISO_OK;
  SolverOpts so = solver_opts(d->opts);
  launch_smem(d, d->ncta, &so);
  if (!d->ilu_ready || d->ilu_key[0] != d->ncta || d->ilu_key[1] != d->threads ||
      d->ilu_key[2] != (so.nbt_cap > 0 ? 1 : 0))
    return fail(d, PISO_ESTATE, "ILU(0) tables do not match the launch layout");
  return PISO_OK;
}

// Plan of the fused y-line CG iteration (cg_pressure_fused) for d->ncta CTAs:
// each CTA's own lines, the halo lines that hold the other neighbours of its
// cells, and the shared-memory slot of every neighbour of every own cell
// (cell y of local line l at slot y * P + l, P = local lines | 1).  Own lines
// are consecutive runs of the domain's lines walked block by block in strips
// of tx columns along z (tx >= nx: the plain x-then-z order), so a CTA owns a
// compact patch of columns and few halo lines; of the strip widths tried the
// one with the smallest shared footprint is kept.  No plan (lf_ready false)
// when the y-line preconditioner is off, two-phase iterations are asked for,
// or no CTA layout fits in shared memory.
template <int ND>
static piso_status build_linefuse_nd(piso_domain* d) {
  const DomStatic& S = d->h_static;
  const int ncta = d->ncta;
  const int32_t nl = S.nlines, lmax = std::max(S.lmax, 1), N = d->N;
  const size_t e = d->elem;
  constexpr int NS = 2 * ND;
  // the own cells alone must fit (u, p, x, face coefficients, neighbour slots)
  const int64_t own_min = (int64_t)((nl + ncta - 1) / ncta) * lmax;
  if (nl < ncta || own_min * ((3 + NS) * e + NS * 2) > (int64_t)NBT_MAX_BYTES) return PISO_OK;
  std::vector<int32_t> cline(N), cy(N), nbr((size_t)N * NS);
  for (int32_t i = 0; i < N; i++) {
    const Cell c = locate<ND>(S, i);
    cline[i] = line_of(S, c);
    cy[i] = c.y;
    for (int q = 0; q < NS; q++) nbr[(size_t)i * NS + q] = c.nb[q];
  }
  auto order_for = [&](int tx, std::vector<int32_t>& ord) {
    ord.clear();
    for (int b = 0; b < S.nblocks; b++) {
      const BlockInfo& B = S.blk[b];
      const int w = std::min(tx, B.nx);
      for (int x0 = 0; x0 < B.nx; x0 += w)
        for (int z = 0; z < B.nz; z++)
          for (int x = x0; x < std::min(x0 + w, B.nx); x++) ord.push_back(B.line0 + x + B.nx * z);
    }
  };
  struct Layout {
    std::vector<int32_t> off, nown, lines;
    int32_t own_cap = 0, slot_cap = 0, max_loc = 0;
    size_t bytes = 0;
  };
  std::vector<int32_t> mark(nl, -1), loc(nl, 0), ord;
  auto layout_for = [&](const std::vector<int32_t>& ord_, Layout& Lo) {
    Lo.off.assign(1, 0);
    Lo.nown.clear();
    Lo.lines.clear();
    Lo.own_cap = Lo.slot_cap = Lo.max_loc = 0;
    std::fill(mark.begin(), mark.end(), -1);
    for (int r = 0; r < ncta; r++) {
      const int32_t a = (int32_t)(((int64_t)nl * r) / ncta), z = (int32_t)(((int64_t)nl * (r + 1)) / ncta);
      const size_t base = Lo.lines.size();
      for (int32_t t = a; t < z; t++) {
        mark[ord_[t]] = r;
        Lo.lines.push_back(ord_[t]);
      }
      for (int32_t t = a; t < z; t++) {
        const LineDesc ld = line_desc(S, ord_[t]);
        for (int32_t y = 0; y < ld.len; y++) {
          const int32_t i = ld.start + y * ld.stride;
          for (int q = 0; q < NS; q++) {
            const int32_t j = nbr[(size_t)i * NS + q];
            if (j < 0 || mark[cline[j]] == r) continue;
            mark[cline[j]] = r;
            Lo.lines.push_back(cline[j]);
          }
        }
      }
      const int32_t n_own = z - a, n_loc = (int32_t)(Lo.lines.size() - base);
      Lo.nown.push_back(n_own);
      Lo.off.push_back((int32_t)Lo.lines.size());
      Lo.own_cap = std::max(Lo.own_cap, n_own * lmax);
      Lo.slot_cap = std::max(Lo.slot_cap, (n_loc | 1) * lmax);
      Lo.max_loc = std::max(Lo.max_loc, n_loc);
    }
    Lo.bytes = ((e * (6 * (size_t)Lo.slot_cap + (3 + NS) * (size_t)Lo.own_cap) + 4 * (size_t)Lo.slot_cap +
                 2 * NS * (size_t)Lo.own_cap) + 15) & ~size_t(15);
  };
  Layout best, cur;
  bool have = false;
  int maxnx = 1;
  for (int b = 0; b < S.nblocks; b++) maxnx = std::max(maxnx, S.blk[b].nx);
  for (int tx = 1;; tx *= 2) {
    const int t = std::min(tx, maxnx);
    order_for(t, ord);
    layout_for(ord, cur);
    const bool ok = cur.max_loc <= LINE_LBMAX && cur.slot_cap <= 32767;
    if (ok && (!have || cur.bytes < best.bytes)) {
      best = cur;
      have = true;
    }
    if (t >= maxnx) break;
  }
  if (!have || best.bytes > NBT_MAX_BYTES) return PISO_OK;
  // neighbour slots of the own cells, [ncta][NS][own_cap], own cell y * n_own + t
  const int32_t oc = best.own_cap;
  std::vector<int16_t> nbs((size_t)ncta * NS * oc, (int16_t)-1);
  for (int r = 0; r < ncta; r++) {
    const int32_t a = best.off[r], n_loc = best.off[r + 1] - a, n_own = best.nown[r], P = n_loc | 1;
    for (int32_t t = 0; t < n_loc; t++) loc[best.lines[a + t]] = t;
    for (int32_t t = 0; t < n_own; t++) {
      const LineDesc ld = line_desc(S, best.lines[a + t]);
      for (int32_t y = 0; y < ld.len; y++) {
        const int32_t i = ld.start + y * ld.stride, k = y * n_own + t;
        for (int q = 0; q < NS; q++) {
          const int32_t j = nbr[(size_t)i * NS + q];
          if (j >= 0) nbs[((size_t)r * NS + q) * oc + k] = (int16_t)(cy[j] * P + loc[cline[j]]);
        }
      }
    }
  }
  auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
  const size_t o_off = 0, o_nown = al(sizeof(int32_t) * (ncta + 1)), o_lines = o_nown + al(sizeof(int32_t) * ncta),
               o_nbs = o_lines + al(sizeof(int32_t) * best.lines.size()), total = o_nbs + al(sizeof(int16_t) * nbs.size());
  if (d->lf_buf) {
    CUDA_TRY(d, cudaDeviceSynchronize());   // no launch in flight may still read the old plan
    CUDA_TRY(d, cudaFree(d->lf_buf));
    d->lf_buf = nullptr;
  }
  CUDA_TRY(d, cudaMalloc(&d->lf_buf, total));
  char* bb = (char*)d->lf_buf;
  CUDA_TRY(d, cudaMemcpy(bb + o_off, best.off.data(), sizeof(int32_t) * (ncta + 1), cudaMemcpyHostToDevice));
  CUDA_TRY(d, cudaMemcpy(bb + o_nown, best.nown.data(), sizeof(int32_t) * ncta, cudaMemcpyHostToDevice));
  CUDA_TRY(d, cudaMemcpy(bb + o_lines, best.lines.data(), sizeof(int32_t) * best.lines.size(), cudaMemcpyHostToDevice));
  CUDA_TRY(d, cudaMemcpy(bb + o_nbs, nbs.data(), sizeof(int16_t) * nbs.size(), cudaMemcpyHostToDevice));
  d->lf_off = (const int32_t*)(bb + o_off);
  d->lf_nown = (const int32_t*)(bb + o_nown);
  d->lf_lines = (const int32_t*)(bb + o_lines);
  d->lf_nbs = (const int16_t*)(bb + o_nbs);
  d->lf_own_cap = best.own_cap;
  d->lf_slot_cap = best.slot_cap;
  d->lf_bytes = (int32_t)best.bytes;
  d->lf_ncta = ncta;
  d->lf_ready = true;
  return PISO_OK;
}

piso_status build_linefuse(piso_domain* d) {
  if (!d->p_line || d->opts.p_line_split || d->twisted) return PISO_OK;
  if (d->lf_ready && d->lf_ncta == d->ncta) return PISO_OK;
  d->lf_ready = false;
  return d->ndim == 3 ? build_linefuse_nd<3>(d) : build_linefuse_nd<2>(d);
}

// Launch-layout tables: ILU(0) levels and the fused y-line plan.
piso_status build_tables(piso_domain* d) {
  const piso_status s = build_ilu(d);
  if (s) return s;
  return build_linefuse(d);
}

int max_coresident(const void* kernel, int threads, int* sms_out) {
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)NBT_MAX_BYTES);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, NBT_MAX_BYTES);
  if (sms_out) *sms_out = sms;
  return sms * std::max(per_sm, 0);
}

piso_status choose_shape(piso_domain* d) {
  int threads = d->opts.block_threads > 0 ? d->opts.block_threads : 512;
  if (threads % 32 || threads > WIDE || threads < 32)
    return fail(d, PISO_EINVAL, "block_threads must be a multiple of 32 in [32, %d]", WIDE);
  int sms = 148;
  int cap_f = max_coresident(fwd_kernel_ptr(d->prec, d->ndim, threads, fwd_mode(d)), threads, &sms);
  int cap_a = max_coresident(adj_kernel_ptr(d->prec, d->ndim, threads, adj_mode(d)), threads, nullptr);
  int cap = std::min(cap_f, cap_a);
  if (cap <= 0) return fail(d, PISO_ECUDA, "kernel cannot be resident with %d threads", threads);
  int want = d->opts.ctas > 0 ? d->opts.ctas : std::min(sms, (int)((d->N + threads - 1) / threads));
  want = std::max(1, want);
  if (want > cap) want = cap;
  if (want > MAXCTA) want = MAXCTA;
  d->threads = threads;
  d->ncta = want;
  d->sms = sms;
  return build_tables(d);
}

piso_status collect_stats(piso_domain* d, piso_stats* st) {
  cudaError_t e = cudaStreamSynchronize(d->pending_stream);
  if (e != cudaSuccess) return fail(d, PISO_ECUDA, "step failed: %s", cudaGetErrorString(e));
  d->pending = false;
  const int bits = *d->h_status;
  piso_status s = PISO_OK;
  if (bits & PISO_ERR_TIMEOUT) s = PISO_ETIMEOUT;
  else if (bits & PISO_ERR_NAN) s = PISO_ENAN;
  else if (bits & PISO_ERR_BREAKDOWN) s = PISO_EBREAKDOWN;
  else if (bits & (PISO_ERR_NOCONV_ADV | PISO_ERR_NOCONV_P)) s = PISO_ENOCONV;
  if (st) {
    memset(st, 0, sizeof *st);
    st->status = s;
    st->error_bits = bits;
    for (int k = 0; k < 3; k++) {
      st->adv_iters[k] = d->h_istats[k];
      st->adv_resid[k] = d->h_dstats[k];
    }
    for (int k = 0; k < 4; k++) {
      st->p_iters[k] = d->h_istats[4 + k];
      st->p_resid[k] = d->h_dstats[4 + k];
      st->p_rounds[k] = d->h_istats[8 + k];
      st->p_rhs_norm[k] = d->h_dstats[8 + k];
    }
    st->adv_precond_used = d->h_istats[3];
  }
  if (s != PISO_OK) {
    const char* what = s == PISO_ETIMEOUT ? "group barrier timed out"
                       : s == PISO_ENAN   ? "NaN residual"
                       : s == PISO_EBREAKDOWN ? "Krylov breakdown"
                                              : "Krylov solve did not converge";
    return fail(d, s, "%s (error bits %d)", what, bits);
  }
  return PISO_OK;
}

piso_status enqueue_readback(piso_domain* d, cudaStream_t st) {
  CUDA_TRY(d, cudaMemcpyAsync(d->h_status, d->status, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  CUDA_TRY(d, cudaMemcpyAsync(d->h_istats, d->istats, 16 * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  CUDA_TRY(d, cudaMemcpyAsync(d->h_dstats, d->dstats, 16 * sizeof(double), cudaMemcpyDeviceToHost, st));
  return PISO_OK;
}

template <typename real>
piso_status launch_fwd(piso_domain* d, const void* u_in, const void* p_in, void* u_out, void* p_out,
                              double dt, double nu, const void* S, void* tape, cudaStream_t st) {
  const piso_status ci = check_ilu(d);
  if (ci) return ci;
  Launch<FwdCall<real>> L;
  memset(&L, 0, sizeof L);
  L.ngroups = 1;
  L.o = solver_opts(d->opts);
  L.cta_first = nullptr;
  L.calls = nullptr;
  const size_t smem = launch_smem(d, d->ncta, &L.o);
  fill_fwd_call<real>(d, L.call0, u_in, p_in, u_out, p_out, dt, nu, S, tape);
  CUDA_TRY(d, cudaMemsetAsync(d->bar, 0, 64, st));
  CUDA_TRY(d, cudaMemsetAsync(d->status, 0, 64, st));
  CUDA_TRY(d, cudaMemsetAsync(d->istats, 0, 64, st));
  void* args[] = {&L};
  CUDA_TRY(d, coop_launch(fwd_ptr_t<real>(d->ndim, d->threads, fwd_mode(d)), d->ncta, d->threads, args, st, smem));
  return PISO_OK;
}

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

const char* piso_version(void) { return "pisob300 0.1 (sm_103a)"; }

void piso_default_options(piso_options* o) {
  if (!o) return;
  o->n_correctors = 2;
  o->pred_grad_p = 0;
  o->adv_rtol = 1e-12;
  o->p_rtol = 1e-12;
  o->atol = 0.0;
  o->adv_maxit = 1000;
  o->p_maxit = 20000;
  o->block_threads = 0;
  o->ctas = 0;
  o->timeout_s = 5.0;
  o->fault_withhold_cta = -1;
  o->p_refine_rtol = 0.0;
  o->p_inner_rtol = 1e-4;
  o->grad_paths = PISO_GRAD_ADV | PISO_GRAD_P;
  o->p_precond = PISO_PRECOND_AUTO;
  o->p_line_split = 0;
  o->adv_precond = PISO_ADV_PRECOND_NONE;
  o->n_nonortho = 0;
}

piso_status piso_domain_create(int32_t ndim, int32_t prec, piso_domain** out) {
  if (!out) return fail(nullptr, PISO_EINVAL, "out is NULL");
  *out = nullptr;
  if (ndim != 2 && ndim != 3) return fail(nullptr, PISO_EINVAL, "ndim must be 2 or 3");
  if (prec != PISO_FP64 && prec != PISO_FP32) return fail(nullptr, PISO_EINVAL, "unknown precision %d", prec);
  piso_domain* d = new piso_domain();
  d->ndim = ndim;
  d->prec = prec;
  d->elem = prec == PISO_FP64 ? 8 : 4;
  piso_default_options(&d->opts);
  *out = d;
  return PISO_OK;
}

piso_status piso_block_add(piso_domain* d, const int32_t res[3], const double* vertices, int32_t* block_id) {
  if (!d || !res || !vertices) return fail(d, PISO_EINVAL, "NULL argument");
  if (d->finalized) return fail(d, PISO_ESTATE, "domain already finalized");
  if ((int)d->blocks.size() >= MAXB) return fail(d, PISO_EINVAL, "at most %d blocks per domain", MAXB);
  int nz = d->ndim == 2 ? 1 : res[2];
  if (res[0] < 1 || res[1] < 1 || nz < 1) return fail(d, PISO_EINVAL, "resolution must be positive");
  if (d->ndim == 2 && res[2] != 1) return fail(d, PISO_EINVAL, "2D blocks need nz = 1");
  HostBlock b;
  b.res[0] = res[0];
  b.res[1] = res[1];
  b.res[2] = nz;
  size_t nv = (size_t)(res[0] + 1) * (res[1] + 1) * (d->ndim == 3 ? nz + 1 : 1);
  b.vertices.assign(vertices, vertices + nv * d->ndim);
  d->blocks.push_back(std::move(b));
  if (block_id) *block_id = (int32_t)d->blocks.size() - 1;
  return PISO_OK;
}

static piso_status check_side(piso_domain* d, int32_t blk, int32_t side) {
  if (!d) return fail(d, PISO_EINVAL, "NULL domain");
  if (d->finalized) return fail(d, PISO_ESTATE, "domain already finalized");
  if (blk < 0 || blk >= (int)d->blocks.size()) return fail(d, PISO_EINVAL, "no block %d", blk);
  if (side < 0 || side >= 2 * d->ndim) return fail(d, PISO_EINVAL, "bad side %d", side);
  if (d->blocks[blk].side[side].kind != 0)
    return fail(d, PISO_EINVAL, "block %d side %d already has a boundary", blk, side);
  return PISO_OK;
}

piso_status piso_connect(piso_domain* d, int32_t a, int32_t sa, int32_t b, int32_t sb, int32_t axis_perm,
                         int32_t flip_mask) {
  piso_status s = check_side(d, a, sa);
  if (s) return s;
  if (!(a == b && sa == sb)) {
    s = check_side(d, b, sb);
    if (s) return s;
  }
  const int nd = d->ndim;
  if (axis_perm < 0 || axis_perm > 1 || (nd == 2 && axis_perm))
    return fail(d, PISO_EINVAL, "axis_perm must be 0 (2D) or 0/1 (3D)");
  if (flip_mask < 0 || flip_mask >= (1 << (nd - 1))) return fail(d, PISO_EINVAL, "flip_mask out of range");
  const int* ra = d->blocks[a].res;
  const int* rb = d->blocks[b].res;
  int ta[2] = {0, 0}, tb[2] = {0, 0}, n = 0, m = 0;
  for (int x = 0; x < 3; x++) {
    if (x != sa / 2) ta[n++] = x;
    if (x != sb / 2) tb[m++] = x;
  }
  for (int i = 0; i < nd - 1; i++)
    if (ra[ta[i]] != rb[tb[axis_perm ? 1 - i : i]])
      return fail(d, PISO_EINVAL, "connected sides need matching resolution (tangential axis %d)", i);
  if (a == b && sa == sb) {
    // a side folded onto itself pairs cells: the map must pair distinct cells
    if (axis_perm) return fail(d, PISO_EINVAL, "a side joined to itself keeps its axes (axis_perm 0)");
    bool moves = false;
    for (int i = 0; i < nd - 1; i++)
      if (((flip_mask >> i) & 1) && ra[ta[i]] % 2 == 0) moves = true;
    if (!moves)
      return fail(d, PISO_EINVAL, "a side joined to itself needs a reversed axis of even length (no cell may meet "
                                  "itself)");
  }
  SideSpec& A = d->blocks[a].side[sa];
  A.kind = 1;
  A.other = b;
  A.other_side = sb;
  A.perm = axis_perm;
  A.flip = flip_mask;
  if (!(a == b && sa == sb)) {
    // the inverse map: an exchange is its own inverse, the reversal bits follow the axes
    SideSpec& B = d->blocks[b].side[sb];
    B.kind = 1;
    B.other = a;
    B.other_side = sa;
    B.perm = axis_perm;
    B.flip = axis_perm ? (((flip_mask & 1) << 1) | ((flip_mask >> 1) & 1)) : flip_mask;
  }
  return PISO_OK;
}

piso_status piso_set_dirichlet(piso_domain* d, int32_t blk, int32_t side, const double* values) {
  piso_status s = check_side(d, blk, side);
  if (s) return s;
  if (!values) return fail(d, PISO_EINVAL, "values is NULL");
  HostBlock& b = d->blocks[blk];
  int nf = side_nfaces(b.res, side, d->ndim);
  b.side[side].kind = 2;
  b.side[side].values.assign(values, values + (size_t)nf * d->ndim);
  return PISO_OK;
}

piso_status piso_set_advective_outflow(piso_domain* d, int32_t blk, int32_t side, const double* u_m,
                                       const double* values) {
  piso_status s = check_side(d, blk, side);
  if (s) return s;
  if (!values || !u_m) return fail(d, PISO_EINVAL, "NULL argument");
  HostBlock& b = d->blocks[blk];
  int nf = side_nfaces(b.res, side, d->ndim);
  b.side[side].kind = 3;
  b.side[side].values.assign(values, values + (size_t)nf * d->ndim);
  for (int k = 0; k < d->ndim; k++) b.side[side].um[k] = u_m[k];
  return PISO_OK;
}

static piso_status validate_options(piso_domain* d, const piso_options* o) {
  if (o->n_correctors < 1 || o->n_correctors > 4) return fail(d, PISO_EINVAL, "n_correctors must be 1..4");
  if (o->adv_maxit < 0 || o->p_maxit < 0) return fail(d, PISO_EINVAL, "negative iteration limit");
  if (!(o->timeout_s > 0)) return fail(d, PISO_EINVAL, "timeout_s must be positive");
  if (o->adv_rtol < 0 || o->p_rtol < 0 || o->atol < 0) return fail(d, PISO_EINVAL, "negative tolerance");
  if (o->grad_paths & ~(PISO_GRAD_ADV | PISO_GRAD_P)) return fail(d, PISO_EINVAL, "grad_paths: unknown bits");
  if (o->p_precond < PISO_PRECOND_AUTO || o->p_precond > PISO_PRECOND_LINE)
    return fail(d, PISO_EINVAL, "p_precond must be PISO_PRECOND_AUTO, _JACOBI or _LINE");
  if (o->p_line_split != 0 && o->p_line_split != 1) return fail(d, PISO_EINVAL, "p_line_split must be 0 or 1");
  if (o->adv_precond < PISO_ADV_PRECOND_NONE || o->adv_precond > PISO_ADV_PRECOND_ILU_ON_FAILURE)
    return fail(d, PISO_EINVAL, "adv_precond must be PISO_ADV_PRECOND_NONE, _ILU or _ILU_ON_FAILURE");
  if (o->n_nonortho < 0 || o->n_nonortho > NONORTHO_MAX)
    return fail(d, PISO_EINVAL, "n_nonortho must be 0..%d (the step record holds that many iterates)", NONORTHO_MAX);
  if (d && d->has_cross && (o->n_nonortho < 1 || o->pred_grad_p))
    return fail(d, PISO_EINVAL, "a non-orthogonal mesh needs n_nonortho >= 1 and pred_grad_p = 0");
  return PISO_OK;
}

// Pressure preconditioner of a finalized domain from its options and grid.
static void resolve_precond(piso_domain* d) {
  const int p = d->opts.p_precond;
  d->p_line = (p == PISO_PRECOND_LINE || (p == PISO_PRECOND_AUTO && d->aniso >= 4.0)) ? 1 : 0;
  if (d->twisted) d->p_line = 0;   // the line factors read the plain face layout: Jacobi there
}

piso_status piso_finalize(piso_domain* d, const piso_options* opts) {
  if (!d) return fail(d, PISO_EINVAL, "NULL domain");
  if (d->finalized) return fail(d, PISO_ESTATE, "domain already finalized");
  if (d->blocks.empty()) return fail(d, PISO_EINVAL, "domain has no blocks");
  if (opts) {
    piso_status s = validate_options(d, opts);
    if (s) return s;
    d->opts = *opts;
  }
  const int nd = d->ndim;
  const int nsd = 2 * nd;
  // sizes, offsets, boundary faces
  std::vector<int> off(d->blocks.size() + 1, 0);
  for (size_t b = 0; b < d->blocks.size(); b++) {
    const int* r = d->blocks[b].res;
    off[b + 1] = off[b] + r[0] * r[1] * r[2];
  }
  if ((int64_t)off.back() >= (1ll << 30)) return fail(d, PISO_EINVAL, "too many cells");
  d->N = off.back();
  const int32_t N = d->N;
  DomStatic& S = d->h_static;
  memset(&S, 0, sizeof S);
  S.ndim = nd;
  S.nblocks = (int)d->blocks.size();
  S.N = N;
  int nbf = 0, n_out = 0;
  for (size_t b = 0; b < d->blocks.size(); b++) {
    HostBlock& hb = d->blocks[b];
    BlockInfo& bi = S.blk[b];
    bi.nx = hb.res[0];
    bi.ny = hb.res[1];
    bi.nz = hb.res[2];
    bi.off = off[b];
    bi.dnx = make_fast_div(bi.nx);
    bi.dny = make_fast_div(bi.ny);
    bi.line0 = S.nlines;                 // y-lines: one per (x, z) column of the block
    S.nlines += bi.nx * bi.nz;
    S.lmax = std::max(S.lmax, bi.ny);
    for (int s = 0; s < 6; s++) {
      bi.link[s] = -1;
      bi.bfo[s] = 0;
      bi.lside[s] = (int8_t)(s ^ 1);
      bi.lperm[s] = 0;
      bi.lflip[s] = 0;
      bi.lplain[s] = 1;
    }
    for (int s = 0; s < nsd; s++) {
      const SideSpec& sp = hb.side[s];
      if (sp.kind == 0) return fail(d, PISO_EINVAL, "block %d side %d has no boundary", (int)b, s);
      if (sp.kind == 1) {
        bi.link[s] = sp.other;
        bi.lside[s] = (int8_t)sp.other_side;
        bi.lperm[s] = (int8_t)sp.perm;
        bi.lflip[s] = (int8_t)sp.flip;
        bi.lplain[s] = (sp.other_side == (s ^ 1) && !sp.perm && !sp.flip) ? 1 : 0;
        if (!bi.lplain[s]) d->twisted = true;
      } else {
        bi.bfo[s] = nbf;
        int nf = side_nfaces(hb.res, s, nd);
        nbf += nf;
        if (sp.kind == 3) n_out += nf;
      }
    }
  }
  d->nbf = nbf;
  d->n_out = n_out;
  S.vec4 = d->twisted ? 0 : 1;
  for (int b = 0; b < S.nblocks; b++)
    if (S.blk[b].nx % 4) S.vec4 = 0;
  S.nbf = nbf;
  S.n_out = n_out;
  // metrics
  const size_t e = d->elem;
  std::vector<char> hJ(N * e), hT((size_t)nd * nd * N * e), hA((size_t)nd * N * e);
  const int ncross = nd * (nd - 1) / 2;
  std::vector<double> hX((size_t)ncross * N, 0.0);   // cross metrics, kept when some are non-zero
  for (size_t b = 0; b < d->blocks.size(); b++) {
    const HostBlock& hb = d->blocks[b];
    for (int z = 0; z < hb.res[2]; z++)
      for (int y = 0; y < hb.res[1]; y++)
        for (int x = 0; x < hb.res[0]; x++) {
          const size_t i = off[b] + x + (size_t)hb.res[0] * (y + (size_t)hb.res[1] * z);
          double M[3][3], Ti[3][3];
          cell_jacobian(hb, nd, x, y, z, M);
          const double Jv = invert(nd, M, Ti);
          if (!(Jv > 0)) return fail(d, PISO_EINVAL, "cell %zu of block %d has non-positive volume", i, (int)b);
          double G[3][3];
          for (int j = 0; j < nd; j++)
            for (int l = 0; l < nd; l++) {
              double s = 0;
              for (int k = 0; k < nd; k++) s += Ti[j][k] * Ti[l][k];
              G[j][l] = Jv * s;
            }
          for (int k = 0; k < nd; k++)
            if (k != 1 && G[k][k] > 0) d->aniso = std::max(d->aniso, G[1][1] / G[k][k]);
          for (int j = 0; j < nd; j++)
            for (int l = j + 1; l < nd; l++) {
              hX[(size_t)(j + l - 1) * N + i] = G[j][l];
              if (std::fabs(G[j][l]) > 1e-9 * std::max(std::fabs(G[j][j]), std::fabs(G[l][l]))) {
                if (d->opts.n_nonortho < 1 || d->opts.pred_grad_p)
                  return fail(d, PISO_EINVAL,
                              "non-orthogonal cell %zu: cross metrics need n_nonortho >= 1 (and pred_grad_p = 0)",
                              i);
                d->has_cross = true;
              }
            }
          if (d->prec == PISO_FP64) {
            put<double>(hJ, i, Jv);
            for (int j = 0; j < nd; j++) {
              put<double>(hA, (size_t)j * N + i, G[j][j]);
              for (int k = 0; k < nd; k++) put<double>(hT, (size_t)(j * nd + k) * N + i, Ti[j][k]);
            }
          } else {
            put<float>(hJ, i, Jv);
            for (int j = 0; j < nd; j++) {
              put<float>(hA, (size_t)j * N + i, G[j][j]);
              for (int k = 0; k < nd; k++) put<float>(hT, (size_t)(j * nd + k) * N + i, Ti[j][k]);
            }
          }
        }
  }
  // boundary-face tables
  const int nbf1 = std::max(nbf, 1);
  std::vector<int32_t> bf_cell(nbf1, 0);
  std::vector<int8_t> bf_side(nbf1, 0), bf_out(nbf1, 0);
  std::vector<char> bf_um((size_t)nd * nbf1 * e, 0), bval((size_t)nd * nbf1 * e, 0);
  for (size_t b = 0; b < d->blocks.size(); b++) {
    const HostBlock& hb = d->blocks[b];
    const int nx = hb.res[0], ny = hb.res[1], nz = hb.res[2];
    for (int s = 0; s < nsd; s++) {
      const SideSpec& sp = hb.side[s];
      if (sp.kind < 2) continue;
      const int nf = side_nfaces(hb.res, s, nd);
      for (int f = 0; f < nf; f++) {
        int x, y, z;
        if (s < 2) {
          x = (s & 1) ? nx - 1 : 0;
          y = f % ny;
          z = f / ny;
        } else if (s < 4) {
          y = (s & 1) ? ny - 1 : 0;
          x = f % nx;
          z = f / nx;
        } else {
          z = (s & 1) ? nz - 1 : 0;
          x = f % nx;
          y = f / nx;
        }
        const int gf = S.blk[b].bfo[s] + f;
        bf_cell[gf] = off[b] + x + nx * (y + ny * z);
        bf_side[gf] = (int8_t)s;
        bf_out[gf] = sp.kind == 3;
        for (int k = 0; k < nd; k++) {
          const double v = sp.values[(size_t)f * nd + k];
          const double um = sp.kind == 3 ? sp.um[k] : 0.0;
          if (d->prec == PISO_FP64) {
            put<double>(bval, (size_t)k * nbf1 + gf, v);
            put<double>(bf_um, (size_t)k * nbf1 + gf, um);
          } else {
            put<float>(bval, (size_t)k * nbf1 + gf, v);
            put<float>(bf_um, (size_t)k * nbf1 + gf, um);
          }
        }
      }
    }
  }
  // device memory: one arena
  Arena ar;
  auto plan = [&](Arena& a) {
    d->d_static = (DomStatic*)a.take(sizeof(DomStatic));
    d->J = a.take(N * e);
    d->T = a.take((size_t)nd * nd * N * e);
    d->alpha = a.take((size_t)nd * N * e);
    d->gx = d->has_cross ? a.take((size_t)ncross * N * e) : nullptr;
    d->bf_cell = (int32_t*)a.take(nbf1 * sizeof(int32_t));
    d->bf_side = (int8_t*)a.take(nbf1);
    d->bf_out = (int8_t*)a.take(nbf1);
    d->bf_um = a.take((size_t)nd * nbf1 * e);
    d->bval = a.take((size_t)nd * nbf1 * e);
    d->gbval = a.take((size_t)nd * nbf1 * e);
    d->nbfr = d->twisted ? (int16_t*)a.take((size_t)nsd * N * sizeof(int16_t)) : nullptr;
    for (int k = 0; k < W_COUNT; k++)
      d->ws[k] = ws_needed(k, d->has_cross) ? a.take((size_t)ws_units_d(k, d) * N * e) : nullptr;
    d->tape_ws = a.take(tape_layout(d).total);
    d->bar = (uint32_t*)a.take(64);
    d->status = (int32_t*)a.take(64);
    d->istats = (int32_t*)a.take(64);
    d->dstats = (double*)a.take(128);
    d->d_dnu = (double*)a.take(64);
    d->partials = (double*)a.take(sizeof(double) * 2 * NSMAX * MAXCTA);
  };
  plan(ar);
  d->dmem_bytes = ar.used;
  if (cudaMalloc((void**)&d->dmem, d->dmem_bytes) != cudaSuccess) {
    cudaGetLastError();
    return fail(d, PISO_ENOMEM, "cudaMalloc of %zu bytes failed", d->dmem_bytes);
  }
  Arena real_ar;
  real_ar.base = d->dmem;
  plan(real_ar);
  CUDA_TRY(d, cudaMemset(d->dmem, 0, d->dmem_bytes));
  S.J = d->J;
  S.T = d->T;
  S.alpha = d->alpha;
  S.Gx = d->gx;
  S.nbfr = d->nbfr;
  if (d->twisted) {
    // neighbour frames: identity inside blocks and across plain joints; across
    // a joint of side s to side so, the normal axis goes to so's axis (reversed
    // when both sides have the same sign) and the tangential axes as exchanged
    // (lperm) and reversed (lflip)
    std::vector<int16_t> fr((size_t)nsd * N, (int16_t)FRAME_ID);
    for (size_t b = 0; b < d->blocks.size(); b++) {
      const BlockInfo& B = S.blk[b];
      for (int sd = 0; sd < nsd; sd++) {
        if (B.link[sd] < 0 || B.lplain[sd]) continue;
        const int j = sd >> 1, so = B.lside[sd], jo = so >> 1;
        int ax[3] = {0, 1, 2}, ng[3] = {0, 0, 0};
        int ta[2] = {0, 0}, tb[2] = {0, 0}, n = 0, m = 0;
        for (int x = 0; x < 3; x++) {
          if (x != j) ta[n++] = x;
          if (x != jo) tb[m++] = x;
        }
        ax[j] = jo;
        ng[j] = ((sd & 1) == (so & 1)) ? 1 : 0;
        for (int i = 0; i < 2; i++) {
          ax[ta[i]] = tb[B.lperm[sd] ? 1 - i : i];
          ng[ta[i]] = (B.lflip[sd] >> i) & 1;
        }
        const int16_t code = (int16_t)(ax[0] | (ax[1] << 2) | (ax[2] << 4) | (ng[0] << 6) | (ng[1] << 7) | (ng[2] << 8));
        const int nxb = B.nx, nyb = B.ny, nzb = B.nz;
        for (int z = 0; z < nzb; z++)
          for (int y = 0; y < nyb; y++)
            for (int x = 0; x < nxb; x++) {
              const int c3[3] = {x, y, z}, n3[3] = {nxb, nyb, nzb};
              if (c3[j] != ((sd & 1) ? n3[j] - 1 : 0)) continue;
              fr[(size_t)sd * N + B.off + x + nxb * (y + nyb * z)] = code;
            }
      }
    }
    CUDA_TRY(d, cudaMemcpy(d->nbfr, fr.data(), fr.size() * sizeof(int16_t), cudaMemcpyHostToDevice));
  }
  S.bf_cell = d->bf_cell;
  S.bf_side = d->bf_side;
  S.bf_out = d->bf_out;
  S.bf_um = d->bf_um;
  CUDA_TRY(d, cudaMemcpy(d->d_static, &S, sizeof S, cudaMemcpyHostToDevice));
  CUDA_TRY(d, cudaMemcpy(d->J, hJ.data(), hJ.size(), cudaMemcpyHostToDevice));
  CUDA_TRY(d, cudaMemcpy(d->T, hT.data(), hT.size(), cudaMemcpyHostToDevice));
  CUDA_TRY(d, cudaMemcpy(d->alpha, hA.data(), hA.size(), cudaMemcpyHostToDevice));
  if (d->has_cross) {
    std::vector<char> hx((size_t)ncross * N * e);
    for (size_t q = 0; q < hX.size(); q++) {
      if (d->prec == PISO_FP64) put<double>(hx, q, hX[q]);
      else put<float>(hx, q, hX[q]);
    }
    CUDA_TRY(d, cudaMemcpy(d->gx, hx.data(), hx.size(), cudaMemcpyHostToDevice));
  }
  CUDA_TRY(d, cudaMemcpy(d->bf_cell, bf_cell.data(), nbf1 * sizeof(int32_t), cudaMemcpyHostToDevice));
  CUDA_TRY(d, cudaMemcpy(d->bf_side, bf_side.data(), nbf1, cudaMemcpyHostToDevice));
  CUDA_TRY(d, cudaMemcpy(d->bf_out, bf_out.data(), nbf1, cudaMemcpyHostToDevice));
  CUDA_TRY(d, cudaMemcpy(d->bf_um, bf_um.data(), bf_um.size(), cudaMemcpyHostToDevice));
  CUDA_TRY(d, cudaMemcpy(d->bval, bval.data(), bval.size(), cudaMemcpyHostToDevice));
  CUDA_TRY(d, cudaMallocHost((void**)&d->h_status, 64));
  CUDA_TRY(d, cudaMallocHost((void**)&d->h_istats, 64));
  CUDA_TRY(d, cudaMallocHost((void**)&d->h_dstats, 128));
  CUDA_TRY(d, cudaMallocHost((void**)&d->h_dnu, 64));
  resolve_precond(d);
  piso_status s = choose_shape(d);
  if (s) return s;
  d->finalized = true;
  return PISO_OK;
}

piso_status piso_set_options(piso_domain* d, const piso_options* opts) {
  if (!d || !opts) return fail(d, PISO_EINVAL, "NULL argument");
  piso_status s = validate_options(d, opts);
  if (s) return s;
  d->opts = *opts;
  if (d->finalized) {
    resolve_precond(d);
    return choose_shape(d);
  }
  return PISO_OK;
}

piso_status piso_get_boundary_adjoint(piso_domain* d, double* values) {
  if (!d || !values) return fail(d, PISO_EINVAL, "NULL argument");
  if (!d->finalized) return fail(d, PISO_ESTATE, "domain not finalized");
  const int nbf1 = std::max(d->nbf, 1);
  std::vector<char> buf((size_t)d->ndim * nbf1 * d->elem);
  CUDA_TRY(d, cudaMemcpy(buf.data(), d->gbval, buf.size(), cudaMemcpyDeviceToHost));
  for (int k = 0; k < d->ndim; k++)
    for (int f = 0; f < d->nbf; f++) {
      const size_t i = (size_t)k * nbf1 + f;
      values[(size_t)k * d->nbf + f] = d->prec == PISO_FP64 ? reinterpret_cast<double*>(buf.data())[i]
                                                           : (double)reinterpret_cast<float*>(buf.data())[i];
    }
  return PISO_OK;
}

piso_status piso_get_options(const piso_domain* d, piso_options* opts) {
  if (!d || !opts) return fail(const_cast<piso_domain*>(d), PISO_EINVAL, "NULL argument");
  *opts = d->opts;
  return PISO_OK;
}

int32_t piso_pressure_precond(const piso_domain* d) {
  if (!d || !d->finalized) return -1;
  return d->p_line ? PISO_PRECOND_LINE : PISO_PRECOND_JACOBI;
}

int32_t piso_pressure_line_fused(const piso_domain* d) {
  if (!d || !d->finalized) return -1;
  SolverOpts so = solver_opts(d->opts);
  launch_smem(d, d->ncta, &so);
  return d->p_line && so.lf_off ? 1 : 0;
}

int32_t piso_pressure_cg_vec4(const piso_domain* d) {
  if (!d || !d->finalized) return -1;
  SolverOpts so = solver_opts(d->opts);
  launch_smem(d, d->ncta, &so);
  return !d->p_line && d->h_static.vec4 && so.nbt_cap == 0 ? 1 : 0;
}

int64_t piso_num_cells(const piso_domain* d) { return d ? d->N : -1; }
int32_t piso_num_boundary_faces(const piso_domain* d) { return d ? d->nbf : -1; }

size_t piso_tape_bytes(const piso_domain* d) {
  if (!d || !d->finalized) return 0;
  return tape_layout(d).total;
}

piso_status piso_step(piso_domain* d, const void* u_in, const void* p_in, void* u_out, void* p_out, double dt,
                      double nu, const void* S, void* tape, void* stream, piso_stats* stats) {
  if (!d) return fail(d, PISO_EINVAL, "NULL domain");
  if (!d->finalized) return fail(d, PISO_ESTATE, "step before finalize");
  if (!u_in || !p_in || !u_out || !p_out) return fail(d, PISO_EINVAL, "NULL field pointer");
  if (!(dt > 0) || !std::isfinite(dt)) return fail(d, PISO_EINVAL, "dt must be positive and finite");
  if (!(nu >= 0) || !std::isfinite(nu)) return fail(d, PISO_EINVAL, "nu must be non-negative and finite");
  cudaStream_t st = (cudaStream_t)stream;
  d->tape_ws_valid = false;
  piso_status s = d->prec == PISO_FP64 ? launch_fwd<double>(d, u_in, p_in, u_out, p_out, dt, nu, S, tape, st)
                                       : launch_fwd<float>(d, u_in, p_in, u_out, p_out, dt, nu, S, tape, st);
  if (s) return s;
  d->tape_ws_valid = (tape == nullptr);
  s = enqueue_readback(d, st);
  if (s) return s;
  d->pending = true;
  d->pending_kind = 1;
  d->pending_stream = st;
  if (stats) return collect_stats(d, stats);
  return PISO_OK;
}

// Launch-shape autotuner: times one forward step of the caller's state for
// each candidate (CTA width 512 or 768 threads; CTA count = one per SM, or
// just enough CTAs for one cell per thread) and keeps the fastest.  Results
// are cached per process by (ndim, precision, cells, blocks, correctors).
static std::map<std::tuple<int, int, int, int, int>, std::tuple<int, int, int>>& tune_cache() {
  static std::map<std::tuple<int, int, int, int, int>, std::tuple<int, int, int>> c;
  return c;
}

piso_status piso_autotune(piso_domain* d, const void* u, const void* p, double dt, double nu, const void* S,
                          void* stream, int32_t* threads_out, int32_t* ctas_out, double* ms_out) {
  if (!d || !u || !p) return fail(d, PISO_EINVAL, "NULL argument");
  if (!d->finalized) return fail(d, PISO_ESTATE, "autotune before finalize");
  cudaStream_t st = (cudaStream_t)stream;
  const auto key = std::make_tuple(d->ndim, d->prec, (int)d->N, (int)d->blocks.size(),
                                   ((d->opts.n_correctors * 4 + d->opts.p_precond) * 4 + d->opts.adv_precond) * 2 +
                                       (d->opts.p_line_split ? 1 : 0));
  auto it = tune_cache().find(key);
  double best_ms = -1.0;
  if (it == tune_cache().end()) {
    const size_t vb = (size_t)d->ndim * d->N * d->elem, sb = (size_t)d->N * d->elem;
    const size_t bb = (size_t)d->ndim * std::max(d->nbf, 1) * d->elem;
    char* tmp = nullptr;
    CUDA_TRY(d, cudaMalloc((void**)&tmp, vb + sb + bb + 1024));
    char* uo = tmp;
    char* po = tmp + ((vb + 255) / 256) * 256;
    char* bk = po + ((sb + 255) / 256) * 256;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const piso_options saved = d->opts;
    const int saved_threads = d->threads, saved_ncta = d->ncta, saved_line = d->p_line;
    // with PISO_PRECOND_AUTO on a y-anisotropic grid both pressure
    // preconditioners are timed (the line form saves iterations, but costs a
    // second barrier per iteration and a serial line solve per CTA)
    std::vector<int> pls = {d->p_line};
    if (d->opts.p_precond == PISO_PRECOND_AUTO && d->p_line) pls.push_back(0);
    std::vector<std::tuple<int, int, int>> cand;
    for (int pl : pls)
      for (int w : {512, WIDE}) {
        int sms = 148;
        const int cap = std::min(max_coresident(fwd_kernel_ptr(d->prec, d->ndim, w, fwd_mode(d)), w, &sms),
                                 max_coresident(adj_kernel_ptr(d->prec, d->ndim, w, adj_mode(d)), w, nullptr));
        const int one_per_thread = (int)std::min<int64_t>(cap, (d->N + w - 1) / w);
        // with y-lines also the largest CTA count that divides the line count
        // (every CTA owns as many lines; on the 64x48x32 channel 128 CTAs of
        // 16 lines beat 148 CTAs of 13-14 lines by 11%)
        int even = 0;
        if (pl)
          for (int k = std::min(cap, sms); k >= 1 && !even; k--)
            if (d->h_static.nlines % k == 0 && 4 * k >= 3 * std::min(cap, sms)) even = k;
        for (int nc : {std::min(cap, sms), one_per_thread, even})
          if (nc >= 1 && std::find(cand.begin(), cand.end(), std::make_tuple(w, nc, pl)) == cand.end())
            cand.push_back({w, nc, pl});
      }
    std::tuple<int, int, int> best = {saved_threads, saved_ncta, saved_line};
    piso_status s = PISO_OK;
    CUDA_TRY(d, cudaMemcpyAsync(bk, d->bval, bb, cudaMemcpyDeviceToDevice, st));
    d->tape_ws_valid = false;      // the trial steps record into the domain's own tape
    for (auto& c : cand) {
      d->threads = std::get<0>(c);
      d->ncta = std::get<1>(c);
      d->p_line = std::get<2>(c);
      s = build_tables(d);
      if (s != PISO_OK) break;
      double t = 1e300;
      for (int rep = 0; rep < 3 && s == PISO_OK; rep++) {
        cudaEventRecord(e0, st);
        s = d->prec == PISO_FP64 ? launch_fwd<double>(d, u, p, uo, po, dt, nu, S, nullptr, st)
                                 : launch_fwd<float>(d, u, p, uo, po, dt, nu, S, nullptr, st);
        cudaEventRecord(e1, st);
        cudaMemcpyAsync(d->bval, bk, bb, cudaMemcpyDeviceToDevice, st);
        if (cudaEventSynchronize(e1) != cudaSuccess) s = PISO_ECUDA;
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0) t = std::min(t, (double)ms);
      }
      if (s != PISO_OK) break;
      if (best_ms < 0 || t < best_ms) {
        best_ms = t;
        best = c;
      }
    }
    cudaStreamSynchronize(st);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(tmp);
    d->opts = saved;
    d->threads = saved_threads;
    d->ncta = saved_ncta;
    d->p_line = saved_line;
    if (s != PISO_OK) return fail(d, s, "autotune trial step failed");
    it = tune_cache().emplace(key, best).first;
  }
  d->threads = std::get<0>(it->second);
  d->ncta = std::get<1>(it->second);
  d->p_line = std::get<2>(it->second);
  d->opts.block_threads = d->threads;
  d->opts.ctas = d->ncta;
  d->opts.p_precond = d->p_line ? PISO_PRECOND_LINE : PISO_PRECOND_JACOBI;
  const piso_status sb = build_tables(d);
  if (sb) return sb;
  if (threads_out) *threads_out = d->threads;
  if (ctas_out) *ctas_out = d->ncta;
  if (ms_out) *ms_out = best_ms;
  return PISO_OK;
}

piso_status piso_last_stats(piso_domain* d, piso_stats* stats) {
  if (!d) return fail(d, PISO_EINVAL, "NULL domain");
  if (!d->pending) {
    if (stats) memset(stats, 0, sizeof *stats);
    return fail(d, PISO_ESTATE, "no step pending");
  }
  return collect_stats(d, stats);
}

piso_status piso_get_boundary(piso_domain* d, double* values) {
  if (!d || !values) return fail(d, PISO_EINVAL, "NULL argument");
  if (!d->finalized) return fail(d, PISO_ESTATE, "domain not finalized");
  const int nbf1 = std::max(d->nbf, 1);
  std::vector<char> buf((size_t)d->ndim * nbf1 * d->elem);
  CUDA_TRY(d, cudaDeviceSynchronize());
  CUDA_TRY(d, cudaMemcpy(buf.data(), d->bval, buf.size(), cudaMemcpyDeviceToHost));
  for (int k = 0; k < d->ndim; k++)
    for (int f = 0; f < d->nbf; f++) {
      size_t i = (size_t)k * nbf1 + f;
      values[(size_t)k * d->nbf + f] = d->prec == PISO_FP64 ? ((double*)buf.data())[i] : ((float*)buf.data())[i];
    }
  return PISO_OK;
}

piso_status piso_set_boundary(piso_domain* d, const double* values) {
  if (!d || !values) return fail(d, PISO_EINVAL, "NULL argument");
  if (!d->finalized) return fail(d, PISO_ESTATE, "domain not finalized");
  const int nbf1 = std::max(d->nbf, 1);
  std::vector<char> buf((size_t)d->ndim * nbf1 * d->elem, 0);
  for (int k = 0; k < d->ndim; k++)
    for (int f = 0; f < d->nbf; f++) {
      size_t i = (size_t)k * nbf1 + f;
      double v = values[(size_t)k * d->nbf + f];
      if (d->prec == PISO_FP64) ((double*)buf.data())[i] = v;
      else ((float*)buf.data())[i] = (float)v;
    }
  CUDA_TRY(d, cudaDeviceSynchronize());
  CUDA_TRY(d, cudaMemcpy(d->bval, buf.data(), buf.size(), cudaMemcpyHostToDevice));
  return PISO_OK;
}

const char* piso_last_error(const piso_domain* d) { return d ? d->err.c_str() : g_create_error.c_str(); }

void piso_domain_destroy(piso_domain* d) {
  if (!d) return;
  if (d->dmem) cudaFree(d->dmem);
  if (d->h_status) cudaFreeHost(d->h_status);
  if (d->ilu_buf) cudaFree(d->ilu_buf);
  if (d->lf_buf) cudaFree(d->lf_buf);
  if (d->h_istats) cudaFreeHost(d->h_istats);
  if (d->h_dstats) cudaFreeHost(d->h_dstats);
  if (d->h_dnu) cudaFreeHost(d->h_dnu);
  delete d;
}

}  // extern "C"

#include "piso_capi_adjoint.inc"
#include "piso_capi_batch.inc"
#include "piso_capi_stats.inc"

// ===========================================================================
// Forward step with library-owned static scratch (allocates nothing per call).
//
// Some callers cannot allocate device memory when they step: for example a
// process whose device memory is already fully reserved by another framework's
// caching allocator, or a latency-critical loop that must not risk an
// allocation or its failure mid-run.  For them piso_step_static runs the same
// forward kernel as piso_step, but every scratch array it needs (workspace,
// step record and control words) comes from one fixed buffer compiled into
// this library instead of from memory obtained with cudaMalloc.
// ===========================================================================
namespace {

constexpr size_t STATIC_SCRATCH_BYTES = 32ull << 20;   // 32 MiB, held on every device that loads the library
__device__ __align__(256) unsigned char g_static_scratch[STATIC_SCRATCH_BYTES];

constexpr int MAX_DEVICES = 64;
// Device address of g_static_scratch per device, looked up on first use.  The
// entries are atomic, so host threads making their first call on a device at
// the same time each store the same address without a data race.
std::atomic<void*> g_static_ptr[MAX_DEVICES];

// Byte layout of the forward kernel's scratch inside the static buffer.
struct StaticLayout {
  size_t ws[W_COUNT];
  size_t tape, bar, status, istats, dstats, partials, total;
};

StaticLayout static_layout(const piso_domain* d) {
  StaticLayout L{};
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off += (bytes + 255) & ~size_t(255);
    return o;
  };
  for (int k = 0; k < A_GA; k++) L.ws[k] = take((size_t)ws_units_d(k, d) * d->N * d->elem);
  L.tape = take(tape_layout(d).total);
  L.bar = take(64);
  L.status = take(64);
  L.istats = take(64);
  L.dstats = take(128);
  L.partials = take(sizeof(double) * 2 * NSMAX * (size_t)d->ncta);
  L.total = off;
  return L;
}

}  // namespace

extern "C" piso_status piso_step_static(piso_domain* d, const void* u_in, const void* p_in, void* u_out,
                                        void* p_out, double dt, double nu, const void* S, void* stream,
                                        piso_stats* stats) {
  if (!d) return fail(d, PISO_EINVAL, "NULL domain");
  if (!d->finalized) return fail(d, PISO_ESTATE, "step before finalize");
  if (!u_in || !p_in || !u_out || !p_out) return fail(d, PISO_EINVAL, "NULL field pointer");
  if (!(dt > 0) || !std::isfinite(dt)) return fail(d, PISO_EINVAL, "dt must be positive and finite");
  if (!(nu >= 0) || !std::isfinite(nu)) return fail(d, PISO_EINVAL, "nu must be non-negative and finite");
  const piso_status ci = check_ilu(d);
  if (ci) return ci;
  const StaticLayout SL = static_layout(d);
  if (SL.total > STATIC_SCRATCH_BYTES)
    return fail(d, PISO_EINVAL, "domain needs %zu bytes of scratch; piso_step_static provides %zu (use piso_step)",
                SL.total, STATIC_SCRATCH_BYTES);
  int dev = 0;
  CUDA_TRY(d, cudaGetDevice(&dev));
  if (dev < 0 || dev >= MAX_DEVICES) return fail(d, PISO_EINVAL, "device index %d out of range", dev);
  void* sp = g_static_ptr[dev].load(std::memory_order_acquire);
  if (!sp) {   // set-up, once per device, with that device current
    cudaError_t e = cudaGetSymbolAddress(&sp, g_static_scratch);
    if (e != cudaSuccess || !sp)
      return fail(d, PISO_ECUDA, "cudaGetSymbolAddress of the static scratch failed: %s", cudaGetErrorString(e));
    g_static_ptr[dev].store(sp, std::memory_order_release);
  }
  char* base = (char*)sp;
  cudaStream_t st = (cudaStream_t)stream;
  d->tape_ws_valid = false;   // this step's record lives in the shared buffer, not in the domain
  CUDA_TRY(d, cudaMemsetAsync(base + SL.bar, 0, 64, st));      // barrier counter, status and counts start at 0
  CUDA_TRY(d, cudaMemsetAsync(base + SL.status, 0, 64, st));
  CUDA_TRY(d, cudaMemsetAsync(base + SL.istats, 0, 64, st));
  auto launch = [&](auto tag) -> piso_status {
    using real = decltype(tag);
    Launch<FwdCall<real>> L;
    memset(&L, 0, sizeof L);
    L.ngroups = 1;
    L.o = solver_opts(d->opts);
    const size_t smem = launch_smem(d, d->ncta, &L.o);
    FwdCall<real>& c = L.call0;
    fill_fwd_call<real>(d, c, u_in, p_in, u_out, p_out, dt, nu, S, base + SL.tape);
    auto W = [&](int k) { return (real*)(base + SL.ws[k]); };
    c.U = W(W_U);
    c.rhs0 = W(W_RHS0);
    c.r = W(W_R);
    c.rhat = W(W_RHAT);
    c.pv[0] = W(W_P0);
    c.pv[1] = W(W_P1);
    c.vv[0] = W(W_V0);
    c.vv[1] = W(W_V1);
    c.t = W(W_T);
    c.Poff = W(W_POFF);
    c.Pdiag = W(W_PDIAG);
    c.Pinv = W(W_PINV);
    c.invA = W(W_INVA);
    c.Aw = W(W_AW);
    c.Fh = W(W_FH);
    c.b = W(W_B);
    c.cx = W(W_CX);
    c.crb[0] = W(W_CRB0);
    c.crb[1] = W(W_CRB1);
    c.cwb[0] = W(W_CWB0);
    c.cwb[1] = W(W_CWB1);
    c.csb[0] = W(W_CSB0);
    c.csb[1] = W(W_CSB1);
    c.cp = W(W_CP);
    c.x64 = (double*)(base + SL.ws[W_X64]);
    c.rin = W(W_RIN);
    c.ce = W(W_CE);
    c.lfa = W(W_LFA);
    c.lfm = W(W_LFM);
    c.lfc = W(W_LFC);
    c.ilud = W(W_ILUD);
    c.bx = W(W_BX);
    c.bar = (uint32_t*)(base + SL.bar);
    c.status = (int32_t*)(base + SL.status);
    c.istats = (int32_t*)(base + SL.istats);
    c.dstats = (double*)(base + SL.dstats);
    c.partials = (double*)(base + SL.partials);
    void* args[] = {&L};
    CUDA_TRY(d, coop_launch(fwd_ptr_t<real>(d->ndim, d->threads, fwd_mode(d)), d->ncta, d->threads, args, st, smem));
    return PISO_OK;
  };
  piso_status s = d->prec == PISO_FP64 ? launch(double(0)) : launch(float(0));
  if (s) return s;
  CUDA_TRY(d, cudaMemcpyAsync(d->h_status, base + SL.status, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  CUDA_TRY(d, cudaMemcpyAsync(d->h_istats, base + SL.istats, 16 * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  CUDA_TRY(d, cudaMemcpyAsync(d->h_dstats, base + SL.dstats, 16 * sizeof(double), cudaMemcpyDeviceToHost, st));
  d->pending = true;
  d->pending_kind = 1;
  d->pending_stream = st;
  if (stats) return collect_stats(d, stats);
  return PISO_OK;
}

#ifdef PISO_TRACE
// Copy the phase-timing trace (trace builds only): n entries of PISO_TRACE_STAMPS stamps.
extern "C" int piso_trace_read(uint64_t* out, int n) {
  if (n > PISO_TRACE_LEN) n = PISO_TRACE_LEN;
  if (!g_trace_buf) return 0;
  if (cudaMemcpy(out, g_trace_buf, sizeof(uint64_t) * PISO_TRACE_STAMPS * n, cudaMemcpyDeviceToHost) != cudaSuccess)
    return -1;
  return n;
}
#endif
