// Turbulence-statistics operators (arXiv:2505.16992, Sec. 2.5 "Operators for
// Turbulence Statistics"; Sec. 3.3 "Losses from Turbulence Statistics").
//
// A *record* holds, for every plane y = const of a block (homogeneous
// directions x and z), the count n, the means and the central moments of nq
// per-cell fields normalised by the count, in doubles:
//   [n, mean[nq], m2[nq][nq], m3[nq][nq][nq] (order 3 only)]  per plane.
// Kernels:
//   stats_frame_kernel   one frame's record: two passes over the plane (mean,
//                        then central products), CTA = (plane, chunk of the
//                        unique moments), deterministic block sums in double
//   stats_merge_kernel   record of the union of two sample sets (pairwise
//                        update), one thread per plane: averaging over time is
//                        merging the frames' records, nothing else is stored
//   stats_adjoint_kernel dL/dq += (1/n)(G1_l + G2_lj a_j + G3_ljk a_j a_k) per
//                        cell, a = q - mean, the coefficients formed once per
//                        plane from the record and dL/d(record); applied with the
//                        accumulated record it is the derivative of the
//                        time-averaged statistics with respect to one frame
//   cell_gradients_kernel central differences mapped with T (the operator of
//                        Eq. velCorrDiscrete), ghost 2 u_b - u_P at Dirichlet
//                        faces for the velocity, p_P for the pressure
//   stats_budget_kernel  production, dissipation, turbulent transport, viscous
//                        diffusion and velocity pressure-gradient terms per y
#pragma once
#include "piso_device.cuh"

namespace piso {

constexpr int ST_MAXQ = 12;      // fields per record
constexpr int ST_CHUNK = 16;     // unique moments per CTA of the frame kernel
constexpr int ST_MAXU = 128;     // unique moments per record (nq <= 12 at order 2, nq <= 4 at order 3)

struct StatsGeom {
  int32_t nx, ny, nz, N, nq, order, rsize;
  int32_t nuniq;                  // unique moments: pairs i <= j, then triples i <= j <= k
  int8_t ui[ST_MAXU], uj[ST_MAXU], uk[ST_MAXU];   // uk = -1 for a pair
};

__device__ __forceinline__ int32_t st_cell(const StatsGeom& G, int32_t y, int32_t c) {
  const int32_t x = c % G.nx, z = c / G.nx;
  return x + G.nx * (y + G.ny * z);
}

// deterministic block sum of NV doubles per thread; result valid in thread 0
template <int NV>
__device__ __forceinline__ void st_block_sum(double (&v)[NV], double* s_red /* [32][NV] */) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int k = 0; k < NV; k++)
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], off);
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < NV; k++) s_red[warp * NV + k] = v[k];
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int k = 0; k < NV; k++) {
      double t = lane < nw ? s_red[lane * NV + k] : 0.0;
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) t += __shfl_down_sync(0xffffffffu, t, off);
      v[k] = t;
    }
  }
  __syncthreads();
}

// Deterministic block reduction of NV accumulators in their own arithmetic
// (float pairs on the FP32 pipe in the FP32 mode; FP64 is a small fraction of
// FP32 throughput on this GPU), converted to double once, in thread 0.
template <typename real, int NV>
__device__ __forceinline__ void st_acc_reduce(Acc<real> (&a)[NV], double* s_red /* [32][NV] */, double (&out)[NV]) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int k = 0; k < NV; k++) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) a[k].shfl_down_add(off);
    if (lane == 0) s_red[warp * NV + k] = a[k].pack();
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int k = 0; k < NV; k++) {
      Acc<real> t;
      t.zero();
      if (lane < nw) t.unpack_add(s_red[lane * NV + k]);
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) t.shfl_down_add(off);
      out[k] = t.to_double();
    }
  }
  __syncthreads();
}

// grid (ny, chunks); writes the frame's record entries of this chunk (chunk 0
// also n and the means)
template <typename real>
__global__ void __launch_bounds__(256) stats_frame_kernel(const __grid_constant__ StatsGeom G, const real* __restrict__ q,
                                                          double* __restrict__ rec) {
  __shared__ double s_red[32 * ST_CHUNK];
  __shared__ double s_mean[ST_MAXQ];
  const int32_t y = blockIdx.x;
  const int32_t np = G.nx * G.nz;
  const int32_t nq = G.nq;
  // pass 1: plane means
  {
    double v[ST_MAXQ];
#pragma unroll
    for (int i = 0; i < ST_MAXQ; i++) v[i] = 0.0;
    for (int32_t c = threadIdx.x; c < np; c += blockDim.x) {
      const int32_t cell = st_cell(G, y, c);
#pragma unroll
      for (int i = 0; i < ST_MAXQ; i++)
        if (i < nq) v[i] += (double)q[(size_t)i * G.N + cell];
    }
    st_block_sum<ST_MAXQ>(v, s_red);
    if (threadIdx.x == 0)
      for (int i = 0; i < nq; i++) s_mean[i] = v[i] / (double)np;
    __syncthreads();
  }
  // pass 2: this chunk's central products
  const int u0 = blockIdx.y * ST_CHUNK;
  double v[ST_CHUNK];
#pragma unroll
  for (int k = 0; k < ST_CHUNK; k++) v[k] = 0.0;
  for (int32_t c = threadIdx.x; c < np; c += blockDim.x) {
    const int32_t cell = st_cell(G, y, c);
    double a[ST_MAXQ];
#pragma unroll
    for (int i = 0; i < ST_MAXQ; i++) a[i] = i < nq ? (double)q[(size_t)i * G.N + cell] - s_mean[i] : 0.0;
#pragma unroll
    for (int k = 0; k < ST_CHUNK; k++) {
      const int u = u0 + k;
      if (u < G.nuniq) {
        double t = a[G.ui[u]] * a[G.uj[u]];
        if (G.uk[u] >= 0) t *= a[G.uk[u]];
        v[k] += t;
      }
    }
  }
  st_block_sum<ST_CHUNK>(v, s_red);
  if (threadIdx.x == 0) {
    double* R = rec + (size_t)y * G.rsize;
    const double inv = 1.0 / (double)np;
    if (blockIdx.y == 0) {
      R[0] = (double)np;
      for (int i = 0; i < nq; i++) R[1 + i] = s_mean[i];
    }
    double* m2 = R + 1 + nq;
    double* m3 = m2 + nq * nq;
    for (int k = 0; k < ST_CHUNK; k++) {
      const int u = u0 + k;
      if (u >= G.nuniq) break;
      const int i = G.ui[u], j = G.uj[u], l = G.uk[u];
      const double m = v[k] * inv;
      if (l < 0) {
        m2[i * nq + j] = m;
        m2[j * nq + i] = m;
      } else {   // all permutations of (i, j, l)
        m3[(i * nq + j) * nq + l] = m;
        m3[(i * nq + l) * nq + j] = m;
        m3[(j * nq + i) * nq + l] = m;
        m3[(j * nq + l) * nq + i] = m;
        m3[(l * nq + i) * nq + j] = m;
        m3[(l * nq + j) * nq + i] = m;
      }
    }
  }
}

// a <- merge(a, b) for one plane's records; a record with n = 0 in a takes
// b.  mean = mean_a + (nb/n) d, C2 = C2a + C2b + (na nb / n) d d,
// C3 = C3a + C3b + (na nb (na - nb) / n^2) d d d + (1/n) S(na C2b - nb C2a, d)
// with d = mean_b - mean_a, C = n m and S(M, d)_ijk = M_jk d_i + M_ik d_j + M_ij d_k.
__device__ void st_merge(const StatsGeom& G, double* __restrict__ A, const double* __restrict__ B) {
  const int nq = G.nq;
  const double na = A[0], nb = B[0];
  if (nb == 0.0) return;
  if (na == 0.0) {
    for (int k = 0; k < G.rsize; k++) A[k] = B[k];
    return;
  }
  const double n = na + nb;
  double d[ST_MAXQ];
  for (int i = 0; i < nq; i++) d[i] = B[1 + i] - A[1 + i];
  double* m2a = A + 1 + nq;
  const double* m2b = B + 1 + nq;
  if (G.order >= 3) {   // third moments first: they use both records' second moments
    double* m3a = m2a + nq * nq;
    const double* m3b = m2b + nq * nq;
    const double c3 = na * nb * (na - nb) / (n * n);
    for (int i = 0; i < nq; i++)
      for (int j = 0; j < nq; j++)
        for (int k = 0; k < nq; k++) {
          auto M = [&](int p, int r) { return na * nb * (m2b[p * nq + r] - m2a[p * nq + r]); };
          const double S = M(j, k) * d[i] + M(i, k) * d[j] + M(i, j) * d[k];
          const int idx = (i * nq + j) * nq + k;
          const double C3 = na * m3a[idx] + nb * m3b[idx] + c3 * d[i] * d[j] * d[k] + S / n;
          m3a[idx] = C3 / n;
        }
  }
  const double c2 = na * nb / n;
  for (int i = 0; i < nq; i++)
    for (int j = 0; j < nq; j++) {
      const int idx = i * nq + j;
      m2a[idx] = (na * m2a[idx] + nb * m2b[idx] + c2 * d[i] * d[j]) / n;
    }
  for (int i = 0; i < nq; i++) A[1 + i] += (nb / n) * d[i];
  A[0] = n;
}

// The same merge with one CTA per plane and one thread per record entry (the
// serial form above is a long chain of dependent FP64 operations, slow on this
// GPU's FP64 pipe): every thread reads A and B, forms its entries of the merged
// record, and all write after a barrier.  Called by all threads of the CTA.
__device__ void st_merge_block(const StatsGeom& G, double* __restrict__ A, const double* __restrict__ B) {
  constexpr int EPT = 8;   // entries per thread (record_size <= 8 * blockDim)
  const int nq = G.nq;
  const double na = A[0], nb = B[0];
  double nv[EPT];
  const double n = na + nb;
  int cnt = 0;
  for (int e = threadIdx.x; e < G.rsize && cnt < EPT; e += blockDim.x, cnt++) {
    double v;
    if (nb == 0.0) v = A[e];
    else if (na == 0.0) v = B[e];
    else if (e == 0) v = n;
    else if (e <= nq) {
      const int i = e - 1;
      v = A[e] + (nb / n) * (B[e] - A[e]);
    } else if (e <= nq + nq * nq) {
      const int t = e - 1 - nq, i = t / nq, j = t % nq;
      const double di = B[1 + i] - A[1 + i], dj = B[1 + j] - A[1 + j];
      v = (na * A[e] + nb * B[e] + (na * nb / n) * di * dj) / n;
    } else {
      const int t = e - 1 - nq - nq * nq, i = t / (nq * nq), j = (t / nq) % nq, k = t % nq;
      const double di = B[1 + i] - A[1 + i], dj = B[1 + j] - A[1 + j], dk = B[1 + k] - A[1 + k];
      const double* m2a = A + 1 + nq;
      const double* m2b = B + 1 + nq;
      auto M = [&](int p, int r) { return na * nb * (m2b[p * nq + r] - m2a[p * nq + r]); };
      const double S = M(j, k) * di + M(i, k) * dj + M(i, j) * dk;
      v = (na * A[e] + nb * B[e] + (na * nb * (na - nb) / (n * n)) * di * dj * dk + S / n) / n;
    }
    nv[cnt] = v;
  }
  __syncthreads();
  cnt = 0;
  for (int e = threadIdx.x; e < G.rsize && cnt < EPT; e += blockDim.x, cnt++) A[e] = nv[cnt];
  __syncthreads();
}

// a <- merge(a, b): one CTA per plane
__global__ void __launch_bounds__(128) stats_merge_kernel(const __grid_constant__ StatsGeom G, double* __restrict__ a,
                                                          const double* __restrict__ b) {
  st_merge_block(G, a + (size_t)blockIdx.x * G.rsize, b + (size_t)blockIdx.x * G.rsize);
}

// Partial records: grid (ny, S); CTA (y, s) takes the contiguous share s of
// plane y's cells, forms its own mean and central sums in two passes over the
// share (the second pass hits L1/L2) and writes them as a record of its count.
// NQ fields and moments up to ORD are fixed at compile time, so the moment
// list unrolls into registers.  Central values a = q - mean are formed in
// double; the FP32 mode then accumulates a_i a_j (a_k) as float pairs on the
// FP32 pipe (a = hi + lo, products from FMA-exact pieces; ~2^-44 relative),
// the FP64 mode in double.
template <typename real>
struct StAcc {   // FP64 mode: central values and sums in double
  using val = double;
  double v;
  __device__ __forceinline__ static val center(double q, double mean_hi, double mean_lo) { return q - mean_hi; }
  __device__ __forceinline__ static val mul(val a, val b) { return a * b; }
  __device__ __forceinline__ void zero() { v = 0.0; }
  __device__ __forceinline__ void add2(val ai, val aj) { v = fma(ai, aj, v); }
  __device__ __forceinline__ void add3(val aij, val ak) { v = fma(aij, ak, v); }
  __device__ __forceinline__ double get() const { return v; }
};

template <>
struct StAcc<float> {   // FP32 mode: float pairs on the FP32 pipe
  using val = f2;
  f2 v;
  // q - mean with the mean given as a float pair (hi, lo): TwoSum of q and -hi,
  // then -lo added to the error term
  __device__ __forceinline__ static val center(float q, float mean_hi, float mean_lo) {
    float s, e;
    two_sum(q, -mean_hi, s, e);
    return f2_norm(s, e - mean_lo);
  }
  __device__ __forceinline__ static val mul(val a, val b) {   // product of two float pairs, FMA-exact head
    const float p = a.hi * b.hi;
    const float e = fmaf(a.hi, b.hi, -p);
    return f2_norm(p, fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, e)));
  }
  __device__ __forceinline__ void zero() { v = f2{0.f, 0.f}; }
  __device__ __forceinline__ void add2(val ai, val aj) { v = f2_add(v, mul(ai, aj)); }
  __device__ __forceinline__ void add3(val aij, val ak) { v = f2_add(v, mul(aij, ak)); }
  __device__ __forceinline__ double get() const { return (double)v.hi + (double)v.lo; }
};

template <int NQ, int ORD>
struct StCount {
  static constexpr int U2 = NQ * (NQ + 1) / 2;
  static constexpr int U3 = ORD >= 3 ? NQ * (NQ + 1) * (NQ + 2) / 6 : 0;
  static constexpr int U = U2 + U3;
};

template <typename real, int NQ, int ORD>
__global__ void __launch_bounds__(256) stats_part_kernel(const __grid_constant__ StatsGeom G, const real* __restrict__ q,
                                                         double* __restrict__ part) {
  constexpr int U = StCount<NQ, ORD>::U;
  __shared__ double s_red[32 * (U > NQ ? U : NQ)];
  __shared__ double s_mean[NQ];
  const int32_t y = blockIdx.x, S = gridDim.y, sidx = blockIdx.y;
  const int32_t np = G.nx * G.nz;
  const int32_t c0 = (int32_t)(((int64_t)np * sidx) / S), c1 = (int32_t)(((int64_t)np * (sidx + 1)) / S);
  using Val = typename StAcc<real>::val;
  // pass 1: the share's mean (float-pair or double sums of the stored values)
  {
    Acc<real> s1[NQ];
#pragma unroll
    for (int i = 0; i < NQ; i++) s1[i].zero();
    for (int32_t c = c0 + threadIdx.x; c < c1; c += blockDim.x) {
      const int32_t cell = st_cell(G, y, c);
#pragma unroll
      for (int i = 0; i < NQ; i++) s1[i].add(q[(size_t)i * G.N + cell]);
    }
    double v[NQ];
    st_acc_reduce<real, NQ>(s1, s_red, v);
    if (threadIdx.x == 0)
#pragma unroll
      for (int i = 0; i < NQ; i++) s_mean[i] = c1 > c0 ? v[i] / (double)(c1 - c0) : 0.0;
    __syncthreads();
  }
  real mh[NQ], ml[NQ];   // the mean as a pair of storage-precision numbers
#pragma unroll
  for (int i = 0; i < NQ; i++) {
    mh[i] = (real)s_mean[i];
    ml[i] = (real)(s_mean[i] - (double)mh[i]);
  }
  // pass 2: central sums of the unique moments (i <= j, then i <= j <= k)
  StAcc<real> acc[U];
#pragma unroll
  for (int u = 0; u < U; u++) acc[u].zero();
  for (int32_t c = c0 + threadIdx.x; c < c1; c += blockDim.x) {
    const int32_t cell = st_cell(G, y, c);
    Val a[NQ];
#pragma unroll
    for (int i = 0; i < NQ; i++) a[i] = StAcc<real>::center(q[(size_t)i * G.N + cell], mh[i], ml[i]);
    int u = 0;
#pragma unroll
    for (int i = 0; i < NQ; i++)
#pragma unroll
      for (int j = i; j < NQ; j++) acc[u++].add2(a[i], a[j]);
    if (ORD >= 3) {
#pragma unroll
      for (int i = 0; i < NQ; i++)
#pragma unroll
        for (int j = i; j < NQ; j++) {
          const Val aij = StAcc<real>::mul(a[i], a[j]);
#pragma unroll
          for (int k = j; k < NQ; k++) acc[u++].add3(aij, a[k]);
        }
    }
  }
  double v[U];
  {
    Acc<real> ra[U];   // the same sums as reduction accumulators (same member type)
#pragma unroll
    for (int u = 0; u < U; u++) ra[u].v = acc[u].v;
    st_acc_reduce<real, U>(ra, s_red, v);
  }
  if (threadIdx.x == 0) {
    double* R = part + ((size_t)y * S + sidx) * G.rsize;
    const double n = (double)(c1 - c0);
    const double inv = n > 0 ? 1.0 / n : 0.0;
    R[0] = n;
#pragma unroll
    for (int i = 0; i < NQ; i++) R[1 + i] = s_mean[i];
    double* m2 = R + 1 + NQ;
    double* m3 = m2 + NQ * NQ;
    int u = 0;
#pragma unroll
    for (int i = 0; i < NQ; i++)
#pragma unroll
      for (int j = i; j < NQ; j++) {
        const double m = v[u++] * inv;
        m2[i * NQ + j] = m;
        m2[j * NQ + i] = m;
      }
    if (ORD >= 3) {
#pragma unroll
      for (int i = 0; i < NQ; i++)
#pragma unroll
        for (int j = i; j < NQ; j++)
#pragma unroll
          for (int k = j; k < NQ; k++) {
            const double m = v[u++] * inv;
            m3[(i * NQ + j) * NQ + k] = m;
            m3[(i * NQ + k) * NQ + j] = m;
            m3[(j * NQ + i) * NQ + k] = m;
            m3[(j * NQ + k) * NQ + i] = m;
            m3[(k * NQ + i) * NQ + j] = m;
            m3[(k * NQ + j) * NQ + i] = m;
          }
    }
  }
}

// rec[y] = merge of the S partial records of plane y in order; acc[y] (if
// given) <- merge(acc[y], rec[y]).  One CTA per plane.
__global__ void __launch_bounds__(128) stats_combine_kernel(const __grid_constant__ StatsGeom G,
                                                            const double* __restrict__ part, int32_t S,
                                                            double* __restrict__ rec, double* __restrict__ acc) {
  const int32_t y = blockIdx.x;
  double* R = rec + (size_t)y * G.rsize;
  const double* P0 = part + (size_t)y * S * G.rsize;
  for (int e = threadIdx.x; e < G.rsize; e += blockDim.x) R[e] = P0[e];
  __syncthreads();
  for (int s = 1; s < S; s++) st_merge_block(G, R, P0 + (size_t)s * G.rsize);
  if (acc) st_merge_block(G, acc + (size_t)y * G.rsize, R);
}

// dq[l][cell] += (1/n) (G1_l + sum_j G2_lj a_j + sum_jk G3_ljk a_j a_k), a = q - mean,
// with G2_lj = g2_lj + g2_jl, G3_ljk = g3_ljk + g3_jlk + g3_jkl and
// G1_l = gmean_l - sum_jk G3_ljk m2_jk.  Grid (ny, splits): each CTA forms its
// plane's coefficients in shared memory, then walks a share of the plane.
template <typename real>
__global__ void __launch_bounds__(256) stats_adjoint_kernel(const __grid_constant__ StatsGeom G,
                                                            const real* __restrict__ q,
                                                            const double* __restrict__ rec,
                                                            const double* __restrict__ grad, real* __restrict__ dq) {
  __shared__ double s_mean[ST_MAXQ], s_G1[ST_MAXQ];
  __shared__ double s_G2[ST_MAXQ * ST_MAXQ];
  __shared__ double s_G3[4 * 4 * 4];
  const int32_t y = blockIdx.x;
  const int nq = G.nq;
  const double* R = rec + (size_t)y * G.rsize;
  const double* g = grad + (size_t)y * G.rsize;
  const double* m2 = R + 1 + nq;
  const double* g2 = g + 1 + nq;
  const double* g3 = g2 + nq * nq;
  const bool o3 = G.order >= 3;
  for (int t = threadIdx.x; t < nq * nq; t += blockDim.x) {
    const int l = t / nq, j = t % nq;
    s_G2[t] = g2[l * nq + j] + g2[j * nq + l];
  }
  if (o3)
    for (int t = threadIdx.x; t < nq * nq * nq; t += blockDim.x) {
      const int l = t / (nq * nq), j = (t / nq) % nq, k = t % nq;
      s_G3[t] = g3[(l * nq + j) * nq + k] + g3[(j * nq + l) * nq + k] + g3[(j * nq + k) * nq + l];
    }
  __syncthreads();
  if (threadIdx.x < nq) {
    const int l = threadIdx.x;
    double G1 = g[1 + l];
    if (o3)
      for (int j = 0; j < nq; j++)
        for (int k = 0; k < nq; k++) G1 -= s_G3[(l * nq + j) * nq + k] * m2[j * nq + k];
    s_G1[l] = G1;
    s_mean[l] = R[1 + l];
  }
  __syncthreads();
  const double inv = R[0] > 0.0 ? 1.0 / R[0] : 0.0;
  const int32_t np = G.nx * G.nz;
  for (int32_t c = blockIdx.y * blockDim.x + threadIdx.x; c < np; c += gridDim.y * blockDim.x) {
    const int32_t cell = st_cell(G, y, c);
    double a[ST_MAXQ];
#pragma unroll
    for (int i = 0; i < ST_MAXQ; i++) a[i] = i < nq ? (double)q[(size_t)i * G.N + cell] - s_mean[i] : 0.0;
#pragma unroll
    for (int l = 0; l < ST_MAXQ; l++) {
      if (l >= nq) break;
      double v = s_G1[l];
      for (int j = 0; j < nq; j++) {
        v += s_G2[l * nq + j] * a[j];
        if (o3)
          for (int k = 0; k < nq; k++) v += s_G3[(l * nq + j) * nq + k] * a[j] * a[k];
      }
      real* o = dq + (size_t)l * G.N + cell;
      *o = *o + (real)(v * inv);
    }
  }
}

// The adjoint with NQ and ORD fixed at compile time and the per-cell work in
// the storage precision (the coefficients are formed in double once per plane
// and rounded): dq is stored in that precision anyway, and the FP32 mode then
// stays off the FP64 pipe.
template <typename real, int NQ, int ORD>
__global__ void __launch_bounds__(256) stats_adjoint_t_kernel(const __grid_constant__ StatsGeom G,
                                                              const real* __restrict__ q,
                                                              const double* __restrict__ rec,
                                                              const double* __restrict__ grad,
                                                              real* __restrict__ dq) {
  __shared__ real s_mean[NQ], s_G1[NQ], s_G2[NQ * NQ], s_G3[ORD >= 3 ? NQ * NQ * NQ : 1];
  __shared__ real s_inv;
  const int32_t y = blockIdx.x;
  const double* R = rec + (size_t)y * G.rsize;
  const double* g = grad + (size_t)y * G.rsize;
  const double* m2 = R + 1 + NQ;
  const double* g2 = g + 1 + NQ;
  const double* g3 = g2 + NQ * NQ;
  for (int t = threadIdx.x; t < NQ * NQ; t += blockDim.x) {
    const int l = t / NQ, j = t % NQ;
    s_G2[t] = (real)(g2[l * NQ + j] + g2[j * NQ + l]);
  }
  if (threadIdx.x < NQ) {
    const int l = threadIdx.x;
    double G1 = g[1 + l];
    if (ORD >= 3)
      for (int j = 0; j < NQ; j++)
        for (int k = 0; k < NQ; k++) {
          const double G3 = g3[(l * NQ + j) * NQ + k] + g3[(j * NQ + l) * NQ + k] + g3[(j * NQ + k) * NQ + l];
          s_G3[(l * NQ + j) * NQ + k] = (real)G3;
          G1 -= G3 * m2[j * NQ + k];
        }
    s_G1[l] = (real)G1;
    s_mean[l] = (real)R[1 + l];
  }
  if (threadIdx.x == 0) s_inv = (real)(R[0] > 0.0 ? 1.0 / R[0] : 0.0);
  __syncthreads();
  const int32_t np = G.nx * G.nz;
  const real inv = s_inv;
  for (int32_t c = blockIdx.y * blockDim.x + threadIdx.x; c < np; c += gridDim.y * blockDim.x) {
    const int32_t cell = st_cell(G, y, c);
    real a[NQ], o[NQ];
#pragma unroll
    for (int i = 0; i < NQ; i++) a[i] = q[(size_t)i * G.N + cell] - s_mean[i];
#pragma unroll
    for (int l = 0; l < NQ; l++) o[l] = dq[(size_t)l * G.N + cell];
#pragma unroll
    for (int l = 0; l < NQ; l++) {
      real v = s_G1[l];
#pragma unroll
      for (int j = 0; j < NQ; j++) {
        v += s_G2[l * NQ + j] * a[j];
        if (ORD >= 3) {
          real w = 0;
#pragma unroll
          for (int k = 0; k < NQ; k++) w += s_G3[(l * NQ + j) * NQ + k] * a[k];
          v += w * a[j];
        }
      }
      dq[(size_t)l * G.N + cell] = o[l] + v * inv;
    }
  }
}

// d u_i / d x_k and d p / d x_k at cell centres: sum_j T_jk (f(+j) - f(-j)) / 2
// with f(+-j) the neighbour's value, or at a boundary face the ghost
// 2 u_b - u_P (velocity) / p_P (pressure).
template <typename real, int ND>
__global__ void __launch_bounds__(256) cell_gradients_kernel(const DomStatic* __restrict__ Dp, const real* __restrict__ u,
                                                             const real* __restrict__ p, const real* __restrict__ bval,
                                                             real* __restrict__ gu, real* __restrict__ gp) {
  __shared__ DomStatic D;
  for (int k = threadIdx.x; k < (int)(sizeof(DomStatic) / 4); k += blockDim.x)
    reinterpret_cast<int32_t*>(&D)[k] = reinterpret_cast<const int32_t*>(Dp)[k];
  __syncthreads();
  const int32_t N = D.N, nbf = D.nbf;
  const real* T = reinterpret_cast<const real*>(D.T);
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    const Cell c = locate<ND>(D, i);
    real du[ND][ND], dp[ND];   // du[comp][axis j]
#pragma unroll
    for (int j = 0; j < ND; j++) {
      dp[j] = 0;
#pragma unroll
      for (int s2 = 0; s2 < 2; s2++) {
        const int s = 2 * j + s2;
        const real sg = s2 ? real(0.5) : real(-0.5);
        const int32_t F = c.nb[s];
#pragma unroll
        for (int m = 0; m < ND; m++) {
          const real uP = u[(size_t)m * N + i];
          const real v = F >= 0 ? u[(size_t)m * N + F] : real(2) * bval[(size_t)m * nbf + (-1 - F)] - uP;
          if (s2 == 0) du[m][j] = sg * v;
          else du[m][j] += sg * v;
        }
        if (p) dp[j] += sg * (F >= 0 ? p[F] : p[i]);
      }
    }
#pragma unroll
    for (int k = 0; k < ND; k++) {
#pragma unroll
      for (int m = 0; m < ND; m++) {
        real s = 0;
#pragma unroll
        for (int j = 0; j < ND; j++) s += T[(size_t)(j * ND + k) * N + i] * du[m][j];
        if (gu) gu[(size_t)(m * ND + k) * N + i] = s;
      }
      if (gp) {
        real s = 0;
#pragma unroll
        for (int j = 0; j < ND; j++) s += T[(size_t)(j * ND + k) * N + i] * dp[j];
        gp[(size_t)k * N + i] = s;
      }
    }
  }
}

// three-point y-derivatives of a profile on {y0, yc..., y1} with zero wall values
__device__ __forceinline__ void st_dy(const double* f, int stride, int y, int ny, const double* yc, double y0, double y1,
                                      double& d1, double& d2) {
  const double Ym = y > 0 ? yc[y - 1] : y0, Y0 = yc[y], Yp = y < ny - 1 ? yc[y + 1] : y1;
  const double fm = y > 0 ? f[(size_t)(y - 1) * stride] : 0.0, f0 = f[(size_t)y * stride];
  const double fp = y < ny - 1 ? f[(size_t)(y + 1) * stride] : 0.0;
  const double hm = Y0 - Ym, hp = Yp - Y0;
  d1 = (hm * hm * fp - hp * hp * fm + (hp * hp - hm * hm) * f0) / (hm * hp * (hm + hp));
  d2 = 2.0 * (hm * fp - (hm + hp) * f0 + hp * fm) / (hm * hp * (hm + hp));
}

// Budget terms per plane (one thread per plane) from the records of u (nq = d,
// order 3), of grad u (nq = d^2, q index i*d + k, order 2 or 3) and of
// (u, grad p) (nq = 2d, order 2 or 3): out [5][ny][d][d] = P, eps, T, D, Pi.
__global__ void stats_budget_kernel(int32_t ny, int32_t d, const double* __restrict__ ru, int32_t rs_u,
                                    const double* __restrict__ rg, int32_t rs_g, const double* __restrict__ rp,
                                    int32_t rs_p, const double* __restrict__ yc, double y0, double y1, double nu,
                                    double* __restrict__ out) {
  const int32_t y = blockIdx.x * blockDim.x + threadIdx.x;
  if (y >= ny) return;
  const int dd = d * d;
  const double* U = ru + (size_t)y * rs_u;
  const double* R = U + 1 + d;                    // m2 of u
  const int qg = d * d, qp = 2 * d;
  const double* Gm2 = rg + (size_t)y * rs_g + 1 + qg;
  const double* Pm2 = rp + (size_t)y * rs_p + 1 + qp;
  double* P = out + ((size_t)0 * ny + y) * dd;
  double* E = out + ((size_t)1 * ny + y) * dd;
  double* Tt = out + ((size_t)2 * ny + y) * dd;
  double* Dd = out + ((size_t)3 * ny + y) * dd;
  double* Pi = out + ((size_t)4 * ny + y) * dd;
  double dU[3], dummy;
  for (int i = 0; i < d; i++) st_dy(ru + 1 + i, rs_u, y, ny, yc, y0, y1, dU[i], dummy);
  for (int i = 0; i < d; i++)
    for (int j = 0; j < d; j++) {
      P[i * d + j] = -(R[i * d + 1] * dU[j] + R[j * d + 1] * dU[i]);
      double e = 0;
      for (int k = 0; k < d; k++) e += Gm2[(i * d + k) * qg + (j * d + k)];
      E[i * d + j] = 2.0 * nu * e;
      double t1, t2, r1, r2;
      st_dy(ru + 1 + d + dd + (i * d + j) * d + 1, rs_u, y, ny, yc, y0, y1, t1, t2);   // <u_i' u_j' v'>
      Tt[i * d + j] = -t1;
      st_dy(ru + 1 + d + i * d + j, rs_u, y, ny, yc, y0, y1, r1, r2);                  // R_ij
      Dd[i * d + j] = nu * r2;
      Pi[i * d + j] = -(Pm2[i * qp + d + j] + Pm2[j * qp + d + i]);
    }
}

}  // namespace piso
