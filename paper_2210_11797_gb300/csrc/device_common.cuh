// Device helpers shared by the kernels: deterministic grid reductions and the indexing of
// the trace rows of S.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "hmg_internal.cuh"

namespace hmg {

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum over the thread block of NV per-thread values, in a fixed order; the sums are valid in
// warp 0. With blockDim.x <= kRedThreads one warp adds the staged values 8 per lane, then a
// 5-step shuffle tree: 12 FP64 warp instructions per value and block instead of 45 for a
// shuffle tree in every warp (the FP64 pipe is the scarce unit of this GPU's sparse kernels).
template <int NV>
__device__ __forceinline__ void block_sum(const double (&val)[NV], double (&out)[NV]) {
  const int t = threadIdx.x, lane = t & 31;
  const int nt = (int)blockDim.x;
  if (nt <= kRedThreads) {
    __shared__ double sh[NV][kRedThreads];
#pragma unroll
    for (int i = 0; i < NV; ++i) sh[i][t] = val[i];
    __syncthreads();
    if (t < 32) {
#pragma unroll
      for (int i = 0; i < NV; ++i) {
        double v = lane < nt ? sh[i][lane] : 0.0;
        for (int j = lane + 32; j < nt; j += 32) v += sh[i][j];
        out[i] = warp_sum(v);
      }
    }
  } else {
    __shared__ double sw[NV][32];
    const int warp = t >> 5, nwarp = (nt + 31) >> 5;
#pragma unroll
    for (int i = 0; i < NV; ++i) {
      double v = warp_sum(val[i]);
      if (lane == 0) sw[i][warp] = v;
    }
    __syncthreads();
    if (t < 32) {
#pragma unroll
      for (int i = 0; i < NV; ++i) out[i] = warp_sum(lane < nwarp ? sw[i][lane] : 0.0);
    }
  }
}

// Deterministic reduction of NV per-thread values over the whole grid (gridDim.x <=
// kMaxRedBlocks, blockDim.x a multiple of 32, <= 1024). Each block writes its partial sums to
// part[slot][blockIdx.x]; the block that takes the last ticket sums the partials in block
// order and writes scal[slot]. The summation order depends only on the launch shape, so
// repeated runs give bit-identical results. No block waits on another.
template <int NV>
__device__ __forceinline__ void grid_reduce(const double (&val)[NV], const int (&slot)[NV],
                                            double *part, unsigned int *counter, double *scal) {
  __shared__ double sh[NV][32];
  __shared__ bool is_last;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nwarp = (blockDim.x + 31) >> 5;
  double bs[NV];
  block_sum<NV>(val, bs);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int i = 0; i < NV; ++i) part[(int64_t)slot[i] * kMaxRedBlocks + blockIdx.x] = bs[i];
  }
  if (threadIdx.x == 0) {
    __threadfence();
    unsigned int ticket = atomicAdd(&counter[slot[0]], 1u);
    is_last = (ticket == gridDim.x - 1);
  }
  __syncthreads();
  if (!is_last) return;
  __threadfence();
#pragma unroll
  for (int i = 0; i < NV; ++i) {
    double v = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x)
      v += __ldcg(&part[(int64_t)slot[i] * kMaxRedBlocks + b]);
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) sh[i][warp] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
      double s = 0.0;
      for (int w = 0; w < nwarp; ++w) s += sh[i][w];
      scal[slot[i]] = s;
    }
  }
  if (threadIdx.x == 0) counter[slot[0]] = 0u;
}

// Block-level sums of NV per-thread values written to part[slot][blockIdx.x] (no atomics, no
// fences); finalize_kernel reduces them. For one-row-per-thread kernels with ~10^4-10^5
// blocks, where a single ticket counter serialises every block on one atomic.
template <int NV>
__device__ __forceinline__ void block_partials(const double (&val)[NV], const int (&slot)[NV],
                                               double *part) {
  double bs[NV];
  block_sum<NV>(val, bs);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int i = 0; i < NV; ++i) part[(int64_t)slot[i] * kMaxRedBlocks + blockIdx.x] = bs[i];
  }
}

template <typename T>
__device__ __forceinline__ T ld(const T *p) { return __ldg(p); }

// ---- trace rows of S ------------------------------------------------------------------
// h-row (edge e, level k): slot 0 self; 1-3 the other vertical faces of c1 (local faces
// i1+1, i1+2, i1+3 mod 4); 4, 5 bottom/top of cell (c1, k); 6-8 the other vertical faces
// of c2; 9, 10 bottom/top of (c2, k). st = edge_stencil + 8 e = {c1, c2, ea1..3, eb1..3}.
// z-row (column c, interface k): slot 0 self; 1-4 vertical faces e0..e3 of the cell above
// (c, k); 5 its top (k+1); 6-9 vertical faces of the cell below (c, k-1); 10 its bottom.
struct TraceDims {
  int L;          // layers
  int64_t NH;     // h-rows = nedge * L
  int64_t NT;     // all rows
};

// bbar_K = Gamma_K (P^T R)_K for cell K = (column c, layer k) (Algorithm 2 lines 4-5). P^T
// weights: 1/2 on interior faces (both neighbours share the facet), 1 on ground and lid; the
// weights scale exactly, so each FMA rounds as a product-then-add would.
template <typename T>
__device__ __forceinline__ T trace_restrict_cell(const T *__restrict__ R, const T *__restrict__ gamma,
                                                 const int32_t *__restrict__ col_edges, const TraceDims &d,
                                                 int c, int k, int64_t K) {
  const int32_t *ce = col_edges + 4 * (int64_t)c;
  T s = (T)0.5 * (R[(int64_t)__ldg(ce) * d.L + k] + R[(int64_t)__ldg(ce + 1) * d.L + k] +
                  R[(int64_t)__ldg(ce + 2) * d.L + k] + R[(int64_t)__ldg(ce + 3) * d.L + k]);
  const int64_t zb = d.NH + (int64_t)c * (d.L + 1) + k;
  s = fma(k == 0 ? (T)1 : (T)0.5, R[zb], s);
  s = fma(k == d.L - 1 ? (T)1 : (T)0.5, R[zb + 1], s);
  return gamma[K] * s;
}

// acc + sign * (row of S) . x as a chain of fused multiply-adds, one per coefficient: with
// acc = 0, sign = +1 it is S x; with acc = b, sign = -1 it is the residual b - S x without a
// separate subtraction (the FP64 issue rate, not HBM, bounds these kernels on GB300). S is
// larger than L2 and read once per kernel, so its loads are marked evict-first: the gathered
// x values and the other vectors stay in L2.
template <typename TS, typename TX, typename TA, bool NEG>
__device__ __forceinline__ TA s_row_h(const TS *__restrict__ S, const TX *__restrict__ x,
                                      const int32_t *__restrict__ stencil, const TraceDims d,
                                      int64_t row, TA acc) {
  const int e = (int)(row / d.L);
  const int k = (int)(row - (int64_t)e * d.L);
  const int32_t *st = stencil + 8 * (int64_t)e;
  const int c1 = __ldg(st + 0), c2 = __ldg(st + 1);
  const int64_t z1 = d.NH + (int64_t)c1 * (d.L + 1) + k;
  const int64_t z2 = d.NH + (int64_t)c2 * (d.L + 1) + k;
  const int64_t T = d.NT;
  auto term = [&](int slot, int64_t col) {
    const TA a = (TA)__ldcs(S + slot * T + row);   // S streams through once: evict first
    acc = fma(NEG ? -a : a, (TA)ld(x + col), acc);
  };
  term(0, row);
  term(1, (int64_t)__ldg(st + 2) * d.L + k);
  term(2, (int64_t)__ldg(st + 3) * d.L + k);
  term(3, (int64_t)__ldg(st + 4) * d.L + k);
  term(4, z1);
  term(5, z1 + 1);
  term(6, (int64_t)__ldg(st + 5) * d.L + k);
  term(7, (int64_t)__ldg(st + 6) * d.L + k);
  term(8, (int64_t)__ldg(st + 7) * d.L + k);
  term(9, z2);
  term(10, z2 + 1);
  return acc;
}

template <typename TS, typename TX, typename TA, bool NEG>
__device__ __forceinline__ TA s_row_z(const TS *__restrict__ S, const TX *__restrict__ x,
                                      const int32_t *__restrict__ col_edges, const TraceDims d,
                                      int64_t row, TA acc) {
  const int64_t zr = row - d.NH;
  const int c = (int)(zr / (d.L + 1));
  const int k = (int)(zr - (int64_t)c * (d.L + 1));
  const int64_t T = d.NT;
  const int32_t *ce = col_edges + 4 * (int64_t)c;
  auto term = [&](int slot, int64_t col) {
    const TA a = (TA)__ldcs(S + slot * T + row);   // S streams through once: evict first
    acc = fma(NEG ? -a : a, (TA)ld(x + col), acc);
  };
  term(0, row);
  if (k < d.L) {
    term(1, (int64_t)__ldg(ce + 0) * d.L + k);
    term(2, (int64_t)__ldg(ce + 1) * d.L + k);
    term(3, (int64_t)__ldg(ce + 2) * d.L + k);
    term(4, (int64_t)__ldg(ce + 3) * d.L + k);
    term(5, row + 1);
  }
  if (k > 0) {
    term(6, (int64_t)__ldg(ce + 0) * d.L + k - 1);
    term(7, (int64_t)__ldg(ce + 1) * d.L + k - 1);
    term(8, (int64_t)__ldg(ce + 2) * d.L + k - 1);
    term(9, (int64_t)__ldg(ce + 3) * d.L + k - 1);
    term(10, row - 1);
  }
  return acc;
}

// The same rows without the couplings of the smoother's diagonal block D (Algorithm 1:
// D = [diag(S^hh), blockdiag(S^zz_c)]): an h-row without its diagonal (slots 1-10), a z-row
// without the diagonal and its vertical neighbours (slots 1-4 and 6-9), acc - (S - D) x.
template <typename TS, typename TX, typename TA>
__device__ __forceinline__ TA s_row_h_off(const TS *__restrict__ S, const TX *__restrict__ x,
                                          const int32_t *__restrict__ stencil, const TraceDims d,
                                          int64_t row, TA acc) {
  const int e = (int)(row / d.L);
  const int k = (int)(row - (int64_t)e * d.L);
  const int32_t *st = stencil + 8 * (int64_t)e;
  const int c1 = __ldg(st + 0), c2 = __ldg(st + 1);
  const int64_t z1 = d.NH + (int64_t)c1 * (d.L + 1) + k;
  const int64_t z2 = d.NH + (int64_t)c2 * (d.L + 1) + k;
  const int64_t T = d.NT;
  auto term = [&](int slot, int64_t col) {
    const TA a = (TA)__ldcs(S + slot * T + row);
    acc = fma(-a, (TA)ld(x + col), acc);
  };
  term(1, (int64_t)__ldg(st + 2) * d.L + k);
  term(2, (int64_t)__ldg(st + 3) * d.L + k);
  term(3, (int64_t)__ldg(st + 4) * d.L + k);
  term(4, z1);
  term(5, z1 + 1);
  term(6, (int64_t)__ldg(st + 5) * d.L + k);
  term(7, (int64_t)__ldg(st + 6) * d.L + k);
  term(8, (int64_t)__ldg(st + 7) * d.L + k);
  term(9, z2);
  term(10, z2 + 1);
  return acc;
}

template <typename TS, typename TX, typename TA>
__device__ __forceinline__ TA s_row_z_off(const TS *__restrict__ S, const TX *__restrict__ x,
                                          const int32_t *__restrict__ col_edges, const TraceDims d,
                                          int64_t row, TA acc) {
  const int64_t zr = row - d.NH;
  const int c = (int)(zr / (d.L + 1));
  const int k = (int)(zr - (int64_t)c * (d.L + 1));
  const int64_t T = d.NT;
  const int32_t *ce = col_edges + 4 * (int64_t)c;
  auto term = [&](int slot, int64_t col) {
    const TA a = (TA)__ldcs(S + slot * T + row);
    acc = fma(-a, (TA)ld(x + col), acc);
  };
  if (k < d.L) {
    term(1, (int64_t)__ldg(ce + 0) * d.L + k);
    term(2, (int64_t)__ldg(ce + 1) * d.L + k);
    term(3, (int64_t)__ldg(ce + 2) * d.L + k);
    term(4, (int64_t)__ldg(ce + 3) * d.L + k);
  }
  if (k > 0) {
    term(6, (int64_t)__ldg(ce + 0) * d.L + k - 1);
    term(7, (int64_t)__ldg(ce + 1) * d.L + k - 1);
    term(8, (int64_t)__ldg(ce + 2) * d.L + k - 1);
    term(9, (int64_t)__ldg(ce + 3) * d.L + k - 1);
  }
  return acc;
}

// The serial Thomas recurrences of one column held in shared memory (one thread): on entry
// s[o + k] = the scaled right-hand side, lo[o + k] the sub-diagonal / pivot (k >= 1), up[o + k]
// the super-diagonal / pivot (k <= n - 2); on return s[o + k] = the solution. Forward
// y_k = s_k - lo_k y_{k-1}, backward x_k = y_k - up_k x_{k+1}, one FMA per row each, in the
// order of the plain loops; the loads of CH rows are issued ahead of their FMAs, so that only
// the FMA latency stays on the dependent chain.
template <typename T, int CH = 8>
__device__ __forceinline__ void thomas_smem(T *s, const T *lo, const T *up, int o, int n) {
  T y = s[o];
  int k = 1;
  for (; k + CH - 1 < n; k += CH) {
    T l[CH], r[CH];
#pragma unroll
    for (int j = 0; j < CH; ++j) {
      l[j] = lo[o + k + j];
      r[j] = s[o + k + j];
    }
#pragma unroll
    for (int j = 0; j < CH; ++j) {
      y = fma(-l[j], y, r[j]);
      s[o + k + j] = y;
    }
  }
  for (; k < n; ++k) {
    y = fma(-lo[o + k], y, s[o + k]);
    s[o + k] = y;
  }
  T x = y;
  k = n - 2;
  for (; k >= CH - 1; k -= CH) {
    T u[CH], r[CH];
#pragma unroll
    for (int j = 0; j < CH; ++j) {
      u[j] = up[o + k - j];
      r[j] = s[o + k - j];
    }
#pragma unroll
    for (int j = 0; j < CH; ++j) {
      x = fma(-u[j], x, r[j]);
      s[o + k - j] = x;
    }
  }
  for (; k >= 0; --k) {
    x = fma(-up[o + k], x, s[o + k]);
    s[o + k] = x;
  }
}

// A tridiagonal solve with precomputed Thomas factors by one warp (n <= 32 M rows; lane j holds
// rows j M .. j M + M - 1): on entry s = the scaled right-hand side (r omega / pivot), lo the
// sub-diagonal / pivot (0 on row 0), up the super-diagonal / pivot (0 on row n - 1); on return
// s = the solution. The recurrences y_k = s_k - lo_k y_{k-1} and x_k = y_k - up_k x_{k+1} are
// chains of affine maps v -> A + M v: each lane composes its own rows, a warp scan (five shuffle
// steps) composes the lanes before it (after it, backwards), then the lane replays its rows from
// the value it receives. About ten times the serial form's multiply-adds: for FP32 kernels.
template <typename T, int M>
__device__ __forceinline__ void warp_thomas(T (&s)[M], const T (&lo)[M], const T (&up)[M], int lane, int n) {
  constexpr unsigned kAll = 0xffffffffu;
  T A = (T)0, Mf = (T)1;
#pragma unroll
  for (int i = 0; i < M; ++i)
    if (lane * M + i < n) {
      A = fma(-lo[i], A, s[i]);
      Mf = -lo[i] * Mf;
    }
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const T A2 = __shfl_up_sync(kAll, A, off), M2 = __shfl_up_sync(kAll, Mf, off);
    if (lane >= off) {
      A = fma(Mf, A2, A);
      Mf *= M2;
    }
  }
  T y = __shfl_up_sync(kAll, A, 1);
  if (lane == 0) y = (T)0;
#pragma unroll
  for (int i = 0; i < M; ++i)
    if (lane * M + i < n) {
      y = fma(-lo[i], y, s[i]);
      s[i] = y;
    }
  A = (T)0;
  Mf = (T)1;
#pragma unroll
  for (int i = M - 1; i >= 0; --i)
    if (lane * M + i < n) {
      A = fma(-up[i], A, s[i]);
      Mf = -up[i] * Mf;
    }
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const T A2 = __shfl_down_sync(kAll, A, off), M2 = __shfl_down_sync(kAll, Mf, off);
    if (lane + off < 32) {
      A = fma(Mf, A2, A);
      Mf *= M2;
    }
  }
  T x = __shfl_down_sync(kAll, A, 1);
  if (lane == 31) x = (T)0;
#pragma unroll
  for (int i = M - 1; i >= 0; --i)
    if (lane * M + i < n) {
      x = fma(-up[i], x, s[i]);
      s[i] = x;
    }
}

template <typename TS, typename TX, typename TA, bool NEG>
__device__ __forceinline__ TA s_row(const TS *__restrict__ S, const TX *__restrict__ x,
                                    const int32_t *__restrict__ stencil,
                                    const int32_t *__restrict__ col_edges, const TraceDims d,
                                    int64_t row, TA acc) {
  return row < d.NH ? s_row_h<TS, TX, TA, NEG>(S, x, stencil, d, row, acc)
                    : s_row_z<TS, TX, TA, NEG>(S, x, col_edges, d, row, acc);
}

}  // namespace hmg
