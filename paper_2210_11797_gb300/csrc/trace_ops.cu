// Trace-space kernels of the solve: S apply (with fused inner products), the right-hand
// side B_lambda, recovery, the line smoother (Algorithm 1), residual / restriction with the
// coarse scaling, prolongation, and the two preconditioners (configuration 2: line smoother;
// configuration 3c: Algorithm 2).
//
// Paper (arXiv 2210.11797): Eqs. hybrid-S, hybrid-rhs, hybrid-recovery (Sec. 2.4);
// Algorithm 1 and Eq. banded_system; Algorithm 2; Sec. 2.5 intergrid operators
// (P lambda = {{Pi}}, Restrict = P^T) and Eq. scaling_matrix.
#include "device_common.cuh"
#include "hmg_internal.cuh"
#include "precond.cuh"

namespace hmg {

static TraceDims dims_of(const Level &f) { return TraceDims{f.nlev, f.nth, f.ntrace}; }

constexpr int kSpmvRows = 4;   // rows of S per thread in the S apply with fused reductions

// ---- y = S x with optional fused inner products -----------------------------------------
template <int MODE>
__global__ void __launch_bounds__(kRedThreads)
    spmv_kernel(const double *__restrict__ S, const double *__restrict__ x, double *__restrict__ y,
                const double *__restrict__ w, const TraceDims d, const int32_t *__restrict__ stencil,
                const int32_t *__restrict__ col_edges, double *part, int slot0, int slot1) {
  // kSpmvRows rows per thread (block-strided, so each pass stays coalesced, and four rows'
  // gathers in flight per thread): the block's reduction is paid once per kSpmvRows rows.
  // (A persistent grid striding one row per pass, with the partial sums added by the last
  // block, measured 33% slower at C96.)
  double a0 = 0.0, a1 = 0.0;
  const int64_t base = (int64_t)blockIdx.x * blockDim.x * kSpmvRows + threadIdx.x;
#pragma unroll
  for (int j = 0; j < kSpmvRows; ++j) {
    const int64_t row = base + (int64_t)j * blockDim.x;
    if (row < d.NT) {
      if (MODE == 3) {
        const double v = s_row<double, double, double, true>(S, x, stencil, col_edges, d, row, __ldg(w + row));
        a0 = fma(v, v, a0);
      } else {
        const double v = s_row<double, double, double, false>(S, x, stencil, col_edges, d, row, 0.0);
        y[row] = v;
        if (MODE == 1) a0 = fma(__ldg(w + row), v, a0);
        if (MODE == 2) { a0 = fma(v, __ldg(w + row), a0); a1 = fma(v, v, a1); }
      }
    }
  }
  if (MODE == 1 || MODE == 3) {
    const double val[1] = {a0};
    const int sl[1] = {slot0};
    block_partials<1>(val, sl, part);
  } else if (MODE == 2) {
    const double val[2] = {a0, a1};
    const int sl[2] = {slot0, slot1};
    block_partials<2>(val, sl, part);
  }
}

// Sum of the per-block partials of slots s0 (and s1) into scal, in a fixed order.
__global__ void __launch_bounds__(1024)
    finalize_kernel(const double *__restrict__ part, int nblocks, int s0, int s1, double *scal) {
  __shared__ double sh[2][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int q = 0; q < 2; ++q) {
    const int slot = q == 0 ? s0 : s1;
    if (slot < 0) break;
    const double *p = part + (int64_t)slot * kMaxRedBlocks;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    int b = threadIdx.x;
    for (; b + 3 * 1024 < nblocks; b += 4 * 1024) {
      acc[0] += p[b];
      acc[1] += p[b + 1024];
      acc[2] += p[b + 2048];
      acc[3] += p[b + 3072];
    }
    for (; b < nblocks; b += 1024) acc[0] += p[b];
    double v = warp_sum((acc[0] + acc[1]) + (acc[2] + acc[3]));
    if (lane == 0) sh[q][warp] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
      double s = 0.0;
      for (int i = 0; i < 32; ++i) s += sh[q][i];
      scal[slot] = s;
    }
  }
}

int launch_finalize(Ctx *c, int nblocks, int s0, int s1) {
  finalize_kernel<<<1, 1024, 0, c->stream>>>(c->part, nblocks, s0, s1, c->scal);
  HMG_CUDA(c, cudaGetLastError());
  return HMG_OK;
}

int launch_spmv(Ctx *c, const double *x, double *y, int mode, const double *w, int slot0,
                int slot1) {
  const Level &f = c->lv[0];
  const TraceDims d = dims_of(f);
  const unsigned g = grid_for(f.ntrace, kRedThreads * kSpmvRows);
  if (g > (unsigned)kMaxRedBlocks) return fail(c, HMG_ERR_INVALID_ARG, "too many rows for one reduction");
  Prof prof(c, kCompApply);
  switch (mode) {
    case 0: spmv_kernel<0><<<g, kRedThreads, 0, c->stream>>>(c->S, x, y, w, d, f.edge_stencil, f.col_edges, c->part, slot0, slot1); break;
    case 1: spmv_kernel<1><<<g, kRedThreads, 0, c->stream>>>(c->S, x, y, w, d, f.edge_stencil, f.col_edges, c->part, slot0, slot1); break;
    case 2: spmv_kernel<2><<<g, kRedThreads, 0, c->stream>>>(c->S, x, y, w, d, f.edge_stencil, f.col_edges, c->part, slot0, slot1); break;
    default: spmv_kernel<3><<<g, kRedThreads, 0, c->stream>>>(c->S, x, y, w, d, f.edge_stencil, f.col_edges, c->part, slot0, slot1); break;
  }
  if (mode != 0)
    finalize_kernel<<<1, 1024, 0, c->stream>>>(c->part, (int)g, slot0, mode == 2 ? slot1 : -1, c->scal);
  HMG_CUDA(c, cudaGetLastError());
  return HMG_OK;
}

// ---- B_lambda = C^T A^-1 R_X ------------------------------------------------------------
// Row f of B_lambda sums (A_K^-1 R_K)_{i} over the (one or two) cells K having f as local face i.
__device__ __forceinline__ double ainv_row_dot(const double *__restrict__ Ainv, int64_t C, int64_t K,
                                               int i, const double *__restrict__ Rub,
                                               const double *__restrict__ Rpi) {
  double s = 0.0;
#pragma unroll
  for (int j = 0; j < 6; ++j) s += __ldg(Ainv + (7 * i + j) * C + K) * __ldg(Rub + 6 * K + j);
  s += __ldg(Ainv + (7 * i + 6) * C + K) * __ldg(Rpi + K);
  return s;
}

__global__ void trace_rhs_kernel(const double *__restrict__ Ainv, const double *__restrict__ Rub,
                                 const double *__restrict__ Rpi, double *__restrict__ B,
                                 const TraceDims d, int64_t C, const int32_t *__restrict__ stencil,
                                 const int32_t *__restrict__ edge_fc) {
  const int64_t row = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (row >= d.NT) return;
  double v;
  if (row < d.NH) {
    const int e = (int)(row / d.L), k = (int)(row - (int64_t)e * d.L);
    const int64_t K1 = (int64_t)stencil[8 * (int64_t)e] * d.L + k;
    const int64_t K2 = (int64_t)stencil[8 * (int64_t)e + 1] * d.L + k;
    v = ainv_row_dot(Ainv, C, K1, edge_fc[2 * (int64_t)e], Rub, Rpi) +
        ainv_row_dot(Ainv, C, K2, edge_fc[2 * (int64_t)e + 1], Rub, Rpi);
  } else {
    const int64_t zr = row - d.NH;
    const int c = (int)(zr / (d.L + 1)), k = (int)(zr - (int64_t)c * (d.L + 1));
    double va = 0.0, vb = 0.0;
    if (k < d.L) va = ainv_row_dot(Ainv, C, (int64_t)c * d.L + k, 4, Rub, Rpi);
    if (k > 0) vb = ainv_row_dot(Ainv, C, (int64_t)c * d.L + k - 1, 5, Rub, Rpi);
    v = va + vb;
  }
  B[row] = v;
}

int launch_trace_rhs(Ctx *c, const double *Rub, const double *Rpi, double *B) {
  const Level &f = c->lv[0];
  Prof prof(c, kCompRhs);
  trace_rhs_kernel<<<grid_for(f.ntrace, 256), 256, 0, c->stream>>>(
      c->Ainv, Rub, Rpi, B, dims_of(f), f.ncell, f.edge_stencil, f.edge_fc);
  HMG_CUDA(c, cudaGetLastError());
  return HMG_OK;
}

// ---- X_K = A_K^-1 (R_K - K_K lambda_K) ---------------------------------------------------
__global__ void reconstruct_kernel(const double *__restrict__ Ainv, const double *__restrict__ kth,
                                   const double *__restrict__ lam, const double *__restrict__ Rub,
                                   const double *__restrict__ Rpi, double *__restrict__ ub,
                                   double *__restrict__ pi, const TraceDims d, int64_t C,
                                   const int32_t *__restrict__ col_edges) {
  const int64_t K = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (K >= C) return;
  const int c = (int)(K / d.L), k = (int)(K - (int64_t)c * d.L);
  int64_t g[6];
#pragma unroll
  for (int f = 0; f < 4; ++f) g[f] = (int64_t)col_edges[4 * (int64_t)c + f] * d.L + k;
  g[4] = d.NH + (int64_t)c * (d.L + 1) + k;
  g[5] = g[4] + 1;
  double rm[7];
#pragma unroll
  for (int f = 0; f < 6; ++f) rm[f] = Rub[6 * K + f] - kth[f * C + K] * lam[g[f]];
  rm[6] = Rpi[K];
#pragma unroll
  for (int i = 0; i < 7; ++i) {
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < 7; ++j) s += Ainv[(7 * i + j) * C + K] * rm[j];
    if (i < 6) ub[6 * K + i] = s; else pi[K] = s;
  }
}

int launch_reconstruct(Ctx *c, const double *lam, const double *Rub, const double *Rpi,
                       double *ub, double *pi) {
  const Level &f = c->lv[0];
  reconstruct_kernel<<<grid_for(f.ncell, 128), 128, 0, c->stream>>>(
      c->Ainv, c->kth, lam, Rub, Rpi, ub, pi, dims_of(f), f.ncell, f.col_edges);
  HMG_CUDA(c, cudaGetLastError());
  return HMG_OK;
}

// ---- Algorithm 1: one sweep ---------------------------------------------------------------
// lam_out = lam_in + omega D^-1 (b - S lam_in), D = [diag(S^hh), blockdiag(S^zz_c)]. With
// ZERO, lam_in = 0 and the sweep needs no S apply. Blocks [0, nzb) take CPB columns of
// lambda^z each (residual rows staged in shared memory, one thread per column runs the
// Thomas solve with the precomputed factors); the remaining blocks take lambda^h rows.
// On the lambda^z rows the update is evaluated as (1 - omega) lam_in + omega (S^zz_c)^-1
// (b - (S - D) lam_in), equal in exact arithmetic: eight couplings instead of eleven in the
// residual (the sweep is bound by the FP64 issue rate) and three fewer coefficients read.
// lambda^h rows per thread of the sweep (block-strided): four in a sweep from zero (two loads
// and a store per row, no gathers), two in an FP32 sweep (it waits on the gathered iterate
// values rather than on arithmetic), one in an FP64 sweep (FP64 issue-bound)
template <typename T, bool ZERO>
constexpr int kSweepHRows = ZERO ? 4 : (sizeof(T) == 4 ? 2 : 1);

struct SweepArgs {
  TraceDims d;
  int ncol, cpb, nzb;
  const int32_t *stencil, *col_edges;
  double keep;   // 1 - omega
};

template <typename T, typename Tb, typename Tout, bool ZERO>
__global__ void __launch_bounds__(256)
    sweep_kernel(const SweepArgs a, const T *__restrict__ S, const T *__restrict__ zw,
                 const T *__restrict__ zl, const T *__restrict__ zcp, const T *__restrict__ hw,
                 const Tb *__restrict__ b, const T *__restrict__ lam_in, Tout *__restrict__ lam_out) {
  extern __shared__ unsigned char smem_raw[];
  const TraceDims &d = a.d;
  if ((int)blockIdx.x < a.nzb) {
    T *sr = reinterpret_cast<T *>(smem_raw);
    const int L1 = d.L + 1;
    const int ld = L1 | 1;   // column stride in shared memory, odd: conflict-free lanes
    const int c0 = blockIdx.x * a.cpb;
    const int nc = min(a.cpb, a.ncol - c0);
    const int nrow = nc * L1;
    T *sl = sr + a.cpb * ld, *scp = sl + a.cpb * ld;
    const int64_t base = d.NH + (int64_t)c0 * L1;
    // all threads: r omega / pivot and the factors, so that the serial Thomas recurrences
    // below are one FMA per row each (factors from trace_factor_kernel); two rows per pass
    // keep twice the gathers in flight
#pragma unroll 2
    for (int i = threadIdx.x; i < nrow; i += blockDim.x) {
      const int64_t row = base + i;
      T r = (T)__ldg(b + row);
      if (!ZERO) r = s_row_z_off<T, T, T>(S, lam_in, a.col_edges, d, row, r);
      const int j = (i / L1) * ld + i % L1;
      sr[j] = r * __ldg(zw + (row - d.NH));
      sl[j] = __ldg(zl + (row - d.NH));
      scp[j] = __ldg(zcp + (row - d.NH));
    }
    __syncthreads();
    if ((int)threadIdx.x < nc) thomas_smem<T, sizeof(T) == 4 ? 8 : 1>(sr, sl, scp, (int)threadIdx.x * ld, L1);
    __syncthreads();
    for (int i = threadIdx.x; i < nrow; i += blockDim.x) {
      const int64_t row = base + i;
      const T v = sr[(i / L1) * ld + i % L1];
      lam_out[row] = (Tout)(ZERO ? v : fma((T)a.keep, lam_in[row], v));
    }
  } else {
    constexpr int HR = kSweepHRows<T, ZERO>;
    const int64_t base = (int64_t)(blockIdx.x - a.nzb) * blockDim.x * HR + threadIdx.x;
#pragma unroll
    for (int j = 0; j < HR; ++j) {
      const int64_t row = base + (int64_t)j * blockDim.x;
      if (row < d.NH) {
        T r = (T)__ldg(b + row);
        if (!ZERO) r = s_row_h<T, T, T, true>(S, lam_in, a.stencil, d, row, r);
        lam_out[row] = (Tout)(ZERO ? r * __ldg(hw + row) : fma(r, __ldg(hw + row), lam_in[row]));
      }
    }
  }
}

// The same sweep with one warp per lambda^z column (the FP32 preconditioner's form, columns per
// block -1; L + 1 <= 32 M rows): lane j holds rows j M .. j M + M - 1, whose residuals it
// computes, and the Thomas recurrences run as a warp scan (warp_thomas); 8 columns per block of
// 256 threads. The remaining blocks take lambda^h rows as in sweep_kernel.
template <typename T, typename Tb, typename Tout, bool ZERO, int M>
__global__ void __launch_bounds__(256)
    sweep_warp_kernel(const SweepArgs a, const T *__restrict__ S, const T *__restrict__ zw,
                      const T *__restrict__ zl, const T *__restrict__ zcp, const T *__restrict__ hw,
                      const Tb *__restrict__ b, const T *__restrict__ lam_in, Tout *__restrict__ lam_out) {
  const TraceDims &d = a.d;
  if ((int)blockIdx.x < a.nzb) {
    const int64_t col = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (col >= a.ncol) return;   // whole warps
    const int lane = threadIdx.x & 31, L1 = d.L + 1;
    const int64_t base = d.NH + col * L1;
    T s[M], lo[M], up[M];
#pragma unroll
    for (int i = 0; i < M; ++i) {
      const int k = lane * M + i;
      s[i] = lo[i] = up[i] = (T)0;
      if (k < L1) {
        const int64_t row = base + k;
        T r = (T)__ldg(b + row);
        if (!ZERO) r = s_row_z_off<T, T, T>(S, lam_in, a.col_edges, d, row, r);
        s[i] = r * __ldg(zw + (row - d.NH));
        if (k > 0) lo[i] = __ldg(zl + (row - d.NH));
        if (k < L1 - 1) up[i] = __ldg(zcp + (row - d.NH));
      }
    }
    warp_thomas<T, M>(s, lo, up, lane, L1);
#pragma unroll
    for (int i = 0; i < M; ++i) {
      const int k = lane * M + i;
      if (k < L1) {
        const int64_t row = base + k;
        lam_out[row] = (Tout)(ZERO ? s[i] : fma((T)a.keep, lam_in[row], s[i]));
      }
    }
  } else {
    constexpr int HR = kSweepHRows<T, ZERO>;
    const int64_t base = (int64_t)(blockIdx.x - a.nzb) * blockDim.x * HR + threadIdx.x;
#pragma unroll
    for (int j = 0; j < HR; ++j) {
      const int64_t row = base + (int64_t)j * blockDim.x;
      if (row < d.NH) {
        T r = (T)__ldg(b + row);
        if (!ZERO) r = s_row_h<T, T, T, true>(S, lam_in, a.stencil, d, row, r);
        lam_out[row] = (Tout)(ZERO ? r * __ldg(hw + row) : fma(r, __ldg(hw + row), lam_in[row]));
      }
    }
  }
}

// Columns per block of the sweep: at most 64, and the three shared-memory arrays of the
// block's column rows within the default 48 KB (FP64).
static int sweep_cpb_limit(int nlev) {
  const int m = 2048 / ((nlev + 1) | 1);
  return m < 1 ? 1 : (m > 64 ? 64 : m);
}

template <typename T, typename Tb, typename Tout, bool ZERO>
static int launch_sweep(Ctx *c, const Tb *b, const T *lam_in, Tout *lam_out, int cpb_override = 0,
                        int threads_override = 0) {
  const Level &f = c->lv[0];
  SweepArgs a;
  a.d = dims_of(f);
  a.ncol = f.ncol;
  const int cpb_max = sweep_cpb_limit(f.nlev);
  const int cpb_def = cpb_max < 32 ? cpb_max : 32;
  const int pm = sizeof(T) == 4 ? 1 : 0;   // FP32 preconditioner kernels have their own tuned shape
  if constexpr (sizeof(T) == 4) {
    // columns per block -1 (given or tuned): one warp per lambda^z column
    if ((cpb_override == -1 || (cpb_override == 0 && c->tune_sweep_cpb[1] == -1)) && f.nlev + 1 <= 128) {
      a.stencil = f.edge_stencil;
      a.col_edges = f.col_edges;
      a.keep = 1.0 - c->factor_omega;
      a.cpb = 8;
      a.nzb = (int)grid_for((int64_t)f.ncol * 32, 256);
      const unsigned nhb = grid_for(f.nth, 256 * kSweepHRows<T, ZERO>);
      Prof prof(c, ZERO ? kCompPresmooth : kCompSweep);
      const int L1 = f.nlev + 1;
      auto go = [&](auto kern) {
        kern<<<a.nzb + nhb, 256, 0, c->stream>>>(a, Prec<T>::S(c), Prec<T>::Sz_w(c), Prec<T>::Sz_l(c),
                                                 Prec<T>::Sz_cp(c), Prec<T>::Sh_w(c), b, lam_in, lam_out);
      };
      if (L1 <= 32) go(sweep_warp_kernel<T, Tb, Tout, ZERO, 1>);
      else if (L1 <= 64) go(sweep_warp_kernel<T, Tb, Tout, ZERO, 2>);
      else go(sweep_warp_kernel<T, Tb, Tout, ZERO, 4>);
      HMG_CUDA(c, cudaGetLastError());
      return HMG_OK;
    }
  }
  a.cpb = cpb_override > 0 ? cpb_override : (c->tune_sweep_cpb[pm] > 0 ? c->tune_sweep_cpb[pm] : cpb_def);
  if (a.cpb > cpb_max) a.cpb = cpb_max;
  a.nzb = (f.ncol + a.cpb - 1) / a.cpb;
  a.stencil = f.edge_stencil;
  a.col_edges = f.col_edges;
  a.keep = 1.0 - c->factor_omega;   // the omega folded into the factors
  // threads: the column block's rows rounded up to whole warps (at most 256)
  const int tmax = threads_override > 0 ? threads_override : (c->tune_sweep_threads[pm] > 0 ? c->tune_sweep_threads[pm] : 256);
  int threads = ((a.cpb * (f.nlev + 1) + 31) / 32) * 32;
  if (threads > tmax) threads = tmax;
  if (threads < ((a.cpb + 31) / 32) * 32) threads = ((a.cpb + 31) / 32) * 32;   // a lane per column
  const unsigned nhb = grid_for(f.nth, (int64_t)threads * kSweepHRows<T, ZERO>);
  const size_t smem = (size_t)3 * a.cpb * ((f.nlev + 1) | 1) * sizeof(T);
  Prof prof(c, ZERO ? kCompPresmooth : kCompSweep);
  sweep_kernel<T, Tb, Tout, ZERO><<<a.nzb + nhb, threads, smem, c->stream>>>(
      a, Prec<T>::S(c), Prec<T>::Sz_w(c), Prec<T>::Sz_l(c), Prec<T>::Sz_cp(c), Prec<T>::Sh_w(c), b,
      lam_in, lam_out);
  HMG_CUDA(c, cudaGetLastError());
  return HMG_OK;
}

// ---- R = b - S lam (Algorithm 2 line 3) ------------------------------------------------------
// ZSWEEP: lam is one line-smoother sweep from zero, lam = omega D^-1 b, so D lam = omega b and
// R = (1 - omega) b - (S - D) lam (equal in exact arithmetic; ten couplings on a lambda^h row
// and eight on a lambda^z row instead of eleven).
template <typename T, typename Tb, bool ZSWEEP>
__global__ void __launch_bounds__(256)
    residual_kernel(const T *__restrict__ S, const Tb *__restrict__ b, const T *__restrict__ lam,
                    T *__restrict__ R, const TraceDims d, const int32_t *__restrict__ stencil,
                    const int32_t *__restrict__ col_edges, double keep) {
  const int64_t row = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (row >= d.NT) return;
  if (ZSWEEP) {
    const T acc = (T)keep * (T)__ldg(b + row);
    R[row] = row < d.NH ? s_row_h_off<T, T, T>(S, lam, stencil, d, row, acc)
                        : s_row_z_off<T, T, T>(S, lam, col_edges, d, row, acc);
  } else {
    R[row] = s_row<T, T, T, true>(S, lam, stencil, col_edges, d, row, (T)__ldg(b + row));
  }
}

// ---- bbar = Gamma P^T R (Algorithm 2 lines 4-5) -----------------------------------------
template <typename T>
__global__ void restrict_kernel(const T *__restrict__ R, const T *__restrict__ gamma,
                                T *__restrict__ bbar, const TraceDims d, int64_t C,
                                const int32_t *__restrict__ col_edges) {
  const int64_t K = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (K >= C) return;
  // 32-bit index arithmetic (the mesh limits keep every row index below 2^31)
  const unsigned Ku = (unsigned)K, Lu = (unsigned)d.L;
  const int c = (int)(Ku / Lu), k = (int)(Ku - (unsigned)c * Lu);
  bbar[K] = trace_restrict_cell(R, gamma, col_edges, d, c, k, K);
}

// ---- lam_out = lam_in + P dPi (Algorithm 2 line 7) ---------------------------------------
constexpr int kProlongRows = 4;

template <typename T>
__global__ void prolong_kernel(const T *__restrict__ lam_in, const T *__restrict__ dpi,
                               T *__restrict__ lam_out, const TraceDims d,
                               const int32_t *__restrict__ stencil) {
  // kProlongRows rows per thread, block-strided: few operations per row, so the kernel waits on
  // its loads and more rows per thread keep more of them in flight
  const int64_t base = blockIdx.x * (int64_t)blockDim.x * kProlongRows + threadIdx.x;
#pragma unroll
  for (int j = 0; j < kProlongRows; ++j) {
    const int64_t row = base + (int64_t)j * blockDim.x;
    if (row >= d.NT) break;
    // lam_in + (1/2)(a + b) as one FMA: the halving is exact, so it rounds as the add did
    const T li = lam_in[row];
    T out;
    if (row < d.NH) {   // 32-bit index arithmetic (row indices stay below 2^31)
      const unsigned ru = (unsigned)row, Lu = (unsigned)d.L;
      const int e = (int)(ru / Lu), k = (int)(ru - (unsigned)e * Lu);
      out = fma((T)0.5, dpi[(int64_t)__ldg(stencil + 8 * (int64_t)e) * d.L + k] +
                            dpi[(int64_t)__ldg(stencil + 8 * (int64_t)e + 1) * d.L + k], li);
    } else {
      const unsigned zr = (unsigned)(row - d.NH), L1 = (unsigned)d.L + 1u;
      const int c = (int)(zr / L1), k = (int)(zr - (unsigned)c * L1);
      const int64_t K = (int64_t)c * d.L + k;
      if (k == 0) out = li + dpi[K];
      else if (k == d.L) out = li + dpi[K - 1];
      else out = fma((T)0.5, dpi[K - 1] + dpi[K], li);
    }
    lam_out[row] = out;
  }
}

template <typename Tin, typename Tout>
__global__ void convert_kernel(const Tin *__restrict__ in, Tout *__restrict__ out, int64_t n) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) out[i] = (Tout)in[i];
}

// ---- preconditioners -----------------------------------------------------------------------
// Configuration 2: n_smooth sweeps of Algorithm 1 from zero.
template <typename T>
static int line_precond(Ctx *c, const double *r, double *z) {
  const int n = c->opt.n_smooth;
  T *a = static_cast<T *>(c->w1), *b2 = static_cast<T *>(c->w2);
  int st;
  if (n == 1) return launch_sweep<T, double, double, true>(c, r, nullptr, z);
  if ((st = launch_sweep<T, double, T, true>(c, r, nullptr, a))) return st;
  for (int i = 1; i < n - 1; ++i) {
    if ((st = launch_sweep<T, double, T, false>(c, r, a, b2))) return st;
    T *t = a; a = b2; b2 = t;
  }
  return launch_sweep<T, double, double, false>(c, r, a, z);
}

// Configuration 3c: Algorithm 2 with one pressure V-cycle as the coarse solve.
template <typename T>
static int two_level(Ctx *c, const double *r, double *z) {
  const Level &f = c->lv[0];
  const TraceDims d = dims_of(f);
  T *w1 = static_cast<T *>(c->w1), *w2 = static_cast<T *>(c->w2), *w3 = static_cast<T *>(c->w3);
  int st;
  // line 1-2: lambda = 0, presmooth
  if (c->opt.n_pre >= 1) {
    if ((st = launch_sweep<T, double, T, true>(c, r, nullptr, w1))) return st;
    for (int i = 1; i < c->opt.n_pre; ++i) {
      if ((st = launch_sweep<T, double, T, false>(c, r, w1, w2))) return st;
      T *t = w1; w1 = w2; w2 = t;
    }
  } else {
    HMG_CUDA(c, cudaMemsetAsync(w1, 0, sizeof(T) * f.ntrace, c->stream));
  }
  // lines 3-5: R = r - S lambda; bbar = Gamma P^T R (with a plain V-cycle as the coarse solve,
  // the restriction runs inside the V-cycle's first sweep)
  T *cb = static_cast<T *>(c->cb);
  const int cm = c->opt.coarse;
  const bool plain_vcycle =
      !c->collect_x && (cm == HMG_COARSE_VCYCLE ||
                        ((cm == HMG_COARSE_LEARNED || cm == HMG_COARSE_LEARNED_VCYCLE) && c->coarse_fallback));
  {
    Prof pr(c, kCompResidual, plain_vcycle ? 1 : 2);
    if (c->opt.n_pre == 1)   // w1 is one sweep from zero
      residual_kernel<T, double, true><<<grid_for(f.ntrace, 256), 256, 0, c->stream>>>(
          Prec<T>::S(c), r, w1, w2, d, f.edge_stencil, f.col_edges, 1.0 - c->factor_omega);
    else
      residual_kernel<T, double, false><<<grid_for(f.ntrace, 256), 256, 0, c->stream>>>(
          Prec<T>::S(c), r, w1, w2, d, f.edge_stencil, f.col_edges, 0.0);
    if (!plain_vcycle)
      restrict_kernel<T><<<grid_for(f.ncell, 256), 256, 0, c->stream>>>(w2, Prec<T>::gamma(c), cb, d,
                                                                        f.ncell, f.col_edges);
  }
  HMG_CUDA(c, cudaGetLastError());
  // (training pairs for the learned coarse solve, FP64 path only)
  if (c->collect_x && sizeof(T) == 8 && (st = collect_pair(c, reinterpret_cast<const double *>(cb)))) return st;
  // line 6: the coarse solve H dPi = bbar: one V-cycle of the pressure multigrid, the learned
  // model, or the model's output as the V-cycle's initial guess
  T *dpi = nullptr;
  {
    Prof pv(c, kCompVcycle, vcycle_launches(c));
    const bool learned = (cm == HMG_COARSE_LEARNED || cm == HMG_COARSE_LEARNED_VCYCLE) && !c->coarse_fallback;
    if (plain_vcycle) {
      if ((st = vcycle_trace<T>(c, w2, cb, &dpi))) return st;
    } else if (cm == HMG_COARSE_KRYLOV_EXACT || cm == HMG_COARSE_KRYLOV_APPROX) {
      if (sizeof(T) != 8) return fail(c, HMG_ERR_INVALID_ARG, "the Krylov coarse solves run in FP64");
      dpi = w3;
      if ((st = coarse_krylov(c, reinterpret_cast<const double *>(cb), reinterpret_cast<double *>(dpi),
                              cm == HMG_COARSE_KRYLOV_EXACT ? 1e-14 : 1e-2, 500)))
        return st;
    } else if (learned && cm == HMG_COARSE_LEARNED) {
      dpi = w3;
      if ((st = learned_coarse<T>(c, cb, dpi))) return st;
    } else if (learned) {
      if ((st = learned_coarse<T>(c, cb, w3))) return st;
      if ((st = vcycle<T>(c, cb, &dpi, w3))) return st;
    } else {
      if ((st = vcycle<T>(c, cb, &dpi))) return st;
    }
  }
  // line 7: lambda += P dPi
  {
    Prof pp(c, kCompProlong);
    prolong_kernel<T><<<grid_for(f.ntrace, 256 * kProlongRows), 256, 0, c->stream>>>(w1, dpi, w2, d, f.edge_stencil);
  }
  HMG_CUDA(c, cudaGetLastError());
  // line 8: postsmooth
  const int np = c->opt.n_post;
  if (np == 0) {
    convert_kernel<T, double><<<grid_for(f.ntrace, 256), 256, 0, c->stream>>>(w2, z, f.ntrace);
    HMG_CUDA(c, cudaGetLastError());
    return HMG_OK;
  }
  T *cur = w2, *nxt = w3;
  for (int i = 0; i < np - 1; ++i) {
    if ((st = launch_sweep<T, double, T, false>(c, r, cur, nxt))) return st;
    T *t = cur; cur = nxt; nxt = t;
  }
  return launch_sweep<T, double, double, false>(c, r, cur, z);
}

int precond_apply(Ctx *c, const double *r, double *z) {
  if (c->degree >= 1) return ho_precond(c, r, z);
  const bool mixed = c->opt.precision == HMG_PRECISION_MIXED;
  switch (c->opt.precond) {
    case HMG_PRECOND_SCHUR:
      return schur_precond(c, r, z);
    case HMG_PRECOND_NONE:
      HMG_CUDA(c, cudaMemcpyAsync(z, r, sizeof(double) * sys_n(c), cudaMemcpyDeviceToDevice,
                                  c->stream));
      return HMG_OK;
    case HMG_PRECOND_LINESMOOTH:
      return mixed ? line_precond<float>(c, r, z) : line_precond<double>(c, r, z);
    default:
      return mixed ? two_level<float>(c, r, z) : two_level<double>(c, r, z);
  }
}

int line_smooth_fp64(Ctx *c, const double *b, double *lam, int nsweeps) {
  // ping-pong between lam and a work vector; one copy at the end if the count is odd
  double *cur = lam, *nxt = static_cast<double *>(c->w3);
  int st;
  for (int i = 0; i < nsweeps; ++i) {
    if ((st = launch_sweep<double, double, double, false>(c, b, cur, nxt))) return st;
    double *t = cur; cur = nxt; nxt = t;
  }
  if (cur != lam)
    HMG_CUDA(c, cudaMemcpyAsync(lam, cur, sizeof(double) * c->lv[0].ntrace,
                                cudaMemcpyDeviceToDevice, c->stream));
  return HMG_OK;
}

}  // namespace hmg

// ---- line smoothing without any allocation -----------------------------------------------
// hmg_line_smooth keeps its second vector in the context's workspace, which
// hmg_assemble_trace allocates. This variant takes that vector from a fixed array compiled
// into the library instead, so the call itself never allocates device memory. Its size is
// fixed here: every GPU that loads the library holds these 8 MiB until the process exits.
namespace {
constexpr int64_t kNoAllocMaxTrace = int64_t(1) << 20;   // trace unknowns (1,048,576 doubles)
static __device__ __align__(256) double g_sweep_scratch[kNoAllocMaxTrace];
}  // namespace

namespace hmg {
// Device address of g_sweep_scratch in the current device's context, kept in the library
// context. Called by hmg_assemble_trace (set-up, with the context's device current): the
// lookup loads this file's module, and with it the array, at set-up rather than inside the
// first allocation-free call. The name of a __device__ array is only a host-side stand-in
// and must never be handed to a kernel; this address is what the kernels get. It is as
// valid as the context's own device buffers (a cudaDeviceReset invalidates both).
int noalloc_setup(Ctx *c) {
  void *p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_sweep_scratch);
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaGetSymbolAddress(g_sweep_scratch)");
  c->noalloc_scratch = static_cast<double *>(p);
  return HMG_OK;
}
}  // namespace hmg

extern "C" int hmg_line_smooth_noalloc(hmg_ctx *ctx, const double *b, double *lambda,
                                       int32_t nsweeps) {
  using namespace hmg;
  if (!ctx) return HMG_ERR_INVALID_ARG;
  Ctx *c = ctx;
  if (!c->assembled) return fail(c, HMG_ERR_NOT_READY, "call hmg_assemble_trace first");
  if (!b || !lambda || nsweeps < 0) return fail(c, HMG_ERR_INVALID_ARG, "bad arguments");
  if (c->degree != 0) return fail(c, HMG_ERR_INVALID_ARG, "hmg_line_smooth_noalloc sweeps the degree-0 system");
  if (c->lv[0].ntrace > kNoAllocMaxTrace)
    return fail(c, HMG_ERR_INVALID_ARG,
                "hmg_line_smooth_noalloc: ntrace exceeds the built-in scratch of 1048576 trace "
                "unknowns; use hmg_line_smooth");
  HMG_CUDA(c, cudaSetDevice(c->device));
  double *scratch = c->noalloc_scratch;   // looked up by hmg_assemble_trace
  if (!scratch) return fail(c, HMG_ERR_NOT_READY, "the scratch address was not set up; call hmg_assemble_trace");
  // same sweeps as hmg_line_smooth, ping-ponging between lambda and the fixed array; nothing
  // in the array needs to start at zero (each sweep overwrites every entry it later reads)
  int st;
  double *cur = lambda, *nxt = scratch;
  for (int i = 0; i < nsweeps; ++i) {
    if ((st = launch_sweep<double, double, double, false>(c, b, cur, nxt))) return st;
    double *t = cur; cur = nxt; nxt = t;
  }
  if (cur != lambda)
    HMG_CUDA(c, cudaMemcpyAsync(lambda, cur, sizeof(double) * c->lv[0].ntrace,
                                cudaMemcpyDeviceToDevice, c->stream));
  HMG_CUDA(c, cudaStreamSynchronize(c->stream));
  return HMG_OK;
}

// ---- launch-shape autotuning ---------------------------------------------------------------
namespace hmg {

// Best-of-three average time of a full sweep with `cpb` columns per block (-1: one warp per
// column, FP32 only), in FP64 or (fp32) with the FP32 preconditioner's types (FP32 S and
// lambda in, FP64 b and lambda out); the work vectors serve as data.
int time_sweep_cpb(Ctx *c, int cpb, int threads, int fp32, float *ms) {
  const int64_t T = c->lv[0].ntrace;
  double *b = static_cast<double *>(c->w1), *x = static_cast<double *>(c->w2), *y = static_cast<double *>(c->w3);
  HMG_CUDA(c, cudaMemsetAsync(b, 0, sizeof(double) * T, c->stream));
  HMG_CUDA(c, cudaMemsetAsync(x, 0, sizeof(double) * T, c->stream));
  auto run = [&]() {
    return fp32 ? launch_sweep<float, double, double, false>(c, b, reinterpret_cast<const float *>(x), y, cpb, threads)
                : launch_sweep<double, double, double, false>(c, b, x, y, cpb, threads);
  };
  int st;
  if ((st = run())) return st;   // warm-up
  cudaEvent_t e0, e1;
  HMG_CUDA(c, cudaEventCreate(&e0));
  HMG_CUDA(c, cudaEventCreate(&e1));
  // best of three timings of 10 launches each (the candidates differ by a few per cent)
  float best = 1e30f;
  for (int rep = 0; rep < 3 && !st; ++rep) {
    HMG_CUDA(c, cudaEventRecord(e0, c->stream));
    for (int i = 0; i < 10 && !st; ++i) st = run();
    HMG_CUDA(c, cudaEventRecord(e1, c->stream));
    HMG_CUDA(c, cudaEventSynchronize(e1));
    float t = 0.f;
    cudaEventElapsedTime(&t, e0, e1);
    if (t < best) best = t;
  }
  *ms = best / 10.f;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return st;
}

int autotune(Ctx *c) {
  const Level &f = c->lv[0];
  const int profile = c->opt.profile;
  c->opt.profile = 0;
  int st = HMG_OK;
  // FP64 shapes always; FP32 ones when the FP32 preconditioner's coefficients exist
  for (int pm = 0; pm < 2 && !st; ++pm) {
    if (pm == 1 && (!c->S32 || !c->lv[0].H32)) break;
    const int cmax = sweep_cpb_limit(f.nlev);
    int best = cmax < 32 ? cmax : 32, best_t = 256;
    float best_ms = 1e30f;
    for (int cand : {32, 64, 16, 8, 4, 2, 1})
      for (int thr : {256, 128}) {
        if (cand > cmax || st) continue;
        float ms = 0.f;
        if ((st = time_sweep_cpb(c, cand, thr, pm, &ms))) break;
        if (ms < best_ms) { best_ms = ms; best = cand; best_t = thr; }
      }
    if (pm == 1 && !st && f.nlev + 1 <= 128) {   // FP32: one warp per column competes too
      float ms = 0.f;
      if (!(st = time_sweep_cpb(c, -1, 256, pm, &ms)) && ms < best_ms) { best_ms = ms; best = -1; best_t = 256; }
    }
    // threads are not a parameter of the warp-per-column form: 0, as hmg_set_launch_shapes stores
    if (!st) { c->tune_sweep_cpb[pm] = best; c->tune_sweep_threads[pm] = best == -1 ? 0 : best_t; }
    for (int l = 0; l < c->nmg && !st; ++l) {
      const int mmax = mg_cpb_limit(c->lv[l].nlev);
      int mbest = mmax < 32 ? mmax : 32, mbest_t = 256;
      float mbest_ms = 1e30f;
      for (int cand : {32, 64, 16, 8, 4, 2, 1})
        for (int thr : {256, 128}) {
          if (cand > mmax || st) continue;
          float ms = 0.f;
          if ((st = time_mg_cpb(c, l, cand, thr, pm, &ms))) break;
          if (ms < mbest_ms) { mbest_ms = ms; mbest = cand; mbest_t = thr; }
        }
      // the warp-per-column form (columns per block -1) competes too (in FP64 it wins only on
      // small, latency-bound levels: its scan costs ten times the Thomas form's multiply-adds)
      if (!st && c->lv[l].nlev <= 128) {
        float ms = 0.f;
        if (!(st = time_mg_cpb(c, l, -1, 256, pm, &ms)) && ms < mbest_ms) { mbest_ms = ms; mbest = -1; mbest_t = 256; }
      }
      if (!st) { c->tune_mg_cpb[pm][l] = mbest; c->tune_mg_threads[pm][l] = mbest == -1 ? 0 : mbest_t; }
    }
    // then one coordinate-descent pass over the levels, coarsest first, timing whole
    // V-cycles: the fused restriction / injection sweeps of the small levels take the level's
    // shape too, and a shape that suits the plain smoother can starve them of blocks
    for (int l = c->nmg - 1; l >= 0 && !st; --l) {
      const int mmax = mg_cpb_limit(c->lv[l].nlev);
      int bc = c->tune_mg_cpb[pm][l], bt = c->tune_mg_threads[pm][l];
      float bms = 1e30f;
      if ((st = time_vcycle(c, pm, &bms))) break;
      for (int cand : {32, 64, 16, 8, 4, 2, 1, -1})
        for (int thr : {256, 128}) {
          if (cand > mmax || st || (cand == bc && (thr == bt || cand == -1))) continue;
          if (cand == -1 && (thr != 256 || c->lv[l].nlev > 128)) continue;   // the warp form
          c->tune_mg_cpb[pm][l] = cand;
          c->tune_mg_threads[pm][l] = thr;
          float ms = 0.f;
          if ((st = time_vcycle(c, pm, &ms))) break;
          if (ms < 0.98f * bms) { bms = ms; bc = cand; bt = thr; }   // 2%: beyond the timing noise
        }
      c->tune_mg_cpb[pm][l] = bc;
      c->tune_mg_threads[pm][l] = bc == -1 ? 0 : bt;
    }
  }
  c->opt.profile = profile;
  return st;
}

}  // namespace hmg
