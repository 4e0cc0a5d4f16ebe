// Tensor-product pressure multigrid (Sec. 2.3 of arXiv 2210.11797): the 7-point pressure
// operator H, the column block-Jacobi smoother x <- x + omega H_z^-1 (b - H x)
// (Eq. pressure_block_jacobi, Thomas algorithm per column), residual + restriction (sum over
// the four horizontal children) and prolongation (injection), in one V-cycle with
// mg_npre / mg_npost sweeps per level and mg_ncoarse sweeps on the coarsest level. On small
// (latency-bound) levels the restriction runs inside the level's first sweep and the
// injection inside its first post-sweep; with option mg_fused all coarse levels run as one
// cooperative launch. Every block form does the same arithmetic in the same order; the
// warp-per-column form (a per-level launch shape) evaluates the column solves as a warp scan,
// the same iterate up to rounding order.
#include <algorithm>
#include <cmath>

#include "device_common.cuh"
#include "hmg_internal.cuh"
#include "precond.cuh"

namespace hmg {

struct MGArgs {
  int L, ncol, cpb;
  int64_t ncell;
  const int32_t *col_nbr;
  double keep;   // 1 - omega_p: the share of the old iterate a smoothing sweep keeps
};

// Loads of vectors that other blocks of the same launch wrote (the cooperative coarse-level
// kernel, COH) bypass L1; coefficient arrays, never written during a solve, go through the
// read-only path.
template <bool COH, typename T>
__device__ __forceinline__ T ldv(const T *p) {
  if (COH) return __ldcg(p);
  return *p;
}

// acc + sign * (row K of H) . x as one FMA per coefficient (acc = b, sign = -1: the residual);
// xv(col, kk) gives x in column col, layer kk.
template <typename T, bool NEG, typename XV>
__device__ __forceinline__ T h_apply_f(const T *__restrict__ H, const MGArgs &a, int c, int k, T acc, const XV &xv) {
  const int64_t C = a.ncell, K = (int64_t)c * a.L + k;
  auto term = [&](int slot, int col, int kk) {
    const T h = __ldg(H + slot * C + K);
    acc = fma(NEG ? -h : h, xv(col, kk), acc);
  };
  term(0, c, k);
#pragma unroll
  for (int f = 0; f < 4; ++f) term(1 + f, __ldg(a.col_nbr + 4 * (int64_t)c + f), k);
  if (k > 0) term(5, c, k - 1);
  if (k < a.L - 1) term(6, c, k + 1);
  return acc;
}

template <typename T, bool NEG, bool COH = false>
__device__ __forceinline__ T h_apply(const T *__restrict__ H, const T *__restrict__ x, const MGArgs &a,
                                     int c, int k, T acc) {
  return h_apply_f<T, NEG>(H, a, c, k, acc,
                           [&](int col, int kk) { return ldv<COH>(x + (int64_t)col * a.L + kk); });
}

// acc + sign * (horizontal couplings of row K of H) . x: the four neighbour columns at the same
// layer, H_h = H - H_z.
template <typename T, bool NEG, typename XV>
__device__ __forceinline__ T h_apply_horiz_f(const T *__restrict__ H, const MGArgs &a, int c, int k, T acc,
                                             const XV &xv) {
  const int64_t C = a.ncell, K = (int64_t)c * a.L + k;
#pragma unroll
  for (int f = 0; f < 4; ++f) {
    const T h = __ldg(H + (1 + f) * C + K);
    acc = fma(NEG ? -h : h, xv(__ldg(a.col_nbr + 4 * (int64_t)c + f), k), acc);
  }
  return acc;
}

template <typename T, bool NEG, bool COH = false>
__device__ __forceinline__ T h_apply_horiz(const T *__restrict__ H, const T *__restrict__ x, const MGArgs &a,
                                           int c, int k, T acc) {
  return h_apply_horiz_f<T, NEG>(H, a, c, k, acc,
                                 [&](int col, int kk) { return ldv<COH>(x + (int64_t)col * a.L + kk); });
}

// The smoothing sweep x_out = x + omega H_z^-1 (b - H x) of Eq. pressure_block_jacobi is
// evaluated as x_out = (1 - omega) x + omega H_z^-1 (b - H_h x): the same iterate in exact
// arithmetic (H = H_z + H_h), with the four horizontal couplings instead of all seven in the
// residual and one FMA for the update. After one sweep from zero, x = omega H_z^-1 b, so the
// residual is b - H x = (1 - omega) b - H_h x (used by the restriction that follows the
// pre-smoothing). These kernels are bound by the FP64 issue rate, which this form cuts from 11
// to 8 operations per cell (5 instead of 7 for that residual).

// b_coarse(cc, k) = sum over the four children ch of (b - H x)(ch, k); x == nullptr means 0
// (a: the fine level). zsweep: x is the result of one sweep from zero, so b - H x is evaluated
// as (1 - omega) b - H_h x.
template <typename T, bool COH>
__device__ __forceinline__ T restrict_value(const MGArgs &a, const T *__restrict__ H, const T *__restrict__ b,
                                            const T *__restrict__ x, const int32_t *__restrict__ children,
                                            int cc, int k, bool zsweep) {
  T s = (T)0;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int ch = __ldg(children + 4 * (int64_t)cc + i);
    T r = ldv<COH>(b + (int64_t)ch * a.L + k);
    if (x != nullptr) {
      if (zsweep) r = h_apply_horiz<T, true, COH>(H, x, a, ch, k, (T)a.keep * r);
      else r = h_apply<T, true, COH>(H, x, a, ch, k, r);
    }
    s += r;
  }
  return s;
}

// Sources of the smoother's right-hand side per cell: r(c, k, K) is the vector the sweep
// applies omega H_z^-1 to, out(c, k, K, v) the new iterate from that correction v.
template <typename T, bool COH>
struct SrcZero {   // zero start: x_out = omega H_z^-1 b
  const T *b;
  __device__ T r(const MGArgs &, int, int, int64_t K) const { return ldv<COH>(b + K); }
  __device__ T out(const MGArgs &, int, int, int64_t, T v) const { return v; }
};

template <typename T, bool COH>
struct SrcIter {   // x_out = x + omega H_z^-1 (b - H x), as (1 - omega) x + omega H_z^-1 (b - H_h x)
  const T *H, *b, *x;
  __device__ T r(const MGArgs &a, int c, int k, int64_t K) const {
    return h_apply_horiz<T, true, COH>(H, x, a, c, k, ldv<COH>(b + K));
  }
  __device__ T out(const MGArgs &a, int, int, int64_t K, T v) const { return fma((T)a.keep, ldv<COH>(x + K), v); }
};

template <typename T>
struct SrcRestrict {   // zero start on the coarse level, b = the restricted fine residual (also stored)
  MGArgs af;           // the fine level
  const T *Hf, *bf, *xf;
  const int32_t *children;
  T *bc;
  bool zsweep;         // the fine iterate is one sweep from zero
  __device__ T r(const MGArgs &, int c, int k, int64_t K) const {
    const T v = restrict_value<T, false>(af, Hf, bf, xf, children, c, k, zsweep);
    bc[K] = v;
    return v;
  }
  __device__ T out(const MGArgs &, int, int, int64_t, T v) const { return v; }
};

template <typename T>
struct SrcInject {   // x_in = x + P e (injection), then x_out = (1 - omega) x_in + omega H_z^-1 (b - H_h x_in)
  const T *H, *b, *x, *e;
  const int32_t *parent;
  __device__ T xin(const MGArgs &a, int col, int kk) const {
    return x[(int64_t)col * a.L + kk] + e[(int64_t)__ldg(parent + col) * a.L + kk];
  }
  __device__ T r(const MGArgs &a, int c, int k, int64_t K) const {
    return h_apply_horiz_f<T, true>(H, a, c, k, b[K], [&](int col, int kk) { return xin(a, col, kk); });
  }
  __device__ T out(const MGArgs &a, int c, int k, int64_t, T v) const { return fma((T)a.keep, xin(a, c, k), v); }
};

template <typename T>
struct SrcTraceRestrict {   // zero start on the finest level, b = Gamma P^T R from the trace residual (also stored)
  const T *R, *gamma;
  const int32_t *col_edges;
  TraceDims d;
  T *bc;
  __device__ T r(const MGArgs &, int c, int k, int64_t K) const {
    const T v = trace_restrict_cell(R, gamma, col_edges, d, c, k, K);
    bc[K] = v;
    return v;
  }
  __device__ T out(const MGArgs &, int, int, int64_t, T v) const { return v; }
};

// One column block (columns blk * cpb ..) of the block-Jacobi smoother, by the whole thread
// block: x_out = src.out(omega H_z^-1 src.r).
template <typename T, typename Src>
__device__ __forceinline__ void smooth_block_src(const MGArgs &a, const T *__restrict__ hw, const T *__restrict__ hl,
                                                 const T *__restrict__ hcp, const Src &src, T *__restrict__ x_out,
                                                 int blk, unsigned char *smem_raw) {
  // one column per lane in the serial phase: column j at j * ld, ld = L rounded up to odd so
  // that the lanes of a half-warp hit distinct banks
  const int ld = a.L | 1;
  T *sr = reinterpret_cast<T *>(smem_raw);
  T *sl = sr + a.cpb * ld, *scp = sl + a.cpb * ld;
  const int c0 = blk * a.cpb;
  const int nc = min(a.cpb, a.ncol - c0);
  const int n = nc * a.L;
  const int64_t base = (int64_t)c0 * a.L;
  // all threads: r omega / pivot and the factors, so that the serial Thomas recurrences
  // below are one FMA per row each (factors from pressure_factor_kernel)
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const int c = c0 + i / a.L, k = i % a.L;
    const int64_t K = base + i;
    const T r = src.r(a, c, k, K);
    const int j = (c - c0) * ld + k;
    sr[j] = r * __ldg(hw + K);
    sl[j] = __ldg(hl + K);
    scp[j] = __ldg(hcp + K);
  }
  __syncthreads();
  if ((int)threadIdx.x < nc) thomas_smem(sr, sl, scp, (int)threadIdx.x * ld, a.L);
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const int cl = i / a.L, k = i % a.L;
    x_out[base + i] = src.out(a, c0 + cl, k, base + i, sr[cl * ld + k]);
  }
}

// MODE 0: x_out = omega H_z^-1 b (zero start); 1: x_out = x + omega H_z^-1 (b - H x).
template <typename T, int MODE, bool COH>
__device__ __forceinline__ void smooth_block(const MGArgs &a, const T *__restrict__ H, const T *__restrict__ hw,
                                             const T *__restrict__ hl, const T *__restrict__ hcp,
                                             const T *__restrict__ b, const T *__restrict__ x,
                                             T *__restrict__ x_out, int blk, unsigned char *smem_raw) {
  if (MODE == 0) smooth_block_src(a, hw, hl, hcp, SrcZero<T, COH>{b}, x_out, blk, smem_raw);
  else smooth_block_src(a, hw, hl, hcp, SrcIter<T, COH>{H, b, x}, x_out, blk, smem_raw);
}

template <typename T, int MODE>
__global__ void __launch_bounds__(256)
    mg_smooth_kernel(const MGArgs a, const T *__restrict__ H, const T *__restrict__ hw,
                     const T *__restrict__ hl, const T *__restrict__ hcp, const T *__restrict__ b,
                     const T *__restrict__ x, T *__restrict__ x_out) {
  extern __shared__ unsigned char smem_raw[];
  smooth_block<T, MODE, false>(a, H, hw, hl, hcp, b, x, x_out, blockIdx.x, smem_raw);
}

// One column of the block-Jacobi smoother by one warp, the FP32 preconditioner's latency-bound
// form: lane j holds layers j M .. j M + M - 1 (M = 1 for up to 32 layers) and the Thomas
// recurrences run as a warp scan (warp_thomas). No shared memory and no block barrier; in FP32
// the scan's extra multiply-adds cost nothing next to the loads. x_out = src.out(omega H_z^-1
// src.r), as smooth_block_src.
template <typename T, int M, typename Src>
__device__ __forceinline__ void smooth_warp_src(const MGArgs &a, const T *__restrict__ hw, const T *__restrict__ hl,
                                                const T *__restrict__ hcp, const Src &src, T *__restrict__ x_out,
                                                int c) {
  const int lane = threadIdx.x & 31;
  const int64_t base = (int64_t)c * a.L;
  T s[M], lo[M], up[M];
#pragma unroll
  for (int i = 0; i < M; ++i) {
    const int k = lane * M + i;
    s[i] = lo[i] = up[i] = (T)0;
    if (k < a.L) {
      const int64_t K = base + k;
      s[i] = src.r(a, c, k, K) * __ldg(hw + K);
      if (k > 0) lo[i] = __ldg(hl + K);
      if (k < a.L - 1) up[i] = __ldg(hcp + K);
    }
  }
  warp_thomas<T, M>(s, lo, up, lane, a.L);
#pragma unroll
  for (int i = 0; i < M; ++i) {
    const int k = lane * M + i;
    if (k < a.L) x_out[base + k] = src.out(a, c, k, base + k, s[i]);
  }
}

// One warp per column (whole warps leave together, so the shuffles see full warps).
template <typename T, int M, typename Src>
__global__ void __launch_bounds__(256)
    mg_warp_kernel(const MGArgs a, const T *__restrict__ hw, const T *__restrict__ hl, const T *__restrict__ hcp,
                   const Src src, T *__restrict__ x_out) {
  const int64_t c = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  if (c >= a.ncol) return;
  smooth_warp_src<T, M>(a, hw, hl, hcp, src, x_out, (int)c);
}

// x_out = x + P e: injection of the coarse-level correction e (prolongation, Sec. 2.3).
template <typename T, bool COH>
__device__ __forceinline__ void inject_cell(const T *__restrict__ x, const T *__restrict__ e,
                                            const int32_t *__restrict__ parent, int L, int64_t K,
                                            T *__restrict__ x_out) {
  const int c = (int)(K / L), k = (int)(K - (int64_t)c * L);
  x_out[K] = ldv<COH>(x + K) + ldv<COH>(e + (int64_t)__ldg(parent + c) * L + k);
}

constexpr int kInjectCells = 4;

template <typename T>
__global__ void mg_inject_kernel(const T *__restrict__ x, const T *__restrict__ e,
                                 const int32_t *__restrict__ parent, int L, int64_t ncell,
                                 T *__restrict__ x_out) {
  // kInjectCells cells per thread, block-strided: a few loads and one add per cell, so more
  // cells per thread keep more loads in flight
  const int64_t base = blockIdx.x * (int64_t)blockDim.x * kInjectCells + threadIdx.x;
#pragma unroll
  for (int j = 0; j < kInjectCells; ++j) {
    const int64_t K = base + (int64_t)j * blockDim.x;
    if (K >= ncell) break;
    inject_cell<T, false>(x, e, parent, L, K, x_out);
  }
}

template <typename T, bool COH>
__device__ __forceinline__ void restrict_cell(const MGArgs &a, const T *__restrict__ H, const T *__restrict__ b,
                                              const T *__restrict__ x, const int32_t *__restrict__ children,
                                              int64_t Kc, T *__restrict__ bc, bool zsweep) {
  const int cc = (int)(Kc / a.L), k = (int)(Kc - (int64_t)cc * a.L);
  bc[Kc] = restrict_value<T, COH>(a, H, b, x, children, cc, k, zsweep);
}

template <typename T>
__global__ void mg_residual_restrict_kernel(const MGArgs a, const T *__restrict__ H,
                                            const T *__restrict__ b, const T *__restrict__ x,
                                            const int32_t *__restrict__ children, int ncol_c,
                                            T *__restrict__ bc, bool zsweep) {
  const int64_t Kc = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (Kc >= (int64_t)ncol_c * a.L) return;
  restrict_cell<T, false>(a, H, b, x, children, Kc, bc, zsweep);
}

// Restriction of the fine residual fused with the coarse level's first, zero-start sweep:
// bc = P^T (b_f - H_f x_f) (stored for the later sweeps) and x_out = omega H_z^-1 bc.
template <typename T>
__global__ void __launch_bounds__(256)
    mg_restrict_smooth_kernel(const MGArgs a, const T *__restrict__ hw, const T *__restrict__ hl,
                              const T *__restrict__ hcp, const MGArgs af, const T *__restrict__ Hf,
                              const T *__restrict__ bf, const T *__restrict__ xf,
                              const int32_t *__restrict__ children, T *__restrict__ bc, T *__restrict__ x_out,
                              bool zsweep) {
  extern __shared__ unsigned char smem_raw[];
  smooth_block_src(a, hw, hl, hcp, SrcRestrict<T>{af, Hf, bf, xf, children, bc, zsweep}, x_out, blockIdx.x,
                   smem_raw);
}

// Algorithm 2 lines 4-5 fused with the V-cycle's first, zero-start sweep on the finest level:
// bc = Gamma P^T R (stored for the later sweeps) and x_out = omega H_z^-1 bc.
template <typename T>
__global__ void __launch_bounds__(256)
    mg_trace_restrict_smooth_kernel(const MGArgs a, const T *__restrict__ hw, const T *__restrict__ hl,
                                    const T *__restrict__ hcp, const T *__restrict__ R,
                                    const T *__restrict__ gamma, const int32_t *__restrict__ col_edges,
                                    const TraceDims d, T *__restrict__ bc, T *__restrict__ x_out) {
  extern __shared__ unsigned char smem_raw[];
  smooth_block_src(a, hw, hl, hcp, SrcTraceRestrict<T>{R, gamma, col_edges, d, bc}, x_out, blockIdx.x, smem_raw);
}

// Injection of the coarse correction e fused with the first post-smoothing sweep:
// x_in = x + P e, x_out = x_in + omega H_z^-1 (b - H x_in) (x_in is not stored).
template <typename T>
__global__ void __launch_bounds__(256)
    mg_inject_smooth_kernel(const MGArgs a, const T *__restrict__ H, const T *__restrict__ hw,
                            const T *__restrict__ hl, const T *__restrict__ hcp, const T *__restrict__ b,
                            const T *__restrict__ x, const T *__restrict__ e, const int32_t *__restrict__ parent,
                            T *__restrict__ x_out) {
  extern __shared__ unsigned char smem_raw[];
  smooth_block_src(a, hw, hl, hcp, SrcInject<T>{H, b, x, e, parent}, x_out, blockIdx.x, smem_raw);
}

template <typename T>
__global__ void mg_residual_kernel(const MGArgs a, const T *__restrict__ H, const T *__restrict__ b,
                                   const T *__restrict__ x, T *__restrict__ r) {
  const int64_t K = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (K >= a.ncell) return;
  const int c = (int)(K / a.L), k = (int)(K - (int64_t)c * a.L);
  r[K] = h_apply<T, true>(H, x, a, c, k, b[K]);
}

template <typename T>
__global__ void mg_apply_kernel(const MGArgs a, const T *__restrict__ H, const T *__restrict__ x,
                                T *__restrict__ y) {
  const int64_t K = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (K >= a.ncell) return;
  const int c = (int)(K / a.L), k = (int)(K - (int64_t)c * a.L);
  y[K] = h_apply<T, false>(H, x, a, c, k, (T)0);
}

// ---- the coarse levels of a V-cycle in one cooperative launch ----------------------------------
// Levels l0 .. nmg-1 (all but the finest) are small and latency-bound as one launch per step;
// here one co-resident grid runs every step (smoothing sweeps, residual + restriction,
// injection) with a grid-wide barrier between steps. Same arithmetic as the per-step kernels.
constexpr uint64_t kGridBarrierLimitNs = 500000000ull;   // a barrier gives up after 0.5 s

// arrival counter and generation on separate 128-byte lines, so that the polling of the
// generation does not contend with the arrivals
struct GridBarrier {
  unsigned int count, pad0[31];
  unsigned int gen, pad1[31];
};

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// All blocks of the co-resident grid meet. Arrival is an acq_rel add at GPU scope (it
// publishes this block's writes, ordered before it by __syncthreads); the last block resets
// the counter and releases the next generation, which the others acquire. A block that waits
// past the limit records it in *flag (reported as HMG_ERR_TIMEOUT) and goes on.
__device__ __forceinline__ void grid_barrier(GridBarrier *gb, unsigned int &gen, int *flag) {
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned int old;
    asm volatile("atom.add.acq_rel.gpu.global.u32 %0, [%1], 1;" : "=r"(old) : "l"(&gb->count) : "memory");
    if (old == gridDim.x - 1) {
      asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(&gb->count), "r"(0u) : "memory");
      asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(&gb->gen), "r"(gen + 1) : "memory");
    } else {
      const uint64_t t0 = global_ns();
      unsigned int g;
      for (;;) {
        asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(g) : "l"(&gb->gen) : "memory");
        if (g != gen) break;
        if (global_ns() - t0 > kGridBarrierLimitNs) {
          atomicExch(flag, 1);
          break;
        }
        __nanosleep(32);
      }
    }
  }
  ++gen;
  __syncthreads();
}

template <typename T>
struct CoarseLevel {
  MGArgs a;
  const T *H, *hw, *hl, *hcp;
  T *vb, *vx, *vy;
  const int32_t *children;   // [ncol][4]: this level's children on the next finer level
  const int32_t *parent;     // [ncol]: the column containing it on the next coarser level
  int nblk;                  // column blocks of the smoother
};

template <typename T>
struct CoarseArgs {
  int l0, nmg, npre, npost, ncoarse;
  bool zsweep;   // one pre-sweep from zero on every level: the residual form of restrict_value
  CoarseLevel<T> lv[kMaxLevels];
  GridBarrier *bar;
  int *flag;
};

template <typename T>
__global__ void __launch_bounds__(256) mg_coarse_kernel(const CoarseArgs<T> p) {
  extern __shared__ unsigned char smem_raw[];
  unsigned int gen = 0;
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x, nthr = (int64_t)gridDim.x * blockDim.x;
  auto smooth_phase = [&](int l, bool zero, const T *xin, T *xout) {
    const CoarseLevel<T> &q = p.lv[l];
    for (int blk = blockIdx.x; blk < q.nblk; blk += gridDim.x) {
      if (zero) smooth_block<T, 0, true>(q.a, q.H, q.hw, q.hl, q.hcp, q.vb, nullptr, xout, blk, smem_raw);
      else smooth_block<T, 1, true>(q.a, q.H, q.hw, q.hl, q.hcp, q.vb, xin, xout, blk, smem_raw);
      __syncthreads();   // the next column block reuses the shared memory
    }
    grid_barrier(p.bar, gen, p.flag);
  };
  auto sweeps_from_zero = [&](int l, int n) {
    T *cur = p.lv[l].vx, *oth = p.lv[l].vy;
    smooth_phase(l, true, nullptr, cur);
    for (int i = 1; i < n; ++i) {
      smooth_phase(l, false, cur, oth);
      T *t = cur; cur = oth; oth = t;
    }
    return cur;
  };
  T *x[kMaxLevels];
  for (int l = p.l0; l < p.nmg - 1; ++l) {
    x[l] = sweeps_from_zero(l, p.npre);
    const CoarseLevel<T> &q = p.lv[l], &cq = p.lv[l + 1];
    for (int64_t Kc = tid; Kc < cq.a.ncell; Kc += nthr)
      restrict_cell<T, true>(q.a, q.H, q.vb, x[l], cq.children, Kc, cq.vb, p.zsweep);
    grid_barrier(p.bar, gen, p.flag);
  }
  const int lc = p.nmg - 1;
  x[lc] = sweeps_from_zero(lc, p.ncoarse);
  for (int l = p.nmg - 2; l >= p.l0; --l) {
    const CoarseLevel<T> &q = p.lv[l];
    T *other = x[l] == q.vx ? q.vy : q.vx;
    for (int64_t K = tid; K < q.a.ncell; K += nthr) inject_cell<T, true>(x[l], x[l + 1], q.parent, q.a.L, K, other);
    grid_barrier(p.bar, gen, p.flag);
    T *cur = other, *nxt = x[l];
    for (int i = 0; i < p.npost; ++i) {
      smooth_phase(l, false, cur, nxt);
      T *t = cur; cur = nxt; nxt = t;
    }
    x[l] = cur;
  }
}

// pm: 0 for the FP64 kernels' tuned shapes, 1 for the FP32 ones
static MGArgs mg_args(const Ctx *c, int l, int pm = 0) {
  const Level &lv = c->lv[l];
  MGArgs a;
  a.L = lv.nlev;
  a.ncol = lv.ncol;
  const int cdef = mg_cpb_limit(lv.nlev) < 32 ? mg_cpb_limit(lv.nlev) : 32;
  const int tc = c->tune_mg_cpb[pm][l];
  a.cpb = tc > 0 && tc <= mg_cpb_limit(lv.nlev) ? tc : cdef;
  a.ncell = lv.ncell;
  a.col_nbr = lv.col_nbr;
  a.keep = 1.0 - c->factor_mg_omega;   // the omega the Thomas factors were built with
  return a;
}

// Launch shape of a smoothing sweep on level l: column blocks of a.cpb columns, threads per
// block, dynamic shared memory.
struct SmoothShape {
  MGArgs a;
  unsigned grid;
  int threads;
  size_t smem;
};

template <typename T>
static SmoothShape smooth_shape(const Ctx *c, int l, int cpb_override = 0, int threads_override = 0) {
  const Level &lv = c->lv[l];
  SmoothShape sh;
  const int pm = sizeof(T) == 4 ? 1 : 0;
  sh.a = mg_args(c, l, pm);
  if (cpb_override > 0 && cpb_override <= mg_cpb_limit(lv.nlev)) sh.a.cpb = cpb_override;
  sh.grid = (unsigned)((lv.ncol + sh.a.cpb - 1) / sh.a.cpb);
  sh.smem = (size_t)3 * sh.a.cpb * (lv.nlev | 1) * sizeof(T);
  const int tt = c->tune_mg_threads[pm][l];
  const int tmax = threads_override > 0 ? threads_override : (tt > 0 ? tt : 256);
  int threads = ((sh.a.cpb * lv.nlev + 31) / 32) * 32;   // the block's cells in whole warps
  if (threads > tmax) threads = tmax;
  if (threads < ((sh.a.cpb + 31) / 32) * 32) threads = ((sh.a.cpb + 31) / 32) * 32;   // a lane per column
  sh.threads = threads;
  return sh;
}

// The warp-per-column form serves level l when the tuned (or given) columns per block of the
// precision is -1 and the level has at most 128 layers.
template <typename T>
static bool warp_form(const Ctx *c, int l, int cpb_override = 0) {
  if (c->lv[l].nlev > 128) return false;
  return cpb_override == -1 || (cpb_override == 0 && c->tune_mg_cpb[sizeof(T) == 4 ? 1 : 0][l] == -1);
}

template <typename T, typename Src>
static int launch_warp(Ctx *c, int l, const Src &src, T *out) {
  const Level &lv = c->lv[l];
  const MGArgs a = mg_args(c, l, sizeof(T) == 4 ? 1 : 0);
  const unsigned grid = grid_for((int64_t)lv.ncol * 32, 256);
  const T *hw = Prec<T>::Hz_w(lv), *hl = Prec<T>::Hz_l(lv), *hcp = Prec<T>::Hz_cp(lv);
  if (lv.nlev <= 32) mg_warp_kernel<T, 1, Src><<<grid, 256, 0, c->stream>>>(a, hw, hl, hcp, src, out);
  else if (lv.nlev <= 64) mg_warp_kernel<T, 2, Src><<<grid, 256, 0, c->stream>>>(a, hw, hl, hcp, src, out);
  else mg_warp_kernel<T, 4, Src><<<grid, 256, 0, c->stream>>>(a, hw, hl, hcp, src, out);
  HMG_CUDA(c, cudaGetLastError());
  return HMG_OK;
}

template <typename T, int MODE>
static int smooth(Ctx *c, int l, const T *b, const T *x, T *out, int cpb_override = 0, int threads_override = 0) {
  const Level &lv = c->lv[l];
  if (warp_form<T>(c, l, cpb_override)) {
    if (MODE == 0) return launch_warp<T>(c, l, SrcZero<T, false>{b}, out);
    return launch_warp<T>(c, l, SrcIter<T, false>{Prec<T>::H(lv), b, x}, out);
  }
  const SmoothShape sh = smooth_shape<T>(c, l, cpb_override > 0 ? cpb_override : 0, threads_override);
  mg_smooth_kernel<T, MODE><<<sh.grid, sh.threads, sh.smem, c->stream>>>(
      sh.a, Prec<T>::H(lv), Prec<T>::Hz_w(lv), Prec<T>::Hz_l(lv), Prec<T>::Hz_cp(lv), b, x, out);
  HMG_CUDA(c, cudaGetLastError());
  return HMG_OK;
}

// Level l+1's restricted right-hand side (into lv[l+1].vb) and its first zero-start sweep
// (into out), from level l's b and x, in one launch.
template <typename T>
static int restrict_smooth(Ctx *c, int l, const T *bf, const T *xf, T *out, bool zsweep) {
  const Level &fine = c->lv[l], &lv = c->lv[l + 1];
  if (warp_form<T>(c, l + 1))
    return launch_warp<T>(c, l + 1, SrcRestrict<T>{mg_args(c, l), Prec<T>::H(fine), bf, xf, lv.children,
                                                   static_cast<T *>(lv.vb), zsweep}, out);
  const SmoothShape sh = smooth_shape<T>(c, l + 1);
  mg_restrict_smooth_kernel<T><<<sh.grid, sh.threads, sh.smem, c->stream>>>(
      sh.a, Prec<T>::Hz_w(lv), Prec<T>::Hz_l(lv), Prec<T>::Hz_cp(lv), mg_args(c, l), Prec<T>::H(fine), bf, xf,
      lv.children, static_cast<T *>(lv.vb), out, zsweep);
  HMG_CUDA(c, cudaGetLastError());
  return HMG_OK;
}

// Gamma P^T R into cb and the finest level's first zero-start sweep (into out), in one launch.
template <typename T>
static int trace_restrict_smooth(Ctx *c, const T *R, T *cb, T *out) {
  const Level &lv = c->lv[0];
  const TraceDims d{lv.nlev, lv.nth, lv.ntrace};
  if (warp_form<T>(c, 0))
    return launch_warp<T>(c, 0, SrcTraceRestrict<T>{R, Prec<T>::gamma(c), lv.col_edges, d, cb}, out);
  const SmoothShape sh = smooth_shape<T>(c, 0);
  mg_trace_restrict_smooth_kernel<T><<<sh.grid, sh.threads, sh.smem, c->stream>>>(
      sh.a, Prec<T>::Hz_w(lv), Prec<T>::Hz_l(lv), Prec<T>::Hz_cp(lv), R, Prec<T>::gamma(c), lv.col_edges, d,
      cb, out);
  HMG_CUDA(c, cudaGetLastError());
  return HMG_OK;
}

// x + P e (e from level l+1) and level l's first post-smoothing sweep from it, in one launch.
template <typename T>
static int inject_smooth(Ctx *c, int l, const T *b, const T *x, const T *e, T *out) {
  const Level &lv = c->lv[l];
  if (warp_form<T>(c, l)) return launch_warp<T>(c, l, SrcInject<T>{Prec<T>::H(lv), b, x, e, lv.parent}, out);
  const SmoothShape sh = smooth_shape<T>(c, l);
  mg_inject_smooth_kernel<T><<<sh.grid, sh.threads, sh.smem, c->stream>>>(
      sh.a, Prec<T>::H(lv), Prec<T>::Hz_w(lv), Prec<T>::Hz_l(lv), Prec<T>::Hz_cp(lv), b, x, e, lv.parent, out);
  HMG_CUDA(c, cudaGetLastError());
  return HMG_OK;
}

// Best-of-three average time of a smoothing sweep on level l with `cpb` columns per block,
// in FP64 (fp32 = 0) or FP32.
template <typename T>
static int time_mg_cpb_t(Ctx *c, int l, int cpb, int threads, float *ms) {
  Level &lv = c->lv[l];
  T *b = static_cast<T *>(lv.vb), *x = static_cast<T *>(lv.vx), *y = static_cast<T *>(lv.vy);
  HMG_CUDA(c, cudaMemsetAsync(b, 0, sizeof(T) * lv.ncell, c->stream));
  HMG_CUDA(c, cudaMemsetAsync(x, 0, sizeof(T) * lv.ncell, c->stream));
  int st = smooth<T, 1>(c, l, b, x, y, cpb, threads);
  cudaEvent_t e0, e1;
  HMG_CUDA(c, cudaEventCreate(&e0));
  HMG_CUDA(c, cudaEventCreate(&e1));
  // best of three timings of 10 launches each (the candidates differ by a few per cent)
  float best = 1e30f;
  for (int rep = 0; rep < 3 && !st; ++rep) {
    HMG_CUDA(c, cudaEventRecord(e0, c->stream));
    for (int i = 0; i < 10 && !st; ++i) st = smooth<T, 1>(c, l, b, x, y, cpb, threads);
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

int time_mg_cpb(Ctx *c, int l, int cpb, int threads, int fp32, float *ms) {
  return fp32 ? time_mg_cpb_t<float>(c, l, cpb, threads, ms) : time_mg_cpb_t<double>(c, l, cpb, threads, ms);
}

// n sweeps on level l from zero, or from x0 (n >= 1); the result ends in *cur (one of
// lv.vx / lv.vy; x0 must be neither).
template <typename T>
static int sweeps_from_zero(Ctx *c, int l, const T *b, int n, T **cur, const T *x0 = nullptr) {
  Level &lv = c->lv[l];
  T *x = static_cast<T *>(lv.vx), *y = static_cast<T *>(lv.vy);
  int st;
  if (x0) st = smooth<T, 1>(c, l, b, x0, x);
  else st = smooth<T, 0>(c, l, b, nullptr, x);
  if (st) return st;
  for (int i = 1; i < n; ++i) {
    if ((st = smooth<T, 1>(c, l, b, x, y))) return st;
    T *t = x; x = y; y = t;
  }
  *cur = x;
  return HMG_OK;
}

// Launches the coarse levels 1 .. nmg-1 of a V-cycle as one cooperative grid; *x1 receives
// level 1's correction (lv[1].vx or vy, the pointer sequence of the kernel replayed here).
template <typename T>
static int launch_coarse(Ctx *c, T **x1) {
  const int nmg = c->nmg;
  CoarseArgs<T> p{};
  p.l0 = 1;
  p.nmg = nmg;
  p.npre = c->opt.mg_npre;
  p.npost = c->opt.mg_npost;
  p.ncoarse = c->opt.mg_ncoarse;
  p.zsweep = c->opt.mg_npre == 1;
  size_t smem = 0;
  int64_t need = 1;
  for (int l = 1; l < nmg; ++l) {
    const Level &lv = c->lv[l];
    CoarseLevel<T> &q = p.lv[l];
    q.a = mg_args(c, l, sizeof(T) == 4 ? 1 : 0);
    q.H = Prec<T>::H(lv);
    q.hw = Prec<T>::Hz_w(lv);
    q.hl = Prec<T>::Hz_l(lv);
    q.hcp = Prec<T>::Hz_cp(lv);
    q.vb = static_cast<T *>(lv.vb);
    q.vx = static_cast<T *>(lv.vx);
    q.vy = static_cast<T *>(lv.vy);
    q.children = lv.children;
    q.parent = lv.parent;
    q.nblk = (lv.ncol + q.a.cpb - 1) / q.a.cpb;
    const size_t sm = (size_t)3 * q.a.cpb * (lv.nlev | 1) * sizeof(T);
    if (sm > smem) smem = sm;
    need = std::max<int64_t>(need, std::max<int64_t>(q.nblk, (lv.ncell + 255) / 256));
  }
  p.bar = reinterpret_cast<GridBarrier *>(c->mg_bar);
  p.flag = c->state + 3;
  int per_sm = 0;
  HMG_CUDA(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, mg_coarse_kernel<T>, 256, smem));
  if (per_sm < 1) return fail(c, HMG_ERR_CUDA, "the coarse-level kernel does not fit on an SM");
  const int64_t grid = std::min<int64_t>(need, (int64_t)per_sm * c->num_sms);
  HMG_CUDA(c, cudaMemsetAsync(c->mg_bar, 0, sizeof(GridBarrier), c->stream));
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3(256);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = c->stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  HMG_CUDA(c, cudaLaunchKernelEx(&cfg, mg_coarse_kernel<T>, p));
  // replay the kernel's choice of work vectors
  T *x[kMaxLevels];
  auto sweeps = [&](int l, int n) {
    T *cur = p.lv[l].vx, *oth = p.lv[l].vy;
    for (int i = 1; i < n; ++i) { T *t = cur; cur = oth; oth = t; }
    return cur;
  };
  for (int l = 1; l < nmg - 1; ++l) x[l] = sweeps(l, p.npre);
  x[nmg - 1] = sweeps(nmg - 1, p.ncoarse);
  for (int l = nmg - 2; l >= 1; --l) {
    T *cur = x[l] == p.lv[l].vx ? p.lv[l].vy : p.lv[l].vx, *nxt = x[l];
    for (int i = 0; i < p.npost; ++i) { T *t = cur; cur = nxt; nxt = t; }
    x[l] = cur;
  }
  *x1 = x[1];
  return HMG_OK;
}

// Levels of at most opt.mg_fuse_cells cells (2^18 by default) are latency-bound: there the
// restriction runs inside the level's first (zero-start) sweep and the injection inside its
// first post-sweep, one launch each instead of two. On larger levels the separate, fully
// parallel restriction and injection kernels are faster (measured on GB300 at C96 and C192,
// 30 layers).
static bool fuse_level(const Ctx *c, int l) { return c->lv[l].ncell <= (int64_t)c->opt.mg_fuse_cells; }

int vcycle_launches(const Ctx *c) {
  const int nmg = c->nmg, npre = c->opt.mg_npre, npost = c->opt.mg_npost;
  if (nmg == 1) return c->opt.mg_ncoarse;
  // finest level: pre-sweeps, restriction, injection and post-sweeps; the coarse levels one launch
  if (c->opt.mg_fused) return npre + 1 + 1 + 1 + npost;
  int n = npre + 1 + npost;   // finest level: pre-sweeps, injection, post-sweeps
  for (int l = 1; l < nmg; ++l) {
    const bool f = fuse_level(c, l);
    n += (l == nmg - 1 ? c->opt.mg_ncoarse : npre) + (f ? 0 : 1);   // sweeps (+ restriction)
    if (l < nmg - 1) n += npost + (f ? 0 : 1);                        // post-sweeps (+ injection)
  }
  return n;
}

// With R (the trace residual), b0 = Gamma P^T R is computed into cb inside the first sweep.
template <typename T>
static int vcycle_impl(Ctx *c, const T *b0, T **x_out, const T *x0, const T *R, T *cb) {
  const int nmg = c->nmg, npre = c->opt.mg_npre, npost = c->opt.mg_npost;
  const T *b[kMaxLevels];
  T *x[kMaxLevels];
  int st;
  const int n0 = nmg == 1 ? c->opt.mg_ncoarse : npre;
  if (R) {
    b[0] = cb;
    T *cur = static_cast<T *>(c->lv[0].vx), *oth = static_cast<T *>(c->lv[0].vy);
    if ((st = trace_restrict_smooth<T>(c, R, cb, cur))) return st;
    for (int i = 1; i < n0; ++i) {
      if ((st = smooth<T, 1>(c, 0, cb, cur, oth))) return st;
      T *t = cur; cur = oth; oth = t;
    }
    x[0] = cur;
  } else {
    b[0] = b0;
    if ((st = sweeps_from_zero<T>(c, 0, b0, n0, &x[0], x0))) return st;
  }
  // the pre-smoothing of a level is one sweep from zero (mg_npre = 1, and on the finest level
  // no initial guess x0): the residual before the restriction takes its shorter form
  const bool zs = npre == 1, zs0 = zs && x0 == nullptr;
  // with mg_fused, only the finest level runs step by step; levels >= 1 are one launch
  const bool fused = c->opt.mg_fused && nmg >= 2;
  if (fused) {
    const Level &coarse = c->lv[1];
    T *bc = static_cast<T *>(coarse.vb);
    mg_residual_restrict_kernel<T><<<grid_for(coarse.ncell, 256), 256, 0, c->stream>>>(
        mg_args(c, 0), Prec<T>::H(c->lv[0]), b[0], x[0], coarse.children, coarse.ncol, bc, zs0);
    HMG_CUDA(c, cudaGetLastError());
    b[1] = bc;
    if ((st = launch_coarse<T>(c, &x[1]))) return st;
  } else {
    for (int l = 0; l + 1 < nmg; ++l) {
      // residual + restriction to level l+1, then its first, zero-start sweep (one launch on
      // small levels)
      const Level &cl = c->lv[l + 1];
      T *cur = static_cast<T *>(cl.vx), *oth = static_cast<T *>(cl.vy);
      const bool zsl = l == 0 ? zs0 : zs;
      if (fuse_level(c, l + 1)) {
        if ((st = restrict_smooth<T>(c, l, b[l], x[l], cur, zsl))) return st;
      } else {
        mg_residual_restrict_kernel<T><<<grid_for(cl.ncell, 256), 256, 0, c->stream>>>(
            mg_args(c, l), Prec<T>::H(c->lv[l]), b[l], x[l], cl.children, cl.ncol, static_cast<T *>(cl.vb), zsl);
        if ((st = smooth<T, 0>(c, l + 1, static_cast<const T *>(cl.vb), nullptr, cur))) return st;
      }
      b[l + 1] = static_cast<const T *>(cl.vb);
      const int n = l + 2 == nmg ? c->opt.mg_ncoarse : npre;
      for (int i = 1; i < n; ++i) {
        if ((st = smooth<T, 1>(c, l + 1, b[l + 1], cur, oth))) return st;
        T *t = cur; cur = oth; oth = t;
      }
      x[l + 1] = cur;
    }
  }
  // options are validated to mg_npre >= 1 and mg_npost >= 1
  for (int l = fused ? 0 : nmg - 2; l >= 0; --l) {
    Level &lv = c->lv[l];
    T *other = x[l] == static_cast<T *>(lv.vx) ? static_cast<T *>(lv.vy) : static_cast<T *>(lv.vx);
    int done = 0;
    if (l >= 1 && fuse_level(c, l)) {
      // the injection rides in the first post-sweep (on the finest level it would add 7 FP64
      // adds per cell to an FP64-bound sweep)
      if ((st = inject_smooth<T>(c, l, b[l], x[l], x[l + 1], other))) return st;
      done = 1;
    } else {
      mg_inject_kernel<T><<<grid_for(lv.ncell, 256 * kInjectCells), 256, 0, c->stream>>>(x[l], x[l + 1], lv.parent, lv.nlev,
                                                                          lv.ncell, other);
      HMG_CUDA(c, cudaGetLastError());
    }
    T *cur = other, *nxt = x[l];
    for (int i = done; i < npost; ++i) {
      if ((st = smooth<T, 1>(c, l, b[l], cur, nxt))) return st;
      T *t = cur; cur = nxt; nxt = t;
    }
    x[l] = cur;
  }
  *x_out = x[0];
  return HMG_OK;
}

template <typename T>
int vcycle(Ctx *c, const T *b0, T **x_out, const T *x0) {
  return vcycle_impl<T>(c, b0, x_out, x0, nullptr, nullptr);
}

template <typename T>
int vcycle_trace(Ctx *c, const T *R, T *cb, T **x_out) {
  return vcycle_impl<T>(c, nullptr, x_out, nullptr, R, cb);
}

template <typename T>
static int time_vcycle_t(Ctx *c, float *ms) {
  T *b = static_cast<T *>(c->lv[0].vb);   // level 0's own b vector is free outside a solve
  HMG_CUDA(c, cudaMemsetAsync(b, 0, sizeof(T) * c->lv[0].ncell, c->stream));
  T *x = nullptr;
  int st = vcycle<T>(c, b, &x);
  cudaEvent_t e0, e1;
  HMG_CUDA(c, cudaEventCreate(&e0));
  HMG_CUDA(c, cudaEventCreate(&e1));
  float best = 1e30f;
  for (int rep = 0; rep < 3 && !st; ++rep) {
    HMG_CUDA(c, cudaEventRecord(e0, c->stream));
    for (int i = 0; i < 10 && !st; ++i) st = vcycle<T>(c, b, &x);
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

int time_vcycle(Ctx *c, int fp32, float *ms) {
  return fp32 ? time_vcycle_t<float>(c, ms) : time_vcycle_t<double>(c, ms);
}

template int vcycle<double>(Ctx *, const double *, double **, const double *);
template int vcycle<float>(Ctx *, const float *, float **, const float *);
template int vcycle_trace<double>(Ctx *, const double *, double *, double **);
template int vcycle_trace<float>(Ctx *, const float *, float *, float **);

int pressure_vcycle_fp64(Ctx *c, const double *b, double *x) {
  double *res = nullptr;
  int st = vcycle<double>(c, b, &res);
  if (st) return st;
  HMG_CUDA(c, cudaMemcpyAsync(x, res, sizeof(double) * c->lv[0].ncell, cudaMemcpyDeviceToDevice,
                              c->stream));
  return HMG_OK;
}

int pressure_residual_fp64(Ctx *c, int l, const double *b, const double *x, double *r) {
  const Level &lv = c->lv[l];
  MGArgs a = mg_args(c, l);
  mg_residual_kernel<double><<<grid_for(lv.ncell, 256), 256, 0, c->stream>>>(a, lv.H, b, x, r);
  HMG_CUDA(c, cudaGetLastError());
  return HMG_OK;
}

int apply_pressure_fp64(Ctx *c, int l, const double *x, double *y) {
  const Level &lv = c->lv[l];
  MGArgs a = mg_args(c, l);
  mg_apply_kernel<double><<<grid_for(lv.ncell, 256), 256, 0, c->stream>>>(a, lv.H, x, y);
  HMG_CUDA(c, cudaGetLastError());
  return HMG_OK;
}


// ---- configurations 3a / 3b: the coarse solve by Krylov iteration ---------------------------
// Right-preconditioned BiCGStab (van der Vorst 1992) on H_0 x = b from x = 0, the pressure
// V-cycle as preconditioner, stopping when ||r|| <= tol ||b|| (Sec. 3.2: 1e-14 for 3a, 1e-2
// for 3b) or after maxit iterations (the approximation is used either way, as for a fixed
// number of V-cycles). The host reads the inner products (one synchronisation each).
__global__ void ck_p_kernel(double *__restrict__ p, const double *__restrict__ r, const double *__restrict__ v,
                            double beta, double omega, int64_t n) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) p[i] = r[i] + beta * (p[i] - omega * v[i]);
}
// y = x + a z
__global__ void ck_axpy_kernel(double *__restrict__ y, const double *__restrict__ x, double a,
                               const double *__restrict__ z, int64_t n) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) y[i] = x[i] + a * z[i];
}
// x += alpha phat + omega shat
__global__ void ck_x_kernel(double *__restrict__ x, const double *__restrict__ ph, const double *__restrict__ sh,
                            double alpha, double omega, int64_t n) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) x[i] = x[i] + alpha * ph[i] + omega * sh[i];
}

int coarse_krylov(Ctx *c, const double *b, double *x, double tol, int maxit) {
  const Level &f = c->lv[0];
  const int64_t n = f.ncell;
  int st;
  if (!c->ck && (st = dev_alloc(c, &c->ck, (size_t)8 * n))) return st;
  double *r = c->ck, *rh = r + n, *p = rh + n, *v = p + n, *s = v + n, *t = s + n, *ph = t + n, *sh = ph + n;
  const unsigned g = grid_for(n, 256);
  constexpr int kSlot = 12;
  auto dot = [&](const double *a, const double *bb, double *out) -> int {
    int e = launch_dot(c, a, bb, n, kSlot);
    if (e) return e;
    HMG_CUDA(c, cudaMemcpyAsync(out, c->scal + kSlot, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    HMG_CUDA(c, cudaStreamSynchronize(c->stream));
    return HMG_OK;
  };
  HMG_CUDA(c, cudaMemsetAsync(x, 0, sizeof(double) * n, c->stream));
  HMG_CUDA(c, cudaMemcpyAsync(r, b, sizeof(double) * n, cudaMemcpyDeviceToDevice, c->stream));
  HMG_CUDA(c, cudaMemcpyAsync(rh, b, sizeof(double) * n, cudaMemcpyDeviceToDevice, c->stream));
  HMG_CUDA(c, cudaMemsetAsync(p, 0, sizeof(double) * n, c->stream));
  HMG_CUDA(c, cudaMemsetAsync(v, 0, sizeof(double) * n, c->stream));
  double bb = 0.0;
  if ((st = dot(b, b, &bb))) return st;
  const double bnorm = std::sqrt(bb);
  if (!(bnorm > 0.0)) return HMG_OK;
  double rho_old = 1.0, alpha = 1.0, omega = 1.0;
  for (int it = 0; it < maxit; ++it) {
    double rho = 0.0, rv = 0.0, tt = 0.0, ts = 0.0, rr = 0.0;
    if ((st = dot(rh, r, &rho))) return st;
    if (rho == 0.0 || !std::isfinite(rho)) break;
    const double beta = (rho / rho_old) * (alpha / omega);
    ck_p_kernel<<<g, 256, 0, c->stream>>>(p, r, v, beta, omega, n);
    HMG_CUDA(c, cudaGetLastError());
    if ((st = pressure_vcycle_fp64(c, p, ph))) return st;
    if ((st = apply_pressure_fp64(c, 0, ph, v))) return st;
    if ((st = dot(rh, v, &rv))) return st;
    if (rv == 0.0 || !std::isfinite(rv)) break;
    alpha = rho / rv;
    ck_axpy_kernel<<<g, 256, 0, c->stream>>>(s, r, -alpha, v, n);
    HMG_CUDA(c, cudaGetLastError());
    if ((st = pressure_vcycle_fp64(c, s, sh))) return st;
    if ((st = apply_pressure_fp64(c, 0, sh, t))) return st;
    if ((st = dot(t, t, &tt))) return st;
    if (tt == 0.0 || !std::isfinite(tt)) {   // s = 0: x += alpha phat is exact
      ck_x_kernel<<<g, 256, 0, c->stream>>>(x, ph, sh, alpha, 0.0, n);
      HMG_CUDA(c, cudaGetLastError());
      break;
    }
    if ((st = dot(t, s, &ts))) return st;
    omega = ts / tt;
    ck_x_kernel<<<g, 256, 0, c->stream>>>(x, ph, sh, alpha, omega, n);
    ck_axpy_kernel<<<g, 256, 0, c->stream>>>(r, s, -omega, t, n);
    HMG_CUDA(c, cudaGetLastError());
    rho_old = rho;
    if ((st = dot(r, r, &rr))) return st;
    const double rel = std::sqrt(rr) / bnorm;
    if (!std::isfinite(rel) || rel <= tol) break;
  }
  return HMG_OK;
}

}  // namespace hmg
