// Learned coarse-level correction: a small network f ~ H^-1 used at Algorithm 2 line 6
// (instead of, or as the initial guess of, the pressure V-cycle), its training on the GPU
// (forward, backward, Adam) and the collection of training pairs from the solver itself.
// The paper has no learned component; this is the growth axis of the hot path.
//
// Network per column over the levels (zero padding at ground and lid), bias-free:
//   h1 = relu(conv(1 -> 32, 3)(x)); h2 = relu(conv(32 -> 32, 3)(h1));
//   h3 = relu(w_c h2 + w_e sum(4 edge neighbours) + w_d sum(4 corner neighbours));
//   y  = conv(32 -> 1, 3)(h3); conv(a -> b, 3): y[o,k] = sum_i sum_d W[o,i,d] x[i,k+d-1].
// Around it the diagonal of H scales input and output: dPi = D^-1/2 f(D^-1/2 bbar).
// Storage: BF16 weights and activations (or FP32 for gradient checks), FP32 accumulation,
// FP32 master weights for Adam. Parameters, flat: W1 [32][1][3], W2 [32][32][3],
// M [32][3] (w_c, w_e, w_d), W3 [1][32][3].
#include <cuda_bf16.h>

#include <cmath>
#include <vector>

#include "device_common.cuh"
#include "hmg_internal.cuh"
#include "precond.cuh"

namespace hmg {

constexpr int kCh = 32;
constexpr int kOffW1 = 0, kOffW2 = 96, kOffM = 96 + 3072, kOffW3 = 96 + 3072 + 96;
constexpr int kNParams = kOffW3 + 96;   // 3360
static_assert(kNParams == kCoarseParams, "parameter count");
constexpr int kMaxL = 128;              // levels a column may have for the network kernels
constexpr int kMaxNnCpb = 16;           // columns per block of the horizontal-mix kernel (at most)

template <typename A>
__device__ __forceinline__ float to_f(A v);
template <>
__device__ __forceinline__ float to_f<float>(float v) { return v; }
template <>
__device__ __forceinline__ float to_f<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }
template <typename A>
__device__ __forceinline__ A from_f(float v);
template <>
__device__ __forceinline__ float from_f<float>(float v) { return v; }
template <>
__device__ __forceinline__ __nv_bfloat16 from_f<__nv_bfloat16>(float v) { return __float2bfloat16(v); }
// value as it is stored (rounded to the storage type), back in FP32
template <typename A>
__device__ __forceinline__ float rnd(float v) { return to_f<A>(from_f<A>(v)); }

// ---- neighbour access -----------------------------------------------------------------------
// On the mesh: edge and corner neighbours from tables. On a training patch (nx x ny columns,
// column j*nx + i of sample s): the regular grid, -1 outside the patch (zero padding).
struct Nbrs {
  const int32_t *edge, *diag;   // mesh tables [ncol][4]; null on patches
  int nx, ny;                   // patch shape
  __device__ __forceinline__ void get(int col, int out_e[4], int out_d[4]) const {
    if (edge) {
#pragma unroll
      for (int s = 0; s < 4; ++s) { out_e[s] = edge[4 * col + s]; out_d[s] = diag[4 * col + s]; }
      return;
    }
    const int P = nx * ny, s0 = (col / P) * P, q = col - s0, i = q % nx, j = q / nx;
    auto at = [&](int di, int dj) {
      const int i2 = i + di, j2 = j + dj;
      return (i2 >= 0 && i2 < nx && j2 >= 0 && j2 < ny) ? s0 + j2 * nx + i2 : -1;
    };
    out_e[0] = at(0, -1); out_e[1] = at(1, 0); out_e[2] = at(0, 1); out_e[3] = at(-1, 0);
    out_d[0] = at(1, -1); out_d[1] = at(1, 1); out_d[2] = at(-1, 1); out_d[3] = at(-1, -1);
  }
};

// ---- forward, column-local layers: x -> h1 -> h2 ---------------------------------------------
// One block per CPB columns; weights and one column block of activations in shared memory.
// x = xin[K] * xscale(K) with xscale = 1/sqrt(diag H) (mesh) or 1 (patches). Stores h2 (and h1
// when training) in A, channel-major [32][ncells].
template <typename A, typename Tin>
__global__ void __launch_bounds__(128)
    nn_front_kernel(const float *__restrict__ wts, const Tin *__restrict__ xin,
                    const double *__restrict__ diagH, const float *__restrict__ diagH32, int ncol,
                    int L, int cpb, A *__restrict__ h1_out, A *__restrict__ h2_out) {
  extern __shared__ float sm[];
  float *W1 = sm, *W2 = W1 + 96;
  float *xs = W2 + 3072;                       // [cpb][L+2]
  float *h1 = xs + cpb * (L + 2);              // [cpb][32][L+2]
  for (int i = threadIdx.x; i < 96; i += blockDim.x) W1[i] = rnd<A>(wts[kOffW1 + i]);
  for (int i = threadIdx.x; i < 3072; i += blockDim.x) W2[i] = rnd<A>(wts[kOffW2 + i]);
  const int c0 = blockIdx.x * cpb, nc = min(cpb, ncol - c0);
  const int64_t C = (int64_t)ncol * L;
  for (int i = threadIdx.x; i < cpb * (L + 2); i += blockDim.x) {
    const int cc = i / (L + 2), k = i % (L + 2) - 1;
    float v = 0.f;
    if (cc < nc && k >= 0 && k < L) {
      const int64_t K = (int64_t)(c0 + cc) * L + k;
      float s = 1.f;
      if (diagH) s = (float)(1.0 / sqrt(diagH[K]));
      else if (diagH32) s = rsqrtf(diagH32[K]);
      v = rnd<A>((float)xin[K] * s);
    }
    xs[i] = v;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < cpb * kCh * (L + 2); i += blockDim.x) {
    const int cc = i / (kCh * (L + 2)), r = i % (kCh * (L + 2)), o = r / (L + 2), k = r % (L + 2) - 1;
    float v = 0.f;
    if (cc < nc && k >= 0 && k < L) {
      const float *x = xs + cc * (L + 2) + k;    // x[k-1..k+1] at x[0..2]
      v = fmaxf(fmaf(W1[3 * o], x[0], fmaf(W1[3 * o + 1], x[1], W1[3 * o + 2] * x[2])), 0.f);
      v = rnd<A>(v);
      if (h1_out) h1_out[(int64_t)o * C + (int64_t)(c0 + cc) * L + k] = from_f<A>(v);
    }
    h1[i] = v;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < nc * kCh * L; i += blockDim.x) {
    const int cc = i / (kCh * L), r = i % (kCh * L), o = r / L, k = r % L;
    const float *hb = h1 + cc * kCh * (L + 2) + k;   // channel i at hb + i*(L+2), taps 0..2
    const float *w = W2 + o * 96;
    float acc = 0.f;
#pragma unroll 8
    for (int ci = 0; ci < kCh; ++ci) {
      const float *hc = hb + ci * (L + 2);
      acc = fmaf(w[3 * ci], hc[0], acc);
      acc = fmaf(w[3 * ci + 1], hc[1], acc);
      acc = fmaf(w[3 * ci + 2], hc[2], acc);
    }
    h2_out[(int64_t)o * C + (int64_t)(c0 + cc) * L + k] = from_f<A>(fmaxf(acc, 0.f));
  }
}

// ---- forward, column-local layers on the tensor cores (inference, BF16) ---------------------
// The cells are laid out in padded rows, R = col (L + 2) + k + 1, with an empty row below and
// above every column (levels -1 and L). Per tile of 128 padded rows,
// h2 = relu(conv(32 -> 32, 3)(h1)) is a GEMM
//   H2[m][o] = sum_d sum_i h1[i](row m + d - 1) W2[o][i][d]
// issued as six tcgen05.mma (M 128, N 32, K 16; K = d * 32 + i): the A operand of tap d is the
// tile's h1 rows shifted by d - 1, i.e. the same shared-memory buffer read from a start address
// d rows further on. h1 is zero on the padded rows, which is the convolution's zero padding at
// ground and lid, so A needs no im2col copy. A: h1 on the tile's rows -1 .. 128 in BF16,
// K-major without swizzle ([8-channel group][row][8 channels]: rows every 16 B, core matrices
// along M every 128 B, along K every 130 x 16 B); B (32 x 96 BF16) in the same core-matrix form.
// The FP32 accumulator lives in 32 TMEM columns and is read back by the four warps (warp w owns
// lanes 32w..32w+31); the results of padded rows are dropped. h2 leaves cell-major, [ncell][32]
// BF16, for nn_mix_out_kernel.
constexpr int kTcM = 128;
constexpr int kTcRows = kTcM + 2;                      // h1 rows of a tile: -1 .. 128
constexpr int kTcLbo = kTcRows * 16;                   // bytes between 8-channel groups
constexpr int kTcB = (4 * kTcLbo + 1023) / 1024 * 1024;   // A: 8,320 B; B from here (6 KB)
constexpr int kTcX = kTcB + 6 * 1024;                  // x (132 floats), W1 (96), levels (132 ints)
constexpr int kTcBar = kTcX + 1536;                    // two mbarriers (16 B), TMEM address (4 B)
constexpr int kTcSmem = kTcBar + 64;
constexpr uint32_t kTcWaitLimit = 1u << 20;   // mbarrier polls before the kernel gives up

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// shared-memory matrix descriptor: start, leading (K) and stride (M/N) byte offsets, no swizzle
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;   // descriptor version of this architecture
  return d;                 // base offset 0, layout type 0 (no swizzle)
}

// instruction descriptor of kind::f16: FP32 D, BF16 A and B, both K-major, M x N
__host__ __device__ constexpr uint32_t umma_idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// W2 -> the B operand image: B[o][d * 32 + i] in BF16, core-matrix order (N = 32: 4 row groups)
__global__ void nn_pack_b_kernel(const float *__restrict__ wts, __nv_bfloat16 *__restrict__ bimg) {
  for (int e = threadIdx.x; e < 32 * 96; e += blockDim.x) {
    const int o = e / 96, kk = e % 96, d = kk / 32, i = kk % 32;
    const int off = ((kk >> 3) * 4 + (o >> 3)) * 64 + (o & 7) * 8 + (kk & 7);   // in elements
    bimg[off] = __float2bfloat16(wts[kOffW2 + (o * 32 + i) * 3 + d]);
  }
}

__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, uint32_t limit = kTcWaitLimit) {
  uint32_t done = 0;
  for (uint32_t it = 0; it < limit && !done; ++it)
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
                 : "=r"(done) : "r"(smem_u32(bar)), "r"(parity) : "memory");
  return done != 0;
}

// TRAIN (the training minibatch's forward, x unscaled): h1 and h2 are stored channel-major
// [32][ncell] BF16 for the backward instead of h2 cell-major, and no scale is kept.
template <typename Tin, bool TRAIN = false>
__global__ void __launch_bounds__(128)
    nn_front_tc_kernel(const float *__restrict__ wts, const __nv_bfloat16 *__restrict__ bimg,
                       const Tin *__restrict__ xin, const double *__restrict__ diagH,
                       const float *__restrict__ diagH32, int ncol, int L,
                       __nv_bfloat16 *__restrict__ h2_out, float *__restrict__ dscale_out,
                       int *__restrict__ wait_flag, __nv_bfloat16 *__restrict__ h1_out = nullptr) {
  extern __shared__ __align__(1024) unsigned char tc_smem[];
  unsigned char *sA = tc_smem, *sB = tc_smem + kTcB;
  float *xs = reinterpret_cast<float *>(tc_smem + kTcX);            // 132 floats
  float *w1s = xs + kTcM + 4;                                        // 96 floats
  int *lev = reinterpret_cast<int *>(w1s + 96);                      // 132 ints: level of x's rows
  uint64_t *bar = reinterpret_cast<uint64_t *>(tc_smem + kTcBar);   // [0] MMA done, [1] B loaded
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(tc_smem + kTcBar + 16);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int P = L + 2, nrows = ncol * P;     // padded rows (the host checks that they fit an int)
  const int R0 = blockIdx.x * kTcM;
  // level of padded row R, or -1 on a pad row or past the mesh
  auto level = [&](int R) {
    if (R < 0 || R >= nrows) return -1;
    const int k = R % P - 1;
    return k < L ? k : -1;
  };

  if (warp == 0) {   // 32 TMEM columns for the 128 x 32 FP32 accumulator
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 32;" ::"r"(smem_u32(tmem_slot)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar + 1)));
    asm volatile("fence.mbarrier_init.release.cluster;");
    // B (6 KB) by the bulk-copy engine
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar + 1)), "r"(6144));
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(smem_u32(sB)), "l"(bimg), "r"(6144), "r"(smem_u32(bar + 1)) : "memory");
  }
  // x on padded rows R0-2 .. R0+129 (scaled by diag(H)^-1/2 in FP32, rounded to BF16), 0 on pad
  // rows and outside the mesh; the scale of the tile's own rows is kept for the output layer
  for (int j = tid; j < kTcM + 4; j += blockDim.x) {
    const int R = R0 - 2 + j, k = level(R);
    lev[j] = k;
    float v = 0.f;
    if (k >= 0) {
      const int64_t q = (int64_t)(R / P) * L + k;
      const float sc = rsqrtf(diagH ? (float)diagH[q] : diagH32 ? diagH32[q] : 1.f);
      v = rnd<__nv_bfloat16>((float)xin[q] * sc);
      if (!TRAIN && j >= 2 && j < kTcM + 2) dscale_out[q] = sc;
    }
    xs[j] = v;
  }
  if (tid < 96) w1s[tid] = rnd<__nv_bfloat16>(wts[kOffW1 + tid]);
  __syncthreads();
  // A: h1 = relu(conv(1 -> 32, 3)(x)) on tile rows -1..128 (buffer rows 0..129), 16 B (8 channels
  // of one row) per store, rows fastest (consecutive 16-byte slots, no bank conflicts)
  for (int e = tid; e < 4 * kTcRows; e += blockDim.x) {
    const int row = e % kTcRows, g = e / kTcRows;
    uint4 pack = make_uint4(0u, 0u, 0u, 0u);
    if (lev[row + 1] >= 0) {
      const float xm = xs[row], x0 = xs[row + 1], xp = xs[row + 2];   // zero on pad rows
      uint32_t wds[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        float hv[2];
#pragma unroll
        for (int t = 0; t < 2; ++t) {
          const float *w = w1s + 3 * (g * 8 + 2 * q + t);
          hv[t] = fmaxf(fmaf(w[0], xm, fmaf(w[1], x0, w[2] * xp)), 0.f);
        }
        const __nv_bfloat162 b2 = __floats2bfloat162_rn(hv[0], hv[1]);
        wds[q] = *reinterpret_cast<const uint32_t *>(&b2);
        if (TRAIN && row >= 1 && row <= kTcM) {   // the tile's own rows: h1 for the backward
          const int64_t C = (int64_t)ncol * L, cell = (int64_t)((R0 - 1 + row) / P) * L + lev[row + 1];
          h1_out[(int64_t)(g * 8 + 2 * q) * C + cell] = b2.x;
          h1_out[(int64_t)(g * 8 + 2 * q + 1) * C + cell] = b2.y;
        }
      }
      pack = make_uint4(wds[0], wds[1], wds[2], wds[3]);
    }
    *reinterpret_cast<uint4 *>(sA + g * kTcLbo + row * 16) = pack;
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // generic writes -> tensor core
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  if (tid == 0) {
    if (mbar_wait(bar + 1, 0)) {
      const uint32_t a0 = smem_u32(sA), b0 = smem_u32(sB);
      const uint32_t idesc = umma_idesc_bf16(kTcM, 32);
      for (int s = 0; s < 6; ++s) {   // tap d = s / 2, channels 16 (s % 2) .. + 15
        const int d = s >> 1, h = s & 1;
        const uint64_t ad = umma_desc(a0 + 2 * h * kTcLbo + d * 16, kTcLbo, 128);
        const uint64_t bd = umma_desc(b0 + s * 2 * 4 * 128, 4 * 128, 128);
        const uint32_t acc = s > 0 ? 1u : 0u;
        asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                     " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(tmem),
                     "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar)));
    } else {
      atomicExch(wait_flag, 1);
      // the bulk copy of B may still be in flight: wait for it once more (bounded) before the
      // block releases its shared memory, then release the waiters without any MMA
      mbar_wait(bar + 1, 0);
      asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)));
    }
  }
  // one decision for the whole block, so that the warp-collective loads below never diverge
  const bool done = __syncthreads_and(mbar_wait(bar, 0) ? 1 : 0) != 0;
  if (!done) {
    // MMAs may still be writing the accumulator: one more bounded wait for their commit before
    // the tensor memory is freed (the launch's outputs are undefined either way)
    if (tid == 0) {
      atomicExch(wait_flag, 1);
      mbar_wait(bar, 0);
    }
    __syncthreads();
  }
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (done) {
    uint32_t r[32];
    const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16);
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                 "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                   "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
                   "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
                   "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    const int R = R0 + warp * 32 + lane, k = lev[warp * 32 + lane + 2];
    if (TRAIN && k >= 0) {   // channel-major: each channel's store coalesced over the warp's cells
      const int64_t C = (int64_t)ncol * L, cell = (int64_t)(R / P) * L + k;
#pragma unroll
      for (int i = 0; i < kCh; ++i) h2_out[(int64_t)i * C + cell] = __float2bfloat16_rn(fmaxf(__uint_as_float(r[i]), 0.f));
    } else if (k >= 0) {   // cell-major: the 32 channels of a cell in 64 contiguous bytes
      const int64_t cell = (int64_t)(R / P) * L + k;
      uint32_t wd[16];
#pragma unroll
      for (int p = 0; p < 16; ++p) {
        const __nv_bfloat162 b2 =
            __floats2bfloat162_rn(fmaxf(__uint_as_float(r[2 * p]), 0.f), fmaxf(__uint_as_float(r[2 * p + 1]), 0.f));
        wd[p] = *reinterpret_cast<const uint32_t *>(&b2);
      }
      uint4 *dst = reinterpret_cast<uint4 *>(h2_out + cell * kCh);
#pragma unroll
      for (int g = 0; g < 4; ++g) dst[g] = make_uint4(wd[4 * g], wd[4 * g + 1], wd[4 * g + 2], wd[4 * g + 3]);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 32;" ::"r"(tmem));
}

// ---- inference: horizontal mix and output layer after the tensor-core layers -----------------
// h2 cell-major [ncell][32] BF16. Four threads per cell, thread q owning channels 8q..8q+7, so
// that one 16-byte load brings a neighbour's share and a warp reads 512 contiguous bytes per
// neighbour; the nine loads are issued before any use. Sums in FP32, two channels per packed
// instruction. A block holds whole columns: h3 goes to shared memory in padded rows ([column]
// [L + 2][36 floats], zero rows at levels -1 and L, so the output convolution needs no edge
// test), and the four partial sums of the output convolution are added by shuffles. The same
// arithmetic as nn_back_kernel's mesh form up to the order of the 96-term output sum.
// out[K] = y * dscale[K], dscale = diag(H)^-1/2 in FP32 as the front kernel computed it.
template <typename Tout>
__global__ void __launch_bounds__(512)
    nn_mix_out_kernel(const float *__restrict__ wts, const __nv_bfloat16 *__restrict__ h2, Nbrs nb, int ncol,
                      int L, int cpb, const float *__restrict__ dscale, Tout *__restrict__ out) {
  extern __shared__ __align__(16) float sm[];
  // weights per channel as float4, channel 8q + t at 9q + t (no bank conflicts across q)
  float4 *Mw4 = reinterpret_cast<float4 *>(sm);          // (w_c, w_e, w_d, 0)
  float4 *W34 = Mw4 + 36;                                // (W3[0][ch][0..2], 0)
  int *snb = reinterpret_cast<int *>(W34 + 36);          // [cpb][8] edge, corner neighbours
  float *h3 = reinterpret_cast<float *>(snb + 8 * cpb);  // [cpb][L + 2][36]
  const int tid = threadIdx.x;
  if (tid < 32) {
    const int w = 9 * (tid >> 3) + (tid & 7);
    const float *m = wts + kOffM + 3 * tid, *w3 = wts + kOffW3 + 3 * tid;
    Mw4[w] = make_float4(rnd<__nv_bfloat16>(m[0]), rnd<__nv_bfloat16>(m[1]), rnd<__nv_bfloat16>(m[2]), 0.f);
    W34[w] = make_float4(rnd<__nv_bfloat16>(w3[0]), rnd<__nv_bfloat16>(w3[1]), rnd<__nv_bfloat16>(w3[2]), 0.f);
  }
  const int c0 = blockIdx.x * cpb, nc = min(cpb, ncol - c0);
  if (tid < nc) {
    int e[4], d[4];
    nb.get(c0 + tid, e, d);
#pragma unroll
    for (int q = 0; q < 4; ++q) { snb[8 * tid + q] = e[q]; snb[8 * tid + 4 + q] = d[q]; }
  }
  for (int e = tid; e < cpb * 72; e += blockDim.x) {   // the pad rows
    const int cc = e / 72, r = e % 72;
    h3[(cc * (L + 2) + (r < 36 ? 0 : L + 1)) * 36 + r % 36] = 0.f;
  }
  // one (cell, channel group) per thread: the host launches at least 4 L cpb threads
  const int j = tid >> 2, q = tid & 3;
  const bool act = j < nc * L;
  const int cc = act ? j / L : 0, k = j - cc * L;
  __syncthreads();
  float *row = h3 + (cc * (L + 2) + k + 1) * 36 + 8 * q;
  if (act) {
    const int *nbr = snb + 8 * cc;
    const unsigned own = (unsigned)(c0 + cc), L4 = 4u * (unsigned)L;
    const uint4 *hv = reinterpret_cast<const uint4 *>(h2) + (4u * (unsigned)k + q);   // + column * 4 L
    uint4 v[9];
    v[0] = hv[own * L4];
#pragma unroll
    for (int s = 0; s < 8; ++s) v[1 + s] = hv[(nbr[s] >= 0 ? (unsigned)nbr[s] : own) * L4];
    auto pair = [](const uint4 &u, int p) {
      const uint32_t w = p == 0 ? u.x : p == 1 ? u.y : p == 2 ? u.z : u.w;
      return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&w));
    };
    float hq[8];
#pragma unroll
    for (int p = 0; p < 4; ++p) {   // channels 8q + 2p, 8q + 2p + 1
      float2 se = make_float2(0.f, 0.f), sd = make_float2(0.f, 0.f);
#pragma unroll
      for (int s = 0; s < 4; ++s) {
        if (nbr[s] >= 0) se = __fadd2_rn(se, pair(v[1 + s], p));
        if (nbr[4 + s] >= 0) sd = __fadd2_rn(sd, pair(v[5 + s], p));
      }
      const float4 ma = Mw4[9 * q + 2 * p], mb = Mw4[9 * q + 2 * p + 1];
      float2 a = __fmul2_rn(make_float2(ma.z, mb.z), sd);
      a = __ffma2_rn(make_float2(ma.y, mb.y), se, a);
      a = __ffma2_rn(make_float2(ma.x, mb.x), pair(v[0], p), a);
      const float2 r = __bfloat1622float2(__floats2bfloat162_rn(fmaxf(a.x, 0.f), fmaxf(a.y, 0.f)));
      hq[2 * p] = r.x;
      hq[2 * p + 1] = r.y;
    }
    reinterpret_cast<float4 *>(row)[0] = make_float4(hq[0], hq[1], hq[2], hq[3]);
    reinterpret_cast<float4 *>(row)[1] = make_float4(hq[4], hq[5], hq[6], hq[7]);
  }
  const float dsc = act && q == 0 ? dscale[(int64_t)c0 * L + j] : 0.f;   // in flight across the barrier
  __syncthreads();
  float y = 0.f;
  if (act) {
    float xm[8], x0[8], xp[8];
    const float4 *rm = reinterpret_cast<const float4 *>(row - 36), *r0 = reinterpret_cast<const float4 *>(row),
                 *rp = reinterpret_cast<const float4 *>(row + 36);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const float4 a = rm[h], b = r0[h], c = rp[h];
      xm[4 * h] = a.x; xm[4 * h + 1] = a.y; xm[4 * h + 2] = a.z; xm[4 * h + 3] = a.w;
      x0[4 * h] = b.x; x0[4 * h + 1] = b.y; x0[4 * h + 2] = b.z; x0[4 * h + 3] = b.w;
      xp[4 * h] = c.x; xp[4 * h + 1] = c.y; xp[4 * h + 2] = c.z; xp[4 * h + 3] = c.w;
    }
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      const float4 w = W34[9 * q + t];
      y = fmaf(w.x, xm[t], fmaf(w.y, x0[t], fmaf(w.z, xp[t], y)));
    }
  }
  y += __shfl_xor_sync(0xffffffffu, y, 1);
  y += __shfl_xor_sync(0xffffffffu, y, 2);
  if (act && q == 0) out[(int64_t)c0 * L + j] = (Tout)(y * dsc);
}

// ---- forward, horizontal mix and output layer: h2 -> h3 -> y ---------------------------------
// mesh: out[K] = y * yscale(K) (yscale = 1/sqrt(diag H)) written as Tout.
// training: also stores h3 and, for the loss, gy = 2 (y - t) / (||t_s||^2 B) and the per-block
// sums of (y - t)^2 / ||t_s||^2 (sample s of the block's columns).
template <typename A, typename Tout>
__global__ void __launch_bounds__(128)
    nn_back_kernel(const float *__restrict__ wts, const A *__restrict__ h2, Nbrs nb, int ncol, int L,
                   int cpb, const double *__restrict__ diagH, const float *__restrict__ diagH32,
                   Tout *__restrict__ out, A *__restrict__ h3_out, const float *__restrict__ target,
                   const float *__restrict__ tnorm2, int patch_cols, float inv_batch,
                   float *__restrict__ gy_out, double *__restrict__ loss_part) {
  extern __shared__ float sm[];
  float *Mw = sm, *W3 = Mw + 96;
  float *h3 = W3 + 96;                          // [cpb][32][L+2]
  __shared__ double red[4];
  __shared__ int snb[kMaxNnCpb][8];             // edge and corner neighbours of the block's columns
  for (int i = threadIdx.x; i < 96; i += blockDim.x) {
    Mw[i] = rnd<A>(wts[kOffM + i]);
    W3[i] = rnd<A>(wts[kOffW3 + i]);
  }
  const int c0 = blockIdx.x * cpb, nc = min(cpb, ncol - c0);
  const int64_t C = (int64_t)ncol * L;
  if ((int)threadIdx.x < nc) {
    int e[4], d[4];
    nb.get(c0 + threadIdx.x, e, d);
#pragma unroll
    for (int q = 0; q < 4; ++q) { snb[threadIdx.x][q] = e[q]; snb[threadIdx.x][4 + q] = d[q]; }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < cpb * kCh * (L + 2); i += blockDim.x) {
    const int cc = i / (kCh * (L + 2)), r = i % (kCh * (L + 2)), ch = r / (L + 2), k = r % (L + 2) - 1;
    float v = 0.f;
    if (cc < nc && k >= 0 && k < L) {
      const int col = c0 + cc;
      const int *e = snb[cc], *d = snb[cc] + 4;
      const A *hc = h2 + (int64_t)ch * C;
      float se = 0.f, sd = 0.f;
#pragma unroll
      for (int s = 0; s < 4; ++s) {
        if (e[s] >= 0) se += to_f<A>(hc[(int64_t)e[s] * L + k]);
        if (d[s] >= 0) sd += to_f<A>(hc[(int64_t)d[s] * L + k]);
      }
      const float a = fmaf(Mw[3 * ch], to_f<A>(hc[(int64_t)col * L + k]), fmaf(Mw[3 * ch + 1], se, Mw[3 * ch + 2] * sd));
      v = rnd<A>(fmaxf(a, 0.f));
      if (h3_out) h3_out[(int64_t)ch * C + (int64_t)col * L + k] = from_f<A>(v);
    }
    h3[i] = v;
  }
  __syncthreads();
  double lsum = 0.0;
  for (int i = threadIdx.x; i < nc * L; i += blockDim.x) {
    const int cc = i / L, k = i % L;
    const float *hb = h3 + cc * kCh * (L + 2) + k;
    float y = 0.f;
#pragma unroll 8
    for (int ch = 0; ch < kCh; ++ch) {
      const float *hc = hb + ch * (L + 2);
      y = fmaf(W3[3 * ch], hc[0], fmaf(W3[3 * ch + 1], hc[1], fmaf(W3[3 * ch + 2], hc[2], y)));
    }
    const int64_t K = (int64_t)(c0 + cc) * L + k;
    if (out) {
      double s = 1.0;
      if (diagH) s = 1.0 / sqrt(diagH[K]);
      else if (diagH32) s = (double)rsqrtf(diagH32[K]);
      out[K] = (Tout)((double)y * s);
    }
    if (gy_out) {
      const int sample = (c0 + cc) / patch_cols;
      const float r = y - target[K];
      const float w = 1.0f / tnorm2[sample];
      gy_out[K] = 2.0f * r * w * inv_batch;
      lsum += (double)(r * r * w);
    }
  }
  if (loss_part) {
    lsum = warp_sum(lsum);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = lsum;
    __syncthreads();
    if (threadIdx.x == 0) {
      double s = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
      loss_part[blockIdx.x] = s;
    }
  }
}

// ---- backward ---------------------------------------------------------------------------------
// B3: gh3 = conv^T(W3, gy), ga3 = gh3 [h3 > 0]; partial gW3[ch][d] = sum gy[k] h3[ch][k+d-1].
// One block per CPB columns; the partial sums of its columns go to part[block][96].
template <typename A>
__global__ void __launch_bounds__(128)
    nn_bwd3_kernel(const float *__restrict__ wts, const A *__restrict__ h3, const float *__restrict__ gy,
                   int ncol, int L, int cpb, float *__restrict__ ga3, float *__restrict__ part) {
  extern __shared__ float sm[];
  float *W3 = sm, *gys = W3 + 96;               // gys [cpb][L+2]
  float *acc = gys + cpb * (L + 2);             // [96] per-block partials
  for (int i = threadIdx.x; i < 96; i += blockDim.x) { W3[i] = rnd<A>(wts[kOffW3 + i]); acc[i] = 0.f; }
  const int c0 = blockIdx.x * cpb, nc = min(cpb, ncol - c0);
  const int64_t C = (int64_t)ncol * L;
  for (int i = threadIdx.x; i < cpb * (L + 2); i += blockDim.x) {
    const int cc = i / (L + 2), k = i % (L + 2) - 1;
    gys[i] = (cc < nc && k >= 0 && k < L) ? gy[(int64_t)(c0 + cc) * L + k] : 0.f;
  }
  __syncthreads();
  // ga3 (one thread per (column, channel, level))
  for (int i = threadIdx.x; i < nc * kCh * L; i += blockDim.x) {
    const int cc = i / (kCh * L), r = i % (kCh * L), ch = r / L, k = r % L;
    const float *g = gys + cc * (L + 2) + k;    // gy[k-1..k+1] at g[0..2]
    // y[k'] += W3[ch][d] h3[ch][k'+d-1]  =>  gh3[ch][k] = sum_d W3[ch][d] gy[k-d+1]
    const float gh = fmaf(W3[3 * ch], g[2], fmaf(W3[3 * ch + 1], g[1], W3[3 * ch + 2] * g[0]));
    const int64_t idx = (int64_t)ch * C + (int64_t)(c0 + cc) * L + k;
    ga3[idx] = to_f<A>(h3[idx]) > 0.f ? gh : 0.f;
  }
  // gW3 partials: thread per (ch, d), loop over the block's positions
  for (int w = threadIdx.x; w < 96; w += blockDim.x) {
    const int ch = w / 3, d = w % 3;
    float s = 0.f;
    for (int cc = 0; cc < nc; ++cc)
      for (int k = 0; k < L; ++k) {
        const int kk = k + d - 1;
        if (kk < 0 || kk >= L) continue;
        s = fmaf(gys[cc * (L + 2) + k + 1], to_f<A>(h3[(int64_t)ch * C + (int64_t)(c0 + cc) * L + kk]), s);
      }
    acc[w] = s;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 96; i += blockDim.x) part[(int64_t)blockIdx.x * 96 + i] = acc[i];
}

// B2: gh2 = w_c ga3 + w_e sum(edge nbrs of ga3) + w_d sum(corner nbrs) (the neighbour relation is
// symmetric on a patch), ga2 = gh2 [h2 > 0]; partials of gM: (ga3 . h2, ga3 . sum_e h2,
// ga3 . sum_d h2) per channel. Thread per cell (consecutive threads on consecutive levels, so every
// channel's loads and stores are coalesced), grid-stride over the cells; blockIdx.y picks 4 of the
// 32 channels. Block x writes entries 12 y .. 12 y + 11 of partial row x.
constexpr int kBw2Ch = 4;
template <typename A>
__global__ void __launch_bounds__(128)
    nn_bwd2_kernel(const float *__restrict__ wts, const A *__restrict__ h2, const float *__restrict__ ga3,
                   Nbrs nb, int ncol, int L, float *__restrict__ ga2, float *__restrict__ part) {
  __shared__ float Mw[3 * kBw2Ch], red[4][3 * kBw2Ch];
  const int ch0 = blockIdx.y * kBw2Ch;
  if (threadIdx.x < 3 * kBw2Ch) Mw[threadIdx.x] = rnd<A>(wts[kOffM + 3 * ch0 + threadIdx.x]);
  __syncthreads();
  const int64_t C = (int64_t)ncol * L;
  float acc[3 * kBw2Ch];
#pragma unroll
  for (int q = 0; q < 3 * kBw2Ch; ++q) acc[q] = 0.f;
  for (int64_t K = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; K < C; K += (int64_t)gridDim.x * blockDim.x) {
    const int col = (int)(K / L), k = (int)(K - (int64_t)col * L);
    int e[4], d[4];
    nb.get(col, e, d);
    int64_t oe[4], od[4];
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      oe[s] = e[s] >= 0 ? (int64_t)e[s] * L + k : -1;
      od[s] = d[s] >= 0 ? (int64_t)d[s] * L + k : -1;
    }
#pragma unroll
    for (int j = 0; j < kBw2Ch; ++j) {
      const float *g = ga3 + (int64_t)(ch0 + j) * C;
      const A *h = h2 + (int64_t)(ch0 + j) * C;
      const float gk = g[K], hk = to_f<A>(h[K]);
      float ge = 0.f, gd = 0.f, he = 0.f, hd = 0.f;
#pragma unroll
      for (int s = 0; s < 4; ++s) {
        if (oe[s] >= 0) { ge += g[oe[s]]; he += to_f<A>(h[oe[s]]); }
        if (od[s] >= 0) { gd += g[od[s]]; hd += to_f<A>(h[od[s]]); }
      }
      const float gh = fmaf(Mw[3 * j], gk, fmaf(Mw[3 * j + 1], ge, Mw[3 * j + 2] * gd));
      ga2[(int64_t)(ch0 + j) * C + K] = hk > 0.f ? gh : 0.f;
      acc[3 * j] = fmaf(gk, hk, acc[3 * j]);
      acc[3 * j + 1] = fmaf(gk, he, acc[3 * j + 1]);
      acc[3 * j + 2] = fmaf(gk, hd, acc[3 * j + 2]);
    }
  }
  // fixed-order reduction: lanes by butterfly, then the four warps
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int q = 0; q < 3 * kBw2Ch; ++q) {
    float v = acc[q];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) red[warp][q] = v;
  }
  __syncthreads();
  if (threadIdx.x < 3 * kBw2Ch)
    part[(int64_t)blockIdx.x * 96 + 3 * ch0 + threadIdx.x] =
        (red[0][threadIdx.x] + red[1][threadIdx.x]) + (red[2][threadIdx.x] + red[3][threadIdx.x]);
}

// B1: gh1 = conv^T(W2, ga2), ga1 = gh1 [h1 > 0]; partials of gW2 = sum ga2[o][k] h1[i][k+d-1]
// and gW1 = sum ga1[o][k] x[k+d-1]. One block per CPB columns; thread-owned weight slots.
template <typename A>
__global__ void __launch_bounds__(256)
    nn_bwd1_kernel(const float *__restrict__ wts, const A *__restrict__ h1, const float *__restrict__ ga2,
                   const float *__restrict__ xin, int ncol, int L, int cpb, float *__restrict__ part2,
                   float *__restrict__ part1) {
  extern __shared__ float sm[];
  float *W2 = sm;                                   // [32][32][3]
  float *g2 = W2 + 3072;                            // [32][L+2] one column of ga2
  float *h1s = g2 + kCh * (L + 2);                  // [32][L+2]
  float *g1 = h1s + kCh * (L + 2);                  // [32][L+2]
  float *xs = g1 + kCh * (L + 2);                   // [L+2]
  for (int i = threadIdx.x; i < 3072; i += blockDim.x) W2[i] = rnd<A>(wts[kOffW2 + i]);
  const int c0 = blockIdx.x * cpb, nc = min(cpb, ncol - c0);
  const int64_t C = (int64_t)ncol * L;
  float a2[12], a1 = 0.f;                           // thread-owned gW2 slots w = tid + 256 j
#pragma unroll
  for (int j = 0; j < 12; ++j) a2[j] = 0.f;
  for (int cc = 0; cc < nc; ++cc) {
    const int col = c0 + cc;
    __syncthreads();
    for (int i = threadIdx.x; i < kCh * (L + 2); i += blockDim.x) {
      const int ch = i / (L + 2), k = i % (L + 2) - 1;
      const bool in = k >= 0 && k < L;
      g2[i] = in ? ga2[(int64_t)ch * C + (int64_t)col * L + k] : 0.f;
      h1s[i] = in ? to_f<A>(h1[(int64_t)ch * C + (int64_t)col * L + k]) : 0.f;
    }
    for (int i = threadIdx.x; i < L + 2; i += blockDim.x) {
      const int k = i - 1;
      xs[i] = (k >= 0 && k < L) ? rnd<A>(xin[(int64_t)col * L + k]) : 0.f;
    }
    __syncthreads();
    // ga1 = (W2^T conv ga2) [h1 > 0]
    for (int i = threadIdx.x; i < kCh * L; i += blockDim.x) {
      const int ci = i / L, k = i % L;
      float s = 0.f;
      for (int o = 0; o < kCh; ++o) {
        const float *g = g2 + o * (L + 2) + k;     // ga2[o][k-1..k+1]
        const float *w = W2 + o * 96 + 3 * ci;
        s = fmaf(w[0], g[2], fmaf(w[1], g[1], fmaf(w[2], g[0], s)));
      }
      g1[ci * (L + 2) + k + 1] = h1s[ci * (L + 2) + k + 1] > 0.f ? s : 0.f;
    }
    for (int i = threadIdx.x; i < kCh; i += blockDim.x) { g1[i * (L + 2)] = 0.f; g1[i * (L + 2) + L + 1] = 0.f; }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < 12; ++j) {
      const int w = threadIdx.x + 256 * j;        // (o, i, d)
      const int o = w / 96, ci = (w % 96) / 3, d = w % 3;
      float s = a2[j];
      for (int k = 0; k < L; ++k) s = fmaf(g2[o * (L + 2) + k + 1], h1s[ci * (L + 2) + k + d], s);
      a2[j] = s;
    }
    if (threadIdx.x < 96) {
      const int o = threadIdx.x / 3, d = threadIdx.x % 3;
      float s = a1;
      for (int k = 0; k < L; ++k) s = fmaf(g1[o * (L + 2) + k + 1], xs[k + d], s);
      a1 = s;
    }
  }
#pragma unroll
  for (int j = 0; j < 12; ++j) part2[(int64_t)blockIdx.x * 3072 + threadIdx.x + 256 * j] = a2[j];
  if (threadIdx.x < 96) part1[(int64_t)blockIdx.x * 96 + threadIdx.x] = a1;
}

// ---- the training backward of the 32 -> 32 convolution on the tensor cores -----------------------
// BF16 minibatch on patches: h1 [32][C] BF16 and ga2 [32][C] FP32 channel-major, x [C]. Per tile of
// 128 padded rows (R = col (L + 2) + k + 1, rows k = -1 and L empty), two GEMMs on tcgen05.mma:
//   dX: D1[m][i] = sum_{d, o} ga2[o](m + d - 1) W2[o][i][2 - d]   (M 128, N 32, K 96: six MMAs), then
//       ga1 = D1 [h1 > 0] and gW1[i][d] += ga1[m][i] x(m + d - 1) on the CUDA cores;
//   dW: D2[d 32 + i][o] += sum_m h1[i](m + d - 1) ga2[o](m)        (M 128 (96 used), N 32, K = the tile's
//       128 rows: eight MMAs), accumulated in tensor memory over all the CTA's tiles.
// A1 is ga2 on the tile's rows -1 .. 128 in the forward's layout ([8-channel group][row][8 channels]),
// so the three taps are three start addresses a row apart; B1 is W2 transposed and flipped in the
// forward's B layout. A2 ([m / 8][d 32 + i][8 m]) and B2 ([m / 8][o][8 m]) are K-major over the rows.
// ga2 is FP32: it enters as two BF16 parts, hi = bf16(g) and lo = bf16(g - hi), two MMAs into the same
// accumulator, so the products keep about 16 bits (W2 and h1 are BF16 values already).
constexpr int kBwRows = 130;                                  // A1 rows: tile rows -1 .. 128
constexpr int kBwLbo = kBwRows * 16;                          // A1: bytes between 8-channel groups
constexpr int kBwA1 = 4 * kBwLbo;                             // 8,320 B per part
constexpr int kBwB1 = ((2 * kBwA1 + 1023) / 1024) * 1024;     // W2 image (6 KB)
constexpr int kBwA2 = kBwB1 + 6 * 1024;                       // h1 shifted: 16 x 128 x 16 B = 32 KB
constexpr int kBwB2 = kBwA2 + 16 * 128 * 16;                  // ga2 over the rows: 16 x 32 x 16 B = 8 KB per part
constexpr int kBwX = kBwB2 + 2 * 16 * 32 * 16;                // x on rows -1 .. 128 (130 floats)
constexpr int kBwG = kBwX + ((kBwRows * 4 + 15) / 16) * 16;   // ga2 tile, FP32 [32][130]
constexpr int kBwH = kBwG + 32 * kBwRows * 4;                 // h1 tile, BF16 [32][130]
constexpr int kBwCell = kBwH + 32 * kBwRows * 2;              // cell of each row, int32 [130]
constexpr int kBwBar = kBwCell + ((kBwRows * 4 + 15) / 16) * 16;   // mbarrier (8 B), TMEM address (4 B)
constexpr int kBwSmem = kBwBar + 64;
constexpr int kBwRed = kBwA2;                                 // end-of-kernel reduction scratch (reuses A2)

// W2 -> B1[i][kk], kk = d 32 + o, value W2[o][i][2 - d], in the core-matrix order of the forward's B
__global__ void nn_pack_bt_kernel(const float *__restrict__ wts, __nv_bfloat16 *__restrict__ bimg) {
  for (int e = threadIdx.x; e < 32 * 96; e += blockDim.x) {
    const int i = e / 96, kk = e % 96, d = kk / 32, o = kk % 32;
    const int off = ((kk >> 3) * 4 + (i >> 3)) * 64 + (i & 7) * 8 + (kk & 7);   // in elements
    bimg[off] = __float2bfloat16(wts[kOffW2 + (o * 32 + i) * 3 + (2 - d)]);
  }
}

struct BwArgs {
  int ncol, L;
  int64_t C, nrows, ntiles;
};

__device__ __forceinline__ int64_t bw_cell(const BwArgs &a, int64_t R) {   // cell of padded row R, or -1
  if (R < 0 || R >= a.nrows) return -1;
  const int64_t col = R / (a.L + 2);
  const int k = (int)(R - col * (a.L + 2)) - 1;
  return (k >= 0 && k < a.L) ? col * a.L + k : -1;
}

__device__ __forceinline__ uint32_t pack_bf16x2(float a, float b) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<const uint32_t *>(&v);
}

__device__ __forceinline__ void split_bf16(float v, float &hi, float &lo) {
  hi = __bfloat162float(__float2bfloat16(v));
  lo = v - hi;
}

__global__ void __launch_bounds__(128)
    nn_bwd1_tc_kernel(const BwArgs a, const __nv_bfloat16 *__restrict__ bt, const __nv_bfloat16 *__restrict__ h1,
                      const float *__restrict__ ga2, const float *__restrict__ xin, float *__restrict__ part2,
                      float *__restrict__ part1, int *__restrict__ wait_flag) {
  extern __shared__ __align__(1024) unsigned char bw_smem[];
  unsigned char *sA1 = bw_smem, *sB1 = bw_smem + kBwB1, *sA2 = bw_smem + kBwA2, *sB2 = bw_smem + kBwB2;
  float *xs = reinterpret_cast<float *>(bw_smem + kBwX);
  float *Gs = reinterpret_cast<float *>(bw_smem + kBwG);
  __nv_bfloat16 *Hs = reinterpret_cast<__nv_bfloat16 *>(bw_smem + kBwH);
  int *cellr = reinterpret_cast<int *>(bw_smem + kBwCell);
  uint64_t *bar = reinterpret_cast<uint64_t *>(bw_smem + kBwBar);
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bw_smem + kBwBar + 16);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (warp == 0) {   // 64 TMEM columns: D1 at 0, D2 at 32
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 64;" ::"r"(smem_u32(tmem_slot)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  // B1 (the W2 image), and the unused rows 96 .. 127 of A2, once
  for (int e = tid; e < 6 * 1024 / 16; e += blockDim.x)
    reinterpret_cast<uint4 *>(sB1)[e] = reinterpret_cast<const uint4 *>(bt)[e];
  for (int e = tid; e < 16 * 32; e += blockDim.x) {
    const int kg = e / 32, row = 96 + e % 32;
    *reinterpret_cast<uint4 *>(sA2 + kg * 2048 + row * 16) = make_uint4(0u, 0u, 0u, 0u);
  }
  float acc1[96];                   // gW1[i][d] partials of this thread's rows
#pragma unroll
  for (int q = 0; q < 96; ++q) acc1[q] = 0.f;
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  const uint32_t idesc = umma_idesc_bf16(kTcM, 32);
  bool ok = true, first = true;
  uint32_t phase = 0;
  for (int64_t t = blockIdx.x; t < a.ntiles && ok; t += gridDim.x) {
    const int64_t R0 = t * kTcM;
    // the tile's rows R0 - 1 .. R0 + 128 (buffer row r = R - R0 + 1): their cells, then ga2 (FP32),
    // h1 (BF16) and x (BF16-rounded) on them, each value read once from global memory
    for (int r = tid; r < kBwRows; r += blockDim.x) {
      const int64_t cell = bw_cell(a, R0 - 1 + r);
      cellr[r] = (int)cell;
      xs[r] = cell >= 0 ? rnd<__nv_bfloat16>(xin[cell]) : 0.f;
    }
    __syncthreads();
    for (int e = tid; e < 32 * kBwRows; e += blockDim.x) {
      const int ch = e / kBwRows, r = e - ch * kBwRows, cell = cellr[r];
      Gs[e] = cell >= 0 ? ga2[(int64_t)ch * a.C + cell] : 0.f;
      Hs[e] = cell >= 0 ? h1[(int64_t)ch * a.C + cell] : __float2bfloat16(0.f);
    }
    __syncthreads();
    // A1: ga2 on rows -1 .. 128 in the forward's layout, hi and lo parts
    for (int e = tid; e < 4 * kBwRows; e += blockDim.x) {
      const int r = e % kBwRows, g = e / kBwRows;
      uint32_t hw[4], lw[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        float h0, l0, h1v, l1;
        split_bf16(Gs[(8 * g + 2 * q) * kBwRows + r], h0, l0);
        split_bf16(Gs[(8 * g + 2 * q + 1) * kBwRows + r], h1v, l1);
        hw[q] = pack_bf16x2(h0, h1v);
        lw[q] = pack_bf16x2(l0, l1);
      }
      *reinterpret_cast<uint4 *>(sA1 + g * kBwLbo + r * 16) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
      *reinterpret_cast<uint4 *>(sA1 + kBwA1 + g * kBwLbo + r * 16) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
    }
    // A2: h1[i] on rows m + d - 1 (buffer row m + d), row d 32 + i, m = 8 kg .. 8 kg + 7
    for (int e = tid; e < 96 * 16; e += blockDim.x) {
      const int kg = e % 16, row = e / 16, d = row / 32, i = row % 32;
      const __nv_bfloat16 *hr = Hs + i * kBwRows + 8 * kg + d;
      uint32_t w[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) w[q] = pack_bf16x2(__bfloat162float(hr[2 * q]), __bfloat162float(hr[2 * q + 1]));
      *reinterpret_cast<uint4 *>(sA2 + kg * 2048 + row * 16) = make_uint4(w[0], w[1], w[2], w[3]);
    }
    // B2: ga2[o] on rows m (buffer row m + 1), hi and lo parts
    for (int e = tid; e < 32 * 16; e += blockDim.x) {
      const int kg = e % 16, o = e / 16;
      const float *gr = Gs + o * kBwRows + 8 * kg + 1;
      uint32_t hw[4], lw[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        float h0, l0, h1v, l1;
        split_bf16(gr[2 * q], h0, l0);
        split_bf16(gr[2 * q + 1], h1v, l1);
        hw[q] = pack_bf16x2(h0, h1v);
        lw[q] = pack_bf16x2(l0, l1);
      }
      *reinterpret_cast<uint4 *>(sB2 + kg * 512 + o * 16) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
      *reinterpret_cast<uint4 *>(sB2 + 8192 + kg * 512 + o * 16) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // generic writes -> tensor core
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (tid == 0) {
      const uint32_t a1 = smem_u32(sA1), b1 = smem_u32(sB1), a2 = smem_u32(sA2), b2 = smem_u32(sB2);
      for (int part = 0; part < 2; ++part)   // dX: hi, then lo part of ga2
        for (int s6 = 0; s6 < 6; ++s6) {
          const int d = s6 >> 1, h = s6 & 1;
          const uint64_t ad = umma_desc(a1 + part * kBwA1 + 2 * h * kBwLbo + d * 16, kBwLbo, 128);
          const uint64_t bd = umma_desc(b1 + s6 * 2 * 4 * 128, 4 * 128, 128);
          const uint32_t accum = (part | s6) ? 1u : 0u;
          asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                       " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(tmem),
                       "l"(ad), "l"(bd), "r"(idesc), "r"(accum));
        }
      for (int part = 0; part < 2; ++part)   // dW: B = hi, then lo part of ga2
        for (int j = 0; j < 8; ++j) {
          const uint64_t ad = umma_desc(a2 + 2 * j * 2048, 2048, 128);
          const uint64_t bd = umma_desc(b2 + part * 8192 + 2 * j * 512, 512, 128);
          const uint32_t accum = (first && part == 0 && j == 0) ? 0u : 1u;
          asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                       " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(tmem + 32u),
                       "l"(ad), "l"(bd), "r"(idesc), "r"(accum));
        }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar)));
    }
    first = false;
    ok = __syncthreads_and(mbar_wait(bar, phase) ? 1 : 0) != 0;
    if (!ok) {   // the MMAs may still be running: one more bounded wait before anything is freed
      if (tid == 0) {
        atomicExch(wait_flag, 1);
        mbar_wait(bar, phase);
      }
      __syncthreads();
      break;
    }
    phase ^= 1u;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    uint32_t r[32];
    const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16);
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                 "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                   "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
                   "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
                   "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    const int m = warp * 32 + lane;
    if (cellr[m + 1] >= 0) {
      const float x0 = xs[m], x1 = xs[m + 1], x2 = xs[m + 2];   // x(m - 1), x(m), x(m + 1)
#pragma unroll
      for (int i = 0; i < 32; ++i) {
        const float g = __bfloat162float(Hs[i * kBwRows + m + 1]) > 0.f ? __uint_as_float(r[i]) : 0.f;
        acc1[3 * i] = fmaf(g, x0, acc1[3 * i]);
        acc1[3 * i + 1] = fmaf(g, x1, acc1[3 * i + 1]);
        acc1[3 * i + 2] = fmaf(g, x2, acc1[3 * i + 2]);
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();   // the next tile rewrites the operands and D1
  }
  // D2 -> gW2 partials (row d 32 + i, column o), then the gW1 partials reduced over the block
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (ok) {
    uint32_t r[32];
    const uint32_t taddr = tmem + 32u + ((uint32_t)(warp * 32) << 16);
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                 "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                   "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
                   "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
                   "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    const int row = warp * 32 + lane;
    if (row < 96) {
      const int d = row / 32, i = row % 32;
#pragma unroll
      for (int o = 0; o < 32; ++o)
        part2[(int64_t)blockIdx.x * 3072 + (o * 32 + i) * 3 + d] = __uint_as_float(r[o]);
    }
  }
  float *red = reinterpret_cast<float *>(bw_smem + kBwRed);   // [4 warps][96]
#pragma unroll
  for (int q = 0; q < 96; ++q) {
    float v = acc1[q];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    if (lane == 0) red[warp * 96 + q] = v;
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (tid < 96) part1[(int64_t)blockIdx.x * 96 + tid] = (red[tid] + red[96 + tid]) + (red[192 + tid] + red[288 + tid]);
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 64;" ::"r"(tmem));
}

// Sum of per-block partials [nblocks][n] into out[n]: one block per entry, its threads striding the
// partials, then a fixed-order tree (deterministic for a given nblocks).
__global__ void __launch_bounds__(256)
    sum_partials_kernel(const float *__restrict__ part, int nblocks, int n, float *__restrict__ out) {
  const int i = blockIdx.x;
  double s = 0.0;
  for (int b = threadIdx.x; b < nblocks; b += blockDim.x) s += part[(int64_t)b * n + i];
  s = warp_sum(s);
  __shared__ double red[8];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    out[i] = (float)t;
  }
}

__global__ void sum_loss_kernel(const double *__restrict__ part, int n, double *out) {
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += part[i];
  s = warp_sum(s);
  __shared__ double red[32];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    *out = t;
  }
}

// Adam (Kingma & Ba 2015) with bias correction on the FP32 master weights. The scalars that
// depend only on the hyper-parameters and the step (1 - beta, 1 / (1 - beta^t)) come from the
// host in FP64, rounded once: formed in FP32 from a rounded beta2 = 0.999, 1 - beta2^t would
// be off by about 1e-5 relative.
struct AdamScalars {
  float lr, b1, b2, omb1, omb2, bc1, bc2, eps;
};

static AdamScalars adam_scalars(double lr, double b1, double b2, double eps, int t) {
  return AdamScalars{(float)lr, (float)b1, (float)b2, (float)(1.0 - b1), (float)(1.0 - b2),
                     (float)(1.0 / (1.0 - std::pow(b1, (double)t))), (float)(1.0 / (1.0 - std::pow(b2, (double)t))),
                     (float)eps};
}

__global__ void adam_kernel(float *__restrict__ w, const float *__restrict__ g, float *__restrict__ m,
                            float *__restrict__ v, int n, const AdamScalars a) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = fmaf(a.b1, m[i], a.omb1 * gi);
  const float vi = fmaf(a.b2, v[i], a.omb2 * gi * gi);
  m[i] = mi;
  v[i] = vi;
  w[i] -= a.lr * (mi * a.bc1) / (sqrtf(vi * a.bc2) + a.eps);
}

int adam_update(Ctx *c, float *w, const float *g, float *m, float *v, int n, int step, double lr, double b1,
                double b2, double eps) {
  adam_kernel<<<grid_for(n, 256), 256, 0, c->stream>>>(w, g, m, v, n, adam_scalars(lr, b1, b2, eps, step));
  HMG_CUDA(c, cudaGetLastError());
  return HMG_OK;
}

// per-sample ||t_s||^2 of the training targets
__global__ void tnorm_kernel(const float *__restrict__ t, int64_t per_sample, float *__restrict__ out) {
  const int s = blockIdx.x;
  double acc = 0.0;
  for (int64_t i = threadIdx.x; i < per_sample; i += blockDim.x) {
    const double v = t[(int64_t)s * per_sample + i];
    acc += v * v;
  }
  acc = warp_sum(acc);
  __shared__ double red[32];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) a += red[w];
    out[s] = (float)(a > 0.0 ? a : 1.0);
  }
}

// gather patches: out[p][q][k] = src[pair(p)][cols[p][q]][k] for x and t, then both scaled by
// 1 / rms(x patch) (the network is positively homogeneous, so the pair stays consistent)
__global__ void extract_patches_kernel(const float *__restrict__ xs, const float *__restrict__ ts,
                                       int64_t ncell, const int32_t *__restrict__ pair,
                                       const int32_t *__restrict__ cols, int P, int L,
                                       float *__restrict__ xo, float *__restrict__ to) {
  const int p = blockIdx.x;
  const int64_t n = (int64_t)P * L;
  const float *xsrc = xs + (int64_t)pair[p] * ncell, *tsrc = ts + (int64_t)pair[p] * ncell;
  double acc = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    const int q = (int)(i / L), k = (int)(i % L);
    const float v = xsrc[(int64_t)cols[(int64_t)p * P + q] * L + k];
    acc += (double)v * v;
  }
  acc = warp_sum(acc);
  __shared__ double red[32];
  __shared__ float scale;
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) a += red[w];
    const double rms = sqrt(a / (double)n);
    scale = rms > 0.0 ? (float)(1.0 / rms) : 1.f;
  }
  __syncthreads();
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    const int q = (int)(i / L), k = (int)(i % L);
    const int64_t src = (int64_t)cols[(int64_t)p * P + q] * L + k;
    xo[(int64_t)p * n + i] = xsrc[src] * scale;
    to[(int64_t)p * n + i] = tsrc[src] * scale;
  }
}

// gathers the samples order[b0 .. b0+batch) of (x, t, ||t||^2) into contiguous batch buffers
__global__ void gather_samples_kernel(const float *__restrict__ x, const float *__restrict__ t,
                                      const float *__restrict__ tn, const int32_t *__restrict__ order,
                                      int b0, int batch, int64_t per, float *__restrict__ xb,
                                      float *__restrict__ tb, float *__restrict__ tnb) {
  const int q = blockIdx.y;
  const int64_t src = (int64_t)order[b0 + q] * per;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < per; i += (int64_t)gridDim.x * blockDim.x) {
    xb[(int64_t)q * per + i] = x[src + i];
    tb[(int64_t)q * per + i] = t[src + i];
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) tnb[q] = tn[order[b0 + q]];
}

// ---- host side ---------------------------------------------------------------------------------
static int front_smem(int cpb, int L) { return (96 + 3072 + cpb * (L + 2) + cpb * kCh * (L + 2)) * 4; }
static int back_smem(int cpb, int L) { return (96 + 96 + cpb * kCh * (L + 2)) * 4; }
static int mix_smem(int cpb, int L) { return (2 * 36 * 4 + 8 * cpb + cpb * (L + 2) * 36) * 4; }
// diag(H)^-1/2 in FP32 per cell, passed from the tensor-core front kernel to the output layer:
// the activation buffer (sized for 32 FP32 channels) after the 32 BF16 channels of h2
static float *tc_dscale(Ctx *c) {
  return reinterpret_cast<float *>(static_cast<char *>(c->nn_act) + (size_t)64 * c->lv[0].ncell);
}
static int bwd1_smem(int L) { return (3072 + 3 * kCh * (L + 2) + (L + 2)) * 4; }
constexpr int kNnCpb = 4;

// Allows the column-block kernels the dynamic shared memory of their largest use (128 levels).
template <typename A, typename Tin, typename Tout>
static int nn_attrs(Ctx *c) {
  const int big = 200 * 1024;
  HMG_CUDA(c, cudaFuncSetAttribute(nn_front_kernel<A, Tin>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
  HMG_CUDA(c, cudaFuncSetAttribute(nn_back_kernel<A, Tout>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
  return HMG_OK;
}

// TC: the column-local layers on the tensor cores (A must be BF16), else on the CUDA cores.
template <typename A, typename Tin, typename Tout, bool TC>
static int nn_forward_mesh(Ctx *c, const Tin *bbar, Tout *out, const double *dH, const float *dH32) {
  const Level &f = c->lv[0];
  const int L = f.nlev;
  A *h2 = reinterpret_cast<A *>(c->nn_act);
  const unsigned g = (unsigned)((f.ncol + kNnCpb - 1) / kNnCpb);
  if (TC) {
    static_assert(!TC || sizeof(A) == 2, "the tensor-core layers store BF16");
    const int64_t nrows = (int64_t)f.ncol * (L + 2);   // padded rows
    if (nrows > INT32_MAX - 2 * kTcM || 4 * f.ncell >= (int64_t)UINT32_MAX)
      return fail(c, HMG_ERR_INVALID_ARG, "mesh too large for the tensor-core layers");
    nn_front_tc_kernel<Tin><<<grid_for(nrows, kTcM), 128, kTcSmem, c->stream>>>(
        c->nn_w, static_cast<const __nv_bfloat16 *>(c->nn_bimg), bbar, dH, dH32, f.ncol, L,
        reinterpret_cast<__nv_bfloat16 *>(h2), tc_dscale(c), c->state + 3);
  } else {
    nn_front_kernel<A, Tin><<<g, 128, front_smem(kNnCpb, L), c->stream>>>(c->nn_w, bbar, dH, dH32, f.ncol, L,
                                                                          kNnCpb, nullptr, h2);
  }
  Nbrs nb{f.col_nbr, c->nn_diag, 0, 0};
  if (TC) {   // whole columns per block, about 64 cells, four threads per cell
    const int cpb = std::max(1, 64 / L), thr = (4 * cpb * L + 31) / 32 * 32;
    const unsigned gm = (unsigned)((f.ncol + cpb - 1) / cpb);
    nn_mix_out_kernel<Tout><<<gm, thr, mix_smem(cpb, L), c->stream>>>(
        c->nn_w, reinterpret_cast<const __nv_bfloat16 *>(h2), nb, f.ncol, L, cpb, tc_dscale(c), out);
  } else {
    nn_back_kernel<A, Tout><<<g, 128, back_smem(kNnCpb, L), c->stream>>>(
        c->nn_w, h2, nb, f.ncol, L, kNnCpb, dH, dH32, out, nullptr, nullptr, nullptr, 1, 1.f, nullptr, nullptr);
  }
  HMG_CUDA(c, cudaGetLastError());
  return HMG_OK;
}

// The tensor-core layer's B operand from the FP32 weights; run wherever the weights change
// (set, or an optimiser step), so that the forward pass, also when captured in a graph, reads
// an image that matches them.
int nn_pack_weights(Ctx *c) {
  nn_pack_b_kernel<<<1, 256, 0, c->stream>>>(c->nn_w, static_cast<__nv_bfloat16 *>(c->nn_bimg));
  nn_pack_bt_kernel<<<1, 256, 0, c->stream>>>(c->nn_w, static_cast<__nv_bfloat16 *>(c->nn_bimg_t));
  HMG_CUDA(c, cudaGetLastError());
  return HMG_OK;
}

// dPi = D^-1/2 f(D^-1/2 bbar) on the finest mesh, in the preconditioner's precision.
template <typename T>
int learned_coarse(Ctx *c, const T *bbar, T *out) {
  if (!c->nn_w) return fail(c, HMG_ERR_NOT_READY, "no coarse model set");
  const double *dH = nullptr;
  const float *dH32 = nullptr;
  if (sizeof(T) == 8) dH = c->lv[0].H; else dH32 = c->lv[0].H32;   // row 0 of H = its diagonal
  if (c->nn_tc_off)   // a bounded tensor-core wait ran out earlier: BF16 on the CUDA cores
    return nn_forward_mesh<__nv_bfloat16, T, T, false>(c, bbar, out, dH, dH32);
  return nn_forward_mesh<__nv_bfloat16, T, T, true>(c, bbar, out, dH, dH32);
}
template int learned_coarse<double>(Ctx *, const double *, double *);
template int learned_coarse<float>(Ctx *, const float *, float *);

int nn_setup(Ctx *c) {
  if (c->nn_w) return HMG_OK;
  const Level &f = c->lv[0];
  if (f.nlev > kMaxL) return fail(c, HMG_ERR_INVALID_ARG, "the network kernels take at most 128 levels");
  int st;
  if ((st = nn_attrs<__nv_bfloat16, double, double>(c))) return st;
  if ((st = nn_attrs<__nv_bfloat16, float, float>(c))) return st;
  if ((st = nn_attrs<float, double, double>(c))) return st;
  if ((st = nn_attrs<float, float, float>(c))) return st;
  HMG_CUDA(c, cudaFuncSetAttribute(nn_bwd1_kernel<__nv_bfloat16>, cudaFuncAttributeMaxDynamicSharedMemorySize, 100 * 1024));
  HMG_CUDA(c, cudaFuncSetAttribute(nn_front_tc_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmem));
  HMG_CUDA(c, cudaFuncSetAttribute(nn_front_tc_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmem));
  HMG_CUDA(c, cudaFuncSetAttribute(nn_front_tc_kernel<float, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   kTcSmem));
  HMG_CUDA(c, cudaFuncSetAttribute(nn_bwd1_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kBwSmem));
  HMG_CUDA(c, cudaFuncSetAttribute(nn_bwd1_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, 100 * 1024));
  if ((st = dev_alloc(c, &c->nn_w, kNParams))) return st;
  {
    __nv_bfloat16 *bimg;
    if ((st = dev_alloc(c, &bimg, (size_t)32 * 96))) return st;   // cudaMalloc: 256-B aligned
    c->nn_bimg = bimg;
    if ((st = dev_alloc(c, &bimg, (size_t)32 * 96))) return st;
    c->nn_bimg_t = bimg;
  }
  float *tmp;
  if ((st = dev_alloc(c, &tmp, (size_t)kCh * f.ncell))) return st;   // BF16 h2 fits in half
  c->nn_act = tmp;
  // corner neighbours: across face f to n, then across the face of n after the shared one
  std::vector<int32_t> nbr(4 * (size_t)f.ncol), nbf(4 * (size_t)f.ncol), diag(4 * (size_t)f.ncol);
  HMG_CUDA(c, cudaMemcpy(nbr.data(), f.col_nbr, nbr.size() * 4, cudaMemcpyDeviceToHost));
  HMG_CUDA(c, cudaMemcpy(nbf.data(), f.col_nbr_face, nbf.size() * 4, cudaMemcpyDeviceToHost));
  for (int col = 0; col < f.ncol; ++col)
    for (int s = 0; s < 4; ++s) {
      const int n = nbr[4 * col + s], g = (nbf[4 * col + s] + 1) & 3;
      diag[4 * col + s] = nbr[4 * n + g];
    }
  if ((st = dev_alloc(c, &c->nn_diag, diag.size()))) return st;
  HMG_CUDA(c, cudaMemcpy(c->nn_diag, diag.data(), diag.size() * 4, cudaMemcpyHostToDevice));
  return HMG_OK;
}

// One training batch on patches: forward, loss, backward into grad [kNParams] (FP32).
template <typename A>
static int nn_batch_grad(Ctx *c, const float *x, const float *t, const float *tn, int nsamp, int nx, int ny,
                         int L, float *grad, double *loss_dev) {
  TrainBufs &tb = c->train;
  const int P = nx * ny, ncol = nsamp * P;
  const int64_t C = (int64_t)ncol * L;
  if (C > tb.cap_cells) return fail(c, HMG_ERR_INVALID_ARG, "training batch larger than the buffers");
  A *h1 = reinterpret_cast<A *>(tb.h1), *h2 = reinterpret_cast<A *>(tb.h2), *h3 = reinterpret_cast<A *>(tb.h3);
  const unsigned g = (unsigned)((ncol + kNnCpb - 1) / kNnCpb);
  Nbrs nb{nullptr, nullptr, nx, ny};
  if (sizeof(A) == 2) {   // BF16 storage: the column-local layers on the tensor cores, h1 kept
    const int64_t nrows = (int64_t)ncol * (L + 2);
    if (nrows > INT32_MAX - 2 * kTcM) return fail(c, HMG_ERR_INVALID_ARG, "training batch too large");
    nn_front_tc_kernel<float, true><<<grid_for(nrows, kTcM), 128, kTcSmem, c->stream>>>(
        c->nn_w, static_cast<const __nv_bfloat16 *>(c->nn_bimg), x, nullptr, nullptr, ncol, L,
        reinterpret_cast<__nv_bfloat16 *>(h2), nullptr, c->state + 3, reinterpret_cast<__nv_bfloat16 *>(h1));
  } else {
    nn_front_kernel<A, float><<<g, 128, front_smem(kNnCpb, L), c->stream>>>(c->nn_w, x, nullptr, nullptr, ncol, L,
                                                                            kNnCpb, h1, h2);
  }
  nn_back_kernel<A, float><<<g, 128, back_smem(kNnCpb, L), c->stream>>>(
      c->nn_w, h2, nb, ncol, L, kNnCpb, nullptr, nullptr, nullptr, h3, t, tn, P, 1.f / (float)nsamp, tb.gy,
      tb.loss_part);
  sum_loss_kernel<<<1, 256, 0, c->stream>>>(tb.loss_part, (int)g, loss_dev);
  nn_bwd3_kernel<A><<<g, 128, (96 + kNnCpb * (L + 2) + 96) * 4, c->stream>>>(c->nn_w, h3, tb.gy, ncol, L, kNnCpb,
                                                                             tb.ga3, tb.part3);
  const int64_t g2max = (int64_t)2 * c->num_sms, g2need = (C + 127) / 128;   // partial rows: at most 2 per SM
  const unsigned g2 = (unsigned)(g2need < g2max ? g2need : g2max);
  nn_bwd2_kernel<A><<<dim3(g2, kCh / kBw2Ch), 128, 0, c->stream>>>(c->nn_w, h2, tb.ga3, nb, ncol, L, tb.ga2,
                                                                   tb.partM);
  unsigned g1;
  if (sizeof(A) == 2) {   // BF16 storage: the 32 -> 32 convolution's dX and dW on the tensor cores
    BwArgs ba;
    ba.ncol = ncol;
    ba.L = L;
    ba.C = C;
    ba.nrows = (int64_t)ncol * (L + 2);
    ba.ntiles = (ba.nrows + kTcM - 1) / kTcM;
    const int64_t gmax = (int64_t)2 * c->num_sms;
    g1 = (unsigned)(ba.ntiles < gmax ? ba.ntiles : gmax);
    nn_bwd1_tc_kernel<<<g1, 128, kBwSmem, c->stream>>>(ba, static_cast<const __nv_bfloat16 *>(c->nn_bimg_t),
                                                        reinterpret_cast<const __nv_bfloat16 *>(h1), tb.ga2, x,
                                                        tb.part2, tb.part1, c->state + 3);
  } else {
    const int cpb1 = 64;
    g1 = (unsigned)((ncol + cpb1 - 1) / cpb1);
    nn_bwd1_kernel<A><<<g1, 256, bwd1_smem(L), c->stream>>>(c->nn_w, h1, tb.ga2, x, ncol, L, cpb1, tb.part2,
                                                            tb.part1);
  }
  sum_partials_kernel<<<96, 256, 0, c->stream>>>(tb.part1, (int)g1, 96, grad + kOffW1);
  sum_partials_kernel<<<3072, 256, 0, c->stream>>>(tb.part2, (int)g1, 3072, grad + kOffW2);
  sum_partials_kernel<<<96, 256, 0, c->stream>>>(tb.partM, (int)g2, 96, grad + kOffM);
  sum_partials_kernel<<<96, 256, 0, c->stream>>>(tb.part3, (int)g, 96, grad + kOffW3);
  HMG_CUDA(c, cudaGetLastError());
  return HMG_OK;
}

// Per-block partial-sum rows a minibatch of `ncol` columns needs: the column-block kernels' blocks
// and the tensor-core backward's grid (at most two CTAs per SM).
static int partial_blocks(const Ctx *c, int ncol) {
  const int cb = (ncol + kNnCpb - 1) / kNnCpb + 1;
  return cb > 2 * c->num_sms ? cb : 2 * c->num_sms;
}

int train_buffers(Ctx *c, int64_t cells, int nblocks_max) {
  TrainBufs &tb = c->train;
  int st;
  if (tb.cap_cells < cells) {
    void **acts[] = {&tb.h1, &tb.h2, &tb.h3};
    for (void **a : acts) {   // storage for FP32 activations (BF16 uses half of it)
      dev_free(c, *a);
      float *f;
      if ((st = dev_alloc(c, &f, (size_t)kCh * cells))) return st;
      *a = f;
    }
    float **grads[] = {&tb.ga3, &tb.ga2};
    for (float **g : grads) {
      dev_free(c, *g);
      if ((st = dev_alloc(c, g, (size_t)kCh * cells))) return st;
    }
    dev_free(c, tb.gy);
    if ((st = dev_alloc(c, &tb.gy, (size_t)cells))) return st;
    tb.cap_cells = cells;
  }
  if (tb.cap_blocks < nblocks_max) {
    dev_free(c, tb.loss_part);
    if ((st = dev_alloc(c, &tb.loss_part, (size_t)nblocks_max))) return st;
    float **parts[] = {&tb.part3, &tb.partM, &tb.part1};
    for (float **q : parts) {
      dev_free(c, *q);
      if ((st = dev_alloc(c, q, (size_t)nblocks_max * 96))) return st;
    }
    dev_free(c, tb.part2);
    if ((st = dev_alloc(c, &tb.part2, (size_t)nblocks_max * 3072))) return st;
    tb.cap_blocks = nblocks_max;
  }
  if (!tb.grad) {
    if ((st = dev_alloc(c, &tb.grad, (size_t)kNParams))) return st;
    if ((st = dev_alloc(c, &tb.m, (size_t)kNParams))) return st;
    if ((st = dev_alloc(c, &tb.v, (size_t)kNParams))) return st;
    if ((st = dev_alloc(c, &tb.loss, 1))) return st;
  }
  return HMG_OK;
}

int coarse_model_grad(Ctx *c, const float *x, const float *t, int nsamp, int nx, int ny, int fp32,
                      float *grad_host, double *loss_host) {
  const int L = c->lv[0].nlev;
  const int64_t cells = (int64_t)nsamp * nx * ny * L;
  int st;
  if ((st = nn_setup(c))) return st;
  if ((st = train_buffers(c, cells, partial_blocks(c, nsamp * nx * ny)))) return st;
  if ((st = dev_grow(c, &c->train.tn, &c->train.cap_tn, (size_t)nsamp))) return st;
  float *tn = c->train.tn;
  tnorm_kernel<<<nsamp, 256, 0, c->stream>>>(t, (int64_t)nx * ny * L, tn);
  if (fp32) st = nn_batch_grad<float>(c, x, t, tn, nsamp, nx, ny, L, c->train.grad, c->train.loss);
  else st = nn_batch_grad<__nv_bfloat16>(c, x, t, tn, nsamp, nx, ny, L, c->train.grad, c->train.loss);
  if (st) return st;
  HMG_CUDA(c, cudaMemcpyAsync(grad_host, c->train.grad, sizeof(float) * kNParams, cudaMemcpyDeviceToHost, c->stream));
  HMG_CUDA(c, cudaMemcpyAsync(loss_host, c->train.loss, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  HMG_CUDA(c, cudaStreamSynchronize(c->stream));
  *loss_host /= nsamp;   // the kernels sum the per-sample losses; the gradient is of the mean
  return HMG_OK;
}

// SplitMix64 (Steele, Lea & Flood 2014) for the epoch shuffles of the training samples.
static uint64_t splitmix64_next(uint64_t &s) {
  uint64_t z = (s += 0x9E3779B97F4A7C15ULL);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

int train_coarse_model(Ctx *c, const float *x, const float *t, int nsamp, int nx, int ny, int batch, int epochs,
                       double lr, uint64_t seed, double *loss_hist) {
  const int L = c->lv[0].nlev, P = nx * ny;
  const int64_t per = (int64_t)P * L;
  int st;
  if ((st = nn_setup(c))) return st;
  if (batch < 1 || batch > nsamp) return fail(c, HMG_ERR_INVALID_ARG, "bad batch size");
  if ((st = train_buffers(c, (int64_t)batch * per, partial_blocks(c, batch * P)))) return st;
  TrainBufs &T = c->train;
  if ((st = dev_grow(c, &T.tn, &T.cap_tn, (size_t)nsamp))) return st;
  if ((st = dev_grow(c, &T.order, &T.cap_order, (size_t)nsamp))) return st;
  if ((st = dev_grow(c, &T.xb, &T.cap_xb, (size_t)batch * per))) return st;
  if ((st = dev_grow(c, &T.tb, &T.cap_tb, (size_t)batch * per))) return st;
  if ((st = dev_grow(c, &T.tnb, &T.cap_tnb, (size_t)batch))) return st;
  float *tn_all = T.tn, *xb = T.xb, *tb_ = T.tb, *tnb = T.tnb;
  int32_t *order_dev = T.order;
  tnorm_kernel<<<nsamp, 256, 0, c->stream>>>(t, per, tn_all);
  HMG_CUDA(c, cudaMemsetAsync(c->train.m, 0, sizeof(float) * kNParams, c->stream));
  HMG_CUDA(c, cudaMemsetAsync(c->train.v, 0, sizeof(float) * kNParams, c->stream));
  std::vector<int32_t> order(nsamp);
  uint64_t s = seed;
  int step = 0;
  for (int ep = 0; ep < epochs; ++ep) {
    for (int i = 0; i < nsamp; ++i) order[i] = i;
    for (int i = nsamp - 1; i > 0; --i) {           // Fisher-Yates
      const int j = (int)(splitmix64_next(s) % (uint64_t)(i + 1));
      std::swap(order[i], order[j]);
    }
    HMG_CUDA(c, cudaMemcpyAsync(order_dev, order.data(), sizeof(int32_t) * nsamp, cudaMemcpyHostToDevice, c->stream));
    double ep_loss = 0.0;
    int nb = 0;
    for (int b0 = 0; b0 + batch <= nsamp; b0 += batch) {
      gather_samples_kernel<<<dim3(grid_for(per, 256) < 64 ? grid_for(per, 256) : 64, batch), 256, 0, c->stream>>>(
          x, t, tn_all, order_dev, b0, batch, per, xb, tb_, tnb);
      if ((st = nn_batch_grad<__nv_bfloat16>(c, xb, tb_, tnb, batch, nx, ny, L, c->train.grad, c->train.loss))) return st;
      ++step;
      adam_kernel<<<grid_for(kNParams, 256), 256, 0, c->stream>>>(c->nn_w, c->train.grad, c->train.m, c->train.v,
                                                                  kNParams, adam_scalars(lr, 0.9, 0.999, 1e-8, step));
      if ((st = nn_pack_weights(c))) return st;
      double l = 0.0;
      HMG_CUDA(c, cudaMemcpyAsync(&l, c->train.loss, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
      HMG_CUDA(c, cudaStreamSynchronize(c->stream));
      ep_loss += l / batch;
      ++nb;
    }
    if (loss_hist) loss_hist[ep] = nb ? ep_loss / nb : 0.0;
  }
  HMG_CUDA(c, cudaStreamSynchronize(c->stream));
  return HMG_OK;
}

int extract_patches(Ctx *c, const float *xs, const float *ts, int64_t ncell, const int32_t *pair,
                    const int32_t *cols, int npatch, int P, float *xo, float *to) {
  extract_patches_kernel<<<npatch, 256, 0, c->stream>>>(xs, ts, ncell, pair, cols, P, c->lv[0].nlev, xo, to);
  HMG_CUDA(c, cudaGetLastError());
  HMG_CUDA(c, cudaStreamSynchronize(c->stream));
  return HMG_OK;
}

// Self-test of the bounded wait: one CTA waits on an mbarrier that nothing arrives on, gives up
// after `limit` polls, records that in *flag and returns (the context stays usable).
__global__ void wait_selftest_kernel(uint32_t limit, int *flag) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar)));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  __syncthreads();
  const bool done = mbar_wait(&bar, 0, limit);
  if (!done && threadIdx.x == 0) atomicExch(flag, 1);
}

int wait_selftest(Ctx *c, uint32_t limit) {
  wait_selftest_kernel<<<1, 32, 0, c->stream>>>(limit, c->state + 3);
  HMG_CUDA(c, cudaGetLastError());
  HMG_CUDA(c, cudaStreamSynchronize(c->stream));
  return HMG_OK;
}

int apply_coarse_model(Ctx *c, const double *bbar, double *out, int mode) {
  int st = nn_setup(c);
  if (st) return st;
  if (mode == 1) return nn_forward_mesh<float, double, double, false>(c, bbar, out, c->lv[0].H, nullptr);
  if (mode == 2 || c->nn_tc_off) return nn_forward_mesh<__nv_bfloat16, double, double, false>(c, bbar, out, c->lv[0].H, nullptr);
  return nn_forward_mesh<__nv_bfloat16, double, double, true>(c, bbar, out, c->lv[0].H, nullptr);
}

// ---- training pairs from the solver itself -----------------------------------------------------
// out = v D^(+-1/2) in FP32 (up: D^1/2, else D^-1/2)
__global__ void scale_to_float_kernel(const double *__restrict__ v, const double *__restrict__ diagH, bool up,
                                      float *__restrict__ out, int64_t n) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) out[i] = (float)(up ? v[i] * sqrt(diagH[i]) : v[i] / sqrt(diagH[i]));
}

__global__ void add_kernel(double *__restrict__ x, const double *__restrict__ e, int64_t n) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) x[i] += e[i];
}

// For the current preconditioner call: x = D^-1/2 bbar and t = D^1/2 H^-1 bbar, with H^-1 bbar
// from pressure-multigrid V-cycles iterated until ||bbar - H y|| <= 1e-12 ||bbar|| (at most 80).
int collect_pair(Ctx *c, const double *bbar) {
  if (c->collect_n >= c->collect_max) return HMG_OK;
  const Level &f = c->lv[0];
  const int64_t C = f.ncell;
  int st;
  if (!c->collect_r) {
    if ((st = dev_alloc(c, &c->collect_r, (size_t)C))) return st;
    if ((st = dev_alloc(c, &c->collect_y, (size_t)C))) return st;
  }
  const double *dH = f.H;   // row 0 of H: its diagonal
  scale_to_float_kernel<<<grid_for(C, 256), 256, 0, c->stream>>>(bbar, dH, false, c->collect_x + c->collect_n * C, C);
  HMG_CUDA(c, cudaMemsetAsync(c->collect_y, 0, sizeof(double) * C, c->stream));
  if ((st = launch_dot(c, bbar, bbar, C, 10))) return st;
  double bb = 0.0;
  HMG_CUDA(c, cudaMemcpyAsync(&bb, c->scal + 10, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  HMG_CUDA(c, cudaStreamSynchronize(c->stream));
  for (int it = 0; it < 80 && bb > 0.0; ++it) {
    if ((st = pressure_residual_fp64(c, 0, bbar, c->collect_y, c->collect_r))) return st;
    if ((st = launch_dot(c, c->collect_r, c->collect_r, C, 11))) return st;
    double rr = 0.0;
    HMG_CUDA(c, cudaMemcpyAsync(&rr, c->scal + 11, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    HMG_CUDA(c, cudaStreamSynchronize(c->stream));
    if (rr <= 1e-24 * bb) break;
    double *e = nullptr;
    if ((st = vcycle<double>(c, c->collect_r, &e))) return st;
    add_kernel<<<grid_for(C, 256), 256, 0, c->stream>>>(c->collect_y, e, C);
  }
  scale_to_float_kernel<<<grid_for(C, 256), 256, 0, c->stream>>>(c->collect_y, dH, true, c->collect_t + c->collect_n * C, C);
  HMG_CUDA(c, cudaGetLastError());
  ++c->collect_n;
  return HMG_OK;
}

}  // namespace hmg
