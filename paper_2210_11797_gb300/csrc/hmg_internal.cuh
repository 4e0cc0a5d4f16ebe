// Internal declarations of the hmg library: the context, device tables and kernel
// launchers shared by the translation units. Not part of the public C ABI (include/hmg.h).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "hmg.h"

namespace hmg {

constexpr int kMaxLevels = 8;
constexpr int kSlots = 11;      // coefficients per trace row of S
constexpr int kHCoef = 7;       // coefficients per cell of H: diag, e0..e3, below, above
constexpr int kCellData = 55;   // per-cell assembly record (see CellRec)
constexpr int kRedBlocks = 1216;  // blocks of the grid-stride vector reductions (8 per SM)
constexpr int kMaxRedBlocks = 1 << 18;  // partial-sum slots per reduction (one row per thread)
constexpr int kRedThreads = 256;

// Per-cell record written by the geometry kernel on every multigrid level.
// Offsets into a [ncell][kCellData] array.
struct CellRec {
  static constexpr int M = 0;      // 21 entries: upper triangle of M_K, row-major (f <= g)
  static constexpr int B = 21;     // 6: pressure-row couplings b_K(f)
  static constexpr int KTH = 27;   // 6: k * theta_f (diagonal of K_K; G_K = -KTH)
  static constexpr int MPI = 33;   // 1: M3^Pi
  static constexpr int LUMP = 34;  // 6: this cell's share of the lumped mass of each face
  static constexpr int CORI = 40;  // 15: Coriolis part of M_K (antisymmetric), f < g row-major
};

// Reduction slots of the scalar block kept on the device.
struct Scal {
  static constexpr int RHO0 = 0, RHO1 = 1;  // (rhat, r), double-buffered by iteration parity
  static constexpr int RV = 2;              // (rhat, v)
  static constexpr int TS = 3, TT = 4;      // (t, s), (t, t)
  static constexpr int RR = 5;              // (r, r)
  static constexpr int BB = 6;              // (B, B)
  static constexpr int ALPHA = 7, OMEGA = 8;
  static constexpr int AUX = 9;             // scratch for tests / true residual
  static constexpr int N = 16;
};

// Device-side description of one multigrid level.
struct Level {
  int geometry = 0;
  int ncol = 0, nlev = 0, nedge = 0;
  int64_t ncell = 0, nth = 0, ntz = 0, ntrace = 0;
  double radius = 0.0;
  // mesh tables (device)
  int32_t *col_edges = nullptr;     // [ncol][4]
  int32_t *col_nbr = nullptr;       // [ncol][4] column across local face i
  int32_t *col_nbr_face = nullptr;  // [ncol][4] that column's local face index of the edge
  int32_t *edge_stencil = nullptr;  // [nedge][8] c1, c2, 3 other edges of c1, 3 of c2
  int32_t *edge_fc = nullptr;       // [nedge][2] local face of the edge in c1 and in c2
  int32_t *parent = nullptr;        // [ncol] column on level+1 (not on the coarsest)
  int32_t *children = nullptr;      // [ncol][4] columns on level-1 (not on the finest)
  double *corners = nullptr;        // [ncol][4][3]
  double *z = nullptr;              // [nlev+1]
  double *theta_lev = nullptr, *exner_lev = nullptr, *exner = nullptr;
  // assembled pressure operator (device)
  double *H = nullptr;              // [7][ncell]
  // Thomas factors of H_z with the relaxation mg_omega folded in (pivot p_k): omega / p_k,
  // sub_k / p_k and sup_k / p_k, [ncell] each
  double *Hz_w = nullptr, *Hz_l = nullptr, *Hz_cp = nullptr;
  float *H32 = nullptr, *Hz_w32 = nullptr, *Hz_l32 = nullptr, *Hz_cp32 = nullptr;
  // multigrid work vectors, sized for doubles (used as float in the mixed path)
  void *vb = nullptr, *vx = nullptr, *vy = nullptr;
};

// Work buffers of the coarse-model training (learned.cu), grown on demand and reused.
struct TrainBufs {
  int64_t cap_cells = 0, cap_blocks = 0;
  void *h1 = nullptr, *h2 = nullptr, *h3 = nullptr;   // activations (BF16 or FP32)
  float *ga3 = nullptr, *ga2 = nullptr, *gy = nullptr;
  double *loss_part = nullptr, *loss = nullptr;
  float *part3 = nullptr, *partM = nullptr, *part2 = nullptr, *part1 = nullptr;
  float *grad = nullptr, *m = nullptr, *v = nullptr;
  // per-call data (with their capacities): sample norms, the current minibatch, the epoch order
  float *tn = nullptr, *tnb = nullptr, *xb = nullptr, *tb = nullptr;
  int32_t *order = nullptr;
  size_t cap_tn = 0, cap_tnb = 0, cap_xb = 0, cap_tb = 0, cap_order = 0;
};

// The trace system of degree p = 1, 2, 3 (higher_order.cu), finest level only; NB = (p+1)^2
// rows per facet, NF = 6 NB facet dofs per cell, N = the mixed cell matrix's order.
struct HoData {
  int degree = 0;              // the degree the buffers below are laid out for (0: none)
  int64_t ncell = 0;
  int64_t T = 0;               // trace rows: NB per facet
  double *S = nullptr;         // [2 NF][T] two cells x NF facet-dof coefficients per row
  double *Ainv = nullptr;      // [ncell][N][N] A_K^-1
  double *hw = nullptr;        // [NB^2][vertical facets] omega (facet block of S)^-1
  double *zf = nullptr;        // [horizontal facets][3][NB][NB] block Thomas factors of S^zz (transposed)
  double *gamma = nullptr;     // [ncell] Gamma of Eq. scaling_matrix
  double *m = nullptr;         // [ncell] sigma |K|_1 = (H 1)_K
  int8_t *own = nullptr;       // [ncol][4] 1 where the column owns the edge of its face
  double *tab = nullptr;       // reference-element tables
  int *flag = nullptr;         // singular-matrix flag of the assembly
  double factor_omega = 0.0;   // the omega the smoother factors hold
  // FP32 copies for the FP32 preconditioner (precision mixed): S, the smoother factors, Gamma
  float *S32 = nullptr, *hw32 = nullptr, *zf32 = nullptr, *gamma32 = nullptr;
};

// A process-wide counter: a context takes a new value when it is created and whenever its
// captured launches go stale, so (context address, generation) never names two states.
uint64_t next_graph_gen();

struct Ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  hmg_options opt{};
  hmg_scalars sc{};
  std::string err;
  int nmg = 0;
  Level lv[kMaxLevels];
  bool have_mesh = false, have_coeffs = false, assembled = false, have_fp32 = false;
  int degree = 0;              // polynomial degree of the assembled system (0 .. 3)
  HoData ho;
  // finest-level trace system (device)
  double *S = nullptr;        // [11][ntrace]
  // Thomas factors of S^zz with omega folded in (pivot p_k): omega / p_k, sub_k / p_k,
  // sup_k / p_k, [ntz] each; and omega / diag(S^hh) [nth]
  double *Sz_w = nullptr, *Sz_l = nullptr, *Sz_cp = nullptr, *Sh_w = nullptr;
  double factor_omega = 0.0, factor_mg_omega = 0.0;   // the weights the factors were built with
  double *Ainv = nullptr;     // [49][ncell] A_K^-1, entry (i, j) at (7 i + j) * ncell + K
  double *kth = nullptr;      // [6][ncell] diagonal of K_K (k theta on each local face)
  double *gamma = nullptr;    // [ncell]
  float *S32 = nullptr, *Sz_w32 = nullptr, *Sz_l32 = nullptr, *Sz_cp32 = nullptr, *Sh_w32 = nullptr,
        *gamma32 = nullptr;
  // Krylov workspace (FP64, [ntrace] each)
  double *B = nullptr, *r = nullptr, *rhat = nullptr, *p = nullptr, *v = nullptr,
         *s = nullptr, *t = nullptr, *phat = nullptr, *shat = nullptr;
  // preconditioner workspace, sized for doubles ([ntrace] each)
  void *w1 = nullptr, *w2 = nullptr, *w3 = nullptr;
  void *cb = nullptr;          // restricted, scaled residual [ncell]
  // host-visible buffers for stats and the e2e path
  double *scal = nullptr;      // device [Scal::N]
  double *part = nullptr;      // device [Scal::N][kMaxRedBlocks]
  unsigned int *counter = nullptr;  // device [Scal::N] tickets of the last-block reductions
  double *scal_host = nullptr; // pinned [Scal::N]
  double *host_in = nullptr;   // device staging for hmg_solve_host (Rub | Rpi | lambda)
  // device-side iteration state of the Krylov loop: [0] completed iterations, [1] status,
  // [2] continue flag, [3] set by a kernel whose bounded wait ran out;
  // hist[i] = ||r_i|| / ||B|| (i = 0 .. iterations)
  int *state = nullptr;
  double *hist = nullptr;
  int *state_host = nullptr;   // pinned [4]
  double *hist_host = nullptr; // pinned [HMG_MAX_HISTORY]
  cudaEvent_t as_e0 = nullptr, as_e1 = nullptr;   // start / end of an enqueued (async) solve
  cudaEvent_t loop_done = nullptr;   // recorded by the solve graph when its Krylov loop ends
  cudaEvent_t copy_done = nullptr;   // end of the copy of lambda to the host
  cudaStream_t copy_stream = nullptr;   // that copy, overlapping the final residual
  bool stats_pending = false;  // an async solve's results are on their way to the host
  // whole-solve CUDA graph (B_lambda, a WHILE node over BiCGStab iterations, final residual)
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t graph_exec = nullptr;
  cudaGraph_t graph = nullptr;
  struct GraphKey {
    const void *Rub, *Rpi, *lam;
    hmg_options opt;
  } graph_key{};
  uint64_t graph_gen = next_graph_gen();
  // the batched-solve graph this context holds as the first context of a batch, and what it
  // was captured for: each member's address, generation, vectors and options
  struct BatchMember {
    const void *ctx;
    uint64_t gen;
    const void *Rub, *Rpi, *lam;
    hmg_options opt;
  };
  std::vector<BatchMember> batch_key;
  cudaGraphExec_t batch_exec = nullptr;
  cudaGraph_t batch_graph = nullptr;
  // autotuned launch shapes (0 = default): columns per block of the line sweep and of the
  // pressure smoother on each level
  // launch shapes chosen by autotune, [0] for the FP64 kernels, [1] for the FP32 preconditioner's
  int tune_sweep_cpb[2] = {0, 0}, tune_sweep_threads[2] = {0, 0};
  int tune_mg_cpb[2][kMaxLevels] = {}, tune_mg_threads[2][kMaxLevels] = {};
  // learned coarse correction: FP32 master weights, one activation buffer, corner neighbours
  float *nn_w = nullptr;
  void *nn_act = nullptr;
  int32_t *nn_diag = nullptr;
  void *nn_bimg = nullptr;        // W2 as the BF16 B operand image of the tensor-core layer (6 KB)
  void *nn_bimg_t = nullptr;      // W2 transposed and flipped: the B operand of the training's dX (6 KB)
  TrainBufs train;
  bool coarse_fallback = false;   // set by the flexible Krylov loop when it stalls
  // set when a bounded wait of the tensor-core network layer ran out: from then on the
  // context runs those layers in BF16 on the CUDA cores (same arithmetic up to summation order)
  bool nn_tc_off = false;
  // collection of (scaled bbar, scaled H^-1 bbar) pairs at the preconditioner calls
  float *collect_x = nullptr, *collect_t = nullptr;
  int collect_max = 0, collect_n = 0;
  double *collect_r = nullptr, *collect_e = nullptr, *collect_y = nullptr;
  double *ck = nullptr;           // [9][ncell] work vectors of the Krylov coarse solve
  unsigned int *mg_bar = nullptr; // grid barrier of the cooperative coarse-level kernel
  // device address of the allocation-free sweep's built-in scratch array (trace_ops.cu),
  // looked up once by hmg_assemble_trace
  double *noalloc_scratch = nullptr;
  int num_sms = 0;
  int wave_blocks[3] = {0, 0, 0};   // resident blocks (all SMs) of the BiCGStab vector kernels
  // configuration 1 (mixed.cu): the 2x2 operator (velocity block in the 11-slot layout of S,
  // G couplings [2][ntrace], B couplings and M3^Pi [7][ncell]), 1 / lumped mass [ntrace], the
  // solution [ntrace + ncell] and the Step-1 right-hand side [ncell]
  double *mx_Mu = nullptr, *mx_Gx = nullptr, *mx_Bx = nullptr, *mx_ilump = nullptr, *mx_x = nullptr,
         *mx_bp = nullptr;
  bool have_mixed = false;
  // flexible GMRES basis: V [restart+1][ntrace], Z [restart][ntrace], Hessenberg column
  double *gm_V = nullptr, *gm_Z = nullptr, *gm_h = nullptr, *gm_part = nullptr, *gm_y = nullptr;
  int gm_restart = 0;
  int64_t gm_n = 0;            // length of the basis vectors
  int64_t vec_cap = 0, work_cap = 0, host_cap = 0;   // capacities of the solver workspace (doubles)
  std::vector<void *> owned;   // every device allocation, freed by hmg_destroy
  // component timing (hmg_options.profile): event pool and (component, start, end) marks
  std::vector<cudaEvent_t> ev_pool;
  struct Mark { int comp, e0, e1, launches; };
  std::vector<Mark> marks;
  int ev_next = 0;
};

// Records CUDA events around one solver component when profiling is on (no-op otherwise).
class Prof {
 public:
  Prof(Ctx *c, int comp, int launches = 1);
  ~Prof();
 private:
  Ctx *c_;
  int comp_, e0_ = -1, launches_;
};
enum Comp { kCompRhs = 0, kCompApply, kCompPresmooth, kCompSweep, kCompResidual, kCompVcycle,
            kCompProlong, kCompKrylov };

// ---- error helpers --------------------------------------------------------------------
int fail(Ctx *c, int code, const std::string &msg);
int cuda_fail(Ctx *c, cudaError_t e, const char *what);
#define HMG_CUDA(ctx, call)                                   \
  do {                                                        \
    cudaError_t _e = (call);                                  \
    if (_e != cudaSuccess) return ::hmg::cuda_fail(ctx, _e, #call); \
  } while (0)

template <typename T>
int dev_alloc(Ctx *c, T **p, size_t n) {
  void *q = nullptr;
  cudaError_t e = cudaMalloc(&q, n * sizeof(T) > 0 ? n * sizeof(T) : 16);
  if (e != cudaSuccess) {
    *p = nullptr;
    return fail(c, HMG_ERR_OUT_OF_MEMORY, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  }
  c->owned.push_back(q);
  *p = static_cast<T *>(q);
  return HMG_OK;
}

// Releases one device allocation of the context (and forgets it).
inline void dev_free(Ctx *c, void *p) {
  if (!p) return;
  for (size_t i = 0; i < c->owned.size(); ++i)
    if (c->owned[i] == p) {
      c->owned.erase(c->owned.begin() + (long)i);
      break;
    }
  cudaFree(p);
}

// (Re)allocates *p to hold at least n elements (contents not kept); *cap tracks the size.
template <typename T>
int dev_grow(Ctx *c, T **p, size_t *cap, size_t n) {
  if (*p && *cap >= n) return HMG_OK;
  dev_free(c, *p);
  *p = nullptr;
  *cap = 0;
  const int st = dev_alloc(c, p, n);
  if (!st) *cap = n;
  return st;
}

inline unsigned grid_for(int64_t n, int threads) {
  int64_t g = (n + threads - 1) / threads;
  return static_cast<unsigned>(g > 0 ? g : 1);
}

// ---- assembly (assemble.cu) -----------------------------------------------------------
int assemble_all(Ctx *c);
// (Re)builds the relaxation-weighted Thomas factors for the context's omega and mg_omega.
int build_factors(Ctx *c);
int make_fp32(Ctx *c);   // FP32 copies of the assembled operators and factors (no reassembly)

// ---- trace-space kernels (trace_ops.cu) -----------------------------------------------
// y = S x (FP64). mode 0: plain; 1: also (w, y) -> scal[slot0]; 2: also (y, w) -> slot0 and
// (y, y) -> slot1; 3: y is not stored, (b - S x, b - S x) -> slot0 with w = b.
int launch_spmv(Ctx *c, const double *x, double *y, int mode, const double *w, int slot0,
                int slot1);
int launch_trace_rhs(Ctx *c, const double *Rub, const double *Rpi, double *B);
int launch_reconstruct(Ctx *c, const double *lam, const double *Rub, const double *Rpi,
                       double *ub, double *pi);
// preconditioners: z = M^-1 r, r and z FP64 Krylov vectors
int precond_apply(Ctx *c, const double *r, double *z);
int line_smooth_fp64(Ctx *c, const double *b, double *lam, int nsweeps);
// looks up the device address of the allocation-free sweep's scratch array (set-up)
int noalloc_setup(Ctx *c);
int pressure_vcycle_fp64(Ctx *c, const double *b, double *x);
int apply_pressure_fp64(Ctx *c, int level, const double *x, double *y);

// ---- Krylov (krylov.cu) ------------------------------------------------------------------
// allow_async: with opt.async_stats, a graph-launched solve is only enqueued (stats later
// through solve_stats_get)
// host_out (may be null): lambda is also copied into this host buffer, enqueued right behind
// the solve so that one synchronisation covers the solve, the copy and the stats.
int krylov_solve(Ctx *c, const double *Rub, const double *Rpi, double *lambda,
                 hmg_solve_stats *st, bool allow_async, double *host_out = nullptr);
int solve_stats_get(Ctx *c, hmg_solve_stats *st);
int launch_dot(Ctx *c, const double *a, const double *b, int64_t n, int slot);
// sums the per-block partials of slots s0 (and s1 >= 0) into scal (fixed order)
int launch_finalize(Ctx *c, int nblocks, int s0, int s1);

// ---- configuration 1: the unhybridised 2x2 system (mixed.cu) ------------------------------
int build_mixed(Ctx *c, const double *rec0);
// y = Mx x on [u | Pi] vectors (ntrace + ncell), with the fused products of launch_spmv's modes
int launch_mixed_apply(Ctx *c, const double *x, double *y, int mode, const double *w, int slot0, int slot1);
int launch_mixed_rhs(Ctx *c, const double *Rub, const double *Rpi, double *B);
// z = approximate-Schur preconditioner applied to r (Steps 1-3, one pressure V-cycle)
int schur_precond(Ctx *c, const double *r, double *z);
// the Krylov system of the context's configuration: its length, operator and right-hand side
inline bool mixed_system(const Ctx *c) { return c->opt.precond == HMG_PRECOND_SCHUR; }
inline int64_t sys_n(const Ctx *c) {
  if (c->degree >= 1) return c->ho.T;
  return c->lv[0].ntrace + (mixed_system(c) ? c->lv[0].ncell : 0);
}
// Batched solves: one CUDA graph with one branch per context (contexts on one device).
int krylov_solve_batched(hmg_ctx *const *ctxs, int n, const double *const *Rub,
                         const double *const *Rpi, double *const *lambda, hmg_solve_stats *st);
// Releases the context's cached solve graph.
void drop_graph(Ctx *c);

// ---- degree p = 1, 2, 3 (higher_order.cu) -----------------------------------------------------
int64_t ho_trace_size(const Ctx *c, int p);                // (p+1)^2 rows per facet
int ho_assemble(Ctx *c);                                   // needs w1, w2 of ho_trace_size doubles
void ho_free(Ctx *c);
int ho_launch_spmv(Ctx *c, const double *x, double *y, int mode, const double *w, int slot0, int slot1);
int ho_trace_rhs(Ctx *c, const double *Ru, const double *Rp, double *B);
int ho_reconstruct(Ctx *c, const double *lam, const double *Ru, const double *Rp, double *u, double *pi);
int ho_precond(Ctx *c, const double *r, double *z);
int ho_line_smooth(Ctx *c, const double *b, double *lam, int nsweeps);
// rebuilds the degree-p smoother factors when omega changed since they were built, and makes the
// FP32 preconditioner's copies when the precision is mixed (synchronises)
int ho_refactor_if_needed(Ctx *c);
// cell residual sizes of degree p: 3 (p+1)^2 (p+2) velocity and (p+1)^3 pressure dofs per cell
// (6 and 1 at the lowest order)
inline int cell_nu_of(int p) { return 3 * (p + 1) * (p + 1) * (p + 2); }
inline int cell_np_of(int p) { return (p + 1) * (p + 1) * (p + 1); }
inline int cell_nu(const Ctx *c) { return cell_nu_of(c->degree); }
inline int cell_np(const Ctx *c) { return cell_np_of(c->degree); }

// ---- learned coarse correction (learned.cu) ---------------------------------------------
constexpr int kCoarseParams = 3360;
int nn_setup(Ctx *c);
int nn_pack_weights(Ctx *c);
template <typename T>
int learned_coarse(Ctx *c, const T *bbar, T *out);
// mode 0: BF16 on the tensor cores (the solver's form); 1: FP32 and 2: BF16 on the CUDA cores
int apply_coarse_model(Ctx *c, const double *bbar, double *out, int mode);
int coarse_model_grad(Ctx *c, const float *x, const float *t, int nsamp, int nx, int ny, int fp32,
                      float *grad_host, double *loss_host);
int train_coarse_model(Ctx *c, const float *x, const float *t, int nsamp, int nx, int ny, int batch,
                       int epochs, double lr, uint64_t seed, double *loss_hist);
// one Adam step (the training's own kernel) on n FP32 weights: w, m, v updated in place
int adam_update(Ctx *c, float *w, const float *g, float *m, float *v, int n, int step, double lr, double b1,
                double b2, double eps);
int extract_patches(Ctx *c, const float *xs, const float *ts, int64_t ncell, const int32_t *pair,
                    const int32_t *cols, int npatch, int P, float *xo, float *to);
// launches a kernel whose bounded mbarrier wait must run out (sets state[3])
int wait_selftest(Ctx *c, uint32_t limit);
// records (D^-1/2 bbar, D^1/2 H^-1 bbar) for the current preconditioner call (FP64 path)
int collect_pair(Ctx *c, const double *bbar);
// r = b - H_l x (FP64) on level l
int pressure_residual_fp64(Ctx *c, int level, const double *b, const double *x, double *r);
// kernel launches of one V-cycle (for the component timers)
int vcycle_launches(const Ctx *c);
// x = H_0^-1 b by V-cycle-preconditioned BiCGStab to tol (configurations 3a / 3b), host-driven
int coarse_krylov(Ctx *c, const double *b, double *x, double tol, int maxit);
// flexible GMRES(restart) driver (krylov.cu)
int fgmres_solve(Ctx *c, const double *Rub, const double *Rpi, double *lambda, hmg_solve_stats *st);
// Launch-shape autotuning of one context (columns per block of the sweep and MG smoother).
int autotune(Ctx *c);
// Sweep / smoother launches with explicit columns and threads per block (autotuner).
int time_sweep_cpb(Ctx *c, int cpb, int threads, int fp32, float *ms);
int time_mg_cpb(Ctx *c, int level, int cpb, int threads, int fp32, float *ms);
// Best-of-three average time of one whole V-cycle (FP64 or FP32) with the current shapes.
int time_vcycle(Ctx *c, int fp32, float *ms);
// Columns per block of the pressure smoother: at most 64, and its three shared-memory arrays
// (column stride nlev rounded up to odd) within the default 48 KB (FP64).
// layers per column: a one-column block's three shared-memory arrays of the line sweep
// (3 x ((L + 1) | 1) doubles) stay within the default 48 KB of dynamic shared memory
constexpr int kMaxLayers = 2045;

inline int mg_cpb_limit(int nlev) {
  const int m = 2048 / (nlev | 1);
  return m < 1 ? 1 : (m > 64 ? 64 : m);
}

}  // namespace hmg

// The opaque handle of the C ABI is the internal context.
struct hmg_ctx : public hmg::Ctx {};
