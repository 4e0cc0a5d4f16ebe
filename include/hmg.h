/*
 * hmg.h - C ABI of a GB300 (sm_103a) library for the hybridised non-nested multigrid
 * solve of the lowest-order compatible finite element system of
 *   Betteridge, Cotter, Gibson, Griffith, Melvin, Mueller, "Hybridised multigrid
 *   preconditioners for a compatible finite element dynamical core" (arXiv 2210.11797).
 *
 * One context holds one extruded mesh (with its pressure-multigrid hierarchy), one set of
 * background coefficients, the assembled trace operator S and the preconditioner data.
 * A solve takes the cell residuals (R_u^b, R_Pi) and returns the trace multipliers lambda
 * of S lambda = B_lambda (Eq. hybrid_equation), using BiCGStab preconditioned by the
 * non-nested two-level cycle (Algorithm 2) with one pressure V-cycle (configuration 3c).
 *
 * Conventions shared by every call:
 *  - Status: every call returns an int status (HMG_OK = 0). Nothing aborts; device code
 *    never traps. hmg_last_error() gives a one-line description of the last failure.
 *  - Pointers: "host" pointers are read (or written) during the call only and stay owned
 *    by the caller. "device" pointers are caller-owned CUDA global memory on the
 *    context's device (e.g. torch.Tensor.data_ptr()); work on them is ordered on the
 *    context's stream and the call returns after that work has completed.
 *  - The library allocates device memory in hmg_set_mesh, hmg_set_coefficients and
 *    hmg_assemble_trace only; solve/apply/reconstruct allocate nothing.
 *  - Numbering: cells K = column * nlev + level (level 0 at the ground); local faces
 *    e0..e3 (vertical, along the column corners counter-clockwise seen from above: e0 =
 *    corner0->corner1, e1 = corner1->corner2, e2 = corner2->corner3, e3 = corner3->corner0),
 *    then bottom (4) and top (5). Trace dofs lambda = [lambda^h: edge * nlev + level |
 *    lambda^z: nedge * nlev + column * (nlev + 1) + interface], interfaces 0..nlev.
 *  - All arithmetic of the FP64 path is IEEE double; results agree with a plain CPU
 *    implementation up to rounding order, not bit for bit.
 */
#ifndef HMG_H
#define HMG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------------------ */
#define HMG_OK 0
#define HMG_ERR_INVALID_ARG 1   /* bad size, pointer, table entry or option */
#define HMG_ERR_CUDA 2          /* a CUDA runtime call failed (message in hmg_last_error) */
#define HMG_ERR_NOT_READY 3     /* mesh, coefficients or assembly missing */
#define HMG_ERR_NOT_CONVERGED 4 /* max_iter reached or divergence detected */
#define HMG_ERR_BREAKDOWN 5     /* BiCGStab breakdown: (rhat, v) = 0 or (t, t) = 0 */
#define HMG_ERR_NONFINITE 6     /* NaN or Inf in the iteration */
#define HMG_ERR_TIMEOUT 7       /* a bounded device-side wait expired */
#define HMG_ERR_OUT_OF_MEMORY 8 /* device allocation failed */

typedef struct hmg_ctx hmg_ctx; /* opaque, owned by the library */

/* ---- inputs ------------------------------------------------------------------------ */

/* One level of the extruded mesh (finest first). All pointers are host pointers, copied
 * by hmg_set_mesh. The geometry follows Sec. 2.2 (hexahedral cells of an extruded mesh,
 * here with trilinear cells between the level heights). */
typedef struct {
  int32_t geometry;          /* 0: planar, corners are (x, y, 0); 1: sphere, corners are
                                unit vectors and a vertex at height z is corner*(radius+z) */
  int32_t ncol, nlev, nedge; /* columns, layers (1..2045), vertical edges (faces between columns) */
  double radius;             /* sphere radius (geometry 1) */
  const double *corners;     /* [ncol][4][3] column corners, counter-clockwise from above */
  const double *z_levels;    /* [nlev+1] level heights, strictly increasing */
  const int32_t *col_edges;  /* [ncol][4] edge of local face e0..e3 */
  const int32_t *edge_cols;  /* [nedge][2] the two columns; the first is the edge's owner */
  const int8_t *edge_face;   /* [nedge][2] local face index (0..3) in each column */
  const int32_t *parent;     /* [ncol] column of the next coarser level containing this one
                                (2x2 agglomeration); NULL on the coarsest level */
} hmg_mesh_level;

/* Background reference state of one multigrid level (Sec. 2.1-2.2): theta* and the
 * W_theta projection of Exner* at level heights, Exner* at cell centres. Host pointers. */
typedef struct {
  const double *theta_lev; /* [ncol][nlev+1] */
  const double *exner_lev; /* [ncol][nlev+1] */
  const double *exner;     /* [ncol][nlev]   */
} hmg_background;

/* Scalars of Eqs. gh-u .. gh-pi. preset 0: the physical operator with theta elimination
 * (Eq. 2x2system); preset 1: the constant-coefficient Helmholtz operator with
 * G_K = -1, B_K = 1, K_K = I and M3^Pi = sigma |K| (no buoyancy terms). */
typedef struct {
  double dt, tau_u, tau_rho, tau_theta, cp, kappa;
  int32_t preset;
  double sigma;
  double omega;  /* rotation rate (rad/s) of the Coriolis term 2 Omega x u of Eq. gh-u (preset
                    0), about the z axis of the sphere's Earth-centred frame or the vertical of
                    the plane (an f-plane); 0: no rotation. Makes A_K non-symmetric. */
} hmg_scalars;

/* ---- options ----------------------------------------------------------------------- */
#define HMG_PRECISION_FP64 0   /* everything in FP64 */
#define HMG_PRECISION_MIXED 1  /* preconditioner in FP32, Krylov and S apply in FP64 */
#define HMG_PRECOND_NONE 0
#define HMG_PRECOND_LINESMOOTH 1 /* configuration 2: Algorithm 1 from zero, n_smooth sweeps */
#define HMG_PRECOND_NONNESTED 2  /* configuration 3c: Algorithm 2 with one pressure V-cycle */
#define HMG_PRECOND_SCHUR 3      /* configuration 1: the unhybridised 2x2 system (Eq. 2x2system)
                                    with the approximate Schur complement (Sec. 2.3); solved by
                                    hmg_solve_mixed; set before hmg_assemble_trace; FP64 */

typedef struct {
  int32_t precision;    /* HMG_PRECISION_* */
  int32_t precond;      /* HMG_PRECOND_* */
  int32_t n_pre, n_post; /* trace smoother sweeps around the coarse correction (1, 2) */
  int32_t n_smooth;     /* sweeps of the single-level preconditioner (1) */
  double omega;         /* trace smoother relaxation (0.6) */
  int32_t mg_npre, mg_npost, mg_ncoarse; /* pressure MG sweeps (1, 2, 3 on the coarsest) */
  double mg_omega;      /* pressure block-Jacobi relaxation (0.9) */
  double tol;           /* relative residual ||B - S lambda|| / ||B|| to stop (1e-6) */
  int32_t max_iter;     /* BiCGStab iterations (200) */
  double divergence;    /* stop with NOT_CONVERGED if ||r|| > divergence * ||B|| (1e8; BiCGStab on
                           the 2x2 system of configuration 1 passes through residuals of 5e3
                           ||B|| on its way to convergence) */
  int32_t profile;      /* 1: time every solver component with CUDA events (see
                           hmg_solve_stats.comp_ms); 0: no events (default) */
  int32_t graph;        /* 1 (default): the whole solve is one CUDA graph whose BiCGStab loop
                           is a device-side WHILE node (no host round trip per iteration);
                           0: the host drives the loop (always so when profile = 1) */
  int32_t coarse;       /* coarse solve of Algorithm 2 line 6: HMG_COARSE_* */
  int32_t krylov;       /* HMG_KRYLOV_BICGSTAB (default) or HMG_KRYLOV_FGMRES */
  int32_t restart;      /* FGMRES restart length (30) */
  double stall_ratio;   /* FGMRES with a learned coarse solve falls back to the V-cycle for the
                           rest of the solve after two consecutive steps that each reduce the
                           residual estimate by less than this factor (0.9) */
  int32_t mg_fused;     /* 0 (default): one launch per smoothing sweep, restriction and
                           injection; 1: the coarse levels (all but the finest) of each V-cycle
                           run as one cooperative launch with grid-wide barriers (same
                           arithmetic, bitwise the same result; slower inside the solve's
                           CUDA graph on GB300, where launches cost little) */
  int32_t warm_start;   /* 0 (default, the paper): the Krylov iteration starts from zero;
                           1: from the lambda (hmg_solve) or [u | Pi] (hmg_solve_mixed, its
                           internal copy of the last solution) passed in, r_0 = B - S lambda_0
                           (resuming a solve, or a previous time step's solution) */
  int32_t mg_fuse_cells; /* coarse levels of at most this many cells (default 262144) run the
                           restriction inside their first sweep and the injection inside their
                           first post-sweep, one launch instead of two (same arithmetic,
                           bitwise the same result); 0: never. Must be >= 0 */
  int32_t async_stats;  /* 0 (default): hmg_solve synchronises once, to fill its stats.
                           1: a graph-launched BiCGStab solve (graph = 1, profile = 0, no
                           Krylov coarse solve) is only enqueued on the context's stream;
                           hmg_solve returns HMG_OK at once with stats->status set to
                           HMG_ERR_NOT_READY (nothing else filled), and hmg_solve_stats_get
                           gives the stats and the stop reason later.
                           Host-driven and FGMRES solves, hmg_solve_host, hmg_solve_mixed
                           and batched solves stay synchronous */
  int32_t degree;       /* polynomial degree p of the discretisation (Sec. 2.2; the paper's runs and
                           the default: 0, broken RT0 / DG0 / one trace unknown per facet).
                           p = 1, 2, 3: broken RT_p (3 (p+1)^2 (p+2) dofs per cell, 6 (p+1)^2 of
                           them on the facets), DG_p ((p+1)^3) and Q_p trace multipliers
                           ((p+1)^2 per facet): mixed cell matrices of 44 x 44, 135 x 135 and
                           304 x 304 condensed to 24 x 24, 54 x 54 and 96 x 96 (the paper's table
                           of unknowns per cell), for the Helmholtz preset (hmg_scalars.preset =
                           1), with Algorithm 1 on facet blocks and Algorithm 2 on the DG0 coarse
                           space and the lowest-order pressure multigrid; with precision mixed the
                           preconditioner (S, smoother factors, Gamma, V-cycle) runs in FP32 and
                           the Krylov method, its S apply and residuals in FP64. Set before
                           hmg_assemble_trace (a change needs a new assembly; the assembly holds
                           A_K^-1: N^2 doubles per cell, N = 44, 135, 304; HMG_ERR_OUT_OF_MEMORY when the
                           device cannot hold it). With degree p every call that takes cell
                           residuals takes Rub [ncell][3 (p+1)^2 (p+2)] (the cell's RT_p dofs:
                           the outward facet fluxes, face by face e0..e3, bottom, top, node
                           (s, t) at (p+1)^2 f + (p+1) s + t, then the interior dofs component by
                           component) and Rpi [ncell][(p+1)^3] (DG_p, node (i, j, k) at
                           (p+1)^2 i + (p+1) j + k), and lambda has hmg_sizes' ntrace entries:
                           (p+1)^2 per facet, facet by facet in the order of the lowest-order
                           numbering, node (s, t) at + (p+1) s + t (s along a vertical facet in
                           the traversal of the column that owns its edge, t upwards; on a
                           horizontal facet the xi and eta nodes). Batched, mixed-precision,
                           learned, configuration-1 and allocation-free calls stay degree 0 */
} hmg_options;

#define HMG_COARSE_VCYCLE 0         /* one pressure V-cycle (configuration 3c) */
#define HMG_COARSE_LEARNED 1        /* the learned model f ~ H^-1 alone */
#define HMG_COARSE_LEARNED_VCYCLE 2 /* the model's output as the V-cycle's initial guess */
#define HMG_COARSE_KRYLOV_EXACT 3   /* configuration 3a (Sec. 3.2): H dPi = bbar by BiCGStab
                                       preconditioned with the V-cycle, to 1e-14 (FP64 only;
                                       the host drives the inner loop) */
#define HMG_COARSE_KRYLOV_APPROX 4  /* configuration 3b: the same to 1e-2 */
#define HMG_KRYLOV_BICGSTAB 0
#define HMG_KRYLOV_FGMRES 1

#define HMG_MAX_HISTORY 512
/* Solver components timed when hmg_options.profile = 1 (cf. Table time_in_components):
 * 0 B_lambda (forward substitution), 1 S apply in the Krylov loop (hybridised operator),
 * 2 presmoothing sweep from zero, 3 full line-smoother sweeps (Algorithm 1),
 * 4 trace residual + restriction + Gamma (Algorithm 2 lines 3-5), 5 pressure V-cycle,
 * 6 prolongation (Algorithm 2 line 7), 7 Krylov vector updates and inner products. */
#define HMG_NCOMP 8
typedef struct {
  int32_t status;            /* HMG_OK or the reason the iteration stopped */
  int32_t iterations;        /* completed BiCGStab iterations (FGMRES: steps, i.e.
                                preconditioner applications) */
  double rel_residual;       /* recurrence residual ||r_i|| / ||B|| at exit */
  double true_rel_residual;  /* ||B - S lambda|| / ||B|| recomputed in FP64 at exit */
  double solve_ms;           /* device time of the call (CUDA events on the stream) */
  int32_t n_history;         /* entries of history[] used: ||r_i|| / ||B||, i = 0.. */
  double history[HMG_MAX_HISTORY];
  double comp_ms[HMG_NCOMP]; /* device time per component (profile = 1), else 0 */
  int32_t comp_calls[HMG_NCOMP]; /* kernel launches per component (profile = 1) */
  int32_t coarse_fallback;   /* 1 if a learned coarse solve was replaced by the V-cycle */
} hmg_solve_stats;

/* ---- lifecycle --------------------------------------------------------------------- */

/* Fill *opt with the paper's settings (Sec. 3.2): omega 0.6, 1 pre / 2 post sweeps,
 * pressure MG omega 0.9 with 1 pre / 2 post sweeps, tol 1e-6, FP64, configuration 3c. */
int hmg_default_options(hmg_options *opt);

/* Create a context on the current CUDA device. opt: host, copied (NULL = defaults).
 * cuda_stream: a cudaStream_t owned by the caller (NULL = the legacy default stream). */
int hmg_create(hmg_ctx **out, const hmg_options *opt, void *cuda_stream);

/* Replace the options (e.g. the tolerance or precision) without reassembling. On an assembled
 * context, switching to HMG_PRECISION_MIXED makes the FP32 copies of the operators and factors
 * from the assembled FP64 ones (device memory for them is allocated here, once; synchronises);
 * a change of degree needs hmg_assemble_trace. */
int hmg_set_options(hmg_ctx *ctx, const hmg_options *opt);

/* Set the mesh hierarchy: levels[0] finest ... levels[nmg-1] coarsest; every level has
 * the same nlev, level l+1 has ncol/4 columns and each coarse column exactly four children.
 * Tables are validated (INVALID_ARG on an inconsistent table). Host inputs, copied. */
int hmg_set_mesh(hmg_ctx *ctx, int32_t nmg, const hmg_mesh_level *levels);

/* Set the background (one hmg_background per level, host, copied) and the scalars. */
int hmg_set_coefficients(hmg_ctx *ctx, const hmg_scalars *scalars, const hmg_background *levels);

/* Build everything a solve needs (Eqs. bilinear_forms, hybrid-S, elliptic_pressure_system,
 * scaling_matrix): per cell the 7x7 A_K by 3x3x3 Gauss quadrature, its LU with partial
 * pivoting and inverse, S_K = (A_K^-1)_uu K_K; the rows of S (11 coefficients each); the
 * Thomas factors of S^zz and 1/diag(S^hh); H and the Thomas factors of H_z on every level;
 * Gamma = (H 1) / (P^T S P 1). Allocates the solver workspace. */
int hmg_assemble_trace(hmg_ctx *ctx);

/* Sizes: cells and trace unknowns of the finest level (either pointer may be NULL); with
 * degree p >= 1 (assembled) ntrace counts the (p+1)^2 unknowns of every facet. */
int hmg_sizes(const hmg_ctx *ctx, int64_t *ncell, int64_t *ntrace);

void hmg_destroy(hmg_ctx *ctx);
const char *hmg_status_string(int status);
const char *hmg_last_error(const hmg_ctx *ctx);

/* ---- the solve (device pointers) --------------------------------------------------- */

/* B_lambda = C^T A^-1 R_X (Eq. hybrid-rhs). Rub [ncell][6], Rpi [ncell] in; B [ntrace] out. */
int hmg_trace_rhs(hmg_ctx *ctx, const double *Rub, const double *Rpi, double *B);

/* Solve S lambda = B_lambda(Rub, Rpi) to the context tolerance. lambda [ntrace] device,
 * overwritten (the iteration starts from zero); stats host (may be NULL). Returns the
 * stop reason (HMG_OK when converged). */
int hmg_solve(hmg_ctx *ctx, const double *Rub, const double *Rpi, double *lambda,
              hmg_solve_stats *stats);

/* With async_stats = 1: waits for the last enqueued solve of this context (its end event,
 * not the whole stream), fills stats (host, may be NULL) and returns that solve's stop
 * reason. HMG_ERR_NOT_READY when no asynchronous solve is pending. The results of an
 * enqueued solve live in pinned host buffers of the context: a second hmg_solve before this
 * call replaces them, so only the latest solve's stats can be read. */
int hmg_solve_stats_get(hmg_ctx *ctx, hmg_solve_stats *stats);

/* n independent solves (a batch of contexts, all assembled, on the current device, each with
 * its own mesh and options) in ONE CUDA graph launch: one branch per context, each branch
 * B_lambda -> a device-side WHILE loop of BiCGStab iterations -> the final residual, the
 * branches running concurrently. Rub[i], Rpi[i], lambda[i] are device pointers of context
 * i; stats (host, may be NULL) has n entries. Returns the first non-OK status of any solve
 * (details in that solve's stats). The graph runs on ctxs[0]'s stream. ctxs[0] keeps the
 * instantiated graph and launches it again while the next call passes the same contexts in
 * the same order, the same vector pointers and unchanged options and launch shapes (new
 * values in those vectors are read at launch); any change captures it again. Destroying a
 * context releases the batch graph it holds. */
int hmg_solve_batched(hmg_ctx *const *ctxs, int32_t n, const double *const *Rub,
                      const double *const *Rpi, double *const *lambda, hmg_solve_stats *stats);

/* Time the candidate launch shapes of the line sweep and of the pressure smoother on each
 * level (columns per thread block: 1-64; threads per block: 128 or 256; also one warp per
 * column, up to 128 rows per column: the smoother in both precisions, the sweep in FP32) on this
 * context's mesh and keep the fastest; later launches of this context use them. Needs an assembled context; the sweep
 * timings overwrite the context's work vectors. */
int hmg_autotune(hmg_ctx *ctx);

/* Read / set the launch shapes of a context (host int32 arrays): sweep[2] = {columns per
 * block, threads per block} of the line sweep; mg[2 * nmg] = the same for the pressure
 * smoother on each level. 0 means the default (32 columns, 256 threads, within the shared
 * memory limit); columns -1 selects one warp per column (Thomas recurrences as a warp scan:
 * the same iterate up to rounding order): for a smoother level of at most 128 layers in both
 * precisions, for the sweep (at most 127 layers) in the FP32 preconditioner's kernels only, the
 * FP64 sweep taking the default. hmg_get_launch_shapes reports the shapes of the kernels the
 * preconditioner runs: the FP32 kernels' under precision mixed, else the FP64 kernels';
 * hmg_set_launch_shapes sets both (so the shapes read from a context set the same kernels'
 * shapes on another context of the same mesh and precision; columns -1 come with threads 0,
 * which that form does not use). hmg_set_launch_shapes rejects
 * other columns outside 1..64 and threads other than 0, 128 and 256. */
int hmg_get_launch_shapes(hmg_ctx *ctx, int32_t *sweep, int32_t *mg, int32_t nmg);
int hmg_set_launch_shapes(hmg_ctx *ctx, const int32_t *sweep, const int32_t *mg, int32_t nmg);

/* Configuration 1 (Sec. 2.3, Sec. 3.2): BiCGStab on the unhybridised 2x2 system for the
 * continuous normal velocity u and the Exner increment Pi (Eq. 2x2system), preconditioned by
 * the approximate Schur complement: lumped velocity mass, Step 1 (Eq. pressure_rhs), one
 * pressure-multigrid V-cycle on Eq. elliptic_pressure_system, Step 3 (Eq. velocity_recovery).
 * Needs a context assembled with precond = HMG_PRECOND_SCHUR. Rub, Rpi as for hmg_solve (the
 * continuous residual of facet f is the sum of its cells' oriented broken residuals). u
 * [ntrace] device: the normal velocity per facet in the trace numbering, oriented out of
 * edge_cols[e][0] on vertical facets and upwards on horizontal ones, 0 on ground and lid;
 * pi [ncell] device. The Krylov vectors are [u | Pi]; stats as for hmg_solve. */
int hmg_solve_mixed(hmg_ctx *ctx, const double *Rub, const double *Rpi, double *u, double *pi,
                    hmg_solve_stats *stats);

/* y = (2x2 operator) x on [u | Pi] vectors of ntrace + ncell values (device; configuration 1
 * contexts; ground and lid rows are the identity). */
int hmg_apply_mixed(hmg_ctx *ctx, const double *x, double *y);

/* The same solve with HOST buffers: the inputs are copied to the device, the result back. */
int hmg_solve_host(hmg_ctx *ctx, const double *Rub_host, const double *Rpi_host,
                   double *lambda_host, hmg_solve_stats *stats);

/* X_K = A_K^-1 (R_X - K lambda) per cell (Eq. hybrid-recovery): broken velocity ub
 * [ncell][6] (outward fluxes) and Exner increment pi [ncell]. Device pointers. */
int hmg_reconstruct(hmg_ctx *ctx, const double *lambda, const double *Rub, const double *Rpi,
                    double *ub, double *pi);

/* ---- single steps (device pointers), for tests and benchmarks ----------------------- */

/* y = S x (Eq. hybrid-S), FP64. x, y [ntrace]; x and y must not overlap. */
int hmg_apply_trace(hmg_ctx *ctx, const double *x, double *y);

/* z = M^-1 r: one application of the configured preconditioner (Algorithm 2 for
 * HMG_PRECOND_NONNESTED) in the configured precision. r, z [ntrace] (HMG_PRECOND_SCHUR:
 * [ntrace + ncell], the approximate Schur complement of configuration 1), no overlap. */
int hmg_precond_apply(hmg_ctx *ctx, const double *r, double *z);

/* nsweeps of Algorithm 1 on S lambda = b, updating lambda [ntrace] in place (FP64). */
int hmg_line_smooth(hmg_ctx *ctx, const double *b, double *lambda, int32_t nsweeps);

/* The same sweeps as hmg_line_smooth, for callers that must not allocate device memory at
 * call time: for instance code whose device memory is all handed to another allocator (a
 * framework's caching pool), code with a fixed memory budget decided at start-up, or
 * latency-bound loops that cannot afford cudaMalloc/cudaFree, which synchronise the device.
 * The paper has no counterpart; this is a property of the library, not of the method.
 * The second vector of the ping-pong comes from an 8 MiB array compiled into the library
 * (held by every GPU that loads it until the process exits), so ntrace must be at most
 * 1048576; a larger mesh gets HMG_ERR_INVALID_ARG. The call allocates nothing: no
 * cudaMalloc, cudaFree or allocating library routine. hmg_assemble_trace (set-up, with the
 * context's device current) looks up the array's device address with cudaGetSymbolAddress
 * and keeps it in the context; that lookup also loads the library code holding the array, so
 * the array's memory is taken then, not during a call of this function. The address is as
 * valid as the context's own buffers: after a cudaDeviceReset, destroy the context and build
 * a new one. All calls in the process share the one array and it keeps the last call's
 * contents (nothing in it needs to start at zero), so calls whose GPU work overlaps in time,
 * on any streams or contexts of the same device, race and give wrong results. */
int hmg_line_smooth_noalloc(hmg_ctx *ctx, const double *b, double *lambda, int32_t nsweeps);

/* y = H_l x on multigrid level l (Eq. elliptic_pressure_system), FP64, [ncell_l]. */
int hmg_apply_pressure(hmg_ctx *ctx, int32_t level, const double *x, double *y);

/* x = one pressure-multigrid V-cycle for H_0 x = b from zero (Sec. 2.3), FP64, [ncell]. */
int hmg_pressure_vcycle(hmg_ctx *ctx, const double *b, double *x);

/* Gamma [ncell] of Eq. scaling_matrix (device, FP64). */
int hmg_get_gamma(hmg_ctx *ctx, double *gamma);

/* Copy the assembled S (Eq. hybrid-S) as 11 coefficient slots per trace row, slot-major:
 * slots [11][ntrace] device, FP64. A lambda^h row (edge e joining columns c1, c2 through
 * their local faces i1, i2; level k): slot 0 the diagonal; 1-3 the faces i1+1, i1+2, i1+3
 * (mod 4) of cell (c1, k); 4, 5 its bottom and top; 6-8 the faces i2+1..3 of (c2, k);
 * 9, 10 its bottom and top. A lambda^z row (column c, interface k): slot 0 the diagonal;
 * 1-4 faces e0..e3 of the cell above (c, k); 5 its top; 6-9 faces e0..e3 of the cell
 * below (c, k-1); 10 its bottom. Slots of a missing cell (ground, lid) hold 0. */
int hmg_get_trace_operator(hmg_ctx *ctx, double *slots);

/* ---- learned coarse correction ------------------------------------------------------ */
/* The paper has no learned component. These calls replace (HMG_COARSE_LEARNED) or seed
 * (HMG_COARSE_LEARNED_VCYCLE) the coarse solve H dPi = bbar of Algorithm 2 line 6 with a
 * small network f: dPi = D^-1/2 f(D^-1/2 bbar), D = diag(H_0). f acts per column over the
 * levels (zero padding at ground and lid), bias-free:
 *   h1 = relu(conv(1 -> 32, 3)), h2 = relu(conv(32 -> 32, 3)),
 *   h3 = relu(w_c h2 + w_e * (sum of the 4 edge neighbours) + w_d * (sum of the 4 corner
 *        neighbours)) per channel, y = conv(32 -> 1, 3); conv(a -> b, 3): y[o][k] =
 *   sum_i sum_d W[o][i][d] x[i][k + d - 1].
 * Parameters (FP32, flat): W1 [32][1][3] at 0, W2 [32][32][3] at 96, (w_c, w_e, w_d) [32][3]
 * at 3168, W3 [1][32][3] at 3264; 3360 in all. Inference and training store weights and
 * activations in BF16 and accumulate in FP32 (fp32 = 1 keeps them in FP32, for checks).
 * Use it with HMG_KRYLOV_FGMRES (the map is not linear). Corner neighbours: across local
 * face i to column n, then across the face of n that follows the shared one (mod 4). */

/* Self-test of the bounded device-side waits of the tensor-core kernels: one kernel waits
 * on an mbarrier that nothing arrives on, gives up after `polls` polls (1..2^24), records
 * the expiry in a device flag and returns; the call then reports HMG_ERR_TIMEOUT (the
 * expected result) and leaves the context usable. Anything else is a failure. */
int hmg_check_device_wait(hmg_ctx *ctx, int32_t polls);

/* Number of parameters (3360). */
int32_t hmg_coarse_model_size(void);

/* Set / read the parameters (host arrays of n = hmg_coarse_model_size() floats). Needs the
 * mesh (at most 128 levels); the first call allocates the model's device buffers. */
int hmg_set_coarse_model(hmg_ctx *ctx, const float *params, int32_t n);
int hmg_get_coarse_model(hmg_ctx *ctx, float *params, int32_t n);

/* out = D^-1/2 f(D^-1/2 bbar) on the finest mesh; bbar, out [ncell] device FP64. mode 0: the
 * solver's form, the 32 -> 32 convolution on the tensor cores (tcgen05.mma, BF16 operands,
 * FP32 accumulator in tensor memory); 1: FP32 on the CUDA cores; 2: BF16 storage on the CUDA
 * cores. Returns HMG_ERR_TIMEOUT if a bounded wait for the tensor cores ran out; the output
 * of that call (or of the solve in which it happened) is then undefined, and the context runs
 * the network's column layers in the mode-2 form (BF16 on the CUDA cores) for the rest of its
 * life, in this call's mode 0 and inside solves alike. */
int hmg_apply_coarse_model(hmg_ctx *ctx, const double *bbar, double *out, int32_t mode);

/* Training samples are nx x ny patches of columns (column q = j nx + i of a patch, the
 * regular grid's edge and corner neighbours, zero outside the patch): x, t [nsamp][nx ny]
 * [nlev] device FP32, with t the target of f(x). Loss = mean over the samples of
 * ||f(x_s) - t_s||^2 / ||t_s||^2. hmg_coarse_model_grad writes that loss (host) and its
 * gradient (host, [3360]); hmg_train_coarse_model runs `epochs` passes of Adam
 * (beta 0.9 / 0.999, eps 1e-8, learning rate lr) over minibatches of `batch` samples in an
 * order shuffled per epoch by SplitMix64(seed), updating the model in place, and writes the
 * mean loss of each epoch to loss_hist (host [epochs], may be NULL). */
int hmg_coarse_model_grad(hmg_ctx *ctx, const float *x, const float *t, int32_t nsamp, int32_t nx,
                          int32_t ny, int32_t fp32, float *grad, double *loss);
int hmg_train_coarse_model(hmg_ctx *ctx, const float *x, const float *t, int32_t nsamp, int32_t nx,
                           int32_t ny, int32_t batch, int32_t epochs, double lr, uint64_t seed,
                           double *loss_hist);

/* One step of Adam (Kingma & Ba 2015, with bias correction) on n FP32 values, by the same
 * kernel hmg_train_coarse_model runs after each minibatch: m = beta1 m + (1 - beta1) g,
 * v = beta2 v + (1 - beta2) g^2, w -= lr (m / (1 - beta1^step)) / (sqrt(v / (1 - beta2^step))
 * + eps) in FP32, with 1 - beta1, 1 - beta2 and the two bias corrections 1 / (1 - beta^step)
 * formed on the host in FP64 and rounded once. w, m, v (updated in place) and grad are device arrays of n floats on
 * the context's device; step >= 1 is the step number after this update. For checking the
 * optimiser against a reference (the training itself keeps its moments internally). */
int hmg_adam_step(hmg_ctx *ctx, float *w, const float *grad, float *m, float *v, int32_t n, int32_t step,
                  double lr, double beta1, double beta2, double eps);

/* One solve (FP64, HMG_PRECOND_NONNESTED, host-driven loop) that also records, at each of its
 * first max_pairs preconditioner applications, the pair x = D^-1/2 bbar and
 * t = D^1/2 H^-1 bbar, with H^-1 bbar from pressure V-cycles iterated to a relative residual
 * of 1e-12 (at most 80): x_out, t_out [max_pairs][ncell] device FP32; *n_out = pairs taken. */
int hmg_collect_coarse_pairs(hmg_ctx *ctx, const double *Rub, const double *Rpi, double *lambda,
                             int32_t max_pairs, float *x_out, float *t_out, int32_t *n_out,
                             hmg_solve_stats *stats);

/* Cut training patches out of collected pairs: patch p takes the columns cols[p][0..P) of pair
 * pair[p] (device int32 arrays, checked on the host), scaling x and t by 1 / rms(x patch):
 * xo, to [npatch][P][nlev] device FP32. xs, ts [npairs][ncell]. */
int hmg_extract_patches(hmg_ctx *ctx, const float *xs, const float *ts, int32_t npairs,
                        const int32_t *pair, const int32_t *cols, int32_t npatch, int32_t patch_cols,
                        float *xo, float *to);

#ifdef __cplusplus
}
#endif
#endif /* HMG_H */
