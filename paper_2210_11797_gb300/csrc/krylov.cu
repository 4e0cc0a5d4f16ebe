// Outer Krylov iteration on S lambda = B_lambda: right-preconditioned BiCGStab
// (van der Vorst 1992; Saad 2003 Alg. 7.7 with x = M^-1 y) from lambda = 0, stopping when
// the recurrence residual satisfies ||r_i|| <= tol ||B_lambda|| (Sec. 3.1 of arXiv
// 2210.11797: BiCGStab reducing the residual two-norm by the tolerance).
//
// Everything the loop decides lives on the device: the inner products are deterministic
// reductions into ctx->scal, the vector kernels compute alpha, beta and omega from them,
// and a check kernel appends ||r_i|| / ||B|| to a history array and decides whether to go
// on. With hmg_options.graph the whole solve is one CUDA graph in which a WHILE conditional
// node repeats the iteration body until the check kernel clears its condition, so a solve
// costs one graph launch and one synchronisation. Batched solves put one such branch per
// context into a single graph. With graph = 0 (or profile = 1) the host drives the loop.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <vector>

#include "device_common.cuh"
#include "hmg_internal.cuh"

namespace hmg {

// Two CUDA events around a solve on the context's stream, destroyed on every return path.
struct SolveTimer {
  cudaEvent_t e0 = nullptr, e1 = nullptr, e2 = nullptr;
  ~SolveTimer() {
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (e2) cudaEventDestroy(e2);
  }
  int start(Ctx *c) {
    HMG_CUDA(c, cudaEventCreate(&e0));
    HMG_CUDA(c, cudaEventCreate(&e1));
    HMG_CUDA(c, cudaEventCreate(&e2));
    HMG_CUDA(c, cudaEventRecord(e0, c->stream));
    return HMG_OK;
  }
  int stop(Ctx *c, float *ms) {
    HMG_CUDA(c, cudaEventRecord(e1, c->stream));
    HMG_CUDA(c, cudaEventSynchronize(e1));
    *ms = 0.f;
    cudaEventElapsedTime(ms, e0, e1);
    return HMG_OK;
  }
};

static unsigned red_grid(int64_t n) {
  unsigned g = grid_for(n, kRedThreads);
  return g < (unsigned)kRedBlocks ? g : (unsigned)kRedBlocks;
}

enum { kIt = 0, kStatus = 1, kContinue = 2, kWaitFlag = 3 };

// The system the Krylov loop iterates on: S lambda = B_lambda (hybridised configurations) or
// the 2x2 system on [u | Pi] (configuration 1).
static int sys_apply(Ctx *c, const double *x, double *y, int mode, const double *w, int s0, int s1) {
  if (c->degree >= 1) return ho_launch_spmv(c, x, y, mode, w, s0, s1);
  return mixed_system(c) ? launch_mixed_apply(c, x, y, mode, w, s0, s1) : launch_spmv(c, x, y, mode, w, s0, s1);
}
static int sys_rhs(Ctx *c, const double *Rub, const double *Rpi, double *B) {
  if (c->degree >= 1) return ho_trace_rhs(c, Rub, Rpi, B);
  return mixed_system(c) ? launch_mixed_rhs(c, Rub, Rpi, B) : launch_trace_rhs(c, Rub, Rpi, B);
}

__global__ void __launch_bounds__(kRedThreads)
    dot_kernel(const double *__restrict__ a, const double *__restrict__ b, int64_t n, double *part,
               unsigned int *counter, double *scal, int slot) {
  double s = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    s = fma(a[i], b[i], s);
  const double v[1] = {s};
  const int sl[1] = {slot};
  grid_reduce<1>(v, sl, part, counter, scal);
}

int launch_dot(Ctx *c, const double *a, const double *b, int64_t n, int slot) {
  dot_kernel<<<red_grid(n), kRedThreads, 0, c->stream>>>(a, b, n, c->part, c->counter, c->scal, slot);
  HMG_CUDA(c, cudaGetLastError());
  return HMG_OK;
}

// x = 0, r = rhat = B, p = v = 0
__global__ void bicg_init_kernel(const double *__restrict__ B, double *__restrict__ x,
                                 double *__restrict__ r, double *__restrict__ rhat,
                                 double *__restrict__ p, double *__restrict__ v, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double b = B[i];
    x[i] = 0.0;
    r[i] = b;
    rhat[i] = b;
    p[i] = 0.0;
    v[i] = 0.0;
  }
}

struct LoopParams {
  double tol, divergence;
  int max_iter;
  int warm;   // the iteration starts from the lambda passed in (r_0 = B - S lambda_0)
};

// warm start: r = B - y (y = S x_0 on entry in r), rhat = r, p = v = 0; x is kept
__global__ void bicg_init_warm_kernel(const double *__restrict__ B, double *__restrict__ r,
                                      double *__restrict__ rhat, double *__restrict__ p,
                                      double *__restrict__ v, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double ri = B[i] - r[i];
    r[i] = ri;
    rhat[i] = ri;
    p[i] = 0.0;
    v[i] = 0.0;
  }
}

// rho_0 = (B, B), rho_-1 = alpha = omega = 1; iteration state and history[0]; the loop runs
// while B != 0 is finite, the tolerance is not met and iterations are allowed.
template <bool GRAPH>
__global__ void bicg_start_kernel(double *scal, int *state, double *hist, LoopParams lp,
                                  cudaGraphConditionalHandle handle) {
  const double bb = scal[Scal::BB];
  const double rr0 = lp.warm ? scal[Scal::RR] : bb;   // (rhat, r_0) = ||r_0||^2
  scal[Scal::RHO0] = rr0;
  scal[Scal::RHO1] = 1.0;
  scal[Scal::ALPHA] = 1.0;
  scal[Scal::OMEGA] = 1.0;
  const double rel0 = bb > 0.0 ? sqrt(rr0 / bb) : 0.0;
  int status = isfinite(bb) && isfinite(rr0) ? HMG_OK : HMG_ERR_NONFINITE;
  const bool work = status == HMG_OK && bb > 0.0 && rel0 > lp.tol;
  if (work && lp.max_iter <= 0) status = HMG_ERR_NOT_CONVERGED;
  const int cont = work && lp.max_iter > 0;
  state[kIt] = 0;
  state[kStatus] = status;
  state[kContinue] = cont;
  hist[0] = rel0;
  if (GRAPH) cudaGraphSetConditional(handle, cont);
}

// Vector updates take kVecUnroll grid-stride elements per pass, loads first, so that each
// thread keeps several independent loads in flight (HBM latency x bandwidth).
constexpr int kVecUnroll = 4;
constexpr int kXrUnroll = 2;   // six input vectors: 2 keeps bicg_xr_kernel at 8 blocks per SM

// p = r + beta (p - omega v), beta = (rho_i / rho_{i-1}) (alpha / omega)
__global__ void bicg_p_kernel(const double *__restrict__ r, double *__restrict__ p,
                              const double *__restrict__ v, const double *__restrict__ scal,
                              const int *__restrict__ state, int64_t n) {
  // the coefficients once per block (FP64 divides are long sequences on the narrow FP64 pipe)
  __shared__ double coef[2];
  if (threadIdx.x == 0) {
    const int par = state[kIt] & 1;
    const double rho = scal[par], rho_prev = scal[1 - par];
    const double alpha = scal[Scal::ALPHA], omega = scal[Scal::OMEGA];
    coef[0] = (rho / rho_prev) * (alpha / omega);
    coef[1] = omega;
  }
  __syncthreads();
  const double beta = coef[0], omega = coef[1];
  const int64_t st = (int64_t)gridDim.x * blockDim.x;
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  for (; i + (kVecUnroll - 1) * st < n; i += kVecUnroll * st) {   // all loads of the group first
    double rr[kVecUnroll], pp[kVecUnroll], vv[kVecUnroll];
#pragma unroll
    for (int u = 0; u < kVecUnroll; ++u) {
      rr[u] = r[i + u * st];
      pp[u] = p[i + u * st];
      vv[u] = v[i + u * st];
    }
#pragma unroll
    for (int u = 0; u < kVecUnroll; ++u) p[i + u * st] = fma(beta, fma(-omega, vv[u], pp[u]), rr[u]);
  }
  for (; i < n; i += st) p[i] = fma(beta, fma(-omega, v[i], p[i]), r[i]);
}

// alpha = rho_i / (rhat, v); s = r - alpha v
__global__ void bicg_s_kernel(const double *__restrict__ r, const double *__restrict__ v,
                              double *__restrict__ s, double *scal, const int *__restrict__ state,
                              int64_t n) {
  __shared__ double coef;
  if (threadIdx.x == 0) coef = scal[state[kIt] & 1] / scal[Scal::RV];
  __syncthreads();
  const double alpha = coef;
  const int64_t st = (int64_t)gridDim.x * blockDim.x;
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  for (; i + (kVecUnroll - 1) * st < n; i += kVecUnroll * st) {
    double rr[kVecUnroll], vv[kVecUnroll];
#pragma unroll
    for (int u = 0; u < kVecUnroll; ++u) {
      rr[u] = r[i + u * st];
      vv[u] = v[i + u * st];
    }
#pragma unroll
    for (int u = 0; u < kVecUnroll; ++u) s[i + u * st] = fma(-alpha, vv[u], rr[u]);
  }
  for (; i < n; i += st) s[i] = fma(-alpha, v[i], r[i]);
  if (blockIdx.x == 0 && threadIdx.x == 0) scal[Scal::ALPHA] = alpha;
}

// omega = (t, s) / (t, t); x += alpha phat + omega shat; r = s - omega t;
// (rhat, r) -> scal[1 - par] (rho_{i+1}), (r, r) -> scal[RR]
__global__ void __launch_bounds__(kRedThreads)
    bicg_xr_kernel(double *__restrict__ x, double *__restrict__ r, const double *__restrict__ s,
                   const double *__restrict__ t, const double *__restrict__ phat,
                   const double *__restrict__ shat, const double *__restrict__ rhat, double *scal,
                   double *part, unsigned int *counter, const int *__restrict__ state, int64_t n) {
  const int par = state[kIt] & 1;
  const double alpha = scal[Scal::ALPHA];
  __shared__ double coef;
  if (threadIdx.x == 0) coef = scal[Scal::TS] / scal[Scal::TT];
  __syncthreads();
  const double omega = coef;
  double a0 = 0.0, a1 = 0.0;
  const int64_t st = (int64_t)gridDim.x * blockDim.x;
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  // the partial sums accumulate in the same order (i, i + st, ...) as a plain grid-stride loop
  for (; i + (kXrUnroll - 1) * st < n; i += kXrUnroll * st) {
    double xx[kXrUnroll], sh[kXrUnroll], ph[kXrUnroll], tt[kXrUnroll], ss[kXrUnroll], rh[kXrUnroll];
#pragma unroll
    for (int u = 0; u < kXrUnroll; ++u) {
      xx[u] = x[i + u * st];
      sh[u] = shat[i + u * st];
      ph[u] = phat[i + u * st];
      tt[u] = t[i + u * st];
      ss[u] = s[i + u * st];
      rh[u] = rhat[i + u * st];
    }
#pragma unroll
    for (int u = 0; u < kXrUnroll; ++u) {
      x[i + u * st] = fma(omega, sh[u], fma(alpha, ph[u], xx[u]));
      const double ri = fma(-omega, tt[u], ss[u]);
      r[i + u * st] = ri;
      a0 = fma(rh[u], ri, a0);
      a1 = fma(ri, ri, a1);
    }
  }
  for (; i < n; i += st) {
    x[i] = fma(omega, shat[i], fma(alpha, phat[i], x[i]));
    const double ri = fma(-omega, t[i], s[i]);
    r[i] = ri;
    a0 = fma(rhat[i], ri, a0);
    a1 = fma(ri, ri, a1);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) scal[Scal::OMEGA] = omega;
  const double val[2] = {a0, a1};
  const int sl[2] = {1 - par, Scal::RR};
  grid_reduce<2>(val, sl, part, counter, scal);
}

// End of an iteration: record ||r_i|| / ||B||, decide the status, continue or stop.
template <bool GRAPH>
__global__ void bicg_check_kernel(const double *scal, int *state, double *hist, LoopParams lp,
                                  cudaGraphConditionalHandle handle) {
  const int it = state[kIt] + 1;        // iterations completed after this one
  const int par_next = it & 1;          // slot holding rho_{i+1}
  const double bnorm = sqrt(scal[Scal::BB]);
  const double rel = sqrt(scal[Scal::RR]) / bnorm;
  hist[it < HMG_MAX_HISTORY ? it : HMG_MAX_HISTORY - 1] = rel;
  int status = HMG_OK, cont = 0;
  if (!isfinite(rel) || !isfinite(scal[Scal::ALPHA]) || !isfinite(scal[Scal::OMEGA])) {
    status = HMG_ERR_NONFINITE;
  } else if (rel <= lp.tol) {
    status = HMG_OK;
  } else if (scal[Scal::RV] == 0.0 || scal[Scal::TT] == 0.0 || scal[par_next] == 0.0) {
    status = HMG_ERR_BREAKDOWN;
  } else if (rel > lp.divergence || it >= lp.max_iter) {
    status = HMG_ERR_NOT_CONVERGED;
  } else {
    cont = 1;
  }
  state[kIt] = it;
  state[kStatus] = status;
  state[kContinue] = cont;
  if (GRAPH) cudaGraphSetConditional(handle, cont);
}

static LoopParams loop_params(const Ctx *c) {
  return LoopParams{c->opt.tol, c->opt.divergence, c->opt.max_iter, c->opt.warm_start ? 1 : 0};
}

// B_lambda, (B, B), x = 0, r = rhat = B, loop state
static int solve_head(Ctx *c, const double *Rub, const double *Rpi, double *x, bool graph,
                      cudaGraphConditionalHandle h) {
  const int64_t n = sys_n(c);
  int s;
  if ((s = sys_rhs(c, Rub, Rpi, c->B))) return s;
  Prof pk(c, kCompKrylov, 3);
  if ((s = launch_dot(c, c->B, c->B, n, Scal::BB))) return s;
  if (c->opt.warm_start) {
    if ((s = sys_apply(c, x, c->r, 0, nullptr, 0, 0))) return s;
    bicg_init_warm_kernel<<<red_grid(n), kRedThreads, 0, c->stream>>>(c->B, c->r, c->rhat, c->p, c->v, n);
    if ((s = launch_dot(c, c->r, c->r, n, Scal::RR))) return s;
  } else {
    bicg_init_kernel<<<red_grid(n), kRedThreads, 0, c->stream>>>(c->B, x, c->r, c->rhat, c->p, c->v, n);
  }
  if (graph) bicg_start_kernel<true><<<1, 1, 0, c->stream>>>(c->scal, c->state, c->hist, loop_params(c), h);
  else bicg_start_kernel<false><<<1, 1, 0, c->stream>>>(c->scal, c->state, c->hist, loop_params(c), h);
  HMG_CUDA(c, cudaGetLastError());
  return HMG_OK;
}

// Blocks of a grid-stride vector kernel: one wave of resident blocks (no partial second
// wave), at most one row per thread; fixed per device, so the reductions stay deterministic.
static int wave_grid(Ctx *c, int which, const void *kernel, int64_t n, unsigned *g) {
  if (!c->wave_blocks[which]) {
    int per_sm = 0;
    HMG_CUDA(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kRedThreads, 0));
    c->wave_blocks[which] = std::max(1, std::min(per_sm * c->num_sms, kRedBlocks));
  }
  *g = (unsigned)std::min<int64_t>(c->wave_blocks[which], grid_for(n, kRedThreads));
  return HMG_OK;
}

// one BiCGStab iteration and its check
static int solve_body(Ctx *c, double *x, bool graph, cudaGraphConditionalHandle h) {
  const int64_t n = sys_n(c);
  unsigned gp, gs, gx;
  int s;
  if ((s = wave_grid(c, 0, (const void *)bicg_p_kernel, n, &gp))) return s;
  if ((s = wave_grid(c, 1, (const void *)bicg_s_kernel, n, &gs))) return s;
  if ((s = wave_grid(c, 2, (const void *)bicg_xr_kernel, n, &gx))) return s;
  {
    Prof pk(c, kCompKrylov);
    bicg_p_kernel<<<gp, kRedThreads, 0, c->stream>>>(c->r, c->p, c->v, c->scal, c->state, n);
    HMG_CUDA(c, cudaGetLastError());
  }
  if ((s = precond_apply(c, c->p, c->phat))) return s;
  if ((s = sys_apply(c, c->phat, c->v, 1, c->rhat, Scal::RV, 0))) return s;
  {
    Prof pk(c, kCompKrylov);
    bicg_s_kernel<<<gs, kRedThreads, 0, c->stream>>>(c->r, c->v, c->s, c->scal, c->state, n);
    HMG_CUDA(c, cudaGetLastError());
  }
  if ((s = precond_apply(c, c->s, c->shat))) return s;
  if ((s = sys_apply(c, c->shat, c->t, 2, c->s, Scal::TS, Scal::TT))) return s;
  {
    Prof pk(c, kCompKrylov, 2);
    bicg_xr_kernel<<<gx, kRedThreads, 0, c->stream>>>(x, c->r, c->s, c->t, c->phat, c->shat, c->rhat,
                                                      c->scal, c->part, c->counter, c->state, n);
    if (graph) bicg_check_kernel<true><<<1, 1, 0, c->stream>>>(c->scal, c->state, c->hist, loop_params(c), h);
    else bicg_check_kernel<false><<<1, 1, 0, c->stream>>>(c->scal, c->state, c->hist, loop_params(c), h);
    HMG_CUDA(c, cudaGetLastError());
  }
  return HMG_OK;
}

// ||B - S x||^2 recomputed in FP64 from the final iterate
static int solve_tail(Ctx *c, const double *x) { return sys_apply(c, x, nullptr, 3, c->B, Scal::AUX, 0); }

// ---- graph construction ------------------------------------------------------------------
// Adds one solve (head -> WHILE(body) -> tail) to graph g, without dependencies on other
// nodes of g: the head is captured into g, the WHILE node is added after the head's last
// nodes, the body is captured into the WHILE node's graph on a second stream, and the tail
// is captured after the WHILE node.
static int add_solve_branch(Ctx *c, cudaGraph_t g, const double *Rub, const double *Rpi, double *x) {
  if (!c->cap_stream) HMG_CUDA(c, cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
  cudaGraphConditionalHandle h;
  HMG_CUDA(c, cudaGraphConditionalHandleCreate(&h, g, 0, cudaGraphCondAssignDefault));
  cudaStream_t saved = c->stream;
  HMG_CUDA(c, cudaStreamBeginCaptureToGraph(c->cap_stream, g, nullptr, nullptr, 0,
                                            cudaStreamCaptureModeThreadLocal));
  c->stream = c->cap_stream;
  int st = solve_head(c, Rub, Rpi, x, true, h);
  if (!st) {
    cudaStreamCaptureStatus cs;
    const cudaGraphNode_t *deps = nullptr;
    size_t nd = 0;
    cudaGraphNode_t wnode = nullptr;
    cudaError_t e = cudaStreamGetCaptureInfo(c->cap_stream, &cs, nullptr, nullptr, &deps, nullptr, &nd);
    cudaGraphNodeParams p = {};
    p.type = cudaGraphNodeTypeConditional;
    p.conditional.handle = h;
    p.conditional.type = cudaGraphCondTypeWhile;
    p.conditional.size = 1;
    if (e == cudaSuccess) e = cudaGraphAddNode(&wnode, g, deps, nullptr, nd, &p);
    if (e == cudaSuccess) e = cudaStreamUpdateCaptureDependencies(c->cap_stream, &wnode, nullptr, 1,
                                                                 cudaStreamSetCaptureDependencies);
    if (e != cudaSuccess) st = cuda_fail(c, e, "graph conditional node");
    if (!st) {
      cudaGraph_t body = p.conditional.phGraph_out[0];
      cudaStream_t s2 = nullptr;
      e = cudaStreamCreateWithFlags(&s2, cudaStreamNonBlocking);
      if (e == cudaSuccess)
        e = cudaStreamBeginCaptureToGraph(s2, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
      if (e != cudaSuccess) {
        st = cuda_fail(c, e, "capture of the iteration body");
      } else {
        c->stream = s2;
        st = solve_body(c, x, true, h);
        cudaGraph_t tmp;
        e = cudaStreamEndCapture(s2, &tmp);
        if (!st && e != cudaSuccess) st = cuda_fail(c, e, "end of the body capture");
      }
      if (s2) cudaStreamDestroy(s2);
      c->stream = c->cap_stream;
      // an event node after the loop: a copy of lambda to the host can overlap the tail
      if (!st) {
        e = cudaEventRecordWithFlags(c->loop_done, c->cap_stream, cudaEventRecordExternal);
        if (e != cudaSuccess) st = cuda_fail(c, e, "loop-end event node");
      }
      if (!st) st = solve_tail(c, x);
    }
  }
  c->stream = saved;
  cudaGraph_t out;
  cudaError_t e = cudaStreamEndCapture(c->cap_stream, &out);
  if (st) return st;
  HMG_CUDA(c, e);
  return HMG_OK;
}

static bool same_key(const Ctx::GraphKey &k, const double *Rub, const double *Rpi, const double *lam,
                     const hmg_options &o) {
  return k.Rub == Rub && k.Rpi == Rpi && k.lam == lam && std::memcmp(&k.opt, &o, sizeof(o)) == 0;
}

uint64_t next_graph_gen() {
  static std::atomic<uint64_t> gen{0};
  return ++gen;
}

static void drop_batch_graph(Ctx *c) {
  if (c->batch_exec) cudaGraphExecDestroy(c->batch_exec);
  if (c->batch_graph) cudaGraphDestroy(c->batch_graph);
  c->batch_exec = nullptr;
  c->batch_graph = nullptr;
  c->batch_key.clear();
}

void drop_graph(Ctx *c) {
  // an enqueued (async_stats) solve may still be running the graph: let it finish first
  if (c->graph_exec && c->stats_pending) cudaEventSynchronize(c->as_e1);
  if (c->graph_exec) cudaGraphExecDestroy(c->graph_exec);
  if (c->graph) cudaGraphDestroy(c->graph);
  c->graph_exec = nullptr;
  c->graph = nullptr;
  // batch graphs that hold this context's launches (its own, or another context's) no longer
  // match its generation
  c->graph_gen = next_graph_gen();
  drop_batch_graph(c);
}

static int ensure_solve_graph(Ctx *c, const double *Rub, const double *Rpi, double *x) {
  if (c->graph_exec && same_key(c->graph_key, Rub, Rpi, x, c->opt)) return HMG_OK;
  drop_graph(c);
  HMG_CUDA(c, cudaGraphCreate(&c->graph, 0));
  int st = add_solve_branch(c, c->graph, Rub, Rpi, x);
  if (st) { drop_graph(c); return st; }
  cudaError_t e = cudaGraphInstantiate(&c->graph_exec, c->graph, 0);
  if (e != cudaSuccess) { drop_graph(c); return cuda_fail(c, e, "cudaGraphInstantiate"); }
  c->graph_key = Ctx::GraphKey{Rub, Rpi, x, c->opt};
  return HMG_OK;
}

// ---- results --------------------------------------------------------------------------------
static int status_message(Ctx *c, int status) {
  if (status == HMG_OK) return HMG_OK;
  const std::string name = c->opt.krylov == HMG_KRYLOV_FGMRES ? "FGMRES" : "BiCGStab";
  const std::string why = status == HMG_ERR_NOT_CONVERGED ? name + " did not converge"
                          : status == HMG_ERR_BREAKDOWN  ? name + " breakdown"
                          : status == HMG_ERR_TIMEOUT    ? "a bounded device-side wait ran out"
                                                         : "non-finite value in " + name;
  return fail(c, status, why);
}

// Copies the loop state, history and scalars to the host (stream-ordered) and fills stats.
// Enqueues the copies of the loop state, history and scalars into the pinned host buffers.
static int enqueue_results(Ctx *c) {
  HMG_CUDA(c, cudaMemcpyAsync(c->scal_host, c->scal, sizeof(double) * Scal::N, cudaMemcpyDeviceToHost, c->stream));
  HMG_CUDA(c, cudaMemcpyAsync(c->state_host, c->state, sizeof(int) * 4, cudaMemcpyDeviceToHost, c->stream));
  HMG_CUDA(c, cudaMemcpyAsync(c->hist_host, c->hist, sizeof(double) * HMG_MAX_HISTORY, cudaMemcpyDeviceToHost, c->stream));
  return HMG_OK;
}

// Stats from the host buffers (the copies have completed) and the solve's stop reason.
static int fill_stats(Ctx *c, hmg_solve_stats *st, float ms) {
  const int it = c->state_host[kIt];
  int status = c->state_host[kStatus];
  if (c->state_host[kWaitFlag]) {   // a bounded device-side wait ran out during the solve
    HMG_CUDA(c, cudaMemsetAsync(c->state + kWaitFlag, 0, sizeof(int), c->stream));
    status = HMG_ERR_TIMEOUT;
    // with a learned coarse solve the wait may have been the tensor-core layer's: the context
    // runs the network on the CUDA cores from now on
    // (captured solve graphs hold the tensor-core launches: they are captured again)
    if ((c->opt.coarse == HMG_COARSE_LEARNED || c->opt.coarse == HMG_COARSE_LEARNED_VCYCLE) && !c->nn_tc_off) {
      drop_graph(c);
      c->nn_tc_off = true;
    }
  }
  if (st) {
    const double bb = c->scal_host[Scal::BB];
    const double bnorm = std::sqrt(bb);
    std::memcpy(st->history, c->hist_host, sizeof(double) * HMG_MAX_HISTORY);
    st->status = status;
    st->iterations = it;
    st->n_history = it + 1 < HMG_MAX_HISTORY ? it + 1 : HMG_MAX_HISTORY;
    st->rel_residual = st->history[st->n_history - 1];
    st->true_rel_residual = bnorm > 0.0 ? std::sqrt(c->scal_host[Scal::AUX]) / bnorm : 0.0;
    st->solve_ms = ms;
    st->coarse_fallback = c->coarse_fallback ? 1 : 0;
    for (int q = 0; q < HMG_NCOMP; ++q) { st->comp_ms[q] = 0.0; st->comp_calls[q] = 0; }
    for (const Ctx::Mark &m : c->marks) {
      float t = 0.f;
      if (cudaEventElapsedTime(&t, c->ev_pool[m.e0], c->ev_pool[m.e1]) == cudaSuccess) {
        st->comp_ms[m.comp] += t;
        st->comp_calls[m.comp] += m.launches;
      }
    }
  }
  return status_message(c, status);
}

static int collect(Ctx *c, hmg_solve_stats *st, float ms) {
  int s;
  if ((s = enqueue_results(c))) return s;
  HMG_CUDA(c, cudaStreamSynchronize(c->stream));
  return fill_stats(c, st, ms);
}

int solve_stats_get(Ctx *c, hmg_solve_stats *st) {
  if (!c->stats_pending) return fail(c, HMG_ERR_NOT_READY, "no asynchronous solve is pending");
  c->stats_pending = false;
  HMG_CUDA(c, cudaEventSynchronize(c->as_e1));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, c->as_e0, c->as_e1);
  c->marks.clear();   // no component timers in a graph-launched solve
  return fill_stats(c, st, ms);
}

// A stop reason of the iteration itself (lambda is then the last iterate), not a failure.
static bool solve_outcome(int r) {
  return r == HMG_OK || r == HMG_ERR_NOT_CONVERGED || r == HMG_ERR_BREAKDOWN || r == HMG_ERR_NONFINITE ||
         r == HMG_ERR_TIMEOUT;
}

static int copy_to_host(Ctx *c, double *host_out, const double *lambda) {
  HMG_CUDA(c, cudaMemcpyAsync(host_out, lambda, sizeof(double) * sys_n(c), cudaMemcpyDeviceToHost, c->stream));
  HMG_CUDA(c, cudaStreamSynchronize(c->stream));
  return HMG_OK;
}

int krylov_solve(Ctx *c, const double *Rub, const double *Rpi, double *lambda, hmg_solve_stats *st,
                 bool allow_async, double *host_out) {
  c->marks.clear();
  c->ev_next = 0;
  c->coarse_fallback = false;
  if (c->opt.krylov == HMG_KRYLOV_FGMRES) {
    c->stats_pending = false;   // its results replace an uncollected enqueued solve's
    const int r = fgmres_solve(c, Rub, Rpi, lambda, st);
    int s2;
    if (host_out && solve_outcome(r) && (s2 = copy_to_host(c, host_out, lambda))) return s2;
    return r;
  }
  SolveTimer timer;
  int s;
  if ((s = timer.start(c))) return s;
  const bool host_coarse = c->opt.precond == HMG_PRECOND_NONNESTED &&
                           (c->opt.coarse == HMG_COARSE_KRYLOV_EXACT || c->opt.coarse == HMG_COARSE_KRYLOV_APPROX);
  if (c->opt.graph && !c->opt.profile && !c->collect_x && !host_coarse) {
    if ((s = ensure_solve_graph(c, Rub, Rpi, lambda))) return s;
    if (allow_async && c->opt.async_stats) {
      // enqueue only: the results travel to the pinned buffers behind the solve
      HMG_CUDA(c, cudaEventRecord(c->as_e0, c->stream));
      HMG_CUDA(c, cudaGraphLaunch(c->graph_exec, c->stream));
      if ((s = enqueue_results(c))) return s;
      // the end event follows the copies: once it completes, the host buffers hold this solve's
      // results (solve_ms includes the few-microsecond copies)
      HMG_CUDA(c, cudaEventRecord(c->as_e1, c->stream));
      c->stats_pending = true;
      if (st) st->status = HMG_ERR_NOT_READY;   // the stats come from hmg_solve_stats_get
      return HMG_OK;
    }
    HMG_CUDA(c, cudaGraphLaunch(c->graph_exec, c->stream));
    // one synchronisation: the solve's end, the copy of lambda to the host (on its own stream,
    // from the end of the Krylov loop, so it overlaps the final residual), the results
    HMG_CUDA(c, cudaEventRecord(timer.e1, c->stream));
    if (host_out) {
      HMG_CUDA(c, cudaStreamWaitEvent(c->copy_stream, c->loop_done, 0));
      HMG_CUDA(c, cudaMemcpyAsync(host_out, lambda, sizeof(double) * sys_n(c), cudaMemcpyDeviceToHost,
                                  c->copy_stream));
      HMG_CUDA(c, cudaEventRecord(c->copy_done, c->copy_stream));
      HMG_CUDA(c, cudaStreamWaitEvent(c->stream, c->copy_done, 0));
    }
    if ((s = enqueue_results(c))) return s;
    HMG_CUDA(c, cudaEventRecord(timer.e2, c->stream));
    HMG_CUDA(c, cudaEventSynchronize(timer.e2));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, timer.e0, timer.e1);
    c->stats_pending = false;   // these results replace an uncollected enqueued solve's
    return fill_stats(c, st, ms);
  } else {
    cudaGraphConditionalHandle none = 0;
    if ((s = solve_head(c, Rub, Rpi, lambda, false, none))) return s;
    for (;;) {
      HMG_CUDA(c, cudaMemcpyAsync(c->state_host, c->state, sizeof(int) * 3, cudaMemcpyDeviceToHost, c->stream));
      HMG_CUDA(c, cudaStreamSynchronize(c->stream));
      if (!c->state_host[kContinue]) break;
      if ((s = solve_body(c, lambda, false, none))) return s;
    }
    if ((s = solve_tail(c, lambda))) return s;
  }
  float ms = 0.f;
  if ((s = timer.stop(c, &ms))) return s;
  c->stats_pending = false;   // these results replace an uncollected enqueued solve's
  const int r = collect(c, st, ms);
  if (host_out && solve_outcome(r) && (s = copy_to_host(c, host_out, lambda))) return s;
  return r;
}

// All contexts on one device; each branch of the graph is one context's whole solve, and
// the branches have no dependencies on one another, so they run concurrently.
int krylov_solve_batched(hmg_ctx *const *ctxs, int n, const double *const *Rub,
                         const double *const *Rpi, double *const *lambda, hmg_solve_stats *st) {
  Ctx *c0 = ctxs[0];
  for (int i = 0; i < n; ++i)
    if (ctxs[i]->opt.krylov != HMG_KRYLOV_BICGSTAB || ctxs[i]->collect_x ||
        ctxs[i]->opt.coarse == HMG_COARSE_KRYLOV_EXACT || ctxs[i]->opt.coarse == HMG_COARSE_KRYLOV_APPROX)
      return fail(c0, HMG_ERR_INVALID_ARG, "batched solves take BiCGStab contexts without pair collection");
  bool profile = false;
  for (int i = 0; i < n; ++i) {
    Ctx *c = ctxs[i];
    c->marks.clear();
    c->ev_next = 0;
    c->coarse_fallback = false;
    if (c->stats_pending) {   // an enqueued solve of this context runs on its own stream
      cudaEventSynchronize(c->as_e1);
      c->stats_pending = false;
    }
    profile = profile || c->opt.profile;
  }
  // the instantiated graph is kept on the first context while the batch (contexts, their
  // generations, vectors and options) stays the same; a profiled batch is captured afresh
  // each call, since its event marks are recorded at capture
  bool cached = !profile && c0->batch_exec && (int)c0->batch_key.size() == n;
  for (int i = 0; cached && i < n; ++i) {
    const Ctx::BatchMember &k = c0->batch_key[i];
    const Ctx *c = ctxs[i];
    cached = k.ctx == c && k.gen == c->graph_gen && k.Rub == Rub[i] && k.Rpi == Rpi[i] && k.lam == lambda[i] &&
             std::memcmp(&k.opt, &c->opt, sizeof(hmg_options)) == 0;
  }
  int s = HMG_OK;
  cudaGraph_t g = nullptr;
  cudaGraphExec_t ex = nullptr;
  if (cached) {
    ex = c0->batch_exec;
  } else {
    drop_batch_graph(c0);
    HMG_CUDA(c0, cudaGraphCreate(&g, 0));
    for (int i = 0; i < n && !s; ++i) {
      Ctx *c = ctxs[i];
      s = add_solve_branch(c, g, Rub[i], Rpi[i], lambda[i]);
      if (s && c != c0) c0->err = c->err;
    }
    if (!s) {
      cudaError_t e = cudaGraphInstantiate(&ex, g, 0);
      if (e != cudaSuccess) s = cuda_fail(c0, e, "cudaGraphInstantiate (batched)");
    }
    if (!s && !profile) {
      c0->batch_graph = g;
      c0->batch_exec = ex;
      for (int i = 0; i < n; ++i)
        c0->batch_key.push_back({ctxs[i], ctxs[i]->graph_gen, Rub[i], Rpi[i], lambda[i], ctxs[i]->opt});
    }
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (!s) {
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, c0->stream);
    cudaError_t e = cudaGraphLaunch(ex, c0->stream);
    if (e != cudaSuccess) s = cuda_fail(c0, e, "cudaGraphLaunch (batched)");
    cudaEventRecord(e1, c0->stream);
    cudaEventSynchronize(e1);
  }
  float ms = 0.f;
  if (!s) cudaEventElapsedTime(&ms, e0, e1);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (!(ex && ex == c0->batch_exec)) {   // not kept: a profiled batch, or one that failed
    if (ex) cudaGraphExecDestroy(ex);
    if (g) cudaGraphDestroy(g);
  }
  if (s) drop_batch_graph(c0);
  if (s) return s;
  int worst = HMG_OK;
  for (int i = 0; i < n; ++i) {
    Ctx *c = ctxs[i];
    cudaStream_t saved = c->stream;
    c->stream = c0->stream;
    const int r = collect(c, st ? &st[i] : nullptr, ms);
    c->stream = saved;
    if (r != HMG_OK && worst == HMG_OK) {
      worst = r;
      c0->err = c->err;
    }
  }
  return worst;
}

// ---- flexible GMRES(m) ----------------------------------------------------------------------
// Right-preconditioned flexible GMRES (Saad 2003 Alg. 9.6) from lambda = 0: z_j = M_j^-1 v_j may
// change from step to step (a learned coarse solve is not a fixed linear map) and the update is
// x += Z_m y_m. The new basis vector is orthogonalised by classical Gram-Schmidt applied twice
// (equal to modified Gram-Schmidt in exact arithmetic and as robust in practice, Giraud et al.
// 2005), so a step costs two multi-vector dot kernels instead of j + 1 dependent reductions.
// The Hessenberg column (j + 2 numbers) goes to the host, which holds the Givens rotations and
// solves the small triangular system: one synchronisation per step, against a preconditioner
// application of about a millisecond. max_iter counts steps (preconditioner applications).
//
// Fallback: with a learned coarse solve, two consecutive steps that each reduce the residual
// estimate by less than the factor stall_ratio, or a step whose Hessenberg column is not
// finite (that step is dropped and the cycle restarts), switch the coarse solve to the
// pressure V-cycle for the rest of the solve.
constexpr int kMaxRestart = 64;
constexpr unsigned kGmBlocks = 608;   // blocks per dot of the multi-vector dot kernel (4 per SM)

__global__ void __launch_bounds__(kRedThreads)
    mdot_kernel(const double *__restrict__ V, int64_t n, const double *__restrict__ w, double *__restrict__ part) {
  const double *v = V + (int64_t)blockIdx.y * n;
  double s = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    s = fma(v[i], w[i], s);
  s = warp_sum(s);
  __shared__ double sh[kRedThreads / 32];
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int q = 0; q < kRedThreads / 32; ++q) t += sh[q];
    part[(int64_t)blockIdx.y * gridDim.x + blockIdx.x] = t;
  }
}

// h[k] = the partials of dot k summed in block order (one block per k); hacc[k] += h[k]
__global__ void mdot_finalize_kernel(const double *__restrict__ part, int nb, double *__restrict__ h,
                                     double *__restrict__ hacc) {
  const int k = blockIdx.x;
  double s = 0.0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) s += part[(int64_t)k * nb + b];
  s = warp_sum(s);
  __shared__ double sh[32];
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += sh[q];
    h[k] = t;
    if (hacc) hacc[k] += t;
  }
}

// w += sign * sum_{k < nk} h[k] V[k]
__global__ void __launch_bounds__(kRedThreads)
    mcomb_kernel(double *__restrict__ w, const double *__restrict__ V, int64_t n, const double *__restrict__ h,
                 int nk, double sign) {
  __shared__ double hs[kMaxRestart + 1];
  for (int k = threadIdx.x; k < nk; k += blockDim.x) hs[k] = sign * h[k];
  __syncthreads();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double s = w[i];
    for (int k = 0; k < nk; ++k) s = fma(hs[k], V[(int64_t)k * n + i], s);
    w[i] = s;
  }
}

// w /= sqrt(nn) (w = 0 when nn = 0); *hout = sqrt(nn)
__global__ void gm_normalize_kernel(double *__restrict__ w, int64_t n, const double *nn, double *hout) {
  __shared__ double coef[2];
  if (threadIdx.x == 0) {
    coef[0] = sqrt(*nn);
    coef[1] = coef[0] > 0.0 ? 1.0 / coef[0] : 0.0;
  }
  __syncthreads();
  const double s = coef[0], inv = coef[1];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    w[i] *= inv;
  if (blockIdx.x == 0 && threadIdx.x == 0) *hout = s;
}

// r = B - y
__global__ void gm_sub_kernel(const double *__restrict__ B, const double *__restrict__ y, double *__restrict__ r,
                              int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    r[i] = B[i] - y[i];
}

static int gm_buffers(Ctx *c, int m) {
  const int64_t n = std::max<int64_t>(c->lv[0].ntrace + c->lv[0].ncell, sys_n(c));   // the longest system
  if (c->gm_V && c->gm_restart >= m && c->gm_n >= n) return HMG_OK;
  dev_free(c, c->gm_V);
  dev_free(c, c->gm_Z);
  c->gm_V = c->gm_Z = nullptr;
  c->gm_restart = 0;
  int s;
  if ((s = dev_alloc(c, &c->gm_V, (size_t)(m + 1) * n))) return s;
  if ((s = dev_alloc(c, &c->gm_Z, (size_t)m * n))) return s;
  if (!c->gm_h) {
    if ((s = dev_alloc(c, &c->gm_h, (size_t)3 * (kMaxRestart + 2)))) return s;
    if ((s = dev_alloc(c, &c->gm_part, (size_t)(kMaxRestart + 1) * kGmBlocks))) return s;
    if ((s = dev_alloc(c, &c->gm_y, (size_t)kMaxRestart))) return s;
  }
  c->gm_restart = m;
  c->gm_n = n;
  return HMG_OK;
}

static unsigned gm_grid(int64_t n) {
  const unsigned g = grid_for(n, kRedThreads);
  return g < kGmBlocks ? g : kGmBlocks;
}

// h[k] = (V_k, w), k < nk (and hacc[k] += h[k])
static int mdot(Ctx *c, const double *V, int nk, const double *w, double *h, double *hacc) {
  const int64_t n = sys_n(c);
  const unsigned nb = gm_grid(n);
  mdot_kernel<<<dim3(nb, (unsigned)nk), kRedThreads, 0, c->stream>>>(V, n, w, c->gm_part);
  mdot_finalize_kernel<<<(unsigned)nk, 256, 0, c->stream>>>(c->gm_part, (int)nb, h, hacc);
  HMG_CUDA(c, cudaGetLastError());
  return HMG_OK;
}

static int mcomb(Ctx *c, double *w, const double *V, const double *h, int nk, double sign) {
  const int64_t n = sys_n(c);
  mcomb_kernel<<<red_grid(n), kRedThreads, 0, c->stream>>>(w, V, n, h, nk, sign);
  HMG_CUDA(c, cudaGetLastError());
  return HMG_OK;
}

// v = v / ||v||, *beta_host = ||v||
static int normalize(Ctx *c, double *v, double *nn_slot, double *h_slot, double *beta_host) {
  const int64_t n = sys_n(c);
  int s;
  if ((s = mdot(c, v, 1, v, nn_slot, nullptr))) return s;
  gm_normalize_kernel<<<red_grid(n), kRedThreads, 0, c->stream>>>(v, n, nn_slot, h_slot);
  HMG_CUDA(c, cudaGetLastError());
  if (beta_host) {
    HMG_CUDA(c, cudaMemcpyAsync(beta_host, h_slot, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    HMG_CUDA(c, cudaStreamSynchronize(c->stream));
  }
  return HMG_OK;
}

int fgmres_solve(Ctx *c, const double *Rub, const double *Rpi, double *x, hmg_solve_stats *st) {
  const int64_t n = sys_n(c);
  const int m = c->opt.restart;
  const bool learned = c->opt.precond == HMG_PRECOND_NONNESTED && c->opt.coarse != HMG_COARSE_VCYCLE;
  int s;
  if ((s = gm_buffers(c, m))) return s;
  double *hd = c->gm_h, *h2 = hd + (kMaxRestart + 2), *sc = h2 + (kMaxRestart + 2);
  double *V = c->gm_V, *Z = c->gm_Z;
  SolveTimer timer;
  if ((s = timer.start(c))) return s;
  if ((s = sys_rhs(c, Rub, Rpi, c->B))) return s;
  double beta = 0.0;
  {
    Prof pk(c, kCompKrylov, 6);
    if ((s = launch_dot(c, c->B, c->B, n, Scal::BB))) return s;
    if (c->opt.warm_start) {   // r_0 = B - S lambda_0
      if ((s = sys_apply(c, x, c->t, 0, nullptr, 0, 0))) return s;
      gm_sub_kernel<<<red_grid(n), kRedThreads, 0, c->stream>>>(c->B, c->t, V, n);
      HMG_CUDA(c, cudaGetLastError());
    } else {
      HMG_CUDA(c, cudaMemsetAsync(x, 0, sizeof(double) * n, c->stream));
      HMG_CUDA(c, cudaMemcpyAsync(V, c->B, sizeof(double) * n, cudaMemcpyDeviceToDevice, c->stream));
    }
    if ((s = normalize(c, V, sc, sc + 1, &beta))) return s;
  }
  double bb_host = 0.0;
  HMG_CUDA(c, cudaMemcpyAsync(&bb_host, c->scal + Scal::BB, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  HMG_CUDA(c, cudaStreamSynchronize(c->stream));
  const double bnorm = std::sqrt(bb_host);
  std::vector<double> hist{bnorm > 0.0 ? beta / bnorm : 0.0};
  const int kRunning = -1;
  int status = !std::isfinite(bnorm) || !std::isfinite(beta) ? HMG_ERR_NONFINITE
               : (bnorm == 0.0 || hist[0] <= c->opt.tol) ? HMG_OK : kRunning;
  if (status == kRunning && c->opt.max_iter <= 0) status = HMG_ERR_NOT_CONVERGED;
  std::vector<double> Hm((size_t)(m + 1) * m), cs(m), sn(m), g(m + 1), col(m + 2), y(m);
  int steps = 0, slow = 0;
  double prev_rel = hist[0];
  while (status == kRunning) {
    std::fill(g.begin(), g.end(), 0.0);
    g[0] = beta;
    int jd = 0;
    for (int j = 0; j < m; ++j) {
      double *vj = V + (int64_t)j * n, *zj = Z + (int64_t)j * n, *w = V + (int64_t)(j + 1) * n;
      if ((s = precond_apply(c, vj, zj))) return s;
      if ((s = sys_apply(c, zj, w, 0, nullptr, 0, 0))) return s;
      {
        Prof pk(c, kCompKrylov, 12);
        if ((s = mdot(c, V, j + 1, w, hd, nullptr))) return s;
        if ((s = mcomb(c, w, V, hd, j + 1, -1.0))) return s;
        if ((s = mdot(c, V, j + 1, w, h2, hd))) return s;
        if ((s = mcomb(c, w, V, h2, j + 1, -1.0))) return s;
        if ((s = normalize(c, w, sc, hd + j + 1, nullptr))) return s;
        HMG_CUDA(c, cudaMemcpyAsync(col.data(), hd, sizeof(double) * (j + 2), cudaMemcpyDeviceToHost, c->stream));
        HMG_CUDA(c, cudaStreamSynchronize(c->stream));
      }
      bool finite = true;
      for (int i = 0; i <= j + 1; ++i) finite = finite && std::isfinite(col[i]);
      if (!finite) {
        if (learned && !c->coarse_fallback) {
          c->coarse_fallback = true;   // drop the step, keep the cycle's first jd steps, restart
          break;
        }
        status = HMG_ERR_NONFINITE;
        break;
      }
      for (int i = 0; i < j; ++i) {
        const double t = cs[i] * col[i] + sn[i] * col[i + 1];
        col[i + 1] = -sn[i] * col[i] + cs[i] * col[i + 1];
        col[i] = t;
      }
      const double den = std::hypot(col[j], col[j + 1]);
      if (den == 0.0) {
        status = HMG_ERR_BREAKDOWN;
        break;
      }
      cs[j] = col[j] / den;
      sn[j] = col[j + 1] / den;
      col[j] = den;
      col[j + 1] = 0.0;
      g[j + 1] = -sn[j] * g[j];
      g[j] = cs[j] * g[j];
      for (int i = 0; i <= j; ++i) Hm[(size_t)i * m + j] = col[i];
      ++steps;
      jd = j + 1;
      const double rel = std::fabs(g[j + 1]) / bnorm;
      hist.push_back(rel);
      if (learned && !c->coarse_fallback) {
        slow = rel > c->opt.stall_ratio * prev_rel ? slow + 1 : 0;
        if (slow >= 2) c->coarse_fallback = true;
      }
      prev_rel = rel;
      if (rel <= c->opt.tol) break;
      if (!(rel <= c->opt.divergence) || steps >= c->opt.max_iter) {
        status = HMG_ERR_NOT_CONVERGED;
        break;
      }
    }
    // x += Z y, y = R^-1 g over the cycle's completed steps
    if (jd > 0) {
      for (int i = jd - 1; i >= 0; --i) {
        double t = g[i];
        for (int k = i + 1; k < jd; ++k) t -= Hm[(size_t)i * m + k] * y[k];
        y[i] = t / Hm[(size_t)i * m + i];
      }
      Prof pk(c, kCompKrylov);
      HMG_CUDA(c, cudaMemcpyAsync(c->gm_y, y.data(), sizeof(double) * jd, cudaMemcpyHostToDevice, c->stream));
      if ((s = mcomb(c, x, Z, c->gm_y, jd, 1.0))) return s;
      HMG_CUDA(c, cudaStreamSynchronize(c->stream));   // y (host) is reused by the next cycle
    }
    if (status != kRunning) break;
    if (hist.back() <= c->opt.tol) {
      status = HMG_OK;
      break;
    }
    // restart from the true residual
    if ((s = sys_apply(c, x, c->t, 0, nullptr, 0, 0))) return s;
    {
      Prof pk(c, kCompKrylov, 4);
      gm_sub_kernel<<<red_grid(n), kRedThreads, 0, c->stream>>>(c->B, c->t, V, n);
      HMG_CUDA(c, cudaGetLastError());
      if ((s = normalize(c, V, sc, sc + 1, &beta))) return s;
    }
    if (!std::isfinite(beta)) status = HMG_ERR_NONFINITE;
  }
  if ((s = solve_tail(c, x))) return s;
  const int nh = (int)hist.size() < HMG_MAX_HISTORY ? (int)hist.size() : HMG_MAX_HISTORY;
  if ((int)hist.size() > HMG_MAX_HISTORY) hist[HMG_MAX_HISTORY - 1] = hist.back();
  c->state_host[kIt] = steps;
  c->state_host[kStatus] = status;
  c->state_host[kContinue] = 0;
  HMG_CUDA(c, cudaMemcpyAsync(c->hist, hist.data(), sizeof(double) * nh, cudaMemcpyHostToDevice, c->stream));
  HMG_CUDA(c, cudaMemcpyAsync(c->state, c->state_host, sizeof(int) * 3, cudaMemcpyHostToDevice, c->stream));
  float ms = 0.f;
  if ((s = timer.stop(c, &ms))) return s;
  return collect(c, st, ms);
}

}  // namespace hmg
