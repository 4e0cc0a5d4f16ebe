// Outer Krylov iteration on S lambda = B_lambda: right-preconditioned BiCGStab
// (van der Vorst 1992; Saad 2003 Alg. 7.7 with x = M^-1 y) from lambda = 0, stopping when
// the recurrence residual satisfies ||r_i|| <= tol ||B_lambda|| (Sec. 3.1 of arXiv
// 2210.11797: BiCGStab reducing the residual two-norm by the tolerance).
//
// Scalars live on the device: every inner product is a deterministic grid reduction into
// ctx->scal, and the vector kernels compute alpha, beta and omega from those sums
// themselves, so an iteration needs one 8-word device-to-host read (for the stopping test).
#include <chrono>
#include <cmath>

#include "device_common.cuh"
#include "hmg_internal.cuh"

namespace hmg {

static unsigned red_grid(int64_t n) {
  unsigned g = grid_for(n, kRedThreads);
  return g < (unsigned)kRedBlocks ? g : (unsigned)kRedBlocks;
}

__global__ void __launch_bounds__(kRedThreads)
    dot_kernel(const double *__restrict__ a, const double *__restrict__ b, int64_t n, double *part,
               unsigned int *counter, double *scal, int slot) {
  double s = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    s += a[i] * b[i];
  const double v[1] = {s};
  const int sl[1] = {slot};
  grid_reduce<1>(v, sl, part, counter, scal);
}

int launch_dot(Ctx *c, const double *a, const double *b, int64_t n, int slot) {
  dot_kernel<<<red_grid(n), kRedThreads, 0, c->stream>>>(a, b, n, c->part, c->counter, c->scal, slot);
  HMG_CUDA(c, cudaGetLastError());
  return HMG_OK;
}

// Start: x = 0, r = rhat = B, p = v = 0, scal[RHO_cur] = (B, B), scal[RHO_prev] = 1,
// alpha = omega = 1.
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

__global__ void bicg_scalars_init_kernel(double *scal) {
  scal[Scal::RHO0] = scal[Scal::BB];
  scal[Scal::RHO1] = 1.0;
  scal[Scal::ALPHA] = 1.0;
  scal[Scal::OMEGA] = 1.0;
}

// p = r + beta (p - omega v), beta = (rho_i / rho_{i-1}) (alpha / omega)
__global__ void bicg_p_kernel(const double *__restrict__ r, double *__restrict__ p,
                              const double *__restrict__ v, const double *__restrict__ scal,
                              int par, int64_t n) {
  const double rho = scal[par], rho_prev = scal[1 - par];
  const double alpha = scal[Scal::ALPHA], omega = scal[Scal::OMEGA];
  const double beta = (rho / rho_prev) * (alpha / omega);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    p[i] = r[i] + beta * (p[i] - omega * v[i]);
}

// alpha = rho_i / (rhat, v); s = r - alpha v
__global__ void bicg_s_kernel(const double *__restrict__ r, const double *__restrict__ v,
                              double *__restrict__ s, double *scal, int par, int64_t n) {
  const double alpha = scal[par] / scal[Scal::RV];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    s[i] = r[i] - alpha * v[i];
  if (blockIdx.x == 0 && threadIdx.x == 0) scal[Scal::ALPHA] = alpha;
}

// omega = (t, s) / (t, t); x += alpha phat + omega shat; r = s - omega t;
// (rhat, r) -> scal[1 - par] (rho_{i+1}), (r, r) -> scal[RR]
__global__ void __launch_bounds__(kRedThreads)
    bicg_xr_kernel(double *__restrict__ x, double *__restrict__ r, const double *__restrict__ s,
                   const double *__restrict__ t, const double *__restrict__ phat,
                   const double *__restrict__ shat, const double *__restrict__ rhat, double *scal,
                   double *part, unsigned int *counter, int par, int64_t n) {
  const double alpha = scal[Scal::ALPHA];
  const double omega = scal[Scal::TS] / scal[Scal::TT];
  double a0 = 0.0, a1 = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    x[i] = x[i] + alpha * phat[i] + omega * shat[i];
    const double ri = s[i] - omega * t[i];
    r[i] = ri;
    a0 += rhat[i] * ri;
    a1 += ri * ri;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) scal[Scal::OMEGA] = omega;
  const double val[2] = {a0, a1};
  const int sl[2] = {1 - par, Scal::RR};
  grid_reduce<2>(val, sl, part, counter, scal);
}

int krylov_solve(Ctx *c, const double *Rub, const double *Rpi, double *lambda, hmg_solve_stats *st) {
  const int64_t n = c->lv[0].ntrace;
  c->marks.clear();
  c->ev_next = 0;
  cudaEvent_t e0, e1;
  HMG_CUDA(c, cudaEventCreate(&e0));
  HMG_CUDA(c, cudaEventCreate(&e1));
  HMG_CUDA(c, cudaEventRecord(e0, c->stream));
  int s;
  if ((s = launch_trace_rhs(c, Rub, Rpi, c->B))) return s;
  const unsigned vg = red_grid(n);
  double *x = lambda;
  {
    Prof pk(c, kCompKrylov, 3);
    if ((s = launch_dot(c, c->B, c->B, n, Scal::BB))) return s;
    bicg_init_kernel<<<vg, kRedThreads, 0, c->stream>>>(c->B, x, c->r, c->rhat, c->p, c->v, n);
    bicg_scalars_init_kernel<<<1, 1, 0, c->stream>>>(c->scal);
    HMG_CUDA(c, cudaGetLastError());
  }
  HMG_CUDA(c, cudaMemcpyAsync(c->scal_host, c->scal, sizeof(double) * Scal::N, cudaMemcpyDeviceToHost, c->stream));
  HMG_CUDA(c, cudaStreamSynchronize(c->stream));
  const double bb = c->scal_host[Scal::BB];
  const double bnorm = std::sqrt(bb);
  int status = HMG_OK, it = 0;
  double rel = bnorm > 0.0 ? 1.0 : 0.0;
  if (st) {
    st->n_history = 0;
    st->history[st->n_history++] = rel;
  }
  if (!std::isfinite(bb)) status = HMG_ERR_NONFINITE;
  const double tol = c->opt.tol;
  while (status == HMG_OK && bnorm > 0.0 && rel > tol) {
    if (it >= c->opt.max_iter) { status = HMG_ERR_NOT_CONVERGED; break; }
    const int par = it & 1;
    {
      Prof pk(c, kCompKrylov);
      bicg_p_kernel<<<vg, kRedThreads, 0, c->stream>>>(c->r, c->p, c->v, c->scal, par, n);
      HMG_CUDA(c, cudaGetLastError());
    }
    if ((s = precond_apply(c, c->p, c->phat))) return s;
    if ((s = launch_spmv(c, c->phat, c->v, 1, c->rhat, Scal::RV, 0))) return s;
    {
      Prof pk(c, kCompKrylov);
      bicg_s_kernel<<<vg, kRedThreads, 0, c->stream>>>(c->r, c->v, c->s, c->scal, par, n);
      HMG_CUDA(c, cudaGetLastError());
    }
    if ((s = precond_apply(c, c->s, c->shat))) return s;
    if ((s = launch_spmv(c, c->shat, c->t, 2, c->s, Scal::TS, Scal::TT))) return s;
    {
      Prof pk(c, kCompKrylov);
      bicg_xr_kernel<<<vg, kRedThreads, 0, c->stream>>>(x, c->r, c->s, c->t, c->phat, c->shat,
                                                        c->rhat, c->scal, c->part, c->counter, par, n);
      HMG_CUDA(c, cudaGetLastError());
    }
    HMG_CUDA(c, cudaMemcpyAsync(c->scal_host, c->scal, sizeof(double) * Scal::N, cudaMemcpyDeviceToHost, c->stream));
    HMG_CUDA(c, cudaStreamSynchronize(c->stream));
    ++it;
    const double *h = c->scal_host;
    rel = std::sqrt(h[Scal::RR]) / bnorm;
    if (st && st->n_history < HMG_MAX_HISTORY) st->history[st->n_history++] = rel;
    if (rel > tol && (h[Scal::RV] == 0.0 || h[Scal::TT] == 0.0 || h[1 - par] == 0.0)) {
      status = HMG_ERR_BREAKDOWN;
      break;
    }
    if (!std::isfinite(rel) || !std::isfinite(h[Scal::ALPHA]) || !std::isfinite(h[Scal::OMEGA])) {
      status = HMG_ERR_NONFINITE;
      break;
    }
    if (rel > c->opt.divergence) { status = HMG_ERR_NOT_CONVERGED; break; }
  }
  // final FP64 residual ||B - S lambda|| recomputed from the iterate
  if ((s = launch_spmv(c, x, nullptr, 3, c->B, Scal::AUX, 0))) return s;
  HMG_CUDA(c, cudaEventRecord(e1, c->stream));
  HMG_CUDA(c, cudaMemcpyAsync(c->scal_host, c->scal, sizeof(double) * Scal::N, cudaMemcpyDeviceToHost, c->stream));
  HMG_CUDA(c, cudaStreamSynchronize(c->stream));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st) {
    for (int q = 0; q < HMG_NCOMP; ++q) { st->comp_ms[q] = 0.0; st->comp_calls[q] = 0; }
    for (const Ctx::Mark &m : c->marks) {
      float t = 0.f;
      if (cudaEventElapsedTime(&t, c->ev_pool[m.e0], c->ev_pool[m.e1]) == cudaSuccess) {
        st->comp_ms[m.comp] += t;
        st->comp_calls[m.comp] += m.launches;
      }
    }
    st->status = status;
    st->iterations = it;
    st->rel_residual = rel;
    st->true_rel_residual = bnorm > 0.0 ? std::sqrt(c->scal_host[Scal::AUX]) / bnorm : 0.0;
    st->solve_ms = ms;
  }
  if (status != HMG_OK) {
    const char *why = status == HMG_ERR_NOT_CONVERGED ? "BiCGStab did not converge"
                      : status == HMG_ERR_BREAKDOWN  ? "BiCGStab breakdown"
                                                     : "non-finite value in BiCGStab";
    return fail(c, status, why);
  }
  return HMG_OK;
}

}  // namespace hmg
