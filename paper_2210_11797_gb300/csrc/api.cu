// C ABI of the library (declared in include/hmg.h): validation of the caller's tables,
// upload of the mesh hierarchy and coefficients, allocation of the solver workspace, and
// the entry points of the solve.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "hmg_internal.cuh"

namespace hmg {

int fail(Ctx *c, int code, const std::string &msg) {
  if (c) c->err = msg;
  return code;
}

int cuda_fail(Ctx *c, cudaError_t e, const char *what) {
  return fail(c, HMG_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

template <typename T>
static int upload(Ctx *c, T **dst, const T *src, size_t n) {
  int st = dev_alloc(c, dst, n);
  if (st) return st;
  HMG_CUDA(c, cudaMemcpy(*dst, src, n * sizeof(T), cudaMemcpyHostToDevice));
  return HMG_OK;
}

static int check_options(Ctx *c, const hmg_options &o) {
  auto bad = [&](const char *m) { return fail(c, HMG_ERR_INVALID_ARG, std::string("options: ") + m); };
  if (o.precision != HMG_PRECISION_FP64 && o.precision != HMG_PRECISION_MIXED) return bad("precision");
  if (o.precond < HMG_PRECOND_NONE || o.precond > HMG_PRECOND_SCHUR) return bad("precond");
  if (o.precond == HMG_PRECOND_SCHUR && o.precision != HMG_PRECISION_FP64)
    return bad("configuration 1 (HMG_PRECOND_SCHUR) runs in FP64");
  if (o.n_pre < 0 || o.n_post < 0 || o.n_smooth < 1) return bad("trace smoother sweep counts");
  if (o.mg_npre < 1 || o.mg_npost < 1 || o.mg_ncoarse < 1) return bad("multigrid sweep counts must be >= 1");
  if (!std::isfinite(o.omega) || !std::isfinite(o.mg_omega)) return bad("relaxation factors");
  if (!(o.tol > 0.0) || o.max_iter < 0 || !(o.divergence > 0.0)) return bad("tol / max_iter / divergence");
  if (o.coarse < HMG_COARSE_VCYCLE || o.coarse > HMG_COARSE_KRYLOV_APPROX) return bad("coarse");
  if ((o.coarse == HMG_COARSE_KRYLOV_EXACT || o.coarse == HMG_COARSE_KRYLOV_APPROX) &&
      o.precision != HMG_PRECISION_FP64)
    return bad("the Krylov coarse solves (configurations 3a, 3b) run in FP64");
  if (o.krylov != HMG_KRYLOV_BICGSTAB && o.krylov != HMG_KRYLOV_FGMRES) return bad("krylov");
  if (o.restart < 1 || o.restart > 64) return bad("restart must be in 1..64");
  if (!(o.stall_ratio > 0.0)) return bad("stall_ratio");
  if (o.warm_start != 0 && o.warm_start != 1) return bad("warm_start must be 0 or 1");
  if (o.mg_fused != 0 && o.mg_fused != 1) return bad("mg_fused must be 0 or 1");
  if (o.mg_fuse_cells < 0) return bad("mg_fuse_cells must be >= 0");
  if (o.async_stats != 0 && o.async_stats != 1) return bad("async_stats must be 0 or 1");
  if (o.degree < 0 || o.degree > 3) return bad("degree must be in 0..3");
  if (o.degree >= 1 && (o.precond == HMG_PRECOND_SCHUR || o.coarse != HMG_COARSE_VCYCLE))
    return bad("degree p >= 1 runs with the trace preconditioners and the V-cycle coarse solve");
  return HMG_OK;
}

static int next_event(Ctx *c) {
  if (c->ev_next >= (int)c->ev_pool.size()) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return -1;
    c->ev_pool.push_back(e);
  }
  return c->ev_next++;
}

// NVTX range names of the components (the names of hmg_solve_stats.comp_ms)
static const char *const kCompNames[HMG_NCOMP] = {"trace_rhs", "trace_apply", "presmooth", "line_sweep",
                                                  "residual_restrict", "pressure_vcycle", "prolong",
                                                  "krylov_vectors"};

Prof::Prof(Ctx *c, int comp, int launches) : c_(c), comp_(comp), launches_(launches) {
  if (!c_->opt.profile) return;
  nvtxRangePushA(kCompNames[comp_]);   // visible to a profiler attached to the process
  e0_ = next_event(c_);
  if (e0_ >= 0) cudaEventRecord(c_->ev_pool[e0_], c_->stream);
}

Prof::~Prof() {
  if (!c_->opt.profile) return;
  nvtxRangePop();
  if (e0_ < 0) return;
  const int e1 = next_event(c_);
  if (e1 < 0) return;
  cudaEventRecord(c_->ev_pool[e1], c_->stream);
  c_->marks.push_back({comp_, e0_, e1, launches_});
}

static void free_all(Ctx *c) {
  drop_graph(c);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  c->cap_stream = nullptr;
  for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
  c->ev_pool.clear();
  for (void *p : c->owned) cudaFree(p);
  c->owned.clear();
  if (c->scal_host) cudaFreeHost(c->scal_host);
  c->scal_host = nullptr;
  if (c->state_host) cudaFreeHost(c->state_host);
  c->state_host = nullptr;
  if (c->hist_host) cudaFreeHost(c->hist_host);
  c->hist_host = nullptr;
  if (c->as_e0) cudaEventDestroy(c->as_e0);
  if (c->as_e1) cudaEventDestroy(c->as_e1);
  c->as_e0 = c->as_e1 = nullptr;
  if (c->loop_done) cudaEventDestroy(c->loop_done);
  if (c->copy_done) cudaEventDestroy(c->copy_done);
  c->loop_done = c->copy_done = nullptr;
  if (c->copy_stream) cudaStreamDestroy(c->copy_stream);
  c->copy_stream = nullptr;
}

}  // namespace hmg

using namespace hmg;

extern "C" {

int hmg_default_options(hmg_options *o) {
  if (!o) return HMG_ERR_INVALID_ARG;
  std::memset(o, 0, sizeof(*o));
  o->precision = HMG_PRECISION_FP64;
  o->precond = HMG_PRECOND_NONNESTED;
  o->n_pre = 1;
  o->n_post = 2;
  o->n_smooth = 1;
  o->omega = 0.6;
  o->mg_npre = 1;
  o->mg_npost = 2;
  o->mg_ncoarse = 3;
  o->mg_omega = 0.9;
  o->tol = 1e-6;
  o->max_iter = 200;
  o->divergence = 1e8;
  o->profile = 0;
  o->graph = 1;
  o->coarse = HMG_COARSE_VCYCLE;
  o->krylov = HMG_KRYLOV_BICGSTAB;
  o->restart = 30;
  o->stall_ratio = 0.9;
  o->mg_fused = 0;
  o->mg_fuse_cells = 1 << 18;
  return HMG_OK;
}

int hmg_create(hmg_ctx **out, const hmg_options *opt, void *cuda_stream) {
  if (!out) return HMG_ERR_INVALID_ARG;
  *out = nullptr;
  hmg_ctx *c = new (std::nothrow) hmg_ctx();
  if (!c) return HMG_ERR_OUT_OF_MEMORY;
  hmg_default_options(&c->opt);
  if (opt) {
    int st = check_options(c, *opt);
    if (st) { delete c; return st; }
    c->opt = *opt;
  }
  c->stream = static_cast<cudaStream_t>(cuda_stream);
  cudaError_t e = cudaGetDevice(&c->device);
  if (e == cudaSuccess) e = cudaMallocHost(&c->scal_host, sizeof(double) * Scal::N);
  if (e == cudaSuccess) e = cudaMallocHost(&c->state_host, sizeof(int) * 4);
  if (e == cudaSuccess) e = cudaMallocHost(&c->hist_host, sizeof(double) * HMG_MAX_HISTORY);
  if (e == cudaSuccess) e = cudaEventCreate(&c->as_e0);
  if (e == cudaSuccess) e = cudaEventCreate(&c->as_e1);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->loop_done, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->copy_done, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    free_all(c);
    delete c;
    return HMG_ERR_CUDA;
  }
  int st = dev_alloc(c, &c->scal, Scal::N);
  if (!st) st = dev_alloc(c, &c->state, 4);
  if (!st) st = dev_alloc(c, &c->hist, HMG_MAX_HISTORY);
  if (!st) st = dev_alloc(c, &c->part, (size_t)Scal::N * kMaxRedBlocks);
  if (!st) st = dev_alloc(c, &c->counter, Scal::N);
  if (!st) st = dev_alloc(c, &c->mg_bar, 64);
  if (!st && cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess)
    st = HMG_ERR_CUDA;
  if (!st && cudaMemset(c->counter, 0, sizeof(unsigned int) * Scal::N) != cudaSuccess) st = HMG_ERR_CUDA;
  if (!st && cudaMemset(c->scal, 0, sizeof(double) * Scal::N) != cudaSuccess) st = HMG_ERR_CUDA;
  if (!st && cudaMemset(c->state, 0, sizeof(int) * 4) != cudaSuccess) st = HMG_ERR_CUDA;
  if (st) {
    free_all(c);
    delete c;
    return st;
  }
  *out = c;
  return HMG_OK;
}

int hmg_set_options(hmg_ctx *c, const hmg_options *opt) {
  if (!c || !opt) return HMG_ERR_INVALID_ARG;
  int st = check_options(c, *opt);
  if (st) return st;
  c->opt = *opt;
  if (c->assembled && c->opt.degree != c->degree) c->assembled = false;   // a new discretisation
  if (c->assembled && c->opt.precision == HMG_PRECISION_MIXED && !c->have_fp32) {
    // the FP32 copies from the assembled FP64 operators (the degree-p ones below)
    HMG_CUDA(c, cudaSetDevice(c->device));
    if ((st = make_fp32(c))) return st;
    HMG_CUDA(c, cudaStreamSynchronize(c->stream));
  }
  if (c->assembled && (c->opt.omega != c->factor_omega || c->opt.mg_omega != c->factor_mg_omega)) {
    HMG_CUDA(c, cudaSetDevice(c->device));
    if ((st = build_factors(c))) return st;
    HMG_CUDA(c, cudaStreamSynchronize(c->stream));
  }
  if (c->assembled && c->degree >= 1) {   // (outside any stream capture: the solve graph replays them)
    HMG_CUDA(c, cudaSetDevice(c->device));
    if ((st = ho_refactor_if_needed(c))) return st;
  }
  return HMG_OK;
}

int hmg_set_mesh(hmg_ctx *c, int32_t nmg, const hmg_mesh_level *levels) {
  if (!c) return HMG_ERR_INVALID_ARG;
  if (c->have_mesh) return fail(c, HMG_ERR_INVALID_ARG, "mesh already set (create a new context)");
  if (nmg < 1 || nmg > kMaxLevels || !levels) return fail(c, HMG_ERR_INVALID_ARG, "nmg out of range");
  HMG_CUDA(c, cudaSetDevice(c->device));
  const int L = levels[0].nlev;
  std::vector<std::vector<int32_t>> children(nmg);
  for (int l = 0; l < nmg; ++l) {
    const hmg_mesh_level &m = levels[l];
    char buf[160];
    auto bad = [&](const char *what) {
      std::snprintf(buf, sizeof buf, "mesh level %d: %s", l, what);
      return fail(c, HMG_ERR_INVALID_ARG, buf);
    };
    if (m.ncol < 1 || m.nlev < 1 || m.nedge < 1) return bad("empty mesh");
    // one column's three Thomas arrays (FP64, L + 1 rows) must fit a block's 48 KB of shared memory
    if (m.nlev > kMaxLayers) return bad("more than 2045 layers");
    if (m.nlev != L) return bad("every level needs the same nlev");
    if (m.geometry != 0 && m.geometry != 1) return bad("geometry must be 0 or 1");
    if (m.geometry == 1 && !(m.radius > 0.0)) return bad("radius must be > 0");
    if (!m.corners || !m.z_levels || !m.col_edges || !m.edge_cols || !m.edge_face) return bad("null table");
    if ((int64_t)m.nedge * 2 != (int64_t)m.ncol * 4) return bad("every column needs 4 edges shared by 2 columns");
    if ((int64_t)m.nedge * m.nlev + (int64_t)m.ncol * (m.nlev + 1) > INT32_MAX / kSlots)
      return bad("mesh too large for 32-bit slot offsets");
    for (int k = 0; k < m.nlev; ++k)
      if (!(m.z_levels[k + 1] > m.z_levels[k])) return bad("z_levels must increase strictly");
    for (int64_t i = 0; i < (int64_t)m.ncol * 4; ++i)
      if (m.col_edges[i] < 0 || m.col_edges[i] >= m.nedge) return bad("col_edges out of range");
    for (int64_t e = 0; e < m.nedge; ++e) {
      for (int s = 0; s < 2; ++s) {
        const int cc = m.edge_cols[2 * e + s], f = m.edge_face[2 * e + s];
        if (cc < 0 || cc >= m.ncol || f < 0 || f > 3) return bad("edge_cols / edge_face out of range");
        if (m.col_edges[4 * (int64_t)cc + f] != e) return bad("col_edges and edge_cols disagree");
      }
      if (m.edge_cols[2 * e] == m.edge_cols[2 * e + 1]) return bad("an edge joins a column to itself");
    }
    if (l + 1 < nmg) {
      if (!m.parent) return bad("parent map missing");
      const int nc = levels[l + 1].ncol;
      std::vector<int32_t> ch((size_t)nc * 4, -1), cnt(nc, 0);
      for (int cc = 0; cc < m.ncol; ++cc) {
        const int p = m.parent[cc];
        if (p < 0 || p >= nc || cnt[p] >= 4) return bad("parent map is not a 2x2 agglomeration");
        ch[4 * (size_t)p + cnt[p]++] = cc;
      }
      for (int p = 0; p < nc; ++p)
        if (cnt[p] != 4) return bad("a coarse column does not have four children");
      children[l + 1] = ch;
    }
  }
  for (int l = 0; l < nmg; ++l) {
    const hmg_mesh_level &m = levels[l];
    Level &lv = c->lv[l];
    lv.geometry = m.geometry;
    lv.ncol = m.ncol;
    lv.nlev = m.nlev;
    lv.nedge = m.nedge;
    lv.radius = m.radius;
    lv.ncell = (int64_t)m.ncol * m.nlev;
    lv.nth = (int64_t)m.nedge * m.nlev;
    lv.ntz = (int64_t)m.ncol * (m.nlev + 1);
    lv.ntrace = lv.nth + lv.ntz;
    std::vector<int32_t> nbr((size_t)m.ncol * 4), nbf((size_t)m.ncol * 4);
    for (int cc = 0; cc < m.ncol; ++cc)
      for (int f = 0; f < 4; ++f) {
        const int e = m.col_edges[4 * (size_t)cc + f];
        const bool first = m.edge_cols[2 * (size_t)e] == cc && m.edge_face[2 * (size_t)e] == f;
        nbr[4 * (size_t)cc + f] = m.edge_cols[2 * (size_t)e + (first ? 1 : 0)];
        nbf[4 * (size_t)cc + f] = m.edge_face[2 * (size_t)e + (first ? 1 : 0)];
      }
    int st;
    if ((st = upload(c, &lv.col_edges, m.col_edges, (size_t)m.ncol * 4))) return st;
    if ((st = upload(c, &lv.col_nbr, nbr.data(), nbr.size()))) return st;
    if ((st = upload(c, &lv.col_nbr_face, nbf.data(), nbf.size()))) return st;
    if ((st = upload(c, &lv.corners, m.corners, (size_t)m.ncol * 12))) return st;
    if ((st = upload(c, &lv.z, m.z_levels, (size_t)m.nlev + 1))) return st;
    if (l + 1 < nmg && (st = upload(c, &lv.parent, m.parent, (size_t)m.ncol))) return st;
    if (l > 0 && (st = upload(c, &lv.children, children[l].data(), children[l].size()))) return st;
    if (l == 0) {
      std::vector<int32_t> sten((size_t)m.nedge * 8), fc((size_t)m.nedge * 2);
      for (int64_t e = 0; e < m.nedge; ++e) {
        const int c1 = m.edge_cols[2 * e], c2 = m.edge_cols[2 * e + 1];
        const int i1 = m.edge_face[2 * e], i2 = m.edge_face[2 * e + 1];
        int32_t *s = &sten[8 * e];
        s[0] = c1;
        s[1] = c2;
        for (int q = 1; q <= 3; ++q) {
          s[1 + q] = m.col_edges[4 * (size_t)c1 + ((i1 + q) & 3)];
          s[4 + q] = m.col_edges[4 * (size_t)c2 + ((i2 + q) & 3)];
        }
        fc[2 * e] = i1;
        fc[2 * e + 1] = i2;
      }
      if ((st = upload(c, &lv.edge_stencil, sten.data(), sten.size()))) return st;
      if ((st = upload(c, &lv.edge_fc, fc.data(), fc.size()))) return st;
    }
    double *tmp;
    if ((st = dev_alloc(c, &tmp, (size_t)lv.ncell))) return st;
    lv.vb = tmp;
    if ((st = dev_alloc(c, &tmp, (size_t)lv.ncell))) return st;
    lv.vx = tmp;
    if ((st = dev_alloc(c, &tmp, (size_t)lv.ncell))) return st;
    lv.vy = tmp;
  }
  c->nmg = nmg;
  c->have_mesh = true;
  return HMG_OK;
}

int hmg_set_coefficients(hmg_ctx *c, const hmg_scalars *sc, const hmg_background *levels) {
  if (!c || !sc || !levels) return HMG_ERR_INVALID_ARG;
  if (!c->have_mesh) return fail(c, HMG_ERR_NOT_READY, "set the mesh first");
  if (sc->preset != 0 && sc->preset != 1) return fail(c, HMG_ERR_INVALID_ARG, "preset must be 0 or 1");
  if (sc->preset == 1 && !(sc->sigma >= 0.0)) return fail(c, HMG_ERR_INVALID_ARG, "sigma must be >= 0");
  if (!std::isfinite(sc->omega)) return fail(c, HMG_ERR_INVALID_ARG, "omega must be finite");
  if (sc->preset == 0 && !(sc->dt > 0.0 && sc->cp > 0.0 && sc->kappa > 0.0 && sc->kappa < 1.0))
    return fail(c, HMG_ERR_INVALID_ARG, "dt, cp > 0 and 0 < kappa < 1 required");
  HMG_CUDA(c, cudaSetDevice(c->device));
  for (int l = 0; l < c->nmg; ++l) {
    Level &lv = c->lv[l];
    const hmg_background &b = levels[l];
    if (!b.theta_lev || !b.exner_lev || !b.exner) return fail(c, HMG_ERR_INVALID_ARG, "null background");
    const size_t nl = (size_t)lv.ncol * (lv.nlev + 1);
    for (size_t i = 0; i < nl; ++i)
      if (!(b.theta_lev[i] > 0.0) || !(b.exner_lev[i] > 0.0))
        return fail(c, HMG_ERR_INVALID_ARG, "theta* and Exner* must be positive");
    for (int64_t i = 0; i < lv.ncell; ++i)
      if (!(b.exner[i] > 0.0)) return fail(c, HMG_ERR_INVALID_ARG, "Exner* must be positive");
    int st;
    if (lv.theta_lev) {
      HMG_CUDA(c, cudaMemcpy(lv.theta_lev, b.theta_lev, nl * 8, cudaMemcpyHostToDevice));
      HMG_CUDA(c, cudaMemcpy(lv.exner_lev, b.exner_lev, nl * 8, cudaMemcpyHostToDevice));
      HMG_CUDA(c, cudaMemcpy(lv.exner, b.exner, (size_t)lv.ncell * 8, cudaMemcpyHostToDevice));
    } else {
      if ((st = upload(c, &lv.theta_lev, b.theta_lev, nl))) return st;
      if ((st = upload(c, &lv.exner_lev, b.exner_lev, nl))) return st;
      if ((st = upload(c, &lv.exner, b.exner, (size_t)lv.ncell))) return st;
    }
  }
  c->sc = *sc;
  c->have_coeffs = true;
  c->assembled = false;
  c->have_fp32 = false;
  return HMG_OK;
}

int hmg_assemble_trace(hmg_ctx *c) {
  if (!c) return HMG_ERR_INVALID_ARG;
  HMG_CUDA(c, cudaSetDevice(c->device));
  const bool need_fp32 = c->opt.precision == HMG_PRECISION_MIXED;
  if (c->have_fp32 && need_fp32) c->have_fp32 = false;  // rebuild copies from fresh FP64 data
  int st = assemble_all(c);
  if (st) return st;
  const Level &f = c->lv[0];
  const int64_t T = f.ntrace, C = f.ncell;
  const int64_t T1 = c->opt.degree >= 1 ? ho_trace_size(c, c->opt.degree) : 0;
  // Krylov vectors long enough for the 2x2 system of configuration 1 ([u | Pi]) and for the
  // degree-p trace system; work vectors for the longer trace system; the host-copy staging area
  // for the cell residuals and lambda of either degree
  const int64_t nvec = std::max(T + C, T1), nwork = std::max(T, T1);
  const int64_t nhost = std::max(7 * C + T, T1 ? (int64_t)(cell_nu_of(c->opt.degree) + cell_np_of(c->opt.degree)) * C + T1 : 0);
  if (c->vec_cap < nvec) {
    double **vecs[] = {&c->B, &c->r, &c->rhat, &c->p, &c->v, &c->s, &c->t, &c->phat, &c->shat};
    for (double **v : vecs) {
      dev_free(c, *v);
      *v = nullptr;
      if ((st = dev_alloc(c, v, (size_t)nvec))) return st;
    }
    c->vec_cap = nvec;
    drop_graph(c);   // a cached solve graph holds the old vectors
  }
  if (c->work_cap < nwork) {
    void **ws[] = {&c->w1, &c->w2, &c->w3};
    for (void **w : ws) {
      dev_free(c, *w);
      double *tmp = nullptr;
      if ((st = dev_alloc(c, &tmp, (size_t)nwork))) return st;
      *w = tmp;
    }
    c->work_cap = nwork;
    drop_graph(c);
  }
  if (!c->cb) {
    double *tmp;
    if ((st = dev_alloc(c, &tmp, (size_t)C))) return st;
    c->cb = tmp;
  }
  if (c->host_cap < nhost) {
    dev_free(c, c->host_in);
    c->host_in = nullptr;
    if ((st = dev_alloc(c, &c->host_in, (size_t)nhost))) return st;
    c->host_cap = nhost;
  }
  c->degree = c->opt.degree;
  if (c->degree >= 1 && (st = ho_assemble(c))) {
    c->degree = 0;
    ho_free(c);
    return st;
  }
  if (c->degree == 0 && c->ho.degree != 0) ho_free(c);   // the degree-p system is no longer in use
  if (!c->noalloc_scratch && (st = noalloc_setup(c))) return st;
  c->assembled = true;
  return HMG_OK;
}

int hmg_sizes(const hmg_ctx *c, int64_t *ncell, int64_t *ntrace) {
  if (!c) return HMG_ERR_INVALID_ARG;
  if (!c->have_mesh) return HMG_ERR_NOT_READY;
  if (ncell) *ncell = c->lv[0].ncell;
  if (ntrace) *ntrace = c->assembled && c->degree >= 1 ? c->ho.T : c->lv[0].ntrace;
  return HMG_OK;
}

void hmg_destroy(hmg_ctx *c) {
  if (!c) return;
  cudaSetDevice(c->device);
  if (c->stream) cudaStreamSynchronize(c->stream); else cudaDeviceSynchronize();
  free_all(c);
  delete c;
}

const char *hmg_status_string(int s) {
  switch (s) {
    case HMG_OK: return "ok";
    case HMG_ERR_INVALID_ARG: return "invalid argument";
    case HMG_ERR_CUDA: return "CUDA error";
    case HMG_ERR_NOT_READY: return "not ready (mesh, coefficients or assembly missing)";
    case HMG_ERR_NOT_CONVERGED: return "not converged";
    case HMG_ERR_BREAKDOWN: return "Krylov breakdown";
    case HMG_ERR_NONFINITE: return "non-finite value";
    case HMG_ERR_TIMEOUT: return "device wait timed out";
    case HMG_ERR_OUT_OF_MEMORY: return "out of device memory";
    default: return "unknown status";
  }
}

const char *hmg_last_error(const hmg_ctx *c) { return c ? c->err.c_str() : "null context"; }

static int ready(hmg_ctx *c) {
  if (!c) return HMG_ERR_INVALID_ARG;
  if (!c->assembled) return fail(c, HMG_ERR_NOT_READY, "call hmg_assemble_trace first");
  HMG_CUDA(c, cudaSetDevice(c->device));
  return HMG_OK;
}

// A kernel whose bounded wait (a tensor-core mbarrier, the grid barrier of the cooperative
// multigrid kernel) ran out sets state[3]; the context stays usable.
static int check_wait_flag(hmg_ctx *c) {
  int flag = 0;
  HMG_CUDA(c, cudaMemcpy(&flag, c->state + 3, sizeof(int), cudaMemcpyDeviceToHost));
  if (!flag) return HMG_OK;
  HMG_CUDA(c, cudaMemset(c->state + 3, 0, sizeof(int)));
  return fail(c, HMG_ERR_TIMEOUT, "a bounded device-side wait ran out");
}

static int finish(hmg_ctx *c, int st) {
  if (st) return st;
  HMG_CUDA(c, cudaStreamSynchronize(c->stream));
  return HMG_OK;
}

int hmg_trace_rhs(hmg_ctx *c, const double *Rub, const double *Rpi, double *B) {
  int st = ready(c);
  if (st) return st;
  if (!Rub || !Rpi || !B) return fail(c, HMG_ERR_INVALID_ARG, "null pointer");
  if (c->degree >= 1) return finish(c, ho_trace_rhs(c, Rub, Rpi, B));
  return finish(c, launch_trace_rhs(c, Rub, Rpi, B));
}

static int reject_schur(hmg_ctx *c) {
  return mixed_system(c) ? fail(c, HMG_ERR_INVALID_ARG, "configuration 1 solves the 2x2 system: use hmg_solve_mixed")
                         : HMG_OK;
}

int hmg_solve(hmg_ctx *c, const double *Rub, const double *Rpi, double *lambda, hmg_solve_stats *stats) {
  int st = ready(c);
  if (st) return st;
  if (!Rub || !Rpi || !lambda) return fail(c, HMG_ERR_INVALID_ARG, "null pointer");
  if ((st = reject_schur(c))) return st;
  return krylov_solve(c, Rub, Rpi, lambda, stats, true);
}

int hmg_solve_stats_get(hmg_ctx *c, hmg_solve_stats *stats) {
  if (!c) return HMG_ERR_INVALID_ARG;
  return solve_stats_get(c, stats);
}

int hmg_solve_mixed(hmg_ctx *c, const double *Rub, const double *Rpi, double *u, double *pi, hmg_solve_stats *stats) {
  int st = ready(c);
  if (st) return st;
  if (!Rub || !Rpi || !u || !pi) return fail(c, HMG_ERR_INVALID_ARG, "null pointer");
  if (!mixed_system(c) || !c->have_mixed)
    return fail(c, HMG_ERR_NOT_READY, "configuration 1 needs precond = HMG_PRECOND_SCHUR before hmg_assemble_trace");
  const int solve_st = krylov_solve(c, Rub, Rpi, c->mx_x, stats, false);
  if (solve_st != HMG_OK && solve_st != HMG_ERR_NOT_CONVERGED && solve_st != HMG_ERR_BREAKDOWN &&
      solve_st != HMG_ERR_NONFINITE && solve_st != HMG_ERR_TIMEOUT)
    return solve_st;
  const Level &f = c->lv[0];
  HMG_CUDA(c, cudaMemcpyAsync(u, c->mx_x, sizeof(double) * f.ntrace, cudaMemcpyDeviceToDevice, c->stream));
  HMG_CUDA(c, cudaMemcpyAsync(pi, c->mx_x + f.ntrace, sizeof(double) * f.ncell, cudaMemcpyDeviceToDevice, c->stream));
  HMG_CUDA(c, cudaStreamSynchronize(c->stream));
  return solve_st;
}

int hmg_apply_mixed(hmg_ctx *c, const double *x, double *y) {
  int st = ready(c);
  if (st) return st;
  if (!x || !y || x == y) return fail(c, HMG_ERR_INVALID_ARG, "bad pointers");
  return finish(c, launch_mixed_apply(c, x, y, 0, nullptr, 0, 0));
}

int hmg_solve_host(hmg_ctx *c, const double *Rub, const double *Rpi, double *lambda, hmg_solve_stats *stats) {
  int st = ready(c);
  if (st) return st;
  if (!Rub || !Rpi || !lambda) return fail(c, HMG_ERR_INVALID_ARG, "null pointer");
  if ((st = reject_schur(c))) return st;
  const Level &f = c->lv[0];
  const int64_t nu = cell_nu(c), np = cell_np(c);
  double *dRub = c->host_in, *dRpi = dRub + nu * f.ncell, *dlam = dRpi + np * f.ncell;
  HMG_CUDA(c, cudaMemcpyAsync(dRub, Rub, sizeof(double) * nu * f.ncell, cudaMemcpyHostToDevice, c->stream));
  HMG_CUDA(c, cudaMemcpyAsync(dRpi, Rpi, sizeof(double) * np * f.ncell, cudaMemcpyHostToDevice, c->stream));
  if (c->opt.warm_start)   // the initial lambda comes from the host buffer too
    HMG_CUDA(c, cudaMemcpyAsync(dlam, lambda, sizeof(double) * sys_n(c), cudaMemcpyHostToDevice, c->stream));
  // lambda comes back to the host behind the solve, under the same synchronisation
  return krylov_solve(c, dRub, dRpi, dlam, stats, false, lambda);
}

int hmg_reconstruct(hmg_ctx *c, const double *lambda, const double *Rub, const double *Rpi, double *ub, double *pi) {
  int st = ready(c);
  if (st) return st;
  if (!lambda || !Rub || !Rpi || !ub || !pi) return fail(c, HMG_ERR_INVALID_ARG, "null pointer");
  if (c->degree >= 1) return finish(c, ho_reconstruct(c, lambda, Rub, Rpi, ub, pi));
  return finish(c, launch_reconstruct(c, lambda, Rub, Rpi, ub, pi));
}

int hmg_apply_trace(hmg_ctx *c, const double *x, double *y) {
  int st = ready(c);
  if (st) return st;
  if (!x || !y || x == y) return fail(c, HMG_ERR_INVALID_ARG, "bad pointers");
  if (c->degree >= 1) return finish(c, ho_launch_spmv(c, x, y, 0, nullptr, 0, 0));
  return finish(c, launch_spmv(c, x, y, 0, nullptr, 0, 0));
}

int hmg_precond_apply(hmg_ctx *c, const double *r, double *z) {
  int st = ready(c);
  if (st) return st;
  if (!r || !z || r == z) return fail(c, HMG_ERR_INVALID_ARG, "bad pointers");
  if ((st = finish(c, precond_apply(c, r, z)))) return st;
  return check_wait_flag(c);
}

int hmg_line_smooth(hmg_ctx *c, const double *b, double *lambda, int32_t nsweeps) {
  int st = ready(c);
  if (st) return st;
  if (!b || !lambda || nsweeps < 0) return fail(c, HMG_ERR_INVALID_ARG, "bad arguments");
  if (c->degree >= 1) return finish(c, ho_line_smooth(c, b, lambda, nsweeps));
  return finish(c, line_smooth_fp64(c, b, lambda, nsweeps));
}

int hmg_apply_pressure(hmg_ctx *c, int32_t level, const double *x, double *y) {
  int st = ready(c);
  if (st) return st;
  if (level < 0 || level >= c->nmg || !x || !y || x == y) return fail(c, HMG_ERR_INVALID_ARG, "bad arguments");
  return finish(c, apply_pressure_fp64(c, level, x, y));
}

int hmg_pressure_vcycle(hmg_ctx *c, const double *b, double *x) {
  int st = ready(c);
  if (st) return st;
  if (!b || !x) return fail(c, HMG_ERR_INVALID_ARG, "bad pointers");
  if ((st = finish(c, pressure_vcycle_fp64(c, b, x)))) return st;
  return check_wait_flag(c);
}

int hmg_get_gamma(hmg_ctx *c, double *gamma) {
  int st = ready(c);
  if (st) return st;
  if (!gamma) return fail(c, HMG_ERR_INVALID_ARG, "null pointer");
  HMG_CUDA(c, cudaMemcpyAsync(gamma, c->degree >= 1 ? c->ho.gamma : c->gamma, sizeof(double) * c->lv[0].ncell,
                              cudaMemcpyDeviceToDevice, c->stream));
  return finish(c, HMG_OK);
}

int hmg_solve_batched(hmg_ctx *const *ctxs, int32_t n, const double *const *Rub,
                      const double *const *Rpi, double *const *lambda, hmg_solve_stats *stats) {
  if (!ctxs || n < 1 || !Rub || !Rpi || !lambda) return HMG_ERR_INVALID_ARG;
  hmg_ctx *c0 = ctxs[0];
  if (!c0) return HMG_ERR_INVALID_ARG;
  for (int i = 0; i < n; ++i) {
    hmg_ctx *c = ctxs[i];
    if (!c) return fail(c0, HMG_ERR_INVALID_ARG, "null context in the batch");
    if (!c->assembled) return fail(c0, HMG_ERR_NOT_READY, "a context of the batch is not assembled");
    if (c->device != c0->device) return fail(c0, HMG_ERR_INVALID_ARG, "batched contexts must share a device");
    if (!Rub[i] || !Rpi[i] || !lambda[i]) return fail(c0, HMG_ERR_INVALID_ARG, "null pointer in the batch");
    if (mixed_system(c)) return fail(c0, HMG_ERR_INVALID_ARG, "batched solves are hybridised solves");
    if (c->degree != 0) return fail(c0, HMG_ERR_INVALID_ARG, "batched solves are degree 0");
    for (int j = 0; j < i; ++j)
      if (ctxs[j] == c) return fail(c0, HMG_ERR_INVALID_ARG, "a context appears twice in the batch");
  }
  HMG_CUDA(c0, cudaSetDevice(c0->device));
  // the batch graph reads inputs that may have been written on the contexts' own streams
  for (int i = 0; i < n; ++i) HMG_CUDA(c0, cudaStreamSynchronize(ctxs[i]->stream));
  return krylov_solve_batched(ctxs, n, Rub, Rpi, lambda, stats);
}

int hmg_autotune(hmg_ctx *c) {
  int st = ready(c);
  if (st) return st;
  drop_graph(c);   // captured launches carry the old shapes
  return finish(c, autotune(c));
}

int hmg_get_launch_shapes(hmg_ctx *c, int32_t *sweep, int32_t *mg, int32_t nmg) {
  if (!c || !sweep || (nmg > 0 && !mg)) return HMG_ERR_INVALID_ARG;
  if (!c->have_mesh || nmg != c->nmg) return fail(c, HMG_ERR_INVALID_ARG, "nmg must equal the mesh's levels");
  // the shapes of the preconditioner's kernels: FP32 ones under precision mixed, else FP64
  const int p = c->opt.precision == HMG_PRECISION_MIXED ? 1 : 0;
  sweep[0] = c->tune_sweep_cpb[p];
  sweep[1] = c->tune_sweep_threads[p];
  for (int l = 0; l < nmg; ++l) {
    mg[2 * l] = c->tune_mg_cpb[p][l];
    mg[2 * l + 1] = c->tune_mg_threads[p][l];
  }
  return HMG_OK;
}

int hmg_set_launch_shapes(hmg_ctx *c, const int32_t *sweep, const int32_t *mg, int32_t nmg) {
  if (!c || !sweep || (nmg > 0 && !mg)) return HMG_ERR_INVALID_ARG;
  if (!c->have_mesh || nmg != c->nmg) return fail(c, HMG_ERR_INVALID_ARG, "nmg must equal the mesh's levels");
  auto ok = [](int32_t cpb, int32_t thr) { return cpb >= 0 && cpb <= 64 && (thr == 0 || thr == 128 || thr == 256); };
  if (!ok(sweep[0], sweep[1]) && !(sweep[0] == -1 && c->lv[0].nlev + 1 <= 128))
    return fail(c, HMG_ERR_INVALID_ARG, "bad sweep launch shape");
  for (int l = 0; l < nmg; ++l)
    if (!ok(mg[2 * l], mg[2 * l + 1]) && !(mg[2 * l] == -1 && c->lv[l].nlev <= 128))
      return fail(c, HMG_ERR_INVALID_ARG, "bad smoother launch shape");
  drop_graph(c);   // captured launches carry the old shapes
  for (int p = 0; p < 2; ++p) {   // the same shapes for the FP64 and FP32 kernels (-1: FP32 only)
    c->tune_sweep_cpb[p] = sweep[0] == -1 ? (p == 1 ? -1 : 0) : sweep[0];
    c->tune_sweep_threads[p] = sweep[0] == -1 ? 0 : sweep[1];
  }
  for (int l = 0; l < nmg; ++l) {
    for (int p = 0; p < 2; ++p) {   // -1: the warp-per-column form for both precisions
      c->tune_mg_cpb[p][l] = mg[2 * l];
      c->tune_mg_threads[p][l] = mg[2 * l] == -1 ? 0 : mg[2 * l + 1];
    }
  }
  return HMG_OK;
}

int hmg_get_trace_operator(hmg_ctx *c, double *slots) {
  int st = ready(c);
  if (st) return st;
  if (!slots) return fail(c, HMG_ERR_INVALID_ARG, "null pointer");
  if (c->degree != 0) return fail(c, HMG_ERR_INVALID_ARG, "the slot layout is that of degree 0");
  HMG_CUDA(c, cudaMemcpyAsync(slots, c->S, sizeof(double) * kSlots * c->lv[0].ntrace,
                              cudaMemcpyDeviceToDevice, c->stream));
  return finish(c, HMG_OK);
}

// ---- learned coarse correction -------------------------------------------------------------

static int mesh_ready(hmg_ctx *c) {
  if (!c) return HMG_ERR_INVALID_ARG;
  if (!c->have_mesh) return fail(c, HMG_ERR_NOT_READY, "call hmg_set_mesh first");
  HMG_CUDA(c, cudaSetDevice(c->device));
  return HMG_OK;
}

int32_t hmg_coarse_model_size(void) { return kCoarseParams; }

int hmg_check_device_wait(hmg_ctx *c, int32_t polls) {
  if (!c) return HMG_ERR_INVALID_ARG;
  if (polls < 1 || polls > (1 << 24)) return fail(c, HMG_ERR_INVALID_ARG, "polls must be in 1..2^24");
  HMG_CUDA(c, cudaSetDevice(c->device));
  int st = wait_selftest(c, (uint32_t)polls);
  if (st) return st;
  return check_wait_flag(c);
}

int hmg_set_coarse_model(hmg_ctx *c, const float *params, int32_t n) {
  int st = mesh_ready(c);
  if (st) return st;
  if (!params || n != kCoarseParams) return fail(c, HMG_ERR_INVALID_ARG, "params must hold hmg_coarse_model_size() floats");
  if ((st = nn_setup(c))) return st;
  HMG_CUDA(c, cudaMemcpyAsync(c->nn_w, params, sizeof(float) * kCoarseParams, cudaMemcpyHostToDevice, c->stream));
  if ((st = nn_pack_weights(c))) return st;
  return finish(c, HMG_OK);
}

int hmg_get_coarse_model(hmg_ctx *c, float *params, int32_t n) {
  int st = mesh_ready(c);
  if (st) return st;
  if (!params || n != kCoarseParams) return fail(c, HMG_ERR_INVALID_ARG, "params must hold hmg_coarse_model_size() floats");
  if (!c->nn_w) return fail(c, HMG_ERR_NOT_READY, "no coarse model set");
  HMG_CUDA(c, cudaMemcpyAsync(params, c->nn_w, sizeof(float) * kCoarseParams, cudaMemcpyDeviceToHost, c->stream));
  return finish(c, HMG_OK);
}

int hmg_apply_coarse_model(hmg_ctx *c, const double *bbar, double *out, int32_t mode) {
  int st = ready(c);
  if (st) return st;
  if (!bbar || !out || bbar == out || mode < 0 || mode > 2) return fail(c, HMG_ERR_INVALID_ARG, "bad arguments");
  if (!c->nn_w) return fail(c, HMG_ERR_NOT_READY, "no coarse model set");
  if ((st = finish(c, apply_coarse_model(c, bbar, out, mode)))) return st;
  st = check_wait_flag(c);
  if (st == HMG_ERR_TIMEOUT && mode == 0 && !c->nn_tc_off) {   // see hmg_apply_coarse_model
    drop_graph(c);   // captured solve graphs hold the tensor-core launches
    c->nn_tc_off = true;
  }
  return st;
}

static int check_patches(hmg_ctx *c, const float *x, const float *t, int32_t nsamp, int32_t nx, int32_t ny) {
  if (!x || !t) return fail(c, HMG_ERR_INVALID_ARG, "null pointer");
  if (nsamp < 1 || nx < 1 || ny < 1 || (int64_t)nsamp * nx * ny > (1 << 26))
    return fail(c, HMG_ERR_INVALID_ARG, "bad patch batch shape");
  if (!c->nn_w) return fail(c, HMG_ERR_NOT_READY, "no coarse model set");
  return HMG_OK;
}

int hmg_coarse_model_grad(hmg_ctx *c, const float *x, const float *t, int32_t nsamp, int32_t nx, int32_t ny,
                          int32_t fp32, float *grad, double *loss) {
  int st = mesh_ready(c);
  if (st) return st;
  if ((st = check_patches(c, x, t, nsamp, nx, ny))) return st;
  if (!grad || !loss) return fail(c, HMG_ERR_INVALID_ARG, "null pointer");
  return coarse_model_grad(c, x, t, nsamp, nx, ny, fp32 ? 1 : 0, grad, loss);
}

int hmg_train_coarse_model(hmg_ctx *c, const float *x, const float *t, int32_t nsamp, int32_t nx, int32_t ny,
                           int32_t batch, int32_t epochs, double lr, uint64_t seed, double *loss_hist) {
  int st = mesh_ready(c);
  if (st) return st;
  if ((st = check_patches(c, x, t, nsamp, nx, ny))) return st;
  if (batch < 1 || batch > nsamp || epochs < 0 || !(lr > 0.0)) return fail(c, HMG_ERR_INVALID_ARG, "bad training settings");
  return train_coarse_model(c, x, t, nsamp, nx, ny, batch, epochs, lr, seed, loss_hist);
}

int hmg_adam_step(hmg_ctx *c, float *w, const float *grad, float *m, float *v, int32_t n, int32_t step,
                  double lr, double beta1, double beta2, double eps) {
  if (!c) return HMG_ERR_INVALID_ARG;
  if (!w || !grad || !m || !v || n < 1 || step < 1 || !(lr > 0.0) || !(beta1 >= 0.0 && beta1 < 1.0) ||
      !(beta2 >= 0.0 && beta2 < 1.0) || !(eps > 0.0))
    return fail(c, HMG_ERR_INVALID_ARG, "bad Adam arguments");
  HMG_CUDA(c, cudaSetDevice(c->device));
  return finish(c, adam_update(c, w, grad, m, v, n, step, lr, beta1, beta2, eps));
}

int hmg_collect_coarse_pairs(hmg_ctx *c, const double *Rub, const double *Rpi, double *lambda, int32_t max_pairs,
                             float *x_out, float *t_out, int32_t *n_out, hmg_solve_stats *stats) {
  int st = ready(c);
  if (st) return st;
  if (!Rub || !Rpi || !lambda || !x_out || !t_out || !n_out || max_pairs < 1)
    return fail(c, HMG_ERR_INVALID_ARG, "bad arguments");
  if (c->opt.precision != HMG_PRECISION_FP64 || c->opt.precond != HMG_PRECOND_NONNESTED || c->degree != 0)
    return fail(c, HMG_ERR_INVALID_ARG, "pairs are collected from the FP64 non-nested preconditioner of degree 0");
  c->collect_x = x_out;
  c->collect_t = t_out;
  c->collect_max = max_pairs;
  c->collect_n = 0;
  st = krylov_solve(c, Rub, Rpi, lambda, stats, false);
  *n_out = c->collect_n;
  c->collect_x = c->collect_t = nullptr;
  c->collect_max = c->collect_n = 0;
  return st;
}

int hmg_extract_patches(hmg_ctx *c, const float *xs, const float *ts, int32_t npairs, const int32_t *pair,
                        const int32_t *cols, int32_t npatch, int32_t patch_cols, float *xo, float *to) {
  int st = ready(c);
  if (st) return st;
  if (!xs || !ts || !pair || !cols || !xo || !to || npairs < 1 || npatch < 1 || patch_cols < 1)
    return fail(c, HMG_ERR_INVALID_ARG, "bad arguments");
  // the gather's indices are checked on the host before the kernel reads through them
  std::vector<int32_t> hp(npatch), hc((size_t)npatch * patch_cols);
  HMG_CUDA(c, cudaMemcpy(hp.data(), pair, sizeof(int32_t) * hp.size(), cudaMemcpyDeviceToHost));
  HMG_CUDA(c, cudaMemcpy(hc.data(), cols, sizeof(int32_t) * hc.size(), cudaMemcpyDeviceToHost));
  for (int32_t v : hp)
    if (v < 0 || v >= npairs) return fail(c, HMG_ERR_INVALID_ARG, "pair index out of range");
  for (int32_t v : hc)
    if (v < 0 || v >= c->lv[0].ncol) return fail(c, HMG_ERR_INVALID_ARG, "column index out of range");
  return extract_patches(c, xs, ts, c->lv[0].ncell, pair, cols, npatch, patch_cols, xo, to);
}

}  // extern "C"
