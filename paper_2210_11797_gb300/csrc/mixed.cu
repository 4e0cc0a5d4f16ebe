// Configuration 1 of arXiv 2210.11797 (Sec. 2.3, Sec. 3.2): BiCGStab on the unhybridised
// 2x2 system (Eq. 2x2system) for the continuous normal velocity u (one value per facet, in the
// trace numbering) and the Exner increment Pi, preconditioned by the approximate Schur
// complement: the velocity mass replaced by its lumped diagonal, Step 1 (Eq. pressure_rhs),
// one pressure-multigrid V-cycle on Eq. elliptic_pressure_system (Step 2) and Step 3
// (Eq. velocity_recovery).
//
// Vectors of the mixed system are [u (ntrace) | Pi (ncell)]. The ground and lid facets carry
// u.n = 0: their rows are the identity and every Krylov vector keeps 0 there. The velocity of
// facet f is oriented out of edge_cols[e][0] on vertical facets and upwards on horizontal
// ones; a cell's outward flux through its local face i is s_K(i) u_f.
//
// Storage, built from the cell records of the assembly: the velocity block in the 11-slot
// row layout of S (slot-major), two pressure couplings per facet row (the G block), seven
// coefficients per cell row (the B block and M3^Pi), and 1 / lumped mass per facet.
#include "device_common.cuh"
#include "hmg_internal.cuh"
#include "precond.cuh"

namespace hmg {

struct MixedArgs {
  int L, ncol;
  int64_t NH, NT, ncell;
  const int32_t *stencil, *edge_fc, *col_edges;
};

// s_K(f): +1 where the cell's outward normal through its local face f agrees with the facet's
// orientation (vertical face owned as the edge's first column; the top face), else -1.
__device__ __forceinline__ double face_sign(const MixedArgs &a, int c, int f) {
  if (f == 4) return -1.0;
  if (f == 5) return 1.0;
  const int e = __ldg(a.col_edges + 4 * (int64_t)c + f);
  return (__ldg(a.stencil + 8 * (int64_t)e) == c && __ldg(a.edge_fc + 2 * (int64_t)e) == f) ? 1.0 : -1.0;
}

// M_K(f, g) of a cell record: the symmetric part (21 entries, f <= g, row-major) plus the
// antisymmetric Coriolis part (15 entries, f < g, row-major)
__device__ __forceinline__ double rec_m(const double *r, int f, int g) {
  const int a = f < g ? f : g, b = f < g ? g : f;
  double v = r[CellRec::M + a * 6 - a * (a - 1) / 2 + (b - a)];
  if (a != b) {
    const double c = r[CellRec::CORI + a * 6 - a * (a + 1) / 2 + (b - a - 1)];
    v += f < g ? c : -c;
  }
  return v;
}

// Facet rows: velocity block (11 slots, sign-applied M_K summed over the facet's cells), the
// two G couplings, 1 / lumped mass. Cell rows: s_K(i) b_K(i) and M3^Pi.
__global__ void mixed_rows_kernel(const MixedArgs a, const double *__restrict__ rec, double *__restrict__ Mu,
                                  double *__restrict__ Gx, double *__restrict__ ilump) {
  const int64_t row = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (row >= a.NT) return;
  const int64_t T = a.NT;
  double v[kSlots], g0 = 0.0, g1 = 0.0, il = 0.0;
#pragma unroll
  for (int m = 0; m < kSlots; ++m) v[m] = 0.0;
  if (row < a.NH) {
    const int e = (int)(row / a.L), k = (int)(row - (int64_t)e * a.L);
    const int c1 = __ldg(a.stencil + 8 * (int64_t)e), c2 = __ldg(a.stencil + 8 * (int64_t)e + 1);
    const int i1 = __ldg(a.edge_fc + 2 * (int64_t)e), i2 = __ldg(a.edge_fc + 2 * (int64_t)e + 1);
    const double *r1 = rec + ((int64_t)c1 * a.L + k) * kCellData, *r2 = rec + ((int64_t)c2 * a.L + k) * kCellData;
    // s_{K1}(i1) = +1, s_{K2}(i2) = -1
    v[0] = rec_m(r1, i1, i1) + rec_m(r2, i2, i2);
    for (int m = 1; m <= 3; ++m) {
      const int j1 = (i1 + m) & 3, j2 = (i2 + m) & 3;
      v[m] = face_sign(a, c1, j1) * rec_m(r1, i1, j1);
      v[5 + m] = -face_sign(a, c2, j2) * rec_m(r2, i2, j2);
    }
    // the bottom / top faces at k = 0 / L-1 are ground / lid facets (u = 0): no coupling
    v[4] = k > 0 ? -rec_m(r1, i1, 4) : 0.0;
    v[5] = k < a.L - 1 ? rec_m(r1, i1, 5) : 0.0;
    v[9] = k > 0 ? rec_m(r2, i2, 4) : 0.0;
    v[10] = k < a.L - 1 ? -rec_m(r2, i2, 5) : 0.0;
    g0 = -r1[CellRec::KTH + i1];          // s A(i, 6) with A(i, 6) = -k theta
    g1 = r2[CellRec::KTH + i2];
    il = 1.0 / (r1[CellRec::LUMP + i1] + r2[CellRec::LUMP + i2]);
  } else {
    const int64_t zr = row - a.NH;
    const int c = (int)(zr / (a.L + 1)), k = (int)(zr - (int64_t)c * (a.L + 1));
    if (k > 0 && k < a.L) {   // ground and lid rows stay zero (identity in the apply)
      const double *ra = rec + ((int64_t)c * a.L + k) * kCellData;      // above: its bottom face
      const double *rb = rec + ((int64_t)c * a.L + k - 1) * kCellData;  // below: its top face
      v[0] = rec_m(ra, 4, 4) + rec_m(rb, 5, 5);
      for (int i = 0; i < 4; ++i) {
        const double si = face_sign(a, c, i);
        v[1 + i] = -si * rec_m(ra, 4, i);
        v[6 + i] = si * rec_m(rb, 5, i);
      }
      v[5] = k + 1 < a.L ? -rec_m(ra, 4, 5) : 0.0;   // the lid above, the ground below: u = 0
      v[10] = k - 1 > 0 ? -rec_m(rb, 5, 4) : 0.0;
      g0 = ra[CellRec::KTH + 4];
      g1 = -rb[CellRec::KTH + 5];
      il = 1.0 / (ra[CellRec::LUMP + 4] + rb[CellRec::LUMP + 5]);
    }
  }
#pragma unroll
  for (int m = 0; m < kSlots; ++m) Mu[m * T + row] = v[m];
  Gx[row] = g0;
  Gx[T + row] = g1;
  ilump[row] = il;
}

__global__ void mixed_cell_rows_kernel(const MixedArgs a, const double *__restrict__ rec, double *__restrict__ Bx) {
  const int64_t K = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (K >= a.ncell) return;
  const int c = (int)(K / a.L), k = (int)(K - (int64_t)c * a.L);
  const double *r = rec + K * kCellData;
#pragma unroll
  for (int i = 0; i < 6; ++i) Bx[(int64_t)i * a.ncell + K] = face_sign(a, c, i) * r[CellRec::B + i];
  if (k == 0) Bx[4 * a.ncell + K] = 0.0;            // ground facet: u = 0
  if (k == a.L - 1) Bx[5 * a.ncell + K] = 0.0;      // lid facet
  Bx[6 * a.ncell + K] = r[CellRec::MPI];
}

// facet of local face i of cell (c, k)
__device__ __forceinline__ int64_t cell_facet(const MixedArgs &a, int c, int k, int i) {
  if (i < 4) return (int64_t)__ldg(a.col_edges + 4 * (int64_t)c + i) * a.L + k;
  return a.NH + (int64_t)c * (a.L + 1) + k + (i == 5 ? 1 : 0);
}

// Row `row` of the mixed operator times x (x = [u | Pi]).
__device__ __forceinline__ double mixed_row(const MixedArgs &a, const TraceDims &d, const double *__restrict__ Mu,
                                            const double *__restrict__ Gx, const double *__restrict__ Bx,
                                            const double *__restrict__ x, int64_t row) {
  const int64_t T = a.NT;
  const double *pi = x + T;
  if (row < a.NH) {
    const int e = (int)(row / a.L), k = (int)(row - (int64_t)e * a.L);
    const int c1 = __ldg(a.stencil + 8 * (int64_t)e), c2 = __ldg(a.stencil + 8 * (int64_t)e + 1);
    double v = fma(__ldg(Gx + row), pi[(int64_t)c1 * a.L + k], 0.0);
    v = fma(__ldg(Gx + T + row), pi[(int64_t)c2 * a.L + k], v);
    return s_row_h<double, double, double, false>(Mu, x, a.stencil, d, row, v);
  }
  if (row < T) {
    const int64_t zr = row - a.NH;
    const int c = (int)(zr / (a.L + 1)), k = (int)(zr - (int64_t)c * (a.L + 1));
    if (k == 0 || k == a.L) return x[row];
    double v = fma(__ldg(Gx + row), pi[(int64_t)c * a.L + k], 0.0);
    v = fma(__ldg(Gx + T + row), pi[(int64_t)c * a.L + k - 1], v);
    return s_row_z<double, double, double, false>(Mu, x, a.col_edges, d, row, v);
  }
  const int64_t K = row - T;
  const int c = (int)(K / a.L), k = (int)(K - (int64_t)c * a.L);
  double v = __ldg(Bx + 6 * a.ncell + K) * pi[K];
#pragma unroll
  for (int i = 0; i < 6; ++i) v = fma(__ldg(Bx + (int64_t)i * a.ncell + K), x[cell_facet(a, c, k, i)], v);
  return v;
}

// y = Mx x with the fused inner products of the Krylov loop (modes as in launch_spmv).
template <int MODE>
__global__ void __launch_bounds__(kRedThreads)
    mixed_apply_kernel(const MixedArgs a, const TraceDims d, const double *__restrict__ Mu,
                       const double *__restrict__ Gx, const double *__restrict__ Bx, const double *__restrict__ x,
                       double *__restrict__ y, const double *__restrict__ w, double *part, int slot0, int slot1) {
  const int64_t n = a.NT + a.ncell;
  const int64_t row = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  double a0 = 0.0, a1 = 0.0;
  if (row < n) {
    const double v = mixed_row(a, d, Mu, Gx, Bx, x, row);
    if (MODE == 3) {
      const double r = __ldg(w + row) - v;
      a0 = r * r;
    } else {
      y[row] = v;
      if (MODE == 1) a0 = __ldg(w + row) * v;
      if (MODE == 2) { a0 = v * __ldg(w + row); a1 = v * v; }
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

// [R_u | R_Pi]: R_u(f) = sum over the facet's cells of s_K(i) R_u^b(K, i), 0 on ground and lid
__global__ void mixed_rhs_kernel(const MixedArgs a, const double *__restrict__ Rub, const double *__restrict__ Rpi,
                                 double *__restrict__ B) {
  const int64_t row = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t T = a.NT;
  if (row >= T + a.ncell) return;
  double v = 0.0;
  if (row < a.NH) {
    const int e = (int)(row / a.L), k = (int)(row - (int64_t)e * a.L);
    const int c1 = __ldg(a.stencil + 8 * (int64_t)e), c2 = __ldg(a.stencil + 8 * (int64_t)e + 1);
    const int i1 = __ldg(a.edge_fc + 2 * (int64_t)e), i2 = __ldg(a.edge_fc + 2 * (int64_t)e + 1);
    v = Rub[6 * ((int64_t)c1 * a.L + k) + i1] - Rub[6 * ((int64_t)c2 * a.L + k) + i2];
  } else if (row < T) {
    const int64_t zr = row - a.NH;
    const int c = (int)(zr / (a.L + 1)), k = (int)(zr - (int64_t)c * (a.L + 1));
    if (k > 0 && k < a.L) v = Rub[6 * ((int64_t)c * a.L + k - 1) + 5] - Rub[6 * ((int64_t)c * a.L + k) + 4];
  } else {
    v = Rpi[row - T];
  }
  B[row] = v;
}

// Step 1: B_K = r_Pi(K) - sum_i s_K(i) b_K(i) r_u(f_i) / Mlump(f_i)
__global__ void schur_step1_kernel(const MixedArgs a, const double *__restrict__ Bx, const double *__restrict__ ilump,
                                   const double *__restrict__ r, double *__restrict__ bp) {
  const int64_t K = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (K >= a.ncell) return;
  const int c = (int)(K / a.L), k = (int)(K - (int64_t)c * a.L);
  double v = r[a.NT + K];
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    const int64_t f = cell_facet(a, c, k, i);
    v = fma(-__ldg(Bx + (int64_t)i * a.ncell + K), __ldg(ilump + f) * r[f], v);
  }
  bp[K] = v;
}

// Step 3: u(f) = (r_u(f) - sum over the facet's cells of s_K(i) G_K(i) Pi_K) / Mlump(f);
// identity on the ground and lid; z_Pi = Pi
__global__ void schur_step3_kernel(const MixedArgs a, const double *__restrict__ Gx, const double *__restrict__ ilump,
                                   const double *__restrict__ r, const double *__restrict__ pi, double *__restrict__ z) {
  const int64_t row = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t T = a.NT;
  if (row >= T + a.ncell) return;
  if (row >= T) {
    z[row] = pi[row - T];
    return;
  }
  int64_t K1 = -1, K2 = -1;
  if (row < a.NH) {
    const int e = (int)(row / a.L), k = (int)(row - (int64_t)e * a.L);
    K1 = (int64_t)__ldg(a.stencil + 8 * (int64_t)e) * a.L + k;
    K2 = (int64_t)__ldg(a.stencil + 8 * (int64_t)e + 1) * a.L + k;
  } else {
    const int64_t zr = row - a.NH;
    const int c = (int)(zr / (a.L + 1)), k = (int)(zr - (int64_t)c * (a.L + 1));
    if (k == 0 || k == a.L) {
      z[row] = r[row];
      return;
    }
    K1 = (int64_t)c * a.L + k;
    K2 = K1 - 1;
  }
  double v = fma(-__ldg(Gx + row), pi[K1], r[row]);
  v = fma(-__ldg(Gx + T + row), pi[K2], v);
  z[row] = __ldg(ilump + row) * v;
}

static MixedArgs mixed_args(const Ctx *c) {
  const Level &f = c->lv[0];
  return MixedArgs{f.nlev, f.ncol, f.nth, f.ntrace, f.ncell, f.edge_stencil, f.edge_fc, f.col_edges};
}

int build_mixed(Ctx *c, const double *rec0) {
  const Level &f = c->lv[0];
  const int64_t T = f.ntrace, C = f.ncell;
  int st;
  if (!c->mx_Mu) {
    if ((st = dev_alloc(c, &c->mx_Mu, (size_t)kSlots * T))) return st;
    if ((st = dev_alloc(c, &c->mx_Gx, (size_t)2 * T))) return st;
    if ((st = dev_alloc(c, &c->mx_Bx, (size_t)7 * C))) return st;
    if ((st = dev_alloc(c, &c->mx_ilump, (size_t)T))) return st;
    if ((st = dev_alloc(c, &c->mx_x, (size_t)(T + C)))) return st;
    if ((st = dev_alloc(c, &c->mx_bp, (size_t)C))) return st;
  }
  const MixedArgs a = mixed_args(c);
  mixed_rows_kernel<<<grid_for(T, 256), 256, 0, c->stream>>>(a, rec0, c->mx_Mu, c->mx_Gx, c->mx_ilump);
  mixed_cell_rows_kernel<<<grid_for(C, 256), 256, 0, c->stream>>>(a, rec0, c->mx_Bx);
  HMG_CUDA(c, cudaGetLastError());
  c->have_mixed = true;
  return HMG_OK;
}

int launch_mixed_apply(Ctx *c, const double *x, double *y, int mode, const double *w, int slot0, int slot1) {
  if (!c->have_mixed) return fail(c, HMG_ERR_NOT_READY, "assemble with precond = HMG_PRECOND_SCHUR first");
  const Level &f = c->lv[0];
  const MixedArgs a = mixed_args(c);
  const TraceDims d{f.nlev, f.nth, f.ntrace};
  const unsigned g = grid_for(f.ntrace + f.ncell, kRedThreads);
  if (g > (unsigned)kMaxRedBlocks) return fail(c, HMG_ERR_INVALID_ARG, "too many rows for one reduction");
  Prof prof(c, kCompApply, mode ? 2 : 1);
  switch (mode) {
    case 0: mixed_apply_kernel<0><<<g, kRedThreads, 0, c->stream>>>(a, d, c->mx_Mu, c->mx_Gx, c->mx_Bx, x, y, w, c->part, slot0, slot1); break;
    case 1: mixed_apply_kernel<1><<<g, kRedThreads, 0, c->stream>>>(a, d, c->mx_Mu, c->mx_Gx, c->mx_Bx, x, y, w, c->part, slot0, slot1); break;
    case 2: mixed_apply_kernel<2><<<g, kRedThreads, 0, c->stream>>>(a, d, c->mx_Mu, c->mx_Gx, c->mx_Bx, x, y, w, c->part, slot0, slot1); break;
    default: mixed_apply_kernel<3><<<g, kRedThreads, 0, c->stream>>>(a, d, c->mx_Mu, c->mx_Gx, c->mx_Bx, x, y, w, c->part, slot0, slot1); break;
  }
  HMG_CUDA(c, cudaGetLastError());
  if (mode != 0) return launch_finalize(c, (int)g, slot0, mode == 2 ? slot1 : -1);
  return HMG_OK;
}

int launch_mixed_rhs(Ctx *c, const double *Rub, const double *Rpi, double *B) {
  if (!c->have_mixed) return fail(c, HMG_ERR_NOT_READY, "assemble with precond = HMG_PRECOND_SCHUR first");
  const Level &f = c->lv[0];
  Prof prof(c, kCompRhs);
  mixed_rhs_kernel<<<grid_for(f.ntrace + f.ncell, 256), 256, 0, c->stream>>>(mixed_args(c), Rub, Rpi, B);
  HMG_CUDA(c, cudaGetLastError());
  return HMG_OK;
}

int schur_precond(Ctx *c, const double *r, double *z) {
  if (!c->have_mixed) return fail(c, HMG_ERR_NOT_READY, "assemble with precond = HMG_PRECOND_SCHUR first");
  const Level &f = c->lv[0];
  const MixedArgs a = mixed_args(c);
  int st;
  {
    Prof pr(c, kCompResidual);
    schur_step1_kernel<<<grid_for(f.ncell, 256), 256, 0, c->stream>>>(a, c->mx_Bx, c->mx_ilump, r, c->mx_bp);
    HMG_CUDA(c, cudaGetLastError());
  }
  double *pi = nullptr;
  {
    Prof pv(c, kCompVcycle, vcycle_launches(c));
    if ((st = vcycle<double>(c, c->mx_bp, &pi))) return st;
  }
  Prof pp(c, kCompProlong);
  schur_step3_kernel<<<grid_for(f.ntrace + f.ncell, 256), 256, 0, c->stream>>>(a, c->mx_Gx, c->mx_ilump, r, pi, z);
  HMG_CUDA(c, cudaGetLastError());
  return HMG_OK;
}

}  // namespace hmg
