// Assembly kernels (setup phase): per-cell local matrices by Gauss quadrature, local
// condensation, the rows of the trace operator S, the pressure operator H on every
// multigrid level, Thomas factors of the column systems and the coarse scaling Gamma.
//
// Paper (arXiv 2210.11797): Sec. 2.2 Eq. bilinear_forms and the quadrature rule (3 Gauss
// points per direction for volume terms at p = 0; one-point cell-centre rule for q32,
// m3^rho, m3^Pi); Eq. 2x2system (B = Q32 + M3^rho M3^-1 D); Sec. 2.4 Eqs. hybrid-A,
// hybrid-K, hybrid-S (S = C^T A^-1 K); Sec. 2.3 Eq. elliptic_pressure_system
// (H = -B Mlump^-1 G + M3^Pi); Sec. 2.5 Eq. scaling_matrix (Gamma).
#include <cmath>
#include <cstring>

#include "device_common.cuh"
#include "hmg_internal.cuh"

namespace hmg {

struct CellArgs {
  int geometry, ncol, L;
  int64_t ncell;
  double radius;
  const double *corners, *z, *theta_lev, *exner_lev, *exner;
  const int32_t *col_nbr;
  hmg_scalars sc;
};

// Trilinear shape function values and derivatives at the 27 Gauss points (3 per direction):
// [q][v] = {N_v, dN_v/dxi, dN_v/deta, dN_v/dzeta}, q = qi + 3 qj + 9 qk, vertex v = (v&1,
// v>>1&1, v>>2). They depend on the point only, so they are formed once on the host (with the
// same expressions and order of operations a per-cell evaluation would use) instead of in
// every cell.
__constant__ double c_shape[27][8][4];

static int upload_shape_functions(Ctx *c) {
  static thread_local double h[27][8][4];
  const double gq = std::sqrt(15.0) / 10.0;
  const double gx[3] = {0.5 - gq, 0.5, 0.5 + gq};
  for (int q = 0; q < 27; ++q) {
    const double xi = gx[q % 3], eta = gx[(q / 3) % 3], zeta = gx[q / 9];
    for (int v = 0; v < 8; ++v) {
      const int av = v & 1, bv = (v >> 1) & 1, cv = (v >> 2) & 1;
      const double fx = av ? xi : 1.0 - xi, fy = bv ? eta : 1.0 - eta, fz = cv ? zeta : 1.0 - zeta;
      const double sx = av ? 1.0 : -1.0, sy = bv ? 1.0 : -1.0, sz = cv ? 1.0 : -1.0;
      h[q][v][0] = fx * fy * fz;
      h[q][v][1] = sx * fy * fz;
      h[q][v][2] = fx * sy * fz;
      h[q][v][3] = fx * fy * sz;
    }
  }
  HMG_CUDA(c, cudaMemcpyToSymbol(c_shape, h, sizeof(h)));
  return HMG_OK;
}

// Corner of the column at reference (xi, eta) in {0,1}^2: (0,0)->0, (1,0)->1, (1,1)->2, (0,1)->3.
__device__ __forceinline__ int corner_of(int a, int b) { return b ? (a ? 2 : 3) : (a ? 1 : 0); }

// Geometry and coefficients of one cell; writes its CellRec.
//  M_K(f,g) = sum_q w_q / det J_q * s_f s_g [ (J^T J)_{d_f d_g} + c22 (r.J)_{d_f} (r.J)_{d_g} ],
// where the RT0 reference function of face f is s_f(xi) e_{d_f} (outward unit flux) and the
// contravariant Piola map gives v_f = J s_f e_{d_f} / det J.
__global__ void __launch_bounds__(128) cell_kernel(const CellArgs a, double *__restrict__ rec) {
  const int64_t K = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (K >= a.ncell) return;
  const int c = (int)(K / a.L), k = (int)(K - (int64_t)c * a.L);
  const double z0 = a.z[k], z1 = a.z[k + 1];
  double vx[8], vy[8], vz[8];
#pragma unroll
  for (int v = 0; v < 8; ++v) {
    const int ci = corner_of(v & 1, (v >> 1) & 1);
    const double *cp = a.corners + 12 * (int64_t)c + 3 * ci;
    const double h = (v >> 2) ? z1 : z0;
    if (a.geometry == 1) {
      const double s = a.radius + h;
      vx[v] = cp[0] * s; vy[v] = cp[1] * s; vz[v] = cp[2] * s;
    } else {
      vx[v] = cp[0]; vy[v] = cp[1]; vz[v] = h;
    }
  }
  const int L1 = a.L + 1;
  const double th0 = a.theta_lev[(int64_t)c * L1 + k], th1 = a.theta_lev[(int64_t)c * L1 + k + 1];
  const double pi0 = a.exner_lev[(int64_t)c * L1 + k], pi1 = a.exner_lev[(int64_t)c * L1 + k + 1];
  const double dz = z1 - z0;
  const bool helm = a.sc.preset == 1;
  const double c22 = helm ? 0.0
                          : -a.sc.tau_u * a.sc.tau_theta * a.sc.dt * a.sc.dt * a.sc.cp *
                                ((pi1 - pi0) / dz) * ((th1 - th0) / dz);
  const int dir[6] = {1, 0, 1, 0, 2, 2};
  const double gq = sqrt(15.0) / 10.0;
  const double gx[3] = {0.5 - gq, 0.5, 0.5 + gq};
  const double gw[3] = {5.0 / 18.0, 8.0 / 18.0, 5.0 / 18.0};
  double M[21], Cor[15];
#pragma unroll
  for (int i = 0; i < 21; ++i) M[i] = 0.0;
#pragma unroll
  for (int i = 0; i < 15; ++i) Cor[i] = 0.0;
  // Coriolis vector tau_u dt 2 Omega about z (Eq. gh-u); none for the Helmholtz preset
  const double cz = helm ? 0.0 : a.sc.tau_u * a.sc.dt * 2.0 * a.sc.omega;
  double vol = 0.0;
  for (int q = 0; q < 27; ++q) {
    const int qi = q % 3, qj = (q / 3) % 3, qk = q / 9;
    const double xi = gx[qi], eta = gx[qj], zeta = gx[qk];
    const double w = gw[qi] * gw[qj] * gw[qk];
    double J[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    double x[3] = {0, 0, 0};
#pragma unroll
    for (int v = 0; v < 8; ++v) {
      const double n = c_shape[q][v][0];
      const double d0 = c_shape[q][v][1], d1 = c_shape[q][v][2], d2 = c_shape[q][v][3];
      x[0] += n * vx[v]; x[1] += n * vy[v]; x[2] += n * vz[v];
      J[0][0] += vx[v] * d0; J[0][1] += vx[v] * d1; J[0][2] += vx[v] * d2;
      J[1][0] += vy[v] * d0; J[1][1] += vy[v] * d1; J[1][2] += vy[v] * d2;
      J[2][0] += vz[v] * d0; J[2][1] += vz[v] * d1; J[2][2] += vz[v] * d2;
    }
    const double det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
                       J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
                       J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
    double r[3];
    if (a.geometry == 1) {
      const double inv = 1.0 / sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
      r[0] = x[0] * inv; r[1] = x[1] * inv; r[2] = x[2] * inv;
    } else {
      r[0] = 0.0; r[1] = 0.0; r[2] = 1.0;
    }
    const double wd = w / det;
    // H[d][e] = w / det * (G[d][e] + c22 (r.J)_d (r.J)_e), G = J^T J: 6 distinct entries,
    // formed once per point; each of the 21 entries of M then costs a multiply and an FMA
    double rJ[3], H[3][3];
#pragma unroll
    for (int d = 0; d < 3; ++d) rJ[d] = r[0] * J[0][d] + r[1] * J[1][d] + r[2] * J[2][d];
#pragma unroll
    for (int d = 0; d < 3; ++d)
#pragma unroll
      for (int e = d; e < 3; ++e) {
        const double g = J[0][d] * J[0][e] + J[1][d] * J[1][e] + J[2][d] * J[2][e];
        H[d][e] = H[e][d] = wd * fma(c22 * rJ[d], rJ[e], g);
      }
    const double s[6] = {eta - 1.0, xi, eta, xi - 1.0, zeta - 1.0, zeta};
    int idx = 0;
#pragma unroll
    for (int f = 0; f < 6; ++f) {
#pragma unroll
      for (int g = f; g < 6; ++g) {
        M[idx] = fma(s[f], s[g] * H[dir[f]][dir[g]], M[idx]);
        ++idx;
      }
    }
    if (cz != 0.0) {
      // v_f . (c x v_g) = s_f s_g c . (J_dg x J_df) / det^2: X[d][e] = (c x-products of the
      // columns of J), antisymmetric; c = (0, 0, cz)
      double X[3][3];
#pragma unroll
      for (int d = 0; d < 3; ++d)
#pragma unroll
        for (int e = 0; e < 3; ++e) X[d][e] = wd * cz * (J[0][e] * J[1][d] - J[1][e] * J[0][d]);
      int ci = 0;
#pragma unroll
      for (int f = 0; f < 6; ++f)
#pragma unroll
        for (int g = f + 1; g < 6; ++g) {
          Cor[ci] = fma(s[f], s[g] * X[dir[f]][dir[g]], Cor[ci]);
          ++ci;
        }
    }
    vol += w * det;
  }
  // cell centre: one-point volume |K|_1 and zhat.v_f
  double Jc[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}}, xc[3] = {0, 0, 0};
#pragma unroll
  for (int v = 0; v < 8; ++v) {
    const double sx = (v & 1) ? 1.0 : -1.0, sy = ((v >> 1) & 1) ? 1.0 : -1.0, sz = ((v >> 2) & 1) ? 1.0 : -1.0;
    xc[0] += 0.125 * vx[v]; xc[1] += 0.125 * vy[v]; xc[2] += 0.125 * vz[v];
    Jc[0][0] += 0.25 * sx * vx[v]; Jc[0][1] += 0.25 * sy * vx[v]; Jc[0][2] += 0.25 * sz * vx[v];
    Jc[1][0] += 0.25 * sx * vy[v]; Jc[1][1] += 0.25 * sy * vy[v]; Jc[1][2] += 0.25 * sz * vy[v];
    Jc[2][0] += 0.25 * sx * vz[v]; Jc[2][1] += 0.25 * sy * vz[v]; Jc[2][2] += 0.25 * sz * vz[v];
  }
  const double vol1 = Jc[0][0] * (Jc[1][1] * Jc[2][2] - Jc[1][2] * Jc[2][1]) -
                      Jc[0][1] * (Jc[1][0] * Jc[2][2] - Jc[1][2] * Jc[2][0]) +
                      Jc[0][2] * (Jc[1][0] * Jc[2][1] - Jc[1][1] * Jc[2][0]);
  double rc[3];
  if (a.geometry == 1) {
    const double inv = 1.0 / sqrt(xc[0] * xc[0] + xc[1] * xc[1] + xc[2] * xc[2]);
    rc[0] = xc[0] * inv; rc[1] = xc[1] * inv; rc[2] = xc[2] * inv;
  } else {
    rc[0] = 0.0; rc[1] = 0.0; rc[2] = 1.0;
  }
  double rJc[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) rJc[d] = rc[0] * Jc[0][d] + rc[1] * Jc[1][d] + rc[2] * Jc[2][d];
  const double sc_[6] = {-0.5, 0.5, 0.5, -0.5, -0.5, 0.5};
  // single-valued theta on each face: vertical faces average the two columns' layer means
  const double mean_own = 0.5 * (th0 + th1);
  double theta[6];
#pragma unroll
  for (int f = 0; f < 4; ++f) {
    const int oc = a.col_nbr[4 * (int64_t)c + f];
    const double mo = 0.5 * (a.theta_lev[(int64_t)oc * L1 + k] + a.theta_lev[(int64_t)oc * L1 + k + 1]);
    theta[f] = 0.5 * (mean_own + mo);
  }
  theta[4] = th0;
  theta[5] = th1;
  double *out = rec + (int64_t)K * kCellData;
  double kk, m;
  double b[6];
  if (helm) {
    kk = 1.0;
    m = a.sc.sigma * vol1;
#pragma unroll
    for (int f = 0; f < 6; ++f) { theta[f] = 1.0; b[f] = 1.0; }
  } else {
    kk = a.sc.tau_u * a.sc.dt * a.sc.cp;
    const double dlog = ((th1 - th0) / dz) / mean_own;
    const double base = a.sc.tau_rho * a.sc.dt * vol1 / vol;   // M3^rho M3^-1 D
#pragma unroll
    for (int f = 0; f < 6; ++f) {
      const double zv = sc_[f] * rJc[dir[f]] / vol1;               // (zhat.v_f)(x_c)
      b[f] = base + a.sc.tau_theta * a.sc.dt * (vol1 * dlog) * zv; // + q32
    }
    m = (1.0 - a.sc.kappa) / a.sc.kappa * vol1 / a.exner[K];
  }
#pragma unroll
  for (int i = 0; i < 21; ++i) out[CellRec::M + i] = M[i];
#pragma unroll
  for (int i = 0; i < 15; ++i) out[CellRec::CORI + i] = Cor[i];
#pragma unroll
  for (int f = 0; f < 6; ++f) {
    out[CellRec::B + f] = b[f];
    out[CellRec::KTH + f] = kk * theta[f];
  }
  out[CellRec::MPI] = m;
  // lumped mass share: |M(f,f)| + |M(f, opposite f)|
  const double Mff[6] = {M[0], M[6], M[11], M[15], M[18], M[20]};
  const double Mopp[6] = {M[2], M[8], M[2], M[8], M[19], M[19]};  // (0,2) (1,3) (4,5)
#pragma unroll
  for (int f = 0; f < 6; ++f) out[CellRec::LUMP + f] = fabs(Mff[f]) + fabs(Mopp[f]);
}

__device__ __forceinline__ double mget(const double *M, int f, int g) {
  if (f > g) { int t = f; f = g; g = t; }
  return M[f * 6 - f * (f - 1) / 2 + (g - f)];
}

// A_K = [[M, g], [b^T, m]] with g = -KTH (Eq. hybrid-A). A_K^-1 by block elimination:
// M^-1 from the LU factors of the equilibrated velocity block D M D (D = diag(M)^-1/2; its
// symmetric part is positive definite, the Coriolis part antisymmetric), y = M^-1 g,
// z = M^-T b, pressure Schur complement s = m - b.y, then
// A^-1 = [[M^-1 + y z^T / s, -y / s], [-z^T / s, 1 / s]]. The rows of
// A_K span ~20 orders of magnitude on the sphere; this form keeps every entry within a few
// ulps of its row's scale, where pivoting on A_K itself can lose 1e-12.
// Outputs: Ainv entry-major ((7 i + j) * ncell + K), S_K = (A^-1)_uu diag(KTH) entry-major,
// KTH and S_K 1 face-major. A non-positive pivot (M not positive definite) or s == 0 sets *singular.
__global__ void __launch_bounds__(128) condense_kernel(int64_t ncell, const double *__restrict__ rec,
                                                       double *__restrict__ Ainv,
                                                       double *__restrict__ SK,
                                                       double *__restrict__ kth_out,
                                                       double *__restrict__ sk1,
                                                       int *__restrict__ singular) {
  const int64_t K = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (K >= ncell) return;
  const double *r = rec + K * kCellData;
  // M_K = symmetric part (21 stored) + Coriolis part (antisymmetric, 15 stored)
  auto mfull = [&](int f, int g) {
    double v = mget(r + CellRec::M, f, g);
    if (f < g) v += r[CellRec::CORI + f * 6 - f * (f + 1) / 2 + (g - f - 1)];
    else if (f > g) v -= r[CellRec::CORI + g * 6 - g * (g + 1) / 2 + (f - g - 1)];
    return v;
  };
  double d[6], A[6][6];
#pragma unroll
  for (int f = 0; f < 6; ++f) {
    const double mff = fabs(mget(r + CellRec::M, f, f));
    if (!(mff > 0.0)) { atomicExch(singular, 1); return; }
    d[f] = 1.0 / sqrt(mff);
  }
#pragma unroll
  for (int i = 0; i < 6; ++i)
#pragma unroll
    for (int j = 0; j < 6; ++j) A[i][j] = d[i] * mfull(i, j) * d[j];
  // LU of the equilibrated D M D without pivoting (its symmetric part is positive definite,
  // so every pivot is positive; with no rotation this is the symmetric case), in place
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    if (!(A[k][k] > 0.0)) { atomicExch(singular, 1); return; }
    const double inv = 1.0 / A[k][k];
#pragma unroll
    for (int i = k + 1; i < 6; ++i) {
      const double l = A[i][k] * inv;
      A[i][k] = l;
#pragma unroll
      for (int j = k + 1; j < 6; ++j) A[i][j] -= l * A[k][j];
    }
  }
  // M^-1 = D (LU)^-1 D, column by column
  double Mi[6][6];
#pragma unroll
  for (int c = 0; c < 6; ++c) {
    double y[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      double t = i == c ? 1.0 : 0.0;
#pragma unroll
      for (int q = 0; q < i; ++q) t -= A[i][q] * y[q];
      y[i] = t;
    }
#pragma unroll
    for (int i = 5; i >= 0; --i) {
      double t = y[i];
#pragma unroll
      for (int q = i + 1; q < 6; ++q) t -= A[i][q] * y[q];
      y[i] = t / A[i][i];
    }
#pragma unroll
    for (int i = 0; i < 6; ++i) Mi[i][c] = d[i] * y[i] * d[c];
  }
  double kth[6], g[6], b[6], y[6], z[6];
#pragma unroll
  for (int f = 0; f < 6; ++f) {
    kth[f] = r[CellRec::KTH + f];
    kth_out[(int64_t)f * ncell + K] = kth[f];
    g[f] = -kth[f];
    b[f] = r[CellRec::B + f];
  }
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    double ty = 0.0, tz = 0.0;
#pragma unroll
    for (int j = 0; j < 6; ++j) { ty += Mi[i][j] * g[j]; tz += Mi[j][i] * b[j]; }   // y = M^-1 g, z = M^-T b
    y[i] = ty;
    z[i] = tz;
  }
  double s = r[CellRec::MPI];
#pragma unroll
  for (int j = 0; j < 6; ++j) s -= b[j] * y[j];
  if (s == 0.0) { atomicExch(singular, 1); return; }
  const double is = 1.0 / s;
#pragma unroll
  for (int i = 0; i < 6; ++i) {
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      const double a = Mi[i][j] + y[i] * z[j] * is;
      Ainv[(int64_t)(7 * i + j) * ncell + K] = a;
      SK[(int64_t)(6 * i + j) * ncell + K] = a * kth[j];
    }
    Ainv[(int64_t)(7 * i + 6) * ncell + K] = -y[i] * is;
    Ainv[(int64_t)(42 + i) * ncell + K] = -z[i] * is;
    // S_K 1 = m (A^-1)_{u,p}: from G_K = -K_K 1, A [0; -1] = [K_K 1; -m], so the row sums of
    // S_K follow without the cancellation of summing its entries
    sk1[(int64_t)i * ncell + K] = r[CellRec::MPI] * (-y[i] * is);
  }
  Ainv[(int64_t)48 * ncell + K] = is;
}

struct RowArgs {
  int L;
  int64_t NH, NT, ncell;
  const int32_t *stencil, *edge_fc, *col_edges, *col_nbr, *col_nbr_face;
};

// Rows of S: the sum of the (at most two) cells' S_K rows, in the slot order of s_row.
__global__ void trace_rows_kernel(const RowArgs a, const double *__restrict__ SK,
                                  double *__restrict__ S) {
  const int64_t row = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (row >= a.NT) return;
  const int64_t C = a.ncell, T = a.NT;
  double v[kSlots];
  auto sk = [&](int64_t K, int i, int j) { return SK[(int64_t)(6 * i + j) * C + K]; };
  if (row < a.NH) {
    const int e = (int)(row / a.L), k = (int)(row - (int64_t)e * a.L);
    const int c1 = a.stencil[8 * (int64_t)e], c2 = a.stencil[8 * (int64_t)e + 1];
    const int i1 = a.edge_fc[2 * (int64_t)e], i2 = a.edge_fc[2 * (int64_t)e + 1];
    const int64_t K1 = (int64_t)c1 * a.L + k, K2 = (int64_t)c2 * a.L + k;
    v[0] = sk(K1, i1, i1) + sk(K2, i2, i2);
    for (int m = 1; m <= 3; ++m) v[m] = sk(K1, i1, (i1 + m) & 3);
    v[4] = sk(K1, i1, 4);
    v[5] = sk(K1, i1, 5);
    for (int m = 1; m <= 3; ++m) v[5 + m] = sk(K2, i2, (i2 + m) & 3);
    v[9] = sk(K2, i2, 4);
    v[10] = sk(K2, i2, 5);
  } else {
    const int64_t zr = row - a.NH;
    const int c = (int)(zr / (a.L + 1)), k = (int)(zr - (int64_t)c * (a.L + 1));
    for (int m = 0; m < kSlots; ++m) v[m] = 0.0;
    double self_a = 0.0, self_b = 0.0;
    if (k < a.L) {
      const int64_t Ka = (int64_t)c * a.L + k;
      self_a = sk(Ka, 4, 4);
      for (int i = 0; i < 4; ++i) v[1 + i] = sk(Ka, 4, i);
      v[5] = sk(Ka, 4, 5);
    }
    if (k > 0) {
      const int64_t Kb = (int64_t)c * a.L + k - 1;
      self_b = sk(Kb, 5, 5);
      for (int i = 0; i < 4; ++i) v[6 + i] = sk(Kb, 5, i);
      v[10] = sk(Kb, 5, 4);
    }
    v[0] = self_a + self_b;
  }
#pragma unroll
  for (int m = 0; m < kSlots; ++m) S[m * T + row] = v[m];
}

// Thomas factors of S^zz_c (rows k = 0..L of column c: sub = slot 10, diag = slot 0,
// sup = slot 5) and 1 / diag(S^hh).
// Thomas factors of every S^zz_j (Algorithm 1) with the relaxation folded in: for pivot
// p_k = d_k - s_k cp_{k-1}, zw = omega / p_k, zl = s_k / p_k (s_k the sub-diagonal) and
// zcp = u_k / p_k (u_k the super-diagonal); and hw = omega / diag(S^hh). The sweeps then do
// y_k = r_k zw_k - zl_k y_{k-1}, x_k = y_k - zcp_k x_{k+1} (one FMA per row each) and
// lambda += x, which is lambda + omega (S^zz)^-1 r.
__global__ void trace_factor_kernel(const RowArgs a, int ncol, const double *__restrict__ S, double omega,
                                    double *__restrict__ zw, double *__restrict__ zl,
                                    double *__restrict__ zcp, double *__restrict__ hw) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t T = a.NT;
  if (i < ncol) {
    const int64_t base = a.NH + i * (a.L + 1);
    double cp = 0.0;
    for (int k = 0; k <= a.L; ++k) {
      const int64_t row = base + k;
      const double sub = k > 0 ? S[10 * T + row] : 0.0;
      const double inv = 1.0 / (S[row] - sub * cp);
      cp = S[5 * T + row] * inv;
      zw[row - a.NH] = omega * inv;
      zl[row - a.NH] = sub * inv;
      zcp[row - a.NH] = cp;
    }
  }
  for (int64_t row = i; row < a.NH; row += (int64_t)gridDim.x * blockDim.x) hw[row] = omega / S[row];
}

struct HArgs {
  int L, ncol;
  int64_t ncell;
  const int32_t *col_nbr, *col_nbr_face;
};

// Row of H = -B Mlump^-1 G + M3^Pi for cell K (7-point): coupling across face f is
// -b_K(f) k theta_f / Mlump_f with Mlump_f the sum of both cells' shares; the diagonal is
// M3^Pi plus b_K(f) k theta_f / Mlump_f over the interior faces.
__global__ void pressure_rows_kernel(const HArgs a, const double *__restrict__ rec,
                                     double *__restrict__ H) {
  const int64_t K = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (K >= a.ncell) return;
  const int c = (int)(K / a.L), k = (int)(K - (int64_t)c * a.L);
  const double *r = rec + K * kCellData;
  double diag = r[CellRec::MPI];
  const int64_t C = a.ncell;
#pragma unroll
  for (int f = 0; f < 4; ++f) {
    const int nb = a.col_nbr[4 * (int64_t)c + f], nf = a.col_nbr_face[4 * (int64_t)c + f];
    const double *rn = rec + ((int64_t)nb * a.L + k) * kCellData;
    const double lump = r[CellRec::LUMP + f] + rn[CellRec::LUMP + nf];
    diag += r[CellRec::B + f] * r[CellRec::KTH + f] / lump;
    H[(1 + f) * C + K] = -r[CellRec::B + f] * rn[CellRec::KTH + nf] / lump;
  }
  if (k > 0) {
    const double *rn = r - kCellData;
    const double lump = r[CellRec::LUMP + 4] + rn[CellRec::LUMP + 5];
    diag += r[CellRec::B + 4] * r[CellRec::KTH + 4] / lump;
    H[5 * C + K] = -r[CellRec::B + 4] * rn[CellRec::KTH + 5] / lump;
  } else {
    H[5 * C + K] = 0.0;
  }
  if (k < a.L - 1) {
    const double *rn = r + kCellData;
    const double lump = r[CellRec::LUMP + 5] + rn[CellRec::LUMP + 4];
    diag += r[CellRec::B + 5] * r[CellRec::KTH + 5] / lump;
    H[6 * C + K] = -r[CellRec::B + 5] * rn[CellRec::KTH + 4] / lump;
  } else {
    H[6 * C + K] = 0.0;
  }
  H[K] = diag;
}

// Thomas factors of H_z per column (sub = below, diag, sup = above) with the block-Jacobi
// relaxation omega folded in, in the form of trace_factor_kernel: w = omega / p_k,
// l = sub / p_k, cp = sup / p_k.
__global__ void pressure_factor_kernel(const HArgs a, const double *__restrict__ H, double omega,
                                       double *__restrict__ w_out, double *__restrict__ l_out,
                                       double *__restrict__ cp_out) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= a.ncol) return;
  const int64_t C = a.ncell;
  double cp = 0.0;
  for (int k = 0; k < a.L; ++k) {
    const int64_t K = c * a.L + k;
    const double sub = k > 0 ? H[5 * C + K] : 0.0;
    const double inv = 1.0 / (H[K] - sub * cp);
    cp = H[6 * C + K] * inv;
    w_out[K] = omega * inv;
    l_out[K] = sub * inv;
    cp_out[K] = cp;
  }
}

// Gamma_K = (H 1)_K / (P^T S P 1)_K (Eq. scaling_matrix). H 1 = M3^Pi 1: G annihilates
// constants on every interior facet (its two cells contribute -k theta and +k theta with the
// same single-valued theta), so the numerator is the cell's M3^Pi, free of the cancellation
// of summing H's row. P 1 = 1; S 1 on each face is the sum of S_K 1 over the (one or two)
// cells sharing it; P^T weights 1/2 on interior faces and 1 on ground and lid faces.
__global__ void gamma_kernel(const RowArgs a, const double *__restrict__ sk1,
                             const double *__restrict__ rec, double *__restrict__ gamma) {
  const int64_t K = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (K >= a.ncell) return;
  const int c = (int)(K / a.L), k = (int)(K - (int64_t)c * a.L);
  const int64_t C = a.ncell;
  const double h1 = rec[K * kCellData + CellRec::MPI];
  double ps1 = 0.0;
  for (int f = 0; f < 4; ++f) {
    const int nb = a.col_nbr[4 * (int64_t)c + f], nf = a.col_nbr_face[4 * (int64_t)c + f];
    ps1 += 0.5 * (sk1[f * C + K] + sk1[nf * C + (int64_t)nb * a.L + k]);
  }
  ps1 += k == 0 ? sk1[4 * C + K] : 0.5 * (sk1[4 * C + K] + sk1[5 * C + K - 1]);
  ps1 += k == a.L - 1 ? sk1[5 * C + K] : 0.5 * (sk1[5 * C + K] + sk1[4 * C + K + 1]);
  gamma[K] = h1 / ps1;
}

__global__ void to_float_kernel(const double *__restrict__ in, float *__restrict__ out, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (float)in[i];
}

static int to_float(Ctx *c, const double *in, float **out, int64_t n) {
  if (!*out) {
    int st = dev_alloc(c, out, (size_t)n);
    if (st) return st;
  }
  to_float_kernel<<<grid_for(n, 256) > 4096 ? 4096 : grid_for(n, 256), 256, 0, c->stream>>>(in, *out, n);
  HMG_CUDA(c, cudaGetLastError());
  return HMG_OK;
}

// The FP32 preconditioner's copies of the assembled lowest-order operators (S, Gamma, H on every
// level, then the factors with their copies through build_factors), made from the FP64 data on
// the device when a context switches to precision mixed: no reassembly.
int make_fp32(Ctx *c) {
  const Level &f = c->lv[0];
  int st;
  if ((st = to_float(c, c->S, &c->S32, (int64_t)kSlots * f.ntrace))) return st;
  if ((st = to_float(c, c->gamma, &c->gamma32, f.ncell))) return st;
  for (int l = 0; l < c->nmg; ++l) {
    Level &lv = c->lv[l];
    if ((st = to_float(c, lv.H, &lv.H32, (int64_t)kHCoef * lv.ncell))) return st;
  }
  c->have_fp32 = true;
  return build_factors(c);
}

// Relaxation-weighted Thomas factors of S^zz, 1/diag S^hh and H_z on every level for the
// current omega and mg_omega (and their FP32 copies when those exist). Rebuilt whenever
// either relaxation weight changes.
int build_factors(Ctx *c) {
  const Level &f = c->lv[0];
  RowArgs ra{f.nlev, f.nth, f.ntrace, f.ncell, f.edge_stencil, f.edge_fc, f.col_edges, f.col_nbr, f.col_nbr_face};
  trace_factor_kernel<<<grid_for(f.ncol, 128), 128, 0, c->stream>>>(ra, f.ncol, c->S, c->opt.omega, c->Sz_w,
                                                                    c->Sz_l, c->Sz_cp, c->Sh_w);
  HMG_CUDA(c, cudaGetLastError());
  for (int l = 0; l < c->nmg; ++l) {
    Level &lv = c->lv[l];
    HArgs ha{lv.nlev, lv.ncol, lv.ncell, lv.col_nbr, lv.col_nbr_face};
    pressure_factor_kernel<<<grid_for(lv.ncol, 128), 128, 0, c->stream>>>(ha, lv.H, c->opt.mg_omega, lv.Hz_w,
                                                                           lv.Hz_l, lv.Hz_cp);
    HMG_CUDA(c, cudaGetLastError());
  }
  int st;
  if (c->have_fp32) {
    if ((st = to_float(c, c->Sz_w, &c->Sz_w32, f.ntz))) return st;
    if ((st = to_float(c, c->Sz_l, &c->Sz_l32, f.ntz))) return st;
    if ((st = to_float(c, c->Sz_cp, &c->Sz_cp32, f.ntz))) return st;
    if ((st = to_float(c, c->Sh_w, &c->Sh_w32, f.nth))) return st;
    for (int l = 0; l < c->nmg; ++l) {
      Level &lv = c->lv[l];
      if ((st = to_float(c, lv.Hz_w, &lv.Hz_w32, lv.ncell))) return st;
      if ((st = to_float(c, lv.Hz_l, &lv.Hz_l32, lv.ncell))) return st;
      if ((st = to_float(c, lv.Hz_cp, &lv.Hz_cp32, lv.ncell))) return st;
    }
  }
  c->factor_omega = c->opt.omega;
  c->factor_mg_omega = c->opt.mg_omega;
  return HMG_OK;
}

int assemble_all(Ctx *c) {
  if (!c->have_mesh || !c->have_coeffs) return fail(c, HMG_ERR_NOT_READY, "mesh or coefficients not set");
  // per-level cell records
  double *rec[kMaxLevels] = {nullptr};
  int st0;
  if ((st0 = upload_shape_functions(c))) return st0;
  for (int l = 0; l < c->nmg; ++l) {
    Level &lv = c->lv[l];
    HMG_CUDA(c, cudaMalloc(&rec[l], (size_t)lv.ncell * kCellData * sizeof(double)));
    CellArgs a{lv.geometry, lv.ncol, lv.nlev, lv.ncell, lv.radius, lv.corners, lv.z,
               lv.theta_lev, lv.exner_lev, lv.exner, lv.col_nbr, c->sc};
    cell_kernel<<<grid_for(lv.ncell, 128), 128, 0, c->stream>>>(a, rec[l]);
    HMG_CUDA(c, cudaGetLastError());
  }
  Level &f = c->lv[0];
  const int64_t C = f.ncell, T = f.ntrace;
  int st;
  if (!c->S) {
    if ((st = dev_alloc(c, &c->S, (size_t)kSlots * T))) return st;
    if ((st = dev_alloc(c, &c->Sz_w, (size_t)f.ntz))) return st;
    if ((st = dev_alloc(c, &c->Sz_l, (size_t)f.ntz))) return st;
    if ((st = dev_alloc(c, &c->Sz_cp, (size_t)f.ntz))) return st;
    if ((st = dev_alloc(c, &c->Sh_w, (size_t)f.nth))) return st;
    if ((st = dev_alloc(c, &c->Ainv, (size_t)49 * C))) return st;
    if ((st = dev_alloc(c, &c->kth, (size_t)6 * C))) return st;
    if ((st = dev_alloc(c, &c->gamma, (size_t)C))) return st;
  }
  double *SK = nullptr, *sk1 = nullptr;
  int *singular = nullptr;
  HMG_CUDA(c, cudaMalloc(&SK, (size_t)36 * C * sizeof(double)));
  HMG_CUDA(c, cudaMalloc(&sk1, (size_t)6 * C * sizeof(double)));
  HMG_CUDA(c, cudaMalloc(&singular, sizeof(int)));
  HMG_CUDA(c, cudaMemsetAsync(singular, 0, sizeof(int), c->stream));
  condense_kernel<<<grid_for(C, 128), 128, 0, c->stream>>>(C, rec[0], c->Ainv, SK, c->kth, sk1, singular);
  HMG_CUDA(c, cudaGetLastError());
  RowArgs ra{f.nlev, f.nth, T, C, f.edge_stencil, f.edge_fc, f.col_edges, f.col_nbr, f.col_nbr_face};
  trace_rows_kernel<<<grid_for(T, 256), 256, 0, c->stream>>>(ra, SK, c->S);
  HMG_CUDA(c, cudaGetLastError());
  for (int l = 0; l < c->nmg; ++l) {
    Level &lv = c->lv[l];
    if (!lv.H) {
      if ((st = dev_alloc(c, &lv.H, (size_t)kHCoef * lv.ncell))) return st;
      if ((st = dev_alloc(c, &lv.Hz_w, (size_t)lv.ncell))) return st;
      if ((st = dev_alloc(c, &lv.Hz_l, (size_t)lv.ncell))) return st;
      if ((st = dev_alloc(c, &lv.Hz_cp, (size_t)lv.ncell))) return st;
    }
    HArgs ha{lv.nlev, lv.ncol, lv.ncell, lv.col_nbr, lv.col_nbr_face};
    pressure_rows_kernel<<<grid_for(lv.ncell, 256), 256, 0, c->stream>>>(ha, rec[l], lv.H);
    HMG_CUDA(c, cudaGetLastError());
  }
  gamma_kernel<<<grid_for(C, 256), 256, 0, c->stream>>>(ra, sk1, rec[0], c->gamma);
  HMG_CUDA(c, cudaGetLastError());
  if (c->opt.precond == HMG_PRECOND_SCHUR && (st = build_mixed(c, rec[0]))) return st;
  if (c->opt.precision == HMG_PRECISION_MIXED && !c->have_fp32) {
    if ((st = to_float(c, c->S, &c->S32, (int64_t)kSlots * T))) return st;
    if ((st = to_float(c, c->gamma, &c->gamma32, C))) return st;
    for (int l = 0; l < c->nmg; ++l) {
      Level &lv = c->lv[l];
      if ((st = to_float(c, lv.H, &lv.H32, (int64_t)kHCoef * lv.ncell))) return st;
    }
    c->have_fp32 = true;
  }
  if ((st = build_factors(c))) return st;
  int sing = 0;
  HMG_CUDA(c, cudaMemcpyAsync(&sing, singular, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  HMG_CUDA(c, cudaStreamSynchronize(c->stream));
  cudaFree(SK);
  cudaFree(sk1);
  cudaFree(singular);
  for (int l = 0; l < c->nmg; ++l) cudaFree(rec[l]);
  if (sing) return fail(c, HMG_ERR_INVALID_ARG, "a velocity mass block M_K is not positive definite or A_K is singular");
  return HMG_OK;
}

}  // namespace hmg
