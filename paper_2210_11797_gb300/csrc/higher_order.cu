// The hybridised system of degree p = 1 (broken RT_1 velocity, DG_1 pressure, Q_1 trace
// multipliers: four per facet) for the constant-coefficient Helmholtz form of the operator,
// and its non-nested two-level preconditioner with the piecewise-constant coarse space.
//
// Paper (arXiv 2210.11797): Sec. 2.2 (spaces of degree p, n = p + 3 Gauss points per
// direction), Sec. 2.4 (Eqs. hybrid-S, hybrid-rhs, hybrid-recovery), Sec. 4.1 and the table
// of unknowns per cell (24 x 24 hybridised and 44 x 44 mixed cell matrices at p = 1),
// Algorithm 1 (here on facet blocks and block-tridiagonal columns), Algorithm 2 with the DG0
// coarse space of Sec. 2.5 (P lambda = {{Pi}}, Restrict = P^T, Eq. scaling_matrix) and the
// lowest-order pressure multigrid as its coarse solve.
//
// Numbering. Cell dofs: the 36 RT_1 dofs (24 facet dofs, face f = e0..e3, bottom, top, node
// (s, t) at 4 f + 2 s + t, each the cell's outward normal flux at a Gauss-Legendre node of the
// facet; then 12 interior dofs), then the 8 DG_1 dofs. Trace rows: four per facet, facet-major:
// vertical facet (edge e, level k) at 4 (e L + k), horizontal facet (column c, interface k) at
// NH + 4 (c (L + 1) + k), node (s, t) at + 2 s + t; on a vertical facet s counts along the edge
// in the traversal of its owner column (the other column's local s is 1 - s).
#include <cmath>
#include <vector>

#include "device_common.cuh"
#include "hmg_internal.cuh"
#include "precond.cuh"

namespace hmg {

constexpr int kHoNu = 36;                 // RT_1 dofs
constexpr int kHoNp = 8;                  // DG_1 dofs
constexpr int kHoN = kHoNu + kHoNp;       // 44: the mixed cell matrix
constexpr int kHoNf = 24;                 // facet dofs (the hybridised cell matrix is 24 x 24)
constexpr int kHoQ = 64;                  // 4 x 4 x 4 Gauss points
constexpr int kHoSlots = 48;              // S coefficients stored per trace row (two cells x 24)
constexpr int kHoTabV = 0, kHoTabPhi = kHoTabV + kHoQ * kHoNu, kHoTabW = kHoTabPhi + kHoQ * kHoNp,
              kHoTabX = kHoTabW + kHoQ, kHoTabG = kHoTabX + 3 * kHoQ, kHoTab = kHoTabG + kHoNu * kHoNp;
constexpr double kHoC = 0.25;             // C_K on a facet dof: the product of two Gauss-Legendre weights 1/2

// ---- reference tables, formed on the host ---------------------------------------------------
// 1-D Lagrange values / derivatives, the RT_1 basis (value of its one nonzero component and its
// divergence) and the DG_1 basis at the 64 Gauss points, and G(f, j) = -int phi_j div v_f.
static void lagrange1d(const double *nodes, int n, double x, double *val, double *der) {
  for (int i = 0; i < n; ++i) {
    double v = 1.0, d = 0.0;
    for (int j = 0; j < n; ++j)
      if (j != i) v *= (x - nodes[j]) / (nodes[i] - nodes[j]);
    for (int m = 0; m < n; ++m) {
      if (m == i) continue;
      double t = 1.0 / (nodes[i] - nodes[m]);
      for (int j = 0; j < n; ++j)
        if (j != i && j != m) t *= (x - nodes[j]) / (nodes[i] - nodes[j]);
      d += t;
    }
    val[i] = v;
    der[i] = d;
  }
}

// component, normal node (0 or 2), sign of the facet dofs of face f; (tangential node indices
// of the two other coordinates in increasing coordinate order) from the facet node (s, t)
static const int kFaceComp[6] = {1, 0, 1, 0, 2, 2};
static const int kFaceEnd[6] = {0, 2, 2, 0, 0, 2};
static const double kFaceSign[6] = {-1.0, 1.0, 1.0, -1.0, -1.0, 1.0};

struct HoDof { int d, a, b, c; double sign; };

static std::vector<HoDof> ho_dofs() {
  std::vector<HoDof> v;
  for (int f = 0; f < 6; ++f)
    for (int s = 0; s < 2; ++s)
      for (int t = 0; t < 2; ++t) {
        const int b = (f == 2 || f == 3) ? 1 - s : s;   // e2, e3 traverse their edge backwards
        v.push_back({kFaceComp[f], kFaceEnd[f], b, t, kFaceSign[f]});
      }
  for (int d = 0; d < 3; ++d)
    for (int b = 0; b < 2; ++b)
      for (int c = 0; c < 2; ++c) v.push_back({d, 1, b, c, 1.0});
  return v;
}

static void ho_tables(std::vector<double> &tab) {
  tab.assign(kHoTab, 0.0);
  const double g = 0.5 / std::sqrt(3.0);
  const double gl[2] = {0.5 - g, 0.5 + g};
  const double gll[3] = {0.0, 0.5, 1.0};
  const double r1 = std::sqrt(3.0 / 7.0 - 2.0 / 7.0 * std::sqrt(6.0 / 5.0));
  const double r2 = std::sqrt(3.0 / 7.0 + 2.0 / 7.0 * std::sqrt(6.0 / 5.0));
  const double w1 = (18.0 + std::sqrt(30.0)) / 36.0, w2 = (18.0 - std::sqrt(30.0)) / 36.0;
  const double qx[4] = {0.5 * (1.0 - r2), 0.5 * (1.0 - r1), 0.5 * (1.0 + r1), 0.5 * (1.0 + r2)};
  const double qw[4] = {0.5 * w2, 0.5 * w1, 0.5 * w1, 0.5 * w2};
  const std::vector<HoDof> dofs = ho_dofs();
  for (int a = 0; a < 4; ++a)
    for (int b = 0; b < 4; ++b)
      for (int c = 0; c < 4; ++c) {
        const int q = (a * 4 + b) * 4 + c;
        const double x[3] = {qx[a], qx[b], qx[c]};
        double tv[3][2], td[3][2], nv[3][3], nd[3][3];
        for (int k = 0; k < 3; ++k) {
          lagrange1d(gl, 2, x[k], tv[k], td[k]);
          lagrange1d(gll, 3, x[k], nv[k], nd[k]);
        }
        tab[kHoTabW + q] = qw[a] * qw[b] * qw[c];
        for (int k = 0; k < 3; ++k) tab[kHoTabX + 3 * q + k] = x[k];
        for (int i = 0; i < kHoNu; ++i) {
          const HoDof &o = dofs[i];
          int t1 = 0, t2 = 0;
          if (o.d == 0) { t1 = 1; t2 = 2; } else if (o.d == 1) { t1 = 0; t2 = 2; } else { t1 = 0; t2 = 1; }
          const double tan = tv[t1][o.b] * tv[t2][o.c];
          tab[kHoTabV + q * kHoNu + i] = o.sign * nv[o.d][o.a] * tan;
          // divergence: the derivative of the one nonzero component along its own coordinate
          const double dv = o.sign * nd[o.d][o.a] * tan;
          for (int ii = 0; ii < 2; ++ii)
            for (int jj = 0; jj < 2; ++jj)
              for (int kk = 0; kk < 2; ++kk) {
                const int j = (ii * 2 + jj) * 2 + kk;
                const double phi = tv[0][ii] * tv[1][jj] * tv[2][kk];
                tab[kHoTabG + i * kHoNp + j] -= tab[kHoTabW + q] * dv * phi;
              }
        }
        for (int ii = 0; ii < 2; ++ii)
          for (int jj = 0; jj < 2; ++jj)
            for (int kk = 0; kk < 2; ++kk)
              tab[kHoTabPhi + q * kHoNp + (ii * 2 + jj) * 2 + kk] = tv[0][ii] * tv[1][jj] * tv[2][kk];
      }
}

__device__ __forceinline__ int ho_comp(int i) {   // the nonzero component of velocity dof i
  if (i < kHoNf) {
    const int f = i >> 2;
    return f == 0 || f == 2 ? 1 : (f == 1 || f == 3 ? 0 : 2);
  }
  return (i - kHoNf) >> 2;
}

// ---- mesh access ------------------------------------------------------------------------------
struct HoGeo {
  int L, ncol;
  int64_t NH;                 // rows of the vertical facets (4 nedge L)
  int64_t nhf, nzf;           // vertical and horizontal facets
  const int32_t *col_edges, *stencil, *edge_fc;
  const int8_t *own;          // [ncol][4] 1 if the column owns the edge of that face
};

// trace row of local facet dof q of cell (c, k)
__device__ __forceinline__ int64_t ho_gid(const HoGeo &g, int c, int k, int q) {
  const int f = q >> 2, s = (q >> 1) & 1, t = q & 1;
  if (f < 4) {
    const int64_t e = g.col_edges[4 * (int64_t)c + f];
    const int sg = g.own[4 * (int64_t)c + f] ? s : 1 - s;
    return 4 * (e * g.L + k) + 2 * sg + t;
  }
  const int kk = k + (f == 5 ? 1 : 0);
  return g.NH + 4 * ((int64_t)c * (g.L + 1) + kk) + 2 * s + t;
}

// The one or two cells of facet F: A (and B), their local faces, and whether a node's local s is
// reversed in B (vertical facets: B traverses the edge backwards).
struct HoFacet {
  int cA, kA, fA, cB, kB, fB;   // cB < 0: a ground or lid facet (one cell)
  bool flipB;
};

__device__ __forceinline__ HoFacet ho_facet(const HoGeo &g, int64_t F) {
  HoFacet r;
  if (F < g.nhf) {
    const int e = (int)(F / g.L), k = (int)(F - (int64_t)e * g.L);
    r.cA = g.stencil[8 * (int64_t)e];
    r.cB = g.stencil[8 * (int64_t)e + 1];
    r.fA = g.edge_fc[2 * (int64_t)e];
    r.fB = g.edge_fc[2 * (int64_t)e + 1];
    r.kA = r.kB = k;
    r.flipB = true;
  } else {
    const int64_t zf = F - g.nhf;
    const int c = (int)(zf / (g.L + 1)), k = (int)(zf - (int64_t)c * (g.L + 1));
    r.cA = c;
    r.flipB = false;
    if (k < g.L) {
      r.kA = k;
      r.fA = 4;                                  // the facet is the bottom of the cell above
      r.cB = k > 0 ? c : -1;
      r.kB = k - 1;
      r.fB = 5;
    } else {
      r.kA = g.L - 1;
      r.fA = 5;                                  // the lid: the top of the last cell
      r.cB = -1;
      r.kB = 0;
      r.fB = 0;
    }
  }
  return r;
}

// acc[n] (+/-)= sum over the stored slots of row 4F + n times x: cell A's 24 facet dofs, then
// cell B's without the shared facet (merged into A's slots when S was assembled). OFFD leaves out
// the couplings inside the smoother's diagonal block D of Algorithm 1 (acc - (S - D) x): on a
// vertical facet its own four nodes, on a horizontal facet the horizontal facets of its column
// (A's bottom and top, B's bottom).
template <bool NEG, bool OFFD = false>
__device__ __forceinline__ void ho_rows(const double *__restrict__ S, const double *__restrict__ x, const HoGeo &g,
                                        int64_t T, int64_t F, double acc[4]) {
  const HoFacet fc = ho_facet(g, F);
  const double *Sr = S + 4 * F;
  const bool vert = F < g.nhf;
#pragma unroll 4
  for (int q = 0; q < kHoNf; ++q) {
    if (OFFD && (vert ? (q >> 2) == fc.fA : (q >> 2) >= 4)) continue;
    const double xv = __ldg(x + ho_gid(g, fc.cA, fc.kA, q));
    const double2 s01 = __ldcs(reinterpret_cast<const double2 *>(Sr + (int64_t)q * T));
    const double2 s23 = __ldcs(reinterpret_cast<const double2 *>(Sr + (int64_t)q * T + 2));
    acc[0] = fma(NEG ? -s01.x : s01.x, xv, acc[0]);
    acc[1] = fma(NEG ? -s01.y : s01.y, xv, acc[1]);
    acc[2] = fma(NEG ? -s23.x : s23.x, xv, acc[2]);
    acc[3] = fma(NEG ? -s23.y : s23.y, xv, acc[3]);
  }
  if (fc.cB < 0) return;
#pragma unroll 4
  for (int q = 0; q < kHoNf; ++q) {
    if ((q >> 2) == fc.fB || (OFFD && !vert && (q >> 2) >= 4)) continue;
    const double xv = __ldg(x + ho_gid(g, fc.cB, fc.kB, q));
    const double2 s01 = __ldcs(reinterpret_cast<const double2 *>(Sr + (int64_t)(kHoNf + q) * T));
    const double2 s23 = __ldcs(reinterpret_cast<const double2 *>(Sr + (int64_t)(kHoNf + q) * T + 2));
    acc[0] = fma(NEG ? -s01.x : s01.x, xv, acc[0]);
    acc[1] = fma(NEG ? -s01.y : s01.y, xv, acc[1]);
    acc[2] = fma(NEG ? -s23.x : s23.x, xv, acc[2]);
    acc[3] = fma(NEG ? -s23.y : s23.y, xv, acc[3]);
  }
}

// ---- assembly -------------------------------------------------------------------------------
struct HoCellArgs {
  int geometry, ncol, L;
  int64_t ncell;
  double radius, sigma;
  const double *corners, *z;
};

// A_K = [[M, G], [-G^T, Mp]] by the 4 x 4 x 4 Gauss rule (M with the contravariant Piola map,
// Mp = sigma int phi_i phi_j), then A_K^-1 by Gauss-Jordan elimination with partial pivoting
// of the symmetrically equilibrated D A_K D, D = |diag A_K|^-1/2: A^-1 = D (D A D)^-1 D.
// One cell per block; m[K] = sigma |K|_1 (the one-point volume), H 1 of the coarse operator.
__global__ void __launch_bounds__(128)
    ho_cell_kernel(const HoCellArgs a, const double *__restrict__ tab, double *__restrict__ Ainv,
                   double *__restrict__ mK, int *singular) {
  __shared__ double X[8][3];
  __shared__ double Kq[kHoQ][6];   // (w / det) J^T J: xx, yy, zz, xy, xz, yz
  __shared__ double wd[kHoQ];      // sigma w det
  __shared__ double Ag[kHoN][2 * kHoN + 1];
  __shared__ double dsc[kHoN], fac[kHoN];
  __shared__ int piv;
  const int64_t K = blockIdx.x;
  const int tid = threadIdx.x;
  const int c = (int)(K / a.L), k = (int)(K - (int64_t)c * a.L);
  if (tid < 8) {
    const int va = tid & 1, vb = (tid >> 1) & 1, vc = (tid >> 2) & 1;
    const int corner = va == 0 ? (vb == 0 ? 0 : 3) : (vb == 0 ? 1 : 2);
    const double *cp = a.corners + (4 * (int64_t)c + corner) * 3;
    const double h = a.z[k + vc];
    if (a.geometry == 1) {
      for (int i = 0; i < 3; ++i) X[tid][i] = cp[i] * (a.radius + h);
    } else {
      X[tid][0] = cp[0];
      X[tid][1] = cp[1];
      X[tid][2] = h;
    }
  }
  __syncthreads();
  auto jacobian = [&](double xi, double eta, double zeta, double J[3][3]) {
    for (int i = 0; i < 3; ++i) J[i][0] = J[i][1] = J[i][2] = 0.0;
    for (int v = 0; v < 8; ++v) {
      const int va = v & 1, vb = (v >> 1) & 1, vc = (v >> 2) & 1;
      const double fx = va ? xi : 1.0 - xi, fy = vb ? eta : 1.0 - eta, fz = vc ? zeta : 1.0 - zeta;
      const double gx = va ? 1.0 : -1.0, gy = vb ? 1.0 : -1.0, gz = vc ? 1.0 : -1.0;
      const double dn[3] = {gx * fy * fz, fx * gy * fz, fx * fy * gz};
      for (int i = 0; i < 3; ++i)
        for (int d = 0; d < 3; ++d) J[i][d] += X[v][i] * dn[d];
    }
  };
  auto det3 = [](const double J[3][3]) {
    return J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) - J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
           J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
  };
  if (tid < kHoQ) {
    const double *xq = tab + kHoTabX + 3 * tid;
    double J[3][3];
    jacobian(xq[0], xq[1], xq[2], J);
    const double det = det3(J), w = tab[kHoTabW + tid];
    double G[3][3];
    for (int p = 0; p < 3; ++p)
      for (int q = 0; q < 3; ++q) G[p][q] = J[0][p] * J[0][q] + J[1][p] * J[1][q] + J[2][p] * J[2][q];
    const double s = w / det;
    Kq[tid][0] = s * G[0][0];
    Kq[tid][1] = s * G[1][1];
    Kq[tid][2] = s * G[2][2];
    Kq[tid][3] = s * G[0][1];
    Kq[tid][4] = s * G[0][2];
    Kq[tid][5] = s * G[1][2];
    wd[tid] = a.sigma * w * det;
  } else if (tid == kHoQ) {
    double J[3][3];
    jacobian(0.5, 0.5, 0.5, J);
    mK[K] = a.sigma * det3(J);
  }
  __syncthreads();
  const double *tv = tab + kHoTabV, *tp = tab + kHoTabPhi, *tg = tab + kHoTabG;
  for (int idx = tid; idx < kHoN * kHoN; idx += blockDim.x) {
    const int i = idx / kHoN, j = idx - i * kHoN;
    double v = 0.0;
    if (i < kHoNu && j < kHoNu) {
      const int di = ho_comp(i), dj = ho_comp(j);
      const int kk = di == dj ? di : (di + dj == 1 ? 3 : (di + dj == 2 ? 4 : 5));
      for (int q = 0; q < kHoQ; ++q) v = fma(__ldg(tv + q * kHoNu + i) * __ldg(tv + q * kHoNu + j), Kq[q][kk], v);
    } else if (i < kHoNu) {
      v = __ldg(tg + i * kHoNp + (j - kHoNu));
    } else if (j < kHoNu) {
      v = -__ldg(tg + j * kHoNp + (i - kHoNu));
    } else {
      for (int q = 0; q < kHoQ; ++q)
        v = fma(wd[q] * __ldg(tp + q * kHoNp + (i - kHoNu)), __ldg(tp + q * kHoNp + (j - kHoNu)), v);
    }
    Ag[i][j] = v;
    Ag[i][kHoN + j] = i == j ? 1.0 : 0.0;
  }
  __syncthreads();
  if (tid < kHoN) dsc[tid] = 1.0 / sqrt(fabs(Ag[tid][tid]));
  __syncthreads();
  for (int idx = tid; idx < kHoN * kHoN; idx += blockDim.x) {
    const int i = idx / kHoN, j = idx - i * kHoN;
    Ag[i][j] *= dsc[i] * dsc[j];
  }
  __syncthreads();
  for (int col = 0; col < kHoN; ++col) {
    if (tid == 0) {
      int p = col;
      double best = fabs(Ag[col][col]);
      for (int r = col + 1; r < kHoN; ++r)
        if (fabs(Ag[r][col]) > best) { best = fabs(Ag[r][col]); p = r; }
      if (!(best > 0.0)) atomicExch(singular, 1);
      piv = p;
    }
    __syncthreads();
    const int p = piv;
    if (p != col)
      for (int j = tid; j < 2 * kHoN; j += blockDim.x) {
        const double t = Ag[col][j];
        Ag[col][j] = Ag[p][j];
        Ag[p][j] = t;
      }
    __syncthreads();
    if (tid < kHoN) fac[tid] = Ag[tid][col];
    __syncthreads();
    const double pinv = 1.0 / fac[col];
    for (int j = tid; j < 2 * kHoN; j += blockDim.x) Ag[col][j] *= pinv;
    __syncthreads();
    for (int idx = tid; idx < kHoN * 2 * kHoN; idx += blockDim.x) {
      const int r = idx / (2 * kHoN), j = idx - r * 2 * kHoN;
      if (r != col) Ag[r][j] = fma(-fac[r], Ag[col][j], Ag[r][j]);
    }
    __syncthreads();
  }
  double *out = Ainv + K * (kHoN * kHoN);
  for (int idx = tid; idx < kHoN * kHoN; idx += blockDim.x) {
    const int i = idx / kHoN, j = idx - i * kHoN;
    out[idx] = dsc[i] * Ag[i][kHoN + j] * dsc[j];
  }
}

// own[c][f] = 1 where column c owns the edge of its face f (each entry written by one edge)
__global__ void ho_own_kernel(const int32_t *__restrict__ stencil, const int32_t *__restrict__ edge_fc, int nedge,
                              int8_t *__restrict__ own) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nedge) return;
  own[4 * (int64_t)stencil[8 * (int64_t)e] + edge_fc[2 * (int64_t)e]] = 1;
  own[4 * (int64_t)stencil[8 * (int64_t)e + 1] + edge_fc[2 * (int64_t)e + 1]] = 0;
}

// Rows of S = sum_K C_K^T A_K^-1 C_K (C_K = 1/4 on every facet dof): row 4F + n holds, in slots
// 0-23, (1/16) A_A^-1 restricted to the facet dofs of cell A (row: the node's local index in A),
// and in slots 24-47 the same of cell B, whose shared-facet entries are added into A's slots.
__global__ void ho_rows_kernel(const HoGeo g, int64_t T, const double *__restrict__ Ainv, double *__restrict__ S) {
  const int64_t row = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (row >= T) return;
  const int64_t F = row >> 2;
  const int n = (int)(row & 3), s = n >> 1, t = n & 1;
  const HoFacet fc = ho_facet(g, F);
  const int qa = 4 * fc.fA + 2 * s + t;
  const double *IA = Ainv + ((int64_t)fc.cA * g.L + fc.kA) * (kHoN * kHoN) + qa * kHoN;
  double v[kHoNf];
  for (int q = 0; q < kHoNf; ++q) v[q] = kHoC * kHoC * IA[q];
  if (fc.cB >= 0) {
    const int sb = fc.flipB ? 1 - s : s;
    const int qb = 4 * fc.fB + 2 * sb + t;
    const double *IB = Ainv + ((int64_t)fc.cB * g.L + fc.kB) * (kHoN * kHoN) + qb * kHoN;
    for (int q = 0; q < kHoNf; ++q) {
      const double w = kHoC * kHoC * IB[q];
      if ((q >> 2) == fc.fB) {   // the shared facet: the same trace row as A's node
        const int sq = (q >> 1) & 1, tq = q & 1;
        const int sa = fc.flipB ? 1 - sq : sq;
        v[4 * fc.fA + 2 * sa + tq] += w;
        S[(int64_t)(kHoNf + q) * T + row] = 0.0;
      } else {
        S[(int64_t)(kHoNf + q) * T + row] = w;
      }
    }
  } else {
    for (int q = 0; q < kHoNf; ++q) S[(int64_t)(kHoNf + q) * T + row] = 0.0;
  }
  for (int q = 0; q < kHoNf; ++q) S[(int64_t)q * T + row] = v[q];
}

// 4 x 4 inverse by Gauss-Jordan elimination with partial pivoting; false if singular
__device__ bool inv4(const double A[4][4], double R[4][4]) {
  double M[4][8];
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) {
      M[i][j] = A[i][j];
      M[i][4 + j] = i == j ? 1.0 : 0.0;
    }
  for (int c = 0; c < 4; ++c) {
    int p = c;
    for (int r = c + 1; r < 4; ++r)
      if (fabs(M[r][c]) > fabs(M[p][c])) p = r;
    if (!(fabs(M[p][c]) > 0.0)) return false;
    if (p != c)
      for (int j = 0; j < 8; ++j) { const double t = M[c][j]; M[c][j] = M[p][j]; M[p][j] = t; }
    const double inv = 1.0 / M[c][c];
    for (int j = 0; j < 8; ++j) M[c][j] *= inv;
    for (int r = 0; r < 4; ++r) {
      if (r == c) continue;
      const double f = M[r][c];
      for (int j = 0; j < 8; ++j) M[r][j] = fma(-f, M[c][j], M[r][j]);
    }
  }
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) R[i][j] = M[i][4 + j];
  return true;
}

// omega times the inverse of each vertical facet's 4 x 4 block of S (the Jacobi part of
// Algorithm 1), entry (n, m) at hw[(4 n + m) nhf + F]. The facet block lives in the slots of
// cell A's face (A owns the edge, so its local nodes are the facet's).
__global__ void ho_hfactor_kernel(const HoGeo g, int64_t T, const double *__restrict__ S, double omega,
                                  double *__restrict__ hw, int *singular) {
  const int64_t F = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (F >= g.nhf) return;
  const HoFacet fc = ho_facet(g, F);
  double D[4][4], R[4][4];
  for (int n = 0; n < 4; ++n)
    for (int m = 0; m < 4; ++m) D[n][m] = S[(int64_t)(4 * fc.fA + m) * T + 4 * F + n];
  if (!inv4(D, R)) atomicExch(singular, 1);
  for (int n = 0; n < 4; ++n)
    for (int m = 0; m < 4; ++m) hw[(int64_t)(4 * n + m) * g.nhf + F] = omega * R[n][m];
}

// Block Thomas factors of each column's block-tridiagonal S^zz (blocks D_k, L_k = coupling of
// facet k to k - 1, U_k to k + 1): G_0 = D_0, G_k = D_k - L_k G_{k-1}^-1 U_{k-1}; stored per
// horizontal facet: omega G_k^-1, G_k^-1 L_k, G_k^-1 U_k ([nzf][48], 16 entries each), so that
// omega (S^zz)^-1 r is y_k = (omega G_k^-1) r_k - (G_k^-1 L_k) y_{k-1}, x_k = y_k - (G_k^-1 U_k) x_{k+1}.
__global__ void ho_zfactor_kernel(const HoGeo g, int64_t T, const double *__restrict__ S, double omega,
                                  double *__restrict__ zf, int *singular) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= g.ncol) return;
  const int L = g.L;
  double GU[4][4];   // G_{k-1}^-1 U_{k-1}
  for (int k = 0; k <= L; ++k) {
    const int64_t F = (int64_t)c * (L + 1) + k, row0 = g.NH + 4 * F;
    double D[4][4], Lk[4][4], U[4][4];
    // slots: cell above (c, k) [A, k < L]: bottom 16-19 (this facet), top 20-23 (facet k + 1);
    // cell below (c, k - 1) [B]: bottom 40-43 (facet k - 1). The lid row's A is the cell below:
    // its top 20-23 is this facet, its bottom 16-19 the facet below.
    for (int n = 0; n < 4; ++n)
      for (int m = 0; m < 4; ++m) {
        const double *r = S + row0 + n;
        if (k < L) {
          D[n][m] = r[(int64_t)(16 + m) * T];
          U[n][m] = r[(int64_t)(20 + m) * T];
          Lk[n][m] = k > 0 ? r[(int64_t)(40 + m) * T] : 0.0;
        } else {
          D[n][m] = r[(int64_t)(20 + m) * T];
          Lk[n][m] = r[(int64_t)(16 + m) * T];
          U[n][m] = 0.0;
        }
      }
    if (k > 0)
      for (int n = 0; n < 4; ++n)
        for (int m = 0; m < 4; ++m) {
          double s = D[n][m];
          for (int j = 0; j < 4; ++j) s = fma(-Lk[n][j], GU[j][m], s);
          D[n][m] = s;
        }
    double Gi[4][4];
    if (!inv4(D, Gi)) atomicExch(singular, 1);
    double GL[4][4];
    for (int n = 0; n < 4; ++n)
      for (int m = 0; m < 4; ++m) {
        double sl = 0.0, su = 0.0;
        for (int j = 0; j < 4; ++j) {
          sl = fma(Gi[n][j], Lk[j][m], sl);
          su = fma(Gi[n][j], U[j][m], su);
        }
        GL[n][m] = sl;
        GU[n][m] = su;
      }
    double *o = zf + 48 * ((int64_t)c * (L + 1) + k);   // facet-major: 48 contiguous factors
    for (int n = 0; n < 4; ++n)
      for (int m = 0; m < 4; ++m) {
        o[4 * n + m] = omega * Gi[n][m];
        o[16 + 4 * n + m] = GL[n][m];
        o[32 + 4 * n + m] = GU[n][m];
      }
  }
}

// ---- the operator, the right-hand side and the recovery --------------------------------------
// y = S x, one thread per facet (its four rows share the gathered values); MODE 1, 2, 3 fuse the
// inner products of the Krylov loop as the lowest-order S apply does (3: (b - S x, b - S x), no y).
template <int MODE>
__global__ void __launch_bounds__(kRedThreads)
    ho_spmv_kernel(const HoGeo g, int64_t T, const double *__restrict__ S, const double *__restrict__ x,
                   double *__restrict__ y, const double *__restrict__ w, double *part, int slot0, int slot1) {
  const int64_t F = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  double a0 = 0.0, a1 = 0.0;
  if (F < g.nhf + g.nzf) {
    double acc[4];
    if (MODE == 3) {
      for (int n = 0; n < 4; ++n) acc[n] = __ldg(w + 4 * F + n);
      ho_rows<true>(S, x, g, T, F, acc);
      for (int n = 0; n < 4; ++n) a0 = fma(acc[n], acc[n], a0);
    } else {
      acc[0] = acc[1] = acc[2] = acc[3] = 0.0;
      ho_rows<false>(S, x, g, T, F, acc);
      for (int n = 0; n < 4; ++n) {
        y[4 * F + n] = acc[n];
        if (MODE == 1) a0 = fma(__ldg(w + 4 * F + n), acc[n], a0);
        if (MODE == 2) { a0 = fma(acc[n], __ldg(w + 4 * F + n), a0); a1 = fma(acc[n], acc[n], a1); }
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

// B_lambda row 4F + n: the sum over the facet's cells of (1/4) (A_K^-1 R_K) at the node's local dof
__global__ void ho_rhs_kernel(const HoGeo g, int64_t T, const double *__restrict__ Ainv,
                              const double *__restrict__ Ru, const double *__restrict__ Rp,
                              double *__restrict__ B) {
  const int64_t row = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (row >= T) return;
  const int64_t F = row >> 2;
  const int n = (int)(row & 3), s = n >> 1, t = n & 1;
  const HoFacet fc = ho_facet(g, F);
  auto cell = [&](int cc, int kk, int q) {
    const int64_t K = (int64_t)cc * g.L + kk;
    const double *I = Ainv + K * (kHoN * kHoN) + q * kHoN;
    double v = 0.0;
    for (int j = 0; j < kHoNu; ++j) v = fma(I[j], Ru[K * kHoNu + j], v);
    for (int j = 0; j < kHoNp; ++j) v = fma(I[kHoNu + j], Rp[K * kHoNp + j], v);
    return kHoC * v;
  };
  double v = cell(fc.cA, fc.kA, 4 * fc.fA + 2 * s + t);
  if (fc.cB >= 0) v += cell(fc.cB, fc.kB, 4 * fc.fB + 2 * (fc.flipB ? 1 - s : s) + t);
  B[row] = v;
}

// X_K = A_K^-1 (R_K - C_K lambda_K): u [ncell][36], pi [ncell][8]; one thread per (cell, dof)
__global__ void ho_reconstruct_kernel(const HoGeo g, int64_t ncell, const double *__restrict__ Ainv,
                                      const double *__restrict__ lam, const double *__restrict__ Ru,
                                      const double *__restrict__ Rp, double *__restrict__ u,
                                      double *__restrict__ pi) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= ncell * kHoN) return;
  const int64_t K = idx / kHoN;
  const int i = (int)(idx - K * kHoN);
  const int c = (int)(K / g.L), k = (int)(K - (int64_t)c * g.L);
  const double *I = Ainv + K * (kHoN * kHoN) + i * kHoN;
  double v = 0.0;
  for (int j = 0; j < kHoNu; ++j) {
    double r = Ru[K * kHoNu + j];
    if (j < kHoNf) r = fma(-kHoC, lam[ho_gid(g, c, k, j)], r);
    v = fma(I[j], r, v);
  }
  for (int j = 0; j < kHoNp; ++j) v = fma(I[kHoNu + j], Rp[K * kHoNp + j], v);
  if (i < kHoNu) u[K * kHoNu + i] = v;
  else pi[K * kHoNp + (i - kHoNu)] = v;
}

// ---- Algorithm 1 at p = 1 -----------------------------------------------------------------------
// lam_out = lam_in + omega D^-1 (b - S lam_in) (ZERO: lam_in = 0), evaluated as
// (1 - omega) lam_in + omega D^-1 (b - (S - D) lam_in): equal in exact arithmetic, without the
// 4 (vertical facets) or 12 (horizontal facets) couplings of a row inside D. Blocks [0, nzb) take CPB
// columns each: the residual rows of their horizontal facets staged in shared memory, then the
// block Thomas recurrences with four lanes per column (lane n computes component n of each 4 x 4
// product from its rows of the stored factors; the four lanes of a column sit in one warp and
// meet at __syncwarp between the steps); the other blocks take one vertical facet per thread
// (4 x 4 block Jacobi).
template <bool ZERO>
__global__ void __launch_bounds__(128)
    ho_sweep_kernel(const HoGeo g, int64_t T, int cpb, int nzb, const double *__restrict__ S,
                    const double *__restrict__ hw, const double *__restrict__ zf, const double *__restrict__ b,
                    const double *__restrict__ lam_in, double *__restrict__ lam_out, double keep) {
  extern __shared__ double sr[];   // [cpb][L+1][4]
  const int L1 = g.L + 1;
  if ((int)blockIdx.x < nzb) {
    const int c0 = blockIdx.x * cpb, nc = min(cpb, g.ncol - c0);
    for (int i = threadIdx.x; i < nc * L1; i += blockDim.x) {
      const int64_t F = g.nhf + (int64_t)c0 * L1 + i;
      double acc[4];
      for (int n = 0; n < 4; ++n) acc[n] = __ldg(b + 4 * F + n);
      if (!ZERO) ho_rows<true, true>(S, lam_in, g, T, F, acc);
      for (int n = 0; n < 4; ++n) sr[4 * i + n] = acc[n];
    }
    __syncthreads();
    const int cc = threadIdx.x >> 2, n = threadIdx.x & 3;
    const unsigned grp = 0xFu << (threadIdx.x & 28);   // the four lanes of this column
    if (cc < nc) {
      double *r = sr + 4 * cc * L1;
      const double *f0 = zf + 48 * ((int64_t)(c0 + cc) * L1);
      // forward: y_k = (omega G_k^-1) r_k - (G_k^-1 L_k) y_{k-1}, y written over r
      double yprev[4] = {0.0, 0.0, 0.0, 0.0};
      for (int k = 0; k < L1; ++k) {
        const double *f = f0 + 48 * k;
        double v = 0.0;
        for (int m = 0; m < 4; ++m) v = fma(__ldg(f + 4 * n + m), r[4 * k + m], v);
        for (int m = 0; m < 4; ++m) v = fma(-__ldg(f + 16 + 4 * n + m), yprev[m], v);
        __syncwarp(grp);
        r[4 * k + n] = v;
        __syncwarp(grp);
        for (int m = 0; m < 4; ++m) yprev[m] = r[4 * k + m];
      }
      // backward: x_k = y_k - (G_k^-1 U_k) x_{k+1}, x written over y
      for (int k = L1 - 2; k >= 0; --k) {
        const double *f = f0 + 48 * k;
        double v = r[4 * k + n];
        for (int m = 0; m < 4; ++m) v = fma(-__ldg(f + 32 + 4 * n + m), yprev[m], v);
        __syncwarp(grp);
        r[4 * k + n] = v;
        __syncwarp(grp);
        for (int m = 0; m < 4; ++m) yprev[m] = r[4 * k + m];
      }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nc * L1 * 4; i += blockDim.x) {
      const int64_t row = g.NH + 4 * (int64_t)c0 * L1 + i;
      lam_out[row] = ZERO ? sr[i] : fma(keep, lam_in[row], sr[i]);
    }
  } else {
    const int64_t F = (int64_t)(blockIdx.x - nzb) * blockDim.x + threadIdx.x;
    if (F >= g.nhf) return;
    double acc[4];
    for (int n = 0; n < 4; ++n) acc[n] = __ldg(b + 4 * F + n);
    if (!ZERO) ho_rows<true, true>(S, lam_in, g, T, F, acc);
    for (int n = 0; n < 4; ++n) {
      double v = ZERO ? 0.0 : keep * lam_in[4 * F + n];
      for (int m = 0; m < 4; ++m) v = fma(hw[(int64_t)(4 * n + m) * g.nhf + F], acc[m], v);
      lam_out[4 * F + n] = v;
    }
  }
}

// R = b - S lam (Algorithm 2 line 3), one thread per facet. ZSWEEP: lam is one sweep from zero,
// lam = omega D^-1 b, so R = (1 - omega) b - (S - D) lam (equal in exact arithmetic).
template <bool ZSWEEP>
__global__ void ho_residual_kernel(const HoGeo g, int64_t T, const double *__restrict__ S,
                                   const double *__restrict__ b, const double *__restrict__ lam,
                                   double *__restrict__ R, double keep) {
  const int64_t F = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (F >= g.nhf + g.nzf) return;
  double acc[4];
  for (int n = 0; n < 4; ++n) acc[n] = ZSWEEP ? keep * __ldg(b + 4 * F + n) : __ldg(b + 4 * F + n);
  ho_rows<true, ZSWEEP>(S, lam, g, T, F, acc);
  for (int n = 0; n < 4; ++n) R[4 * F + n] = acc[n];
}

// bbar_K = Gamma_K (P^T R)_K (Algorithm 2 lines 4-5): P is constant on a facet (all four nodes)
// and averages the facet's cells, so P^T sums the cell's 24 facet nodes with weight 1/2 (1 on
// ground and lid facets)
__global__ void ho_restrict_kernel(const HoGeo g, int64_t ncell, const double *__restrict__ R,
                                   const double *__restrict__ gamma, double *__restrict__ bbar) {
  const int64_t K = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (K >= ncell) return;
  const int c = (int)(K / g.L), k = (int)(K - (int64_t)c * g.L);
  double s = 0.0;
  for (int q = 0; q < kHoNf; ++q) {
    const int f = q >> 2;
    const bool boundary = (f == 4 && k == 0) || (f == 5 && k == g.L - 1);
    s = fma(boundary ? 1.0 : 0.5, R[ho_gid(g, c, k, q)], s);
  }
  bbar[K] = gamma ? gamma[K] * s : s;
}

// lam_out = lam_in + P dPi (Algorithm 2 line 7), one thread per row
__global__ void ho_prolong_kernel(const HoGeo g, int64_t T, const double *__restrict__ lam_in,
                                  const double *__restrict__ dpi, double *__restrict__ lam_out) {
  const int64_t row = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (row >= T) return;
  const HoFacet fc = ho_facet(g, row >> 2);
  const double a = dpi[(int64_t)fc.cA * g.L + fc.kA];
  lam_out[row] = fc.cB >= 0 ? fma(0.5, a + dpi[(int64_t)fc.cB * g.L + fc.kB], lam_in[row]) : lam_in[row] + a;
}

__global__ void ho_fill_kernel(double *__restrict__ x, int64_t n, double v) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) x[i] = v;
}

__global__ void ho_gamma_kernel(int64_t ncell, const double *__restrict__ m, double *__restrict__ gamma) {
  const int64_t K = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (K < ncell) gamma[K] = m[K] / gamma[K];   // gamma holds P^T S P 1 on entry
}

// ---- host side ------------------------------------------------------------------------------------
static HoGeo ho_geo(const Ctx *c) {
  const Level &f = c->lv[0];
  HoGeo g;
  g.L = f.nlev;
  g.ncol = f.ncol;
  g.nhf = (int64_t)f.nedge * f.nlev;
  g.nzf = (int64_t)f.ncol * (f.nlev + 1);
  g.NH = 4 * g.nhf;
  g.col_edges = f.col_edges;
  g.stencil = f.edge_stencil;
  g.edge_fc = f.edge_fc;
  g.own = c->ho.own;
  return g;
}

int64_t ho_trace_size(const Ctx *c) {
  const Level &f = c->lv[0];
  return 4 * ((int64_t)f.nedge * f.nlev + (int64_t)f.ncol * (f.nlev + 1));
}

static int ho_build_factors(Ctx *c) {
  HoData &h = c->ho;
  const HoGeo g = ho_geo(c);
  int *sing = h.flag;
  HMG_CUDA(c, cudaMemsetAsync(sing, 0, sizeof(int), c->stream));
  ho_hfactor_kernel<<<grid_for(g.nhf, 128), 128, 0, c->stream>>>(g, h.T, h.S, c->opt.omega, h.hw, sing);
  ho_zfactor_kernel<<<grid_for(g.ncol, 64), 64, 0, c->stream>>>(g, h.T, h.S, c->opt.omega, h.zf, sing);
  HMG_CUDA(c, cudaGetLastError());
  int s = 0;
  HMG_CUDA(c, cudaMemcpyAsync(&s, sing, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  HMG_CUDA(c, cudaStreamSynchronize(c->stream));
  if (s) return fail(c, HMG_ERR_INVALID_ARG, "a smoother block of the degree-1 trace operator is singular");
  h.factor_omega = c->opt.omega;
  return HMG_OK;
}

int ho_assemble(Ctx *c) {
  const Level &f = c->lv[0];
  HoData &h = c->ho;
  if (c->sc.preset != 1) return fail(c, HMG_ERR_INVALID_ARG, "degree 1 is built for the Helmholtz preset (preset 1)");
  const int64_t C = f.ncell;
  int st;
  if (!h.S) {
    h.T = ho_trace_size(c);
    std::vector<double> tab;
    ho_tables(tab);
    if ((st = dev_alloc(c, &h.tab, tab.size()))) return st;
    HMG_CUDA(c, cudaMemcpy(h.tab, tab.data(), sizeof(double) * tab.size(), cudaMemcpyHostToDevice));
    if ((st = dev_alloc(c, &h.S, (size_t)kHoSlots * h.T))) return st;
    if ((st = dev_alloc(c, &h.Ainv, (size_t)kHoN * kHoN * C))) return st;
    if ((st = dev_alloc(c, &h.hw, (size_t)16 * f.nedge * f.nlev))) return st;
    if ((st = dev_alloc(c, &h.zf, (size_t)48 * f.ncol * (f.nlev + 1)))) return st;
    if ((st = dev_alloc(c, &h.gamma, (size_t)C))) return st;
    if ((st = dev_alloc(c, &h.m, (size_t)C))) return st;
    if ((st = dev_alloc(c, &h.own, (size_t)4 * f.ncol))) return st;
    if ((st = dev_alloc(c, &h.flag, 1))) return st;
  }
  HMG_CUDA(c, cudaMemsetAsync(h.own, 0, 4 * (size_t)f.ncol, c->stream));
  ho_own_kernel<<<grid_for(f.nedge, 256), 256, 0, c->stream>>>(f.edge_stencil, f.edge_fc, f.nedge, h.own);
  HMG_CUDA(c, cudaMemsetAsync(h.flag, 0, sizeof(int), c->stream));
  HoCellArgs a{f.geometry, f.ncol, f.nlev, C, f.radius, c->sc.sigma, f.corners, f.z};
  ho_cell_kernel<<<(unsigned)C, 128, 0, c->stream>>>(a, h.tab, h.Ainv, h.m, h.flag);
  HMG_CUDA(c, cudaGetLastError());
  int sing = 0;
  HMG_CUDA(c, cudaMemcpyAsync(&sing, h.flag, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  HMG_CUDA(c, cudaStreamSynchronize(c->stream));
  if (sing) return fail(c, HMG_ERR_INVALID_ARG, "a degree-1 cell matrix A_K is singular");
  const HoGeo g = ho_geo(c);
  ho_rows_kernel<<<grid_for(h.T, 256), 256, 0, c->stream>>>(g, h.T, h.Ainv, h.S);
  HMG_CUDA(c, cudaGetLastError());
  // Gamma = (H 1) / (P^T S P 1): S applied to the ones vector (P 1 = 1), then P^T
  double *ones = static_cast<double *>(c->w1), *s1 = static_cast<double *>(c->w2);
  ho_fill_kernel<<<grid_for(h.T, 256), 256, 0, c->stream>>>(ones, h.T, 1.0);
  ho_spmv_kernel<0><<<grid_for(g.nhf + g.nzf, kRedThreads), kRedThreads, 0, c->stream>>>(
      g, h.T, h.S, ones, s1, nullptr, c->part, 0, 0);
  ho_restrict_kernel<<<grid_for(C, 256), 256, 0, c->stream>>>(g, C, s1, nullptr, h.gamma);
  ho_gamma_kernel<<<grid_for(C, 256), 256, 0, c->stream>>>(C, h.m, h.gamma);
  HMG_CUDA(c, cudaGetLastError());
  return ho_build_factors(c);
}

int ho_refactor_if_needed(Ctx *c) {
  if (c->ho.factor_omega == c->opt.omega) return HMG_OK;
  return ho_build_factors(c);
}

int ho_launch_spmv(Ctx *c, const double *x, double *y, int mode, const double *w, int slot0, int slot1) {
  const HoData &h = c->ho;
  const HoGeo g = ho_geo(c);
  const unsigned grid = grid_for(g.nhf + g.nzf, kRedThreads);
  if (grid > (unsigned)kMaxRedBlocks) return fail(c, HMG_ERR_INVALID_ARG, "too many facets for one reduction");
  Prof prof(c, kCompApply);
  switch (mode) {
    case 0: ho_spmv_kernel<0><<<grid, kRedThreads, 0, c->stream>>>(g, h.T, h.S, x, y, w, c->part, slot0, slot1); break;
    case 1: ho_spmv_kernel<1><<<grid, kRedThreads, 0, c->stream>>>(g, h.T, h.S, x, y, w, c->part, slot0, slot1); break;
    case 2: ho_spmv_kernel<2><<<grid, kRedThreads, 0, c->stream>>>(g, h.T, h.S, x, y, w, c->part, slot0, slot1); break;
    default: ho_spmv_kernel<3><<<grid, kRedThreads, 0, c->stream>>>(g, h.T, h.S, x, y, w, c->part, slot0, slot1); break;
  }
  HMG_CUDA(c, cudaGetLastError());
  if (mode != 0) return launch_finalize(c, (int)grid, slot0, mode == 2 ? slot1 : -1);
  return HMG_OK;
}

int ho_trace_rhs(Ctx *c, const double *Ru, const double *Rp, double *B) {
  const HoData &h = c->ho;
  Prof prof(c, kCompRhs);
  ho_rhs_kernel<<<grid_for(h.T, 128), 128, 0, c->stream>>>(ho_geo(c), h.T, h.Ainv, Ru, Rp, B);
  HMG_CUDA(c, cudaGetLastError());
  return HMG_OK;
}

int ho_reconstruct(Ctx *c, const double *lam, const double *Ru, const double *Rp, double *u, double *pi) {
  const int64_t C = c->lv[0].ncell;
  ho_reconstruct_kernel<<<grid_for(C * kHoN, 128), 128, 0, c->stream>>>(ho_geo(c), C, c->ho.Ainv, lam, Ru, Rp, u,
                                                                        pi);
  HMG_CUDA(c, cudaGetLastError());
  return HMG_OK;
}

constexpr int kHoCpb = 32;   // columns per block of the sweep's line part (four lanes each)

template <bool ZERO>
static int ho_sweep(Ctx *c, const double *b, const double *lam_in, double *lam_out) {
  const HoData &h = c->ho;
  const HoGeo g = ho_geo(c);
  // columns per block: the block's residual rows (4 (L + 1) doubles per column) within 48 KB
  const int cap = (int)((48 * 1024) / (sizeof(double) * 4 * (g.L + 1)));
  if (cap < 1) return fail(c, HMG_ERR_INVALID_ARG, "degree 1 takes at most 1535 layers");
  const int cpb = cap < kHoCpb ? cap : kHoCpb;
  const int nzb = (g.ncol + cpb - 1) / cpb;
  const unsigned nhb = grid_for(g.nhf, 128);
  const size_t smem = sizeof(double) * 4 * cpb * (g.L + 1);
  Prof prof(c, ZERO ? kCompPresmooth : kCompSweep);
  ho_sweep_kernel<ZERO><<<nzb + nhb, 128, smem, c->stream>>>(g, h.T, cpb, nzb, h.S, h.hw, h.zf, b, lam_in, lam_out,
                                                              1.0 - h.factor_omega);
  HMG_CUDA(c, cudaGetLastError());
  return HMG_OK;
}

int ho_line_smooth(Ctx *c, const double *b, double *lam, int nsweeps) {
  int st;
  if ((st = ho_refactor_if_needed(c))) return st;
  double *cur = lam, *nxt = static_cast<double *>(c->w3);
  for (int i = 0; i < nsweeps; ++i) {
    if ((st = ho_sweep<false>(c, b, cur, nxt))) return st;
    double *t = cur; cur = nxt; nxt = t;
  }
  if (cur != lam)
    HMG_CUDA(c, cudaMemcpyAsync(lam, cur, sizeof(double) * c->ho.T, cudaMemcpyDeviceToDevice, c->stream));
  return HMG_OK;
}

// z = M^-1 r: configuration 3c (Algorithm 2, the V-cycle of the lowest-order pressure operator as
// the coarse solve), configuration 2 (n_smooth sweeps of Algorithm 1 from zero) or none.
int ho_precond(Ctx *c, const double *r, double *z) {
  const HoData &h = c->ho;
  const HoGeo g = ho_geo(c);
  const int64_t T = h.T, C = c->lv[0].ncell;
  int st;
  double *w1 = static_cast<double *>(c->w1), *w2 = static_cast<double *>(c->w2), *w3 = static_cast<double *>(c->w3);
  if (c->opt.precond == HMG_PRECOND_NONE) {
    HMG_CUDA(c, cudaMemcpyAsync(z, r, sizeof(double) * T, cudaMemcpyDeviceToDevice, c->stream));
    return HMG_OK;
  }
  if (c->opt.precond == HMG_PRECOND_LINESMOOTH) {
    const int n = c->opt.n_smooth;
    if (n == 1) return ho_sweep<true>(c, r, nullptr, z);
    if ((st = ho_sweep<true>(c, r, nullptr, w1))) return st;
    double *cur = w1, *nxt = w2;
    for (int i = 1; i < n; ++i) {
      if ((st = ho_sweep<false>(c, r, cur, i == n - 1 ? z : nxt))) return st;
      double *t = cur; cur = nxt; nxt = t;
    }
    return HMG_OK;
  }
  // lines 1-2: presmoothing from zero
  if (c->opt.n_pre >= 1) {
    if ((st = ho_sweep<true>(c, r, nullptr, w1))) return st;
    for (int i = 1; i < c->opt.n_pre; ++i) {
      if ((st = ho_sweep<false>(c, r, w1, w2))) return st;
      double *t = w1; w1 = w2; w2 = t;
    }
  } else {
    HMG_CUDA(c, cudaMemsetAsync(w1, 0, sizeof(double) * T, c->stream));
  }
  double *cb = static_cast<double *>(c->cb);
  {
    Prof pr(c, kCompResidual, 2);
    if (c->opt.n_pre == 1)   // w1 is one sweep from zero                                       // line 3
      ho_residual_kernel<true><<<grid_for(g.nhf + g.nzf, 128), 128, 0, c->stream>>>(g, T, h.S, r, w1, w2,
                                                                                   1.0 - h.factor_omega);
    else
      ho_residual_kernel<false><<<grid_for(g.nhf + g.nzf, 128), 128, 0, c->stream>>>(g, T, h.S, r, w1, w2, 0.0);
    ho_restrict_kernel<<<grid_for(C, 256), 256, 0, c->stream>>>(g, C, w2, h.gamma, cb);          // lines 4-5
    HMG_CUDA(c, cudaGetLastError());
  }
  double *dpi = nullptr;
  {
    Prof pv(c, kCompVcycle, vcycle_launches(c));
    if ((st = vcycle<double>(c, cb, &dpi))) return st;                                            // line 6
  }
  {
    Prof pp(c, kCompProlong);
    ho_prolong_kernel<<<grid_for(T, 256), 256, 0, c->stream>>>(g, T, w1, dpi, w2);                  // line 7
    HMG_CUDA(c, cudaGetLastError());
  }
  const int np = c->opt.n_post;                                                                    // line 8
  if (np == 0) {
    HMG_CUDA(c, cudaMemcpyAsync(z, w2, sizeof(double) * T, cudaMemcpyDeviceToDevice, c->stream));
    return HMG_OK;
  }
  double *cur = w2, *nxt = w3;
  for (int i = 0; i < np - 1; ++i) {
    if ((st = ho_sweep<false>(c, r, cur, nxt))) return st;
    double *t = cur; cur = nxt; nxt = t;
  }
  return ho_sweep<false>(c, r, cur, z);
}

}  // namespace hmg
