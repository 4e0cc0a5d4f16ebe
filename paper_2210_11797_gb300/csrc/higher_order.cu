// The hybridised system of degree p = 1, 2, 3 (broken RT_p velocity, DG_p pressure, Q_p trace
// multipliers: (p+1)^2 per facet) for the constant-coefficient Helmholtz form of the operator,
// and its non-nested two-level preconditioner with the piecewise-constant coarse space.
//
// Paper (arXiv 2210.11797): Sec. 2.2 (spaces of degree p, n = p + 3 Gauss points per
// direction), Sec. 2.4 (Eqs. hybrid-S, hybrid-rhs, hybrid-recovery), Sec. 4.1 and the table
// of unknowns per cell (hybridised cell matrices of 24 x 24, 54 x 54 and 96 x 96, mixed cell
// matrices of 44 x 44, 135 x 135 and 304 x 304 at p = 1, 2, 3), Algorithm 1 (here on facet
// blocks and block-tridiagonal columns), Algorithm 2 with the DG0 coarse space of Sec. 2.5
// (P lambda = {{Pi}}, Restrict = P^T, Eq. scaling_matrix) and the lowest-order pressure
// multigrid as its coarse solve.
//
// Numbering (NT = p + 1, NB = NT^2 nodes per facet, NF = 6 NB facet dofs per cell). Cell dofs:
// the RT_p dofs (NF facet dofs, face f = e0..e3, bottom, top, node (s, t) at NB f + NT s + t,
// each the cell's outward normal flux at a Gauss-Legendre node of the facet; then the
// 3 p NT^2 interior dofs, component-major), then the NT^3 DG_p dofs. Trace rows: NB per facet,
// facet-major: vertical facet (edge e, level k) at NB (e L + k), horizontal facet (column c,
// interface k) at NH + NB (c (L + 1) + k), node (s, t) at + NT s + t; on a vertical facet s
// counts along the edge in the traversal of its owner column (the other column's local s is
// p - s).
#include <cmath>
#include <vector>

#include "device_common.cuh"
#include "hmg_internal.cuh"
#include "precond.cuh"

namespace hmg {

template <int P>
struct Ho {
  static constexpr int NT = P + 1;                    // Gauss-Legendre nodes per direction
  static constexpr int NB = NT * NT;                  // nodes (trace rows) per facet
  static constexpr int NF = 6 * NB;                   // facet dofs: the hybridised cell matrix is NF x NF
  static constexpr int NU = 3 * NT * NT * (P + 2);    // RT_p dofs
  static constexpr int NP = NT * NT * NT;             // DG_p dofs
  static constexpr int N = NU + NP;                   // the mixed cell matrix
  static constexpr int NQ1 = P + 3;                   // volume Gauss points per direction
  static constexpr int Q = NQ1 * NQ1 * NQ1;
  static constexpr int SLOTS = 2 * NF;                // S coefficients stored per trace row
  static constexpr int NINT = P * NT * NT;            // interior dofs per component
  // reference tables: velocity values, pressure values, weights, points, G, facet weights
  static constexpr int TV = 0, TPHI = TV + Q * NU, TW = TPHI + Q * NP, TX = TW + Q, TG = TX + 3 * Q,
                       TC = TG + NU * NP, TAB = TC + NB;
  // the sweep's line part: lanes per column (a group of LPC >= NB lanes of one warp; lane n < NB
  // computes component n of each block product) and columns per warp (p = 2: three groups of
  // nine, five lanes idle)
  static constexpr int LPC = P == 1 ? 4 : (P == 2 ? 9 : 16);
  static constexpr int CPW = 32 / LPC;
};

// ---- reference tables, formed on the host ---------------------------------------------------
// n-point Gauss-Legendre rule on [0, 1]: Newton's method on the Legendre polynomial P_n from the
// initial guesses cos(pi (i + 3/4) / (n + 1/2)), weights 2 / ((1 - x^2) P_n'(x)^2) on [-1, 1],
// halved
static void gauss_legendre01(int n, double *x, double *w) {
  for (int i = 0; i < n; ++i) {
    double z = std::cos(M_PI * (i + 0.75) / (n + 0.5)), dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      // p1 = P_n(z), p0 = P_{n-1}(z) (n = 1: P_1 = z, P_0 = 1)
      dp = n * (z * p1 - p0) / (z * z - 1.0);
      const double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    x[n - 1 - i] = 0.5 * (z + 1.0);   // ascending
    w[n - 1 - i] = 1.0 / ((1.0 - z * z) * dp * dp);
  }
}

// n = 2 .. 5 Gauss-Lobatto points on [0, 1]: the end points and the roots of P'_{n-1}
static void gauss_lobatto01(int n, double *x) {
  x[0] = 0.0;
  x[n - 1] = 1.0;
  if (n == 3) x[1] = 0.5;
  if (n == 4) {
    const double r = 1.0 / std::sqrt(5.0);
    x[1] = 0.5 * (1.0 - r);
    x[2] = 0.5 * (1.0 + r);
  }
  if (n == 5) {
    const double r = std::sqrt(3.0 / 7.0);
    x[1] = 0.5 * (1.0 - r);
    x[2] = 0.5;
    x[3] = 0.5 * (1.0 + r);
  }
}

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

// face f: the component normal to it, whether it is the far end (xi, eta or zeta = 1), the sign
// of the outward normal
static const int kFaceComp[6] = {1, 0, 1, 0, 2, 2};
static const int kFaceFar[6] = {0, 1, 1, 0, 0, 1};
static const double kFaceSign[6] = {-1.0, 1.0, 1.0, -1.0, -1.0, 1.0};

// a velocity dof: its component d, its node a along d (Gauss-Lobatto), its nodes (b, c) across d
// (Gauss-Legendre, the other two coordinates in increasing order), its sign
struct HoDof { int d, a, b, c; double sign; };

template <int P>
static std::vector<HoDof> ho_dofs() {
  using H = Ho<P>;
  std::vector<HoDof> v;
  for (int f = 0; f < 6; ++f)
    for (int s = 0; s < H::NT; ++s)
      for (int t = 0; t < H::NT; ++t) {
        const int b = (f == 2 || f == 3) ? P - s : s;   // e2, e3 traverse their edge backwards
        v.push_back({kFaceComp[f], kFaceFar[f] ? P + 1 : 0, b, t, kFaceSign[f]});
      }
  for (int d = 0; d < 3; ++d)
    for (int a = 1; a <= P; ++a)
      for (int b = 0; b < H::NT; ++b)
        for (int c = 0; c < H::NT; ++c) v.push_back({d, a, b, c, 1.0});
  return v;
}

// the RT_p basis (value of its one nonzero component and its divergence) and the DG_p basis at
// the Q Gauss points, G(f, j) = -int phi_j div v_f, and the facet weights of C_K
template <int P>
static void ho_tables(std::vector<double> &tab) {
  using H = Ho<P>;
  tab.assign(H::TAB, 0.0);
  double gl[H::NT], glw[H::NT], gll[P + 2], qx[H::NQ1], qw[H::NQ1];
  gauss_legendre01(H::NT, gl, glw);
  gauss_lobatto01(P + 2, gll);
  gauss_legendre01(H::NQ1, qx, qw);
  const std::vector<HoDof> dofs = ho_dofs<P>();
  for (int a = 0; a < H::NQ1; ++a)
    for (int b = 0; b < H::NQ1; ++b)
      for (int c = 0; c < H::NQ1; ++c) {
        const int q = (a * H::NQ1 + b) * H::NQ1 + c;
        const double x[3] = {qx[a], qx[b], qx[c]};
        double tv[3][H::NT], td[3][H::NT], nv[3][P + 2], nd[3][P + 2];
        for (int k = 0; k < 3; ++k) {
          lagrange1d(gl, H::NT, x[k], tv[k], td[k]);
          lagrange1d(gll, P + 2, x[k], nv[k], nd[k]);
        }
        const double wq = qw[a] * qw[b] * qw[c];
        tab[H::TW + q] = wq;
        for (int k = 0; k < 3; ++k) tab[H::TX + 3 * q + k] = x[k];
        double phi[H::NP];
        for (int ii = 0; ii < H::NT; ++ii)
          for (int jj = 0; jj < H::NT; ++jj)
            for (int kk = 0; kk < H::NT; ++kk) phi[(ii * H::NT + jj) * H::NT + kk] = tv[0][ii] * tv[1][jj] * tv[2][kk];
        for (int j = 0; j < H::NP; ++j) tab[H::TPHI + q * H::NP + j] = phi[j];
        for (int i = 0; i < H::NU; ++i) {
          const HoDof &o = dofs[i];
          const int t1 = o.d == 0 ? 1 : 0, t2 = o.d == 2 ? 1 : 2;
          const double tan = tv[t1][o.b] * tv[t2][o.c];
          tab[H::TV + q * H::NU + i] = o.sign * nv[o.d][o.a] * tan;
          // divergence: the derivative of the one nonzero component along its own coordinate
          const double dv = o.sign * nd[o.d][o.a] * tan;
          for (int j = 0; j < H::NP; ++j) tab[H::TG + i * H::NP + j] -= wq * dv * phi[j];
        }
      }
  for (int s = 0; s < H::NT; ++s)
    for (int t = 0; t < H::NT; ++t) tab[H::TC + s * H::NT + t] = glw[s] * glw[t];
}

template <int P>
__device__ __forceinline__ int ho_comp(int i) {   // the nonzero component of velocity dof i
  using H = Ho<P>;
  if (i < H::NF) {
    const int f = i / H::NB;
    return f == 0 || f == 2 ? 1 : (f == 1 || f == 3 ? 0 : 2);
  }
  return (i - H::NF) / H::NINT;
}

// ---- mesh access ------------------------------------------------------------------------------
struct HoGeo {
  int L, ncol;
  int64_t NH;                 // rows of the vertical facets (NB nedge L)
  int64_t nhf, nzf;           // vertical and horizontal facets
  const int32_t *col_edges, *stencil, *edge_fc;
  const int8_t *own;          // [ncol][4] 1 if the column owns the edge of that face
};

// trace row of local facet dof q of cell (c, k)
template <int P>
__device__ __forceinline__ int64_t ho_gid(const HoGeo &g, int c, int k, int q) {
  using H = Ho<P>;
  const int f = q / H::NB, r = q - f * H::NB, s = r / H::NT, t = r - s * H::NT;
  if (f < 4) {
    const int64_t e = g.col_edges[4 * (int64_t)c + f];
    const int sg = g.own[4 * (int64_t)c + f] ? s : P - s;
    return H::NB * (e * g.L + k) + H::NT * sg + t;
  }
  const int kk = k + (f == 5 ? 1 : 0);
  return g.NH + H::NB * ((int64_t)c * (g.L + 1) + kk) + H::NT * s + t;
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

// NB consecutive coefficients of one slot (the facet's rows) times x into acc: FP64 coefficients
// as double2 pairs, FP32 ones (the FP32 preconditioner's copy) as float4 quads where NB allows
template <int NB, bool NEG, typename TS, typename TA>
__device__ __forceinline__ void ho_slot(const TS *__restrict__ s, TA xv, TA acc[NB]) {
  if constexpr (sizeof(TS) == 8 && NB % 2 == 0) {
#pragma unroll
    for (int n = 0; n < NB; n += 2) {
      const double2 v = __ldcs(reinterpret_cast<const double2 *>(s + n));
      acc[n] = fma(NEG ? -(TA)v.x : (TA)v.x, xv, acc[n]);
      acc[n + 1] = fma(NEG ? -(TA)v.y : (TA)v.y, xv, acc[n + 1]);
    }
  } else if constexpr (sizeof(TS) == 4 && NB % 4 == 0) {
#pragma unroll
    for (int n = 0; n < NB; n += 4) {
      const float4 v = __ldcs(reinterpret_cast<const float4 *>(s + n));
      acc[n] = fma(NEG ? -(TA)v.x : (TA)v.x, xv, acc[n]);
      acc[n + 1] = fma(NEG ? -(TA)v.y : (TA)v.y, xv, acc[n + 1]);
      acc[n + 2] = fma(NEG ? -(TA)v.z : (TA)v.z, xv, acc[n + 2]);
      acc[n + 3] = fma(NEG ? -(TA)v.w : (TA)v.w, xv, acc[n + 3]);
    }
  } else {
#pragma unroll
    for (int n = 0; n < NB; ++n) {
      const TA v = (TA)__ldcs(s + n);
      acc[n] = fma(NEG ? -v : v, xv, acc[n]);
    }
  }
}

// acc[n] (+/-)= sum over the stored slots of row NB F + n times x: cell A's NF facet dofs, then
// cell B's without the shared facet (merged into A's slots when S was assembled). OFFD leaves out
// the couplings inside the smoother's diagonal block D of Algorithm 1 (acc - (S - D) x): on a
// vertical facet its own nodes, on a horizontal facet the horizontal facets of its column (A's
// bottom and top, B's bottom).
template <int P, bool NEG, bool OFFD = false, typename TS = double, typename TX = double, typename TA = double>
__device__ __forceinline__ void ho_rows(const TS *__restrict__ S, const TX *__restrict__ x, const HoGeo &g,
                                        int64_t T, int64_t F, TA acc[Ho<P>::NB]) {
  using H = Ho<P>;
  const HoFacet fc = ho_facet(g, F);
  const TS *Sr = S + (int64_t)H::NB * F;
  const bool vert = F < g.nhf;
  constexpr int U = P == 1 ? 4 : 2;
#pragma unroll U
  for (int q = 0; q < H::NF; ++q) {
    if (OFFD && (vert ? q / H::NB == fc.fA : q / H::NB >= 4)) continue;
    const TA xv = (TA)__ldg(x + ho_gid<P>(g, fc.cA, fc.kA, q));
    ho_slot<H::NB, NEG>(Sr + (int64_t)q * T, xv, acc);
  }
  if (fc.cB < 0) return;
#pragma unroll U
  for (int q = 0; q < H::NF; ++q) {
    if (q / H::NB == fc.fB || (OFFD && !vert && q / H::NB >= 4)) continue;
    const TA xv = (TA)__ldg(x + ho_gid<P>(g, fc.cB, fc.kB, q));
    ho_slot<H::NB, NEG>(Sr + (int64_t)(H::NF + q) * T, xv, acc);
  }
}

// ---- assembly -------------------------------------------------------------------------------
struct HoCellArgs {
  int geometry, ncol, L;
  int64_t ncell;
  double radius, sigma;
  const double *corners, *z;
};

// Shared memory of the cell kernel: the mixed matrix when it fits (p <= 2), then the per-point
// metric terms and the elimination's vectors.
template <int P>
struct HoCellSmem {
  static constexpr bool IN_SMEM = P <= 2;
  static constexpr size_t MAT = IN_SMEM ? sizeof(double) * Ho<P>::N * Ho<P>::N : 0;
  static constexpr size_t BYTES =
      MAT + sizeof(double) * (Ho<P>::Q * 7 + 3 * Ho<P>::N + 24) + sizeof(int) * (Ho<P>::N + 8);
};

// A_K = [[M, G], [-G^T, Mp]] by the (p+3)^3 Gauss rule (M with the contravariant Piola map,
// Mp = sigma int phi_i phi_j), then A_K^-1 by in-place Gauss-Jordan elimination with partial
// pivoting of the symmetrically equilibrated D A_K D, D = |diag A_K|^-1/2: A^-1 = D (D A D)^-1 D.
// The row interchanges are undone at the end as column interchanges in reverse order. One cell
// per block; the matrix lives in shared memory for p <= 2 and in its output slot (global memory)
// at p = 3. m[K] = sigma |K|_1 (the one-point volume), H 1 of the coarse operator.
template <int P>
__global__ void __launch_bounds__(256)
    ho_cell_kernel(const HoCellArgs a, const double *__restrict__ tab, double *__restrict__ Ainv,
                   double *__restrict__ mK, int *singular) {
  using H = Ho<P>;
  using SM = HoCellSmem<P>;
  constexpr int N = H::N;
  extern __shared__ __align__(16) unsigned char ho_smem[];
  const int64_t K = blockIdx.x;
  double *Ag = SM::IN_SMEM ? reinterpret_cast<double *>(ho_smem) : Ainv + K * (int64_t)(N * N);
  double *Kq = reinterpret_cast<double *>(ho_smem + SM::MAT);   // [Q][6] (w / det) J^T J
  double *wd = Kq + 6 * H::Q;                                     // [Q] sigma w det
  double *dsc = wd + H::Q, *fac = dsc + N, *rowk = fac + N;
  double *X = rowk + N;                                           // [8][3] corners
  int *perm = reinterpret_cast<int *>(X + 24);
  int *piv = perm + N;
  __shared__ double bestv[8];
  __shared__ int besti[8];
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int c = (int)(K / a.L), k = (int)(K - (int64_t)c * a.L);
  if (tid < 8) {
    const int va = tid & 1, vb = (tid >> 1) & 1, vc = (tid >> 2) & 1;
    const int corner = va == 0 ? (vb == 0 ? 0 : 3) : (vb == 0 ? 1 : 2);
    const double *cp = a.corners + (4 * (int64_t)c + corner) * 3;
    const double h = a.z[k + vc];
    if (a.geometry == 1) {
      for (int i = 0; i < 3; ++i) X[3 * tid + i] = cp[i] * (a.radius + h);
    } else {
      X[3 * tid] = cp[0];
      X[3 * tid + 1] = cp[1];
      X[3 * tid + 2] = h;
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
        for (int d = 0; d < 3; ++d) J[i][d] += X[3 * v + i] * dn[d];
    }
  };
  auto det3 = [](const double J[3][3]) {
    return J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) - J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
           J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
  };
  for (int q = tid; q <= H::Q; q += nthr) {
    if (q < H::Q) {
      const double *xq = tab + H::TX + 3 * q;
      double J[3][3];
      jacobian(xq[0], xq[1], xq[2], J);
      const double det = det3(J), w = tab[H::TW + q];
      double G[3][3];
      for (int p = 0; p < 3; ++p)
        for (int r = 0; r < 3; ++r) G[p][r] = J[0][p] * J[0][r] + J[1][p] * J[1][r] + J[2][p] * J[2][r];
      const double s = w / det;
      Kq[6 * q] = s * G[0][0];
      Kq[6 * q + 1] = s * G[1][1];
      Kq[6 * q + 2] = s * G[2][2];
      Kq[6 * q + 3] = s * G[0][1];
      Kq[6 * q + 4] = s * G[0][2];
      Kq[6 * q + 5] = s * G[1][2];
      wd[q] = a.sigma * w * det;
    } else {
      double J[3][3];
      jacobian(0.5, 0.5, 0.5, J);
      mK[K] = a.sigma * det3(J);
    }
  }
  __syncthreads();
  const double *tv = tab + H::TV, *tp = tab + H::TPHI, *tg = tab + H::TG;
  for (int idx = tid; idx < N * N; idx += nthr) {
    const int i = idx / N, j = idx - i * N;
    double v = 0.0;
    if (i < H::NU && j < H::NU) {
      const int di = ho_comp<P>(i), dj = ho_comp<P>(j);
      const int kk = di == dj ? di : (di + dj == 1 ? 3 : (di + dj == 2 ? 4 : 5));
      for (int q = 0; q < H::Q; ++q)
        v = fma(__ldg(tv + q * H::NU + i) * __ldg(tv + q * H::NU + j), Kq[6 * q + kk], v);
    } else if (i < H::NU) {
      v = __ldg(tg + i * H::NP + (j - H::NU));
    } else if (j < H::NU) {
      v = -__ldg(tg + j * H::NP + (i - H::NU));
    } else {
      for (int q = 0; q < H::Q; ++q)
        v = fma(wd[q] * __ldg(tp + q * H::NP + (i - H::NU)), __ldg(tp + q * H::NP + (j - H::NU)), v);
    }
    Ag[idx] = v;
  }
  __syncthreads();
  for (int i = tid; i < N; i += nthr) dsc[i] = 1.0 / sqrt(fabs(Ag[(int64_t)i * N + i]));
  __syncthreads();
  for (int idx = tid; idx < N * N; idx += nthr) {
    const int i = idx / N, j = idx - i * N;
    Ag[idx] *= dsc[i] * dsc[j];
  }
  __syncthreads();
  const int warp = tid >> 5, lane = tid & 31, nwarp = nthr >> 5;
  for (int col = 0; col < N; ++col) {
    // pivot: the largest |A[r][col]|, r >= col (the first such row on ties)
    double bv = -1.0;
    int bi = col;
    for (int r = col + tid; r < N; r += nthr) {
      const double v = fabs(Ag[(int64_t)r * N + col]);
      if (v > bv) { bv = v; bi = r; }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double ov = __shfl_xor_sync(0xffffffffu, bv, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ov > bv || (ov == bv && oi < bi)) { bv = ov; bi = oi; }
    }
    if (lane == 0) { bestv[warp] = bv; besti[warp] = bi; }
    __syncthreads();
    if (tid == 0) {
      double v = bestv[0];
      int p = besti[0];
      for (int w = 1; w < nwarp; ++w)
        if (bestv[w] > v || (bestv[w] == v && besti[w] < p)) { v = bestv[w]; p = besti[w]; }
      if (!(v > 0.0)) atomicExch(singular, 1);
      piv[0] = p;
      perm[col] = p;
    }
    __syncthreads();
    const int p = piv[0];
    if (p != col)
      for (int j = tid; j < N; j += nthr) {
        const double t = Ag[(int64_t)col * N + j];
        Ag[(int64_t)col * N + j] = Ag[(int64_t)p * N + j];
        Ag[(int64_t)p * N + j] = t;
      }
    __syncthreads();
    for (int r = tid; r < N; r += nthr) fac[r] = Ag[(int64_t)r * N + col];
    __syncthreads();
    const double pinv = 1.0 / fac[col];
    for (int j = tid; j < N; j += nthr) {
      const double v = (j == col ? 1.0 : Ag[(int64_t)col * N + j]) * pinv;
      Ag[(int64_t)col * N + j] = v;
      rowk[j] = v;
    }
    __syncthreads();
    for (int idx = tid; idx < N * N; idx += nthr) {
      const int r = idx / N, j = idx - r * N;
      if (r != col) Ag[idx] = fma(-fac[r], rowk[j], j == col ? 0.0 : Ag[idx]);
    }
    __syncthreads();
  }
  for (int col = N - 1; col >= 0; --col) {   // undo the row interchanges: columns, in reverse
    const int p = perm[col];
    if (p != col)
      for (int r = tid; r < N; r += nthr) {
        const double t = Ag[(int64_t)r * N + col];
        Ag[(int64_t)r * N + col] = Ag[(int64_t)r * N + p];
        Ag[(int64_t)r * N + p] = t;
      }
    __syncthreads();
  }
  double *out = Ainv + K * (int64_t)(N * N);
  for (int idx = tid; idx < N * N; idx += nthr) {
    const int i = idx / N, j = idx - i * N;
    out[idx] = dsc[i] * Ag[idx] * dsc[j];
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

// Rows of S = sum_K C_K^T A_K^-1 C_K (C_K diagonal on the facet dofs: w_s w_t of the node): row
// NB F + n holds, in slots 0 .. NF - 1, C A_A^-1 C restricted to the facet dofs of cell A (row:
// the node's local index in A), and in slots NF .. 2 NF - 1 the same of cell B, whose
// shared-facet entries are added into A's slots (and stored as 0).
template <int P>
__global__ void ho_rows_kernel(const HoGeo g, int64_t T, const double *__restrict__ tab,
                               const double *__restrict__ Ainv, double *__restrict__ S) {
  using H = Ho<P>;
  constexpr int N = H::N;
  const int64_t row = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (row >= T) return;
  const int64_t F = row / H::NB;
  const int n = (int)(row - F * H::NB), s = n / H::NT, t = n - s * H::NT;
  const double *Cw = tab + H::TC;
  const HoFacet fc = ho_facet(g, F);
  const int qa = H::NB * fc.fA + n;
  const double *IA = Ainv + ((int64_t)fc.cA * g.L + fc.kA) * (int64_t)(N * N) + (int64_t)qa * N;
  for (int q = 0; q < H::NF; ++q) S[(int64_t)q * T + row] = Cw[n] * Cw[q % H::NB] * IA[q];
  if (fc.cB >= 0) {
    const int sb = fc.flipB ? P - s : s;
    const int nb = H::NT * sb + t;
    const int qb = H::NB * fc.fB + nb;
    const double *IB = Ainv + ((int64_t)fc.cB * g.L + fc.kB) * (int64_t)(N * N) + (int64_t)qb * N;
    for (int q = 0; q < H::NF; ++q) {
      const double w = Cw[nb] * Cw[q % H::NB] * IB[q];
      if (q / H::NB == fc.fB) {   // the shared facet: the same trace row as A's node
        const int r = q % H::NB, sq = r / H::NT, tq = r - sq * H::NT;
        const int sa = fc.flipB ? P - sq : sq;
        S[(int64_t)(H::NB * fc.fA + H::NT * sa + tq) * T + row] += w;
        S[(int64_t)(H::NF + q) * T + row] = 0.0;
      } else {
        S[(int64_t)(H::NF + q) * T + row] = w;
      }
    }
  } else {
    for (int q = 0; q < H::NF; ++q) S[(int64_t)(H::NF + q) * T + row] = 0.0;
  }
}

// Gauss-Jordan elimination with partial pivoting by one warp: W [NB][2 NB] (shared memory) holds
// [A | I] on entry and [I | A^-1] on return; lane j < 2 NB owns column j. Every lane finds the
// same pivot (they read the same values), so the branches are uniform. False if A is singular.
template <int NB>
__device__ bool warp_gauss_jordan(double *W, int lane) {
  constexpr int W2 = 2 * NB;
  static_assert(W2 <= 32, "one lane per column");
  for (int c = 0; c < NB; ++c) {
    int p = c;
    double best = fabs(W[c * W2 + c]);
    for (int r = c + 1; r < NB; ++r) {
      const double v = fabs(W[r * W2 + c]);
      if (v > best) { best = v; p = r; }
    }
    if (!(best > 0.0)) return false;
    if (p != c && lane < W2) {
      const double t = W[c * W2 + lane];
      W[c * W2 + lane] = W[p * W2 + lane];
      W[p * W2 + lane] = t;
    }
    __syncwarp();
    const double inv = 1.0 / W[c * W2 + c];
    double fr[NB];   // column c, read before its owner lane changes it
#pragma unroll
    for (int r = 0; r < NB; ++r) fr[r] = W[r * W2 + c];
    __syncwarp();
    if (lane < W2) {
      const double pv = W[c * W2 + lane] * inv;
      W[c * W2 + lane] = pv;
#pragma unroll
      for (int r = 0; r < NB; ++r)
        if (r != c) W[r * W2 + lane] = fma(-fr[r], pv, W[r * W2 + lane]);
    }
    __syncwarp();
  }
  return true;
}

constexpr int kHoFacWarps = 4;   // warps per block of the factor kernels

// omega times the inverse of each vertical facet's NB x NB block of S (the Jacobi part of
// Algorithm 1), entry (n, m) at hw[(NB n + m) nhf + F]; one warp per facet. The facet block lives
// in the slots of cell A's face (A owns the edge, so its local nodes are the facet's).
template <int P>
__global__ void __launch_bounds__(32 * kHoFacWarps)
    ho_hfactor_kernel(const HoGeo g, int64_t T, const double *__restrict__ S, double omega,
                      double *__restrict__ hw, int *singular) {
  constexpr int NB = Ho<P>::NB, W2 = 2 * NB;
  __shared__ double Wsh[kHoFacWarps][NB * W2];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t F = (int64_t)blockIdx.x * kHoFacWarps + warp;
  if (F >= g.nhf) return;   // whole warps leave
  double *W = Wsh[warp];
  const HoFacet fc = ho_facet(g, F);
  for (int e = lane; e < NB * NB; e += 32) {
    const int n = e / NB, m = e - n * NB;
    W[n * W2 + m] = S[(int64_t)(NB * fc.fA + m) * T + NB * F + n];
    W[n * W2 + NB + m] = n == m ? 1.0 : 0.0;
  }
  __syncwarp();
  if (!warp_gauss_jordan<NB>(W, lane) && lane == 0) atomicExch(singular, 1);
  for (int e = lane; e < NB * NB; e += 32) {
    const int n = e / NB, m = e - n * NB;
    hw[(int64_t)(NB * n + m) * g.nhf + F] = omega * W[n * W2 + NB + m];
  }
}

// Block Thomas factors of each column's block-tridiagonal S^zz (blocks D_k, L_k = coupling of
// facet k to k - 1, U_k to k + 1): G_0 = D_0, G_k = D_k - L_k G_{k-1}^-1 U_{k-1}; stored per
// horizontal facet: omega G_k^-1, G_k^-1 L_k, G_k^-1 U_k ([nzf][3][NB][NB], each transposed: entry
// (n, m) at m NB + n, so that the NB lanes of a column read one contiguous run per m), so that
// omega (S^zz)^-1 r is y_k = (omega G_k^-1) r_k - (G_k^-1 L_k) y_{k-1}, x_k = y_k - (G_k^-1 U_k) x_{k+1}.
// Slots: the cell above (c, k) is A for k < L: its bottom (face 4) is this facet, its top (face 5)
// facet k + 1; the cell below (c, k - 1) is B, its bottom facet k - 1. The lid row's A is the
// cell below: its top is this facet, its bottom the facet below. One warp per column.
template <int P>
__global__ void __launch_bounds__(32 * kHoFacWarps)
    ho_zfactor_kernel(const HoGeo g, int64_t T, const double *__restrict__ S, double omega,
                      double *__restrict__ zf, int *singular) {
  using H = Ho<P>;
  constexpr int NB = H::NB, NB2 = NB * NB, W2 = 2 * NB;
  extern __shared__ double zsh[];   // per warp: GU, Lk, U [NB2] and W [NB][2 NB]
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int c = blockIdx.x * kHoFacWarps + warp;
  if (c >= g.ncol) return;   // whole warps leave
  double *GU = zsh + warp * (3 * NB2 + NB * W2), *Lk = GU + NB2, *U = Lk + NB2, *W = U + NB2;
  const int L = g.L;
  bool ok = true;
  for (int k = 0; k <= L; ++k) {
    const int64_t F = (int64_t)c * (L + 1) + k, row0 = g.NH + NB * F;
    for (int e = lane; e < NB2; e += 32) {
      const int n = e / NB, m = e - n * NB;
      const double *r = S + row0 + n;
      if (k < L) {
        W[n * W2 + m] = r[(int64_t)(4 * NB + m) * T];
        U[e] = r[(int64_t)(5 * NB + m) * T];
        Lk[e] = k > 0 ? r[(int64_t)(H::NF + 4 * NB + m) * T] : 0.0;
      } else {
        W[n * W2 + m] = r[(int64_t)(5 * NB + m) * T];
        Lk[e] = r[(int64_t)(4 * NB + m) * T];
        U[e] = 0.0;
      }
      W[n * W2 + NB + m] = n == m ? 1.0 : 0.0;
    }
    __syncwarp();
    if (k > 0) {
      for (int e = lane; e < NB2; e += 32) {   // G_k = D_k - L_k (G_{k-1}^-1 U_{k-1})
        const int n = e / NB, m = e - n * NB;
        double s = W[n * W2 + m];
        for (int j = 0; j < NB; ++j) s = fma(-Lk[n * NB + j], GU[j * NB + m], s);
        W[n * W2 + m] = s;
      }
      __syncwarp();
    }
    if (!warp_gauss_jordan<NB>(W, lane)) ok = false;
    double *o = zf + 3 * NB2 * F;   // facet-major: 3 NB^2 contiguous factors, each matrix transposed
    for (int e = lane; e < NB2; e += 32) {
      const int n = e / NB, m = e - n * NB;
      double sl = 0.0, su = 0.0;
      for (int j = 0; j < NB; ++j) {
        sl = fma(W[n * W2 + NB + j], Lk[j * NB + m], sl);
        su = fma(W[n * W2 + NB + j], U[j * NB + m], su);
      }
      o[m * NB + n] = omega * W[n * W2 + NB + m];
      o[NB2 + m * NB + n] = sl;
      o[2 * NB2 + m * NB + n] = su;
      GU[e] = su;   // (row-major, for the next level's G; nothing reads GU in this loop)
    }
    __syncwarp();
  }
  if (!ok && lane == 0) atomicExch(singular, 1);
}

// ---- the operator, the right-hand side and the recovery --------------------------------------
// y = S x, one thread per facet (its NB rows share the gathered values); MODE 1, 2, 3 fuse the
// inner products of the Krylov loop as the lowest-order S apply does (3: (b - S x, b - S x), no y).
template <int P, int MODE>
__global__ void __launch_bounds__(kRedThreads)
    ho_spmv_kernel(const HoGeo g, int64_t T, const double *__restrict__ S, const double *__restrict__ x,
                   double *__restrict__ y, const double *__restrict__ w, double *part, int slot0, int slot1) {
  constexpr int NB = Ho<P>::NB;
  const int64_t F = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  double a0 = 0.0, a1 = 0.0;
  if (F < g.nhf + g.nzf) {
    double acc[NB];
    const int64_t r0 = (int64_t)NB * F;
    if (MODE == 3) {
#pragma unroll
      for (int n = 0; n < NB; ++n) acc[n] = __ldg(w + r0 + n);
      ho_rows<P, true>(S, x, g, T, F, acc);
#pragma unroll
      for (int n = 0; n < NB; ++n) a0 = fma(acc[n], acc[n], a0);
    } else {
#pragma unroll
      for (int n = 0; n < NB; ++n) acc[n] = 0.0;
      ho_rows<P, false>(S, x, g, T, F, acc);
#pragma unroll
      for (int n = 0; n < NB; ++n) {
        y[r0 + n] = acc[n];
        if (MODE == 1) a0 = fma(__ldg(w + r0 + n), acc[n], a0);
        if (MODE == 2) { a0 = fma(acc[n], __ldg(w + r0 + n), a0); a1 = fma(acc[n], acc[n], a1); }
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

// B_lambda row NB F + n: the sum over the facet's cells of C_K (A_K^-1 R_K) at the node's local dof
template <int P>
__global__ void ho_rhs_kernel(const HoGeo g, int64_t T, const double *__restrict__ tab,
                              const double *__restrict__ Ainv, const double *__restrict__ Ru,
                              const double *__restrict__ Rp, double *__restrict__ B) {
  using H = Ho<P>;
  constexpr int N = H::N;
  const int64_t row = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (row >= T) return;
  const int64_t F = row / H::NB;
  const int n = (int)(row - F * H::NB), s = n / H::NT, t = n - s * H::NT;
  const HoFacet fc = ho_facet(g, F);
  auto cell = [&](int cc, int kk, int q) {
    const int64_t K = (int64_t)cc * g.L + kk;
    const double *I = Ainv + K * (int64_t)(N * N) + (int64_t)q * N;
    double v = 0.0;
    for (int j = 0; j < H::NU; ++j) v = fma(I[j], Ru[K * H::NU + j], v);
    for (int j = 0; j < H::NP; ++j) v = fma(I[H::NU + j], Rp[K * H::NP + j], v);
    return v;
  };
  double v = cell(fc.cA, fc.kA, H::NB * fc.fA + n);
  if (fc.cB >= 0) v += cell(fc.cB, fc.kB, H::NB * fc.fB + H::NT * (fc.flipB ? P - s : s) + t);
  B[row] = tab[H::TC + n] * v;
}

// X_K = A_K^-1 (R_K - C_K lambda_K): u [ncell][NU], pi [ncell][NP]; one thread per (cell, dof)
template <int P>
__global__ void ho_reconstruct_kernel(const HoGeo g, int64_t ncell, const double *__restrict__ tab,
                                      const double *__restrict__ Ainv, const double *__restrict__ lam,
                                      const double *__restrict__ Ru, const double *__restrict__ Rp,
                                      double *__restrict__ u, double *__restrict__ pi) {
  using H = Ho<P>;
  constexpr int N = H::N;
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= ncell * N) return;
  const int64_t K = idx / N;
  const int i = (int)(idx - K * N);
  const int c = (int)(K / g.L), k = (int)(K - (int64_t)c * g.L);
  const double *I = Ainv + K * (int64_t)(N * N) + (int64_t)i * N;
  double v = 0.0;
  for (int j = 0; j < H::NU; ++j) {
    double r = Ru[K * H::NU + j];
    if (j < H::NF) r = fma(-tab[H::TC + j % H::NB], lam[ho_gid<P>(g, c, k, j)], r);
    v = fma(I[j], r, v);
  }
  for (int j = 0; j < H::NP; ++j) v = fma(I[H::NU + j], Rp[K * H::NP + j], v);
  if (i < H::NU) u[K * H::NU + i] = v;
  else pi[K * H::NP + (i - H::NU)] = v;
}

// ---- Algorithm 1 at p >= 1 ------------------------------------------------------------------------
// lam_out = lam_in + omega D^-1 (b - S lam_in) (ZERO: lam_in = 0), evaluated as
// (1 - omega) lam_in + omega D^-1 (b - (S - D) lam_in): equal in exact arithmetic, without the
// couplings of a row inside D. Two launches per sweep. Part 1, one thread per facet (all facets,
// as parallel as the S apply): the residual rows r = b - (S - D) lam_in; on a vertical facet the
// NB x NB block Jacobi step lam_out = keep lam_in + (omega D_F^-1) r at once, on a horizontal
// facet r is parked in lam_out's rows (ZERO: vertical facets only, r = b). Part 2, the line
// solves: each column's r staged in shared memory, the block Thomas recurrences with LPC lanes
// per column (lane n < NB computes component n of each NB x NB product from its rows of the
// stored factors; the lanes of a column sit in one warp and meet at __syncwarp between the
// steps), lam_out = keep lam_in + omega (S^zz_c)^-1 r. T is the arithmetic and coefficient
// type (double, or float in the FP32 preconditioner, whose b is the FP64 Krylov residual and
// whose last sweep writes FP64).
template <int P, bool ZERO, typename T = double, typename Tb = double, typename Tin = double, typename Tout = double>
__global__ void __launch_bounds__(kRedThreads)
    ho_sweep_rows_kernel(const HoGeo g, int64_t TT, const T *__restrict__ S, const T *__restrict__ hw,
                         const Tb *__restrict__ b, const Tin *__restrict__ lam_in,
                         Tout *__restrict__ lam_out, double keep) {
  constexpr int NB = Ho<P>::NB;
  const int64_t F = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (F >= (ZERO ? g.nhf : g.nhf + g.nzf)) return;
  const int64_t r0 = (int64_t)NB * F;
  T acc[NB];
#pragma unroll
  for (int n = 0; n < NB; ++n) acc[n] = (T)__ldg(b + r0 + n);
  if (!ZERO) ho_rows<P, true, true>(S, lam_in, g, TT, F, acc);
  if (F < g.nhf) {
    for (int n = 0; n < NB; ++n) {
      T v = ZERO ? (T)0 : (T)keep * (T)lam_in[r0 + n];
#pragma unroll
      for (int m = 0; m < NB; ++m) v = fma(hw[(int64_t)(NB * n + m) * g.nhf + F], acc[m], v);
      lam_out[r0 + n] = (Tout)v;
    }
  } else {
#pragma unroll
    for (int n = 0; n < NB; ++n) lam_out[r0 + n] = (Tout)acc[n];
  }
}

// Part 2; r is read from src (lam_out after part 1, b for a sweep from zero)
template <int P, bool ZERO, typename T = double, typename Ts = double, typename Tin = double, typename Tout = double>
__global__ void __launch_bounds__(128)
    ho_sweep_lines_kernel(const HoGeo g, int cpb, const T *__restrict__ zf, const Ts *src,
                          const Tin *__restrict__ lam_in, Tout *lam_out, double keep) {
  using H = Ho<P>;
  constexpr int NB = H::NB, NB2 = NB * NB, LPC = H::LPC;
  extern __shared__ __align__(16) unsigned char ho_lines_smem[];
  T *sr = reinterpret_cast<T *>(ho_lines_smem);   // [cpb][L+1][NB]
  const int L1 = g.L + 1;
  const int c0 = blockIdx.x * cpb, nc = min(cpb, g.ncol - c0);
  const int64_t base = g.NH + (int64_t)NB * c0 * L1;
  for (int i = threadIdx.x; i < nc * L1 * NB; i += blockDim.x) sr[i] = (T)src[base + i];
  __syncthreads();
  const int lane = threadIdx.x & 31, gw = lane / LPC;   // the lane's group within its warp
  const int cc = gw < H::CPW ? (threadIdx.x >> 5) * H::CPW + gw : cpb, n = lane - gw * LPC;
  const unsigned grp = ((1u << LPC) - 1u) << (gw * LPC);   // this column's lanes
  if (cc < nc) {
    T *r = sr + NB * cc * L1;
    const T *f0 = zf + 3 * NB2 * ((int64_t)(c0 + cc) * L1) + n;   // this lane's rows (transposed)
    const bool act = n < NB;
    // forward: y_k = (omega G_k^-1) r_k - (G_k^-1 L_k) y_{k-1}, y written over r; the next level's
    // factor rows are loaded one step ahead (the serial recurrence waits on nothing else)
    T fa[NB], fb[NB];
    if (act) {
#pragma unroll
      for (int m = 0; m < NB; ++m) { fa[m] = __ldg(f0 + NB * m); fb[m] = __ldg(f0 + NB2 + NB * m); }
    }
    for (int k = 0; k < L1; ++k) {
      T na[NB], nb[NB];
      if (act && k + 1 < L1) {
        const T *f = f0 + 3 * NB2 * (k + 1);
#pragma unroll
        for (int m = 0; m < NB; ++m) { na[m] = __ldg(f + NB * m); nb[m] = __ldg(f + NB2 + NB * m); }
      }
      T v = (T)0, u = (T)0;
      if (act) {
#pragma unroll
        for (int m = 0; m < NB; ++m) v = fma(fa[m], r[NB * k + m], v);
        if (k > 0) {
#pragma unroll
          for (int m = 0; m < NB; ++m) u = fma(-fb[m], r[NB * (k - 1) + m], u);
        }
      }
      __syncwarp(grp);
      if (act) r[NB * k + n] = v + u;
      __syncwarp(grp);
#pragma unroll
      for (int m = 0; m < NB; ++m) { fa[m] = na[m]; fb[m] = nb[m]; }
    }
    // backward: x_k = y_k - (G_k^-1 U_k) x_{k+1}, x written over y (row k + 1 is not written in
    // this step, row k only by its own lane); G_k^-1 U_k one step ahead as well
    if (act && L1 >= 2) {
      const T *f = f0 + 3 * NB2 * (L1 - 2) + 2 * NB2;
#pragma unroll
      for (int m = 0; m < NB; ++m) fa[m] = __ldg(f + NB * m);
    }
    for (int k = L1 - 2; k >= 0; --k) {
      T na[NB];
      if (act && k > 0) {
        const T *f = f0 + 3 * NB2 * (k - 1) + 2 * NB2;
#pragma unroll
        for (int m = 0; m < NB; ++m) na[m] = __ldg(f + NB * m);
      }
      if (act) {
        T v = r[NB * k + n];
#pragma unroll
        for (int m = 0; m < NB; ++m) v = fma(-fa[m], r[NB * (k + 1) + m], v);
        r[NB * k + n] = v;
      }
      __syncwarp(grp);
#pragma unroll
      for (int m = 0; m < NB; ++m) fa[m] = na[m];
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < nc * L1 * NB; i += blockDim.x)
    lam_out[base + i] = (Tout)(ZERO ? sr[i] : fma((T)keep, (T)lam_in[base + i], sr[i]));
}

// R = b - S lam (Algorithm 2 line 3), one thread per facet. ZSWEEP: lam is one sweep from zero,
// lam = omega D^-1 b, so R = (1 - omega) b - (S - D) lam (equal in exact arithmetic).
template <int P, bool ZSWEEP, typename T = double>
__global__ void ho_residual_kernel(const HoGeo g, int64_t TT, const T *__restrict__ S,
                                   const double *__restrict__ b, const T *__restrict__ lam,
                                   T *__restrict__ R, double keep) {
  constexpr int NB = Ho<P>::NB;
  const int64_t F = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (F >= g.nhf + g.nzf) return;
  T acc[NB];
#pragma unroll
  for (int n = 0; n < NB; ++n) {
    const T bv = (T)__ldg(b + (int64_t)NB * F + n);
    acc[n] = ZSWEEP ? (T)keep * bv : bv;
  }
  ho_rows<P, true, ZSWEEP>(S, lam, g, TT, F, acc);
#pragma unroll
  for (int n = 0; n < NB; ++n) R[(int64_t)NB * F + n] = acc[n];
}

// bbar_K = Gamma_K (P^T R)_K (Algorithm 2 lines 4-5): P is constant on a facet (all its nodes)
// and averages the facet's cells, so P^T sums the cell's facet nodes with weight 1/2 (1 on
// ground and lid facets)
template <int P, typename T = double>
__global__ void ho_restrict_kernel(const HoGeo g, int64_t ncell, const T *__restrict__ R,
                                   const T *__restrict__ gamma, T *__restrict__ bbar) {
  using H = Ho<P>;
  const int64_t K = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (K >= ncell) return;
  const int c = (int)(K / g.L), k = (int)(K - (int64_t)c * g.L);
  T s = (T)0;
  for (int q = 0; q < H::NF; ++q) {
    const int f = q / H::NB;
    const bool boundary = (f == 4 && k == 0) || (f == 5 && k == g.L - 1);
    s = fma(boundary ? (T)1 : (T)0.5, R[ho_gid<P>(g, c, k, q)], s);
  }
  bbar[K] = gamma ? gamma[K] * s : s;
}

// lam_out = lam_in + P dPi (Algorithm 2 line 7), one thread per row
template <int P, typename T = double>
__global__ void ho_prolong_kernel(const HoGeo g, int64_t TT, const T *__restrict__ lam_in,
                                  const T *__restrict__ dpi, T *__restrict__ lam_out) {
  const int64_t row = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (row >= TT) return;
  const HoFacet fc = ho_facet(g, row / Ho<P>::NB);
  const T a = dpi[(int64_t)fc.cA * g.L + fc.kA];
  lam_out[row] = fc.cB >= 0 ? fma((T)0.5, a + dpi[(int64_t)fc.cB * g.L + fc.kB], lam_in[row]) : lam_in[row] + a;
}

// the FP32 preconditioner's copies of the degree-p operator and factors; the last step's FP32
// result widened to FP64
template <typename Ta, typename Tb>
__global__ void ho_convert_kernel(const Ta *__restrict__ x, Tb *__restrict__ y, int64_t n) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) y[i] = (Tb)x[i];
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
template <int P>
static HoGeo ho_geo(const Ctx *c) {
  const Level &f = c->lv[0];
  HoGeo g;
  g.L = f.nlev;
  g.ncol = f.ncol;
  g.nhf = (int64_t)f.nedge * f.nlev;
  g.nzf = (int64_t)f.ncol * (f.nlev + 1);
  g.NH = (int64_t)Ho<P>::NB * g.nhf;
  g.col_edges = f.col_edges;
  g.stencil = f.edge_stencil;
  g.edge_fc = f.edge_fc;
  g.own = c->ho.own;
  return g;
}

int64_t ho_trace_size(const Ctx *c, int p) {
  const Level &f = c->lv[0];
  return (int64_t)(p + 1) * (p + 1) * ((int64_t)f.nedge * f.nlev + (int64_t)f.ncol * (f.nlev + 1));
}

template <int P>
static int ho_build_factors(Ctx *c) {
  HoData &h = c->ho;
  const HoGeo g = ho_geo<P>(c);
  constexpr int NB = Ho<P>::NB;
  int *sing = h.flag;
  HMG_CUDA(c, cudaMemsetAsync(sing, 0, sizeof(int), c->stream));
  const size_t zsmem = sizeof(double) * kHoFacWarps * (3 * NB * NB + 2 * NB * NB);
  ho_hfactor_kernel<P><<<grid_for(g.nhf, kHoFacWarps), 32 * kHoFacWarps, 0, c->stream>>>(g, h.T, h.S, c->opt.omega,
                                                                                      h.hw, sing);
  ho_zfactor_kernel<P><<<grid_for(g.ncol, kHoFacWarps), 32 * kHoFacWarps, zsmem, c->stream>>>(
      g, h.T, h.S, c->opt.omega, h.zf, sing);
  HMG_CUDA(c, cudaGetLastError());
  if (h.S32) {   // the FP32 preconditioner's copies of the factors follow them
    const int64_t nh = (int64_t)NB * NB * g.nhf, nz = (int64_t)3 * NB * NB * g.nzf;
    ho_convert_kernel<double, float><<<grid_for(nh, 256), 256, 0, c->stream>>>(h.hw, h.hw32, nh);
    ho_convert_kernel<double, float><<<grid_for(nz, 256), 256, 0, c->stream>>>(h.zf, h.zf32, nz);
    HMG_CUDA(c, cudaGetLastError());
  }
  int s = 0;
  HMG_CUDA(c, cudaMemcpyAsync(&s, sing, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  HMG_CUDA(c, cudaStreamSynchronize(c->stream));
  if (s) return fail(c, HMG_ERR_INVALID_ARG, "a smoother block of the degree-p trace operator is singular");
  h.factor_omega = c->opt.omega;
  return HMG_OK;
}

// The FP32 copies of S, Gamma and the smoother factors (allocated once per layout)
template <int P>
static int ho_build_fp32(Ctx *c) {
  using H = Ho<P>;
  HoData &h = c->ho;
  const HoGeo g = ho_geo<P>(c);
  const int64_t C = c->lv[0].ncell, nS = (int64_t)H::SLOTS * h.T;
  const int64_t nh = (int64_t)H::NB * H::NB * g.nhf, nz = (int64_t)3 * H::NB * H::NB * g.nzf;
  int st;
  if (!h.S32) {
    if ((st = dev_alloc(c, &h.S32, (size_t)nS))) return st;
    if ((st = dev_alloc(c, &h.hw32, (size_t)nh))) return st;
    if ((st = dev_alloc(c, &h.zf32, (size_t)nz))) return st;
    if ((st = dev_alloc(c, &h.gamma32, (size_t)C))) return st;
  }
  ho_convert_kernel<double, float><<<grid_for(nS, 256), 256, 0, c->stream>>>(h.S, h.S32, nS);
  ho_convert_kernel<double, float><<<grid_for(nh, 256), 256, 0, c->stream>>>(h.hw, h.hw32, nh);
  ho_convert_kernel<double, float><<<grid_for(nz, 256), 256, 0, c->stream>>>(h.zf, h.zf32, nz);
  ho_convert_kernel<double, float><<<grid_for(C, 256), 256, 0, c->stream>>>(h.gamma, h.gamma32, C);
  HMG_CUDA(c, cudaGetLastError());
  return HMG_OK;
}

void ho_free(Ctx *c) {
  HoData &h = c->ho;
  double **bufs[] = {&h.tab, &h.S, &h.Ainv, &h.hw, &h.zf, &h.gamma, &h.m};
  for (double **b : bufs) {
    dev_free(c, *b);
    *b = nullptr;
  }
  dev_free(c, h.own);
  h.own = nullptr;
  dev_free(c, h.flag);
  h.flag = nullptr;
  float **f32[] = {&h.S32, &h.hw32, &h.zf32, &h.gamma32};
  for (float **b : f32) {
    dev_free(c, *b);
    *b = nullptr;
  }
  h.degree = 0;
  h.ncell = 0;
  h.T = 0;
}

template <int P>
static int ho_assemble_p(Ctx *c) {
  using H = Ho<P>;
  const Level &f = c->lv[0];
  HoData &h = c->ho;
  const int64_t C = f.ncell;
  int st;
  if (C > 0x7fffffff) return fail(c, HMG_ERR_INVALID_ARG, "too many cells for one launch");
  if (h.degree != P || h.ncell != C || h.T != ho_trace_size(c, P)) {   // (re)allocate for this degree and mesh
    ho_free(c);
    std::vector<double> tab;
    ho_tables<P>(tab);
    if ((st = dev_alloc(c, &h.tab, tab.size()))) return st;
    HMG_CUDA(c, cudaMemcpy(h.tab, tab.data(), sizeof(double) * tab.size(), cudaMemcpyHostToDevice));
    const int64_t T = ho_trace_size(c, P);
    if ((st = dev_alloc(c, &h.S, (size_t)H::SLOTS * T))) return st;
    if ((st = dev_alloc(c, &h.Ainv, (size_t)H::N * H::N * C))) return st;
    if ((st = dev_alloc(c, &h.hw, (size_t)H::NB * H::NB * f.nedge * f.nlev))) return st;
    if ((st = dev_alloc(c, &h.zf, (size_t)3 * H::NB * H::NB * f.ncol * (f.nlev + 1)))) return st;
    if ((st = dev_alloc(c, &h.gamma, (size_t)C))) return st;
    if ((st = dev_alloc(c, &h.m, (size_t)C))) return st;
    if ((st = dev_alloc(c, &h.own, (size_t)4 * f.ncol))) return st;
    if ((st = dev_alloc(c, &h.flag, 1))) return st;
    h.degree = P;
    h.ncell = C;
    h.T = T;
  }
  h.factor_omega = 0.0;
  HMG_CUDA(c, cudaMemsetAsync(h.own, 0, 4 * (size_t)f.ncol, c->stream));
  ho_own_kernel<<<grid_for(f.nedge, 256), 256, 0, c->stream>>>(f.edge_stencil, f.edge_fc, f.nedge, h.own);
  HMG_CUDA(c, cudaMemsetAsync(h.flag, 0, sizeof(int), c->stream));
  HoCellArgs a{f.geometry, f.ncol, f.nlev, C, f.radius, c->sc.sigma, f.corners, f.z};
  const size_t smem = HoCellSmem<P>::BYTES;
  HMG_CUDA(c, cudaFuncSetAttribute(ho_cell_kernel<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  ho_cell_kernel<P><<<(unsigned)C, 256, smem, c->stream>>>(a, h.tab, h.Ainv, h.m, h.flag);
  HMG_CUDA(c, cudaGetLastError());
  int sing = 0;
  HMG_CUDA(c, cudaMemcpyAsync(&sing, h.flag, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  HMG_CUDA(c, cudaStreamSynchronize(c->stream));
  if (sing) return fail(c, HMG_ERR_INVALID_ARG, "a degree-p cell matrix A_K is singular");
  const HoGeo g = ho_geo<P>(c);
  ho_rows_kernel<P><<<grid_for(h.T, 256), 256, 0, c->stream>>>(g, h.T, h.tab, h.Ainv, h.S);
  HMG_CUDA(c, cudaGetLastError());
  // Gamma = (H 1) / (P^T S P 1): S applied to the ones vector (P 1 = 1), then P^T
  double *ones = static_cast<double *>(c->w1), *s1 = static_cast<double *>(c->w2);
  ho_fill_kernel<<<grid_for(h.T, 256), 256, 0, c->stream>>>(ones, h.T, 1.0);
  ho_spmv_kernel<P, 0><<<grid_for(g.nhf + g.nzf, kRedThreads), kRedThreads, 0, c->stream>>>(
      g, h.T, h.S, ones, s1, nullptr, c->part, 0, 0);
  ho_restrict_kernel<P, double><<<grid_for(C, 256), 256, 0, c->stream>>>(g, C, s1, nullptr, h.gamma);
  ho_gamma_kernel<<<grid_for(C, 256), 256, 0, c->stream>>>(C, h.m, h.gamma);
  HMG_CUDA(c, cudaGetLastError());
  if ((st = ho_build_factors<P>(c))) return st;
  if (c->opt.precision == HMG_PRECISION_MIXED) return ho_build_fp32<P>(c);
  return HMG_OK;
}

template <int P>
static int ho_launch_spmv_p(Ctx *c, const double *x, double *y, int mode, const double *w, int slot0, int slot1) {
  const HoData &h = c->ho;
  const HoGeo g = ho_geo<P>(c);
  const unsigned grid = grid_for(g.nhf + g.nzf, kRedThreads);
  if (grid > (unsigned)kMaxRedBlocks) return fail(c, HMG_ERR_INVALID_ARG, "too many facets for one reduction");
  Prof prof(c, kCompApply);
  switch (mode) {
    case 0: ho_spmv_kernel<P, 0><<<grid, kRedThreads, 0, c->stream>>>(g, h.T, h.S, x, y, w, c->part, slot0, slot1); break;
    case 1: ho_spmv_kernel<P, 1><<<grid, kRedThreads, 0, c->stream>>>(g, h.T, h.S, x, y, w, c->part, slot0, slot1); break;
    case 2: ho_spmv_kernel<P, 2><<<grid, kRedThreads, 0, c->stream>>>(g, h.T, h.S, x, y, w, c->part, slot0, slot1); break;
    default: ho_spmv_kernel<P, 3><<<grid, kRedThreads, 0, c->stream>>>(g, h.T, h.S, x, y, w, c->part, slot0, slot1); break;
  }
  HMG_CUDA(c, cudaGetLastError());
  if (mode != 0) return launch_finalize(c, (int)grid, slot0, mode == 2 ? slot1 : -1);
  return HMG_OK;
}

template <int P>
static int ho_trace_rhs_p(Ctx *c, const double *Ru, const double *Rp, double *B) {
  const HoData &h = c->ho;
  Prof prof(c, kCompRhs);
  ho_rhs_kernel<P><<<grid_for(h.T, 128), 128, 0, c->stream>>>(ho_geo<P>(c), h.T, h.tab, h.Ainv, Ru, Rp, B);
  HMG_CUDA(c, cudaGetLastError());
  return HMG_OK;
}

template <int P>
static int ho_reconstruct_p(Ctx *c, const double *lam, const double *Ru, const double *Rp, double *u, double *pi) {
  const int64_t C = c->lv[0].ncell;
  ho_reconstruct_kernel<P><<<grid_for(C * Ho<P>::N, 128), 128, 0, c->stream>>>(ho_geo<P>(c), C, c->ho.tab,
                                                                              c->ho.Ainv, lam, Ru, Rp, u, pi);
  HMG_CUDA(c, cudaGetLastError());
  return HMG_OK;
}

// The FP64 operator or the FP32 preconditioner's copies
template <typename T> struct HoPrec;
template <> struct HoPrec<double> {
  static const double *S(const HoData &h) { return h.S; }
  static const double *hw(const HoData &h) { return h.hw; }
  static const double *zf(const HoData &h) { return h.zf; }
  static const double *gamma(const HoData &h) { return h.gamma; }
};
template <> struct HoPrec<float> {
  static const float *S(const HoData &h) { return h.S32; }
  static const float *hw(const HoData &h) { return h.hw32; }
  static const float *zf(const HoData &h) { return h.zf32; }
  static const float *gamma(const HoData &h) { return h.gamma32; }
};

// One sweep of Algorithm 1 in arithmetic T: b (the Krylov residual, FP64) and lam_in (Tin) in,
// lam_out (Tout) out.
template <int P, bool ZERO, typename T = double, typename Tin = double, typename Tout = double>
static int ho_sweep(Ctx *c, const double *b, const Tin *lam_in, Tout *lam_out) {
  using H = Ho<P>;
  const HoData &h = c->ho;
  const HoGeo g = ho_geo<P>(c);
  // columns per block of the line part: 4 warps of CPW columns, and the block's rows
  // (NB (L + 1) values per column) within 48 KB
  const int cap = (int)((48 * 1024) / (sizeof(T) * H::NB * (g.L + 1)));
  if (cap < 1) return fail(c, HMG_ERR_INVALID_ARG, "too many layers for the degree-p line smoother");
  const int cpb = cap < 4 * H::CPW ? cap : 4 * H::CPW;
  const unsigned nzb = (unsigned)((g.ncol + cpb - 1) / cpb);
  const size_t smem = sizeof(T) * H::NB * cpb * (g.L + 1);
  const double keep = 1.0 - h.factor_omega;
  Prof prof(c, ZERO ? kCompPresmooth : kCompSweep, 2);
  ho_sweep_rows_kernel<P, ZERO, T, double, Tin, Tout>
      <<<grid_for(ZERO ? g.nhf : g.nhf + g.nzf, kRedThreads), kRedThreads, 0, c->stream>>>(
          g, h.T, HoPrec<T>::S(h), HoPrec<T>::hw(h), b, lam_in, lam_out, keep);
  if constexpr (ZERO)
    ho_sweep_lines_kernel<P, ZERO, T, double, Tin, Tout><<<nzb, 128, smem, c->stream>>>(g, cpb, HoPrec<T>::zf(h), b,
                                                                                      lam_in, lam_out, keep);
  else
    ho_sweep_lines_kernel<P, ZERO, T, Tout, Tin, Tout><<<nzb, 128, smem, c->stream>>>(
        g, cpb, HoPrec<T>::zf(h), lam_out, lam_in, lam_out, keep);
  HMG_CUDA(c, cudaGetLastError());
  return HMG_OK;
}

template <int P>
static int ho_line_smooth_p(Ctx *c, const double *b, double *lam, int nsweeps) {
  int st;
  if ((st = ho_refactor_if_needed(c))) return st;
  double *cur = lam, *nxt = static_cast<double *>(c->w3);
  for (int i = 0; i < nsweeps; ++i) {
    if ((st = ho_sweep<P, false>(c, b, cur, nxt))) return st;
    double *t = cur;
    cur = nxt;
    nxt = t;
  }
  if (cur != lam)
    HMG_CUDA(c, cudaMemcpyAsync(lam, cur, sizeof(double) * c->ho.T, cudaMemcpyDeviceToDevice, c->stream));
  return HMG_OK;
}

// z = M^-1 r: configuration 3c (Algorithm 2, the V-cycle of the lowest-order pressure operator as
// the coarse solve), configuration 2 (n_smooth sweeps of Algorithm 1 from zero) or none. T = float
// is the FP32 preconditioner: its coefficients, work vectors and V-cycle in FP32, r read and z
// written in FP64 (the Krylov vectors).
template <int P, typename T>
static int ho_precond_p(Ctx *c, const double *r, double *z) {
  const HoData &h = c->ho;
  const HoGeo g = ho_geo<P>(c);
  const int64_t TT = h.T, C = c->lv[0].ncell;
  int st;
  if (!HoPrec<T>::S(h)) return fail(c, HMG_ERR_NOT_READY, "the FP32 copies of the degree-p operator are missing");
  T *w1 = static_cast<T *>(c->w1), *w2 = static_cast<T *>(c->w2), *w3 = static_cast<T *>(c->w3);
  if (c->opt.precond == HMG_PRECOND_NONE) {
    HMG_CUDA(c, cudaMemcpyAsync(z, r, sizeof(double) * TT, cudaMemcpyDeviceToDevice, c->stream));
    return HMG_OK;
  }
  if (c->opt.precond == HMG_PRECOND_LINESMOOTH) {
    const int n = c->opt.n_smooth;
    if (n == 1) return ho_sweep<P, true, T, T, double>(c, r, nullptr, z);
    if ((st = ho_sweep<P, true, T, T, T>(c, r, nullptr, w1))) return st;
    T *cur = w1, *nxt = w2;
    for (int i = 1; i < n; ++i) {
      if (i == n - 1) return ho_sweep<P, false, T, T, double>(c, r, cur, z);
      if ((st = ho_sweep<P, false, T, T, T>(c, r, cur, nxt))) return st;
      T *t = cur;
      cur = nxt;
      nxt = t;
    }
    return HMG_OK;
  }
  // lines 1-2: presmoothing from zero
  if (c->opt.n_pre >= 1) {
    if ((st = ho_sweep<P, true, T, T, T>(c, r, nullptr, w1))) return st;
    for (int i = 1; i < c->opt.n_pre; ++i) {
      if ((st = ho_sweep<P, false, T, T, T>(c, r, w1, w2))) return st;
      T *t = w1;
      w1 = w2;
      w2 = t;
    }
  } else {
    HMG_CUDA(c, cudaMemsetAsync(w1, 0, sizeof(T) * TT, c->stream));
  }
  T *cb = static_cast<T *>(c->cb);
  {
    Prof pr(c, kCompResidual, 2);
    if (c->opt.n_pre == 1)   // w1 is one sweep from zero                                       // line 3
      ho_residual_kernel<P, true, T><<<grid_for(g.nhf + g.nzf, 128), 128, 0, c->stream>>>(
          g, TT, HoPrec<T>::S(h), r, w1, w2, 1.0 - h.factor_omega);
    else
      ho_residual_kernel<P, false, T><<<grid_for(g.nhf + g.nzf, 128), 128, 0, c->stream>>>(
          g, TT, HoPrec<T>::S(h), r, w1, w2, 0.0);
    ho_restrict_kernel<P, T><<<grid_for(C, 256), 256, 0, c->stream>>>(g, C, w2, HoPrec<T>::gamma(h), cb);   // lines 4-5
    HMG_CUDA(c, cudaGetLastError());
  }
  T *dpi = nullptr;
  {
    Prof pv(c, kCompVcycle, vcycle_launches(c));
    if ((st = vcycle<T>(c, cb, &dpi))) return st;                                                 // line 6
  }
  {
    Prof pp(c, kCompProlong);
    ho_prolong_kernel<P, T><<<grid_for(TT, 256), 256, 0, c->stream>>>(g, TT, w1, dpi, w2);          // line 7
    HMG_CUDA(c, cudaGetLastError());
  }
  const int np = c->opt.n_post;                                                                    // line 8
  if (np == 0) {
    ho_convert_kernel<T, double><<<grid_for(TT, 256), 256, 0, c->stream>>>(w2, z, TT);
    HMG_CUDA(c, cudaGetLastError());
    return HMG_OK;
  }
  T *cur = w2, *nxt = w3;
  for (int i = 0; i < np - 1; ++i) {
    if ((st = ho_sweep<P, false, T, T, T>(c, r, cur, nxt))) return st;
    T *t = cur;
    cur = nxt;
    nxt = t;
  }
  return ho_sweep<P, false, T, T, double>(c, r, cur, z);
}

// ---- degree dispatch ------------------------------------------------------------------------------
static int bad_degree(Ctx *c) { return fail(c, HMG_ERR_INVALID_ARG, "the degree-p path takes p = 1, 2, 3"); }

int ho_assemble(Ctx *c) {
  if (c->sc.preset != 1) return fail(c, HMG_ERR_INVALID_ARG, "degree p >= 1 is built for the Helmholtz preset (preset 1)");
  switch (c->degree) {
    case 1: return ho_assemble_p<1>(c);
    case 2: return ho_assemble_p<2>(c);
    case 3: return ho_assemble_p<3>(c);
    default: return bad_degree(c);
  }
}

int ho_refactor_if_needed(Ctx *c) {
  if (c->opt.precision == HMG_PRECISION_MIXED && !c->ho.S32) {   // switched to the FP32 preconditioner
    int st = HMG_OK;
    switch (c->degree) {
      case 1: st = ho_build_fp32<1>(c); break;
      case 2: st = ho_build_fp32<2>(c); break;
      case 3: st = ho_build_fp32<3>(c); break;
      default: return bad_degree(c);
    }
    if (st) return st;
  }
  if (c->ho.factor_omega == c->opt.omega) return HMG_OK;
  switch (c->degree) {
    case 1: return ho_build_factors<1>(c);
    case 2: return ho_build_factors<2>(c);
    case 3: return ho_build_factors<3>(c);
    default: return bad_degree(c);
  }
}

int ho_launch_spmv(Ctx *c, const double *x, double *y, int mode, const double *w, int slot0, int slot1) {
  switch (c->degree) {
    case 1: return ho_launch_spmv_p<1>(c, x, y, mode, w, slot0, slot1);
    case 2: return ho_launch_spmv_p<2>(c, x, y, mode, w, slot0, slot1);
    case 3: return ho_launch_spmv_p<3>(c, x, y, mode, w, slot0, slot1);
    default: return bad_degree(c);
  }
}

int ho_trace_rhs(Ctx *c, const double *Ru, const double *Rp, double *B) {
  switch (c->degree) {
    case 1: return ho_trace_rhs_p<1>(c, Ru, Rp, B);
    case 2: return ho_trace_rhs_p<2>(c, Ru, Rp, B);
    case 3: return ho_trace_rhs_p<3>(c, Ru, Rp, B);
    default: return bad_degree(c);
  }
}

int ho_reconstruct(Ctx *c, const double *lam, const double *Ru, const double *Rp, double *u, double *pi) {
  switch (c->degree) {
    case 1: return ho_reconstruct_p<1>(c, lam, Ru, Rp, u, pi);
    case 2: return ho_reconstruct_p<2>(c, lam, Ru, Rp, u, pi);
    case 3: return ho_reconstruct_p<3>(c, lam, Ru, Rp, u, pi);
    default: return bad_degree(c);
  }
}

int ho_line_smooth(Ctx *c, const double *b, double *lam, int nsweeps) {
  switch (c->degree) {
    case 1: return ho_line_smooth_p<1>(c, b, lam, nsweeps);
    case 2: return ho_line_smooth_p<2>(c, b, lam, nsweeps);
    case 3: return ho_line_smooth_p<3>(c, b, lam, nsweeps);
    default: return bad_degree(c);
  }
}

int ho_precond(Ctx *c, const double *r, double *z) {
  const bool mixed = c->opt.precision == HMG_PRECISION_MIXED;
  switch (c->degree) {
    case 1: return mixed ? ho_precond_p<1, float>(c, r, z) : ho_precond_p<1, double>(c, r, z);
    case 2: return mixed ? ho_precond_p<2, float>(c, r, z) : ho_precond_p<2, double>(c, r, z);
    case 3: return mixed ? ho_precond_p<3, float>(c, r, z) : ho_precond_p<3, double>(c, r, z);
    default: return bad_degree(c);
  }
}

}  // namespace hmg
