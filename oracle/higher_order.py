"""Hybridised discretisation of degree p >= 0 (broken RT_p velocity, DG_p pressure, Q_p trace
multipliers on the facets) of the constant-coefficient Helmholtz form of the operator, and
the non-nested two-level preconditioner with a piecewise-constant coarse space. FP64.

Oracle (test infrastructure only; see oracle/__init__.py).

Paper passages (arXiv 2210.11797):
* Sec. 2.2: the function spaces of degree p on hexahedra and the quadrature rule (n = p + 3
  Gauss points per direction for the volume terms).
* Sec. 2.4, Eqs. hybrid-S, hybrid-rhs, hybrid-recovery: broken velocity, trace multipliers,
  S = sum_K C_K^T A_K^-1 C_K, B_lambda = sum_K C_K^T A_K^-1 R_K, X_K = A_K^-1 (R_K - C_K lambda).
* Sec. 4.1, Table tab:ndofs: 6 (p+1)^2 trace unknowns per cell, hybridised cell matrices of
  24 x 24 (p = 1), 54 x 54 (p = 2) and 96 x 96 (p = 3); mixed cell matrices of 44 x 44,
  135 x 135, 304 x 304.
* Sec. 2.5 and Algorithm 2 with the piecewise-constant coarse space the paper chose (Sec. 4.2):
  P lambda = {{Pi}} (the cell average of the two neighbours, constant on the facet),
  Restrict = P^T, Gamma of Eq. scaling_matrix, and Algorithm 1 as the smoother.

Operator: the Helmholtz preset of the lowest-order build (G_K = -1, B_K = 1, K_K = I,
M3^Pi = sigma |K| at p = 0) at degree p:
    (u, v) - (Pi, div v) + <lambda, v.n>_dK = (R_u, v),   (q, div u) + sigma (q, Pi) = (q, R_Pi),
with sum over K of <mu, u.n>_dK = 0 (continuity of the normal flux), i.e. sigma Pi - lap Pi = f,
u = -grad Pi for R_u = 0, with u.n = 0 at the ground and the lid.

Readings (the paper's experiments are all at p = 0):
* spaces on the reference cube [0,1]^3: RT_[p] = Q_{p+1,p,p} x Q_{p,p+1,p} x Q_{p,p,p+1} with
  nodal bases; along a component's own direction at the p + 2 Gauss-Lobatto points (the end
  points carry the facet dofs), across it at the p + 1 Gauss-Legendre points; DG_p and the
  facet space Q_p nodal at the Gauss-Legendre points. Contravariant Piola map on the
  trilinear cells, as at p = 0;
* a facet dof carries its cell's OUTWARD normal flux (the basis changes sign on the faces at
  xi = 0, eta = 0, zeta = 0), like the RT0 basis of the lowest order; then the trace coupling
  C_K = <mu, v.n>_dK is diagonal, the products of the Gauss-Legendre weights of the facet node;
* facet dof numbering (s, t): on a vertical facet, s along the edge in the traversal of the
  edge's owner column (edge_cols[e][0]; columns are counter-clockwise, so the other column
  traverses the edge backwards and its local s is the owner's p - s), t upwards; on a
  horizontal facet (s, t) are the xi and eta nodes of the column;
* m3^Pi by the n = p + 3 Gauss rule (at p = 0 the lowest order's one-point rule gives the
  same value on affine cells);
* Algorithm 1 at degree p: the Jacobi part inverts the (p+1)^2 x (p+1)^2 block of S on each
  vertical facet (its diagonal at p = 0), the line part the block-tridiagonal restriction of S
  to each column's horizontal facets;
* Algorithm 2's coarse operator is the lowest-order pressure operator H of the same mesh and
  coefficients with its multigrid hierarchy (the piecewise-constant coarse space).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import fem
from .nonnested import bicgstab
from .pressure_mg import PressureMultigrid, pressure_operator_times


# ---- one-dimensional rules and nodal bases on [0, 1] -----------------------------------------
def gauss_legendre(n: int):
    """n-point Gauss-Legendre nodes and weights on [0, 1]."""
    x, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * (x + 1.0), 0.5 * w


def gauss_lobatto(n: int) -> np.ndarray:
    """n >= 2 Gauss-Lobatto points on [0, 1]: the end points and the roots of P'_{n-1}."""
    if n == 2:
        return np.array([0.0, 1.0])
    inner = np.sort(np.real(np.polynomial.legendre.Legendre.basis(n - 1).deriv().roots()))
    return 0.5 * (np.concatenate([[-1.0], inner, [1.0]]) + 1.0)


def lagrange(nodes: np.ndarray, x: float):
    """Values and first derivatives at x of the Lagrange polynomials of `nodes`."""
    n = len(nodes)
    val = np.ones(n)
    der = np.zeros(n)
    for i in range(n):
        for j in range(n):
            if j != i:
                val[i] *= (x - nodes[j]) / (nodes[i] - nodes[j])
        for m in range(n):
            if m == i:
                continue
            term = 1.0 / (nodes[i] - nodes[m])
            for j in range(n):
                if j != i and j != m:
                    term *= (x - nodes[j]) / (nodes[i] - nodes[j])
            der[i] += term
    return val, der


# ---- the reference element -----------------------------------------------------------------
# local faces: e0 (eta = 0), e1 (xi = 1), e2 (eta = 1), e3 (xi = 0), bottom (zeta = 0), top (zeta = 1)
# (component, normal node at the end 0 or 1, outward sign)
_FACE = [(1, 0, -1.0), (0, 1, 1.0), (1, 1, 1.0), (0, 0, -1.0), (2, 0, -1.0), (2, 1, 1.0)]


class Element:
    """Degree-p spaces on the unit cube: RT_[p] dofs (6 (p+1)^2 facet dofs in face order,
    (s, t) within a face, then 3 p (p+1)^2 interior dofs), DG_p dofs (i, j, k), and the
    facet nodes (s, t)."""

    def __init__(self, p: int):
        self.p = p
        self.nt = p + 1                      # tangential (and DG) nodes per direction
        self.nn = p + 2                      # normal nodes of a velocity component
        self.gl_x, self.gl_w = gauss_legendre(self.nt)
        self.gll_x = gauss_lobatto(self.nn)
        nt, nn = self.nt, self.nn
        # velocity dofs: (component, normal node, (tangential node 1, tangential node 2), sign)
        dofs = []
        for f, (d, end, sign) in enumerate(_FACE):
            a = 0 if end == 0 else nn - 1
            for s in range(nt):
                for t in range(nt):
                    if f == 0:
                        tan = (s, t)             # (xi, zeta), traversal +xi
                    elif f == 1:
                        tan = (s, t)             # (eta, zeta), traversal +eta
                    elif f == 2:
                        tan = (p - s, t)         # (xi, zeta), traversal -xi
                    elif f == 3:
                        tan = (p - s, t)         # (eta, zeta), traversal -eta
                    else:
                        tan = (s, t)             # (xi, eta)
                    dofs.append((d, a, tan, sign))
        self.nfacet = len(dofs)                  # 6 (p+1)^2
        for d in range(3):
            for a in range(1, nn - 1):
                for b in range(nt):
                    for c in range(nt):
                        dofs.append((d, a, (b, c), 1.0))
        self.vdofs = dofs
        self.nu = len(dofs)                      # 3 (p+2)(p+1)^2
        self.npr = nt ** 3                       # DG_p
        self.nlam = 6 * nt * nt

    def velocity(self, xi, eta, zeta):
        """Reference velocity basis [nu, 3] and its divergence [nu] at one point."""
        tv = [lagrange(self.gl_x, c) for c in (xi, eta, zeta)]     # tangential (GL) per coordinate
        nv = [lagrange(self.gll_x, c) for c in (xi, eta, zeta)]    # normal (GLL) per coordinate
        V = np.zeros((self.nu, 3))
        div = np.zeros(self.nu)
        for i, (d, a, (b, c), sign) in enumerate(self.vdofs):
            others = [q for q in range(3) if q != d]
            t1, t2 = tv[others[0]][0][b], tv[others[1]][0][c]
            V[i, d] = sign * nv[d][0][a] * t1 * t2
            div[i] = sign * nv[d][1][a] * t1 * t2
        return V, div

    def pressure(self, xi, eta, zeta):
        """Reference DG_p basis [npr] at one point, dof (i, j, k) at i nt^2 + j nt + k with i the
        xi node."""
        a, b, c = (lagrange(self.gl_x, v)[0] for v in (xi, eta, zeta))
        return np.einsum("i,j,k->ijk", a, b, c).ravel()

    def trace_coupling(self) -> np.ndarray:
        """C_K [nu, nlam]: <mu_(f,s,t), v.n> on the reference facets (Piola keeps it), diagonal in
        the facet dofs: the Gauss-Legendre weights w_s w_t (1 at p = 0)."""
        C = np.zeros((self.nu, self.nlam))
        w = self.gl_w
        for f in range(6):
            for s in range(self.nt):
                for t in range(self.nt):
                    q = (f * self.nt + s) * self.nt + t
                    C[q, q] = w[s] * w[t]
        return C


# ---- cell matrices --------------------------------------------------------------------------
def cell_matrices(mesh, el: Element, sigma: float, cells=None):
    """A_K = [[M, G], [B, Mp]] [n, nu+npr, nu+npr] of the Helmholtz form by the n = p+3 Gauss
    rule: M(f,g) = int v_f.v_g (contravariant Piola), G(f,j) = -int phi_j div v_f, B = -G^T,
    Mp = sigma int phi_i phi_j. Also the cell volumes."""
    verts = fem.cell_vertices(mesh, cells)
    n = verts.shape[0]
    nu, npr = el.nu, el.npr
    qx, qw = gauss_legendre(el.p + 3)
    M = np.zeros((n, nu, nu))
    G = np.zeros((nu, npr))
    Mp = np.zeros((n, npr, npr))
    vol = np.zeros(n)
    for a, xa in enumerate(qx):
        for b, xb in enumerate(qx):
            for c, xc in enumerate(qx):
                w = qw[a] * qw[b] * qw[c]
                _N, dN = fem.trilinear_shape(xa, xb, xc)
                J = np.matmul(verts.transpose(0, 2, 1), dN)          # [n,3,3]
                det = np.linalg.det(J)
                V, div = el.velocity(xa, xb, xc)
                phi = el.pressure(xa, xb, xc)
                JV = np.matmul(J, V.T)                                # [n,3,nu]
                M += (w / det)[:, None, None] * np.matmul(JV.transpose(0, 2, 1), JV)
                G -= w * np.outer(div, phi)                           # det cancels (Piola)
                Mp += (sigma * w * det)[:, None, None] * np.outer(phi, phi)[None]
                vol += w * det
    A = np.zeros((n, nu + npr, nu + npr))
    A[:, :nu, :nu] = M
    A[:, :nu, nu:] = G[None]
    A[:, nu:, :nu] = -G.T[None]
    A[:, nu:, nu:] = Mp
    return A, vol


def local_inverse(A: np.ndarray) -> np.ndarray:
    """A_K^-1 by LU with partial pivoting of the symmetrically equilibrated matrix
    D A_K D, D = |diag A_K|^-1/2 (the velocity and pressure blocks live on different scales)."""
    d = 1.0 / np.sqrt(np.abs(np.diagonal(A, axis1=1, axis2=2)))
    return d[:, :, None] * np.linalg.inv(A * d[:, :, None] * d[:, None, :]) * d[:, None, :]


# ---- trace numbering ------------------------------------------------------------------------
def trace_sizes(mesh, el: Element):
    nt2 = el.nt * el.nt
    NH = mesh.nedge * mesh.nlev * nt2
    NZ = mesh.ncol * (mesh.nlev + 1) * nt2
    return NH, NZ, NH + NZ


def trace_dof_ids(mesh, el: Element, cells=None) -> np.ndarray:
    """[n, nlam] global trace dof of each local facet node (f, s, t): lambda^h at
    ((edge L + level) nt + s_owner) nt + t, lambda^z at NH + ((column (L+1) + interface) nt + s) nt
    + t, s_owner = s in the owner column and p - s in the other."""
    if cells is None:
        cells = np.arange(mesh.ncell)
    col, lev = np.divmod(np.asarray(cells), mesh.nlev)
    L, nt, p = mesh.nlev, el.nt, el.p
    NH, _NZ, _T = trace_sizes(mesh, el)
    g = np.zeros((len(col), el.nlam), np.int64)
    for f in range(6):
        for s in range(nt):
            for t in range(nt):
                q = (f * nt + s) * nt + t
                if f < 4:
                    e = mesh.col_edges[col, f].astype(np.int64)
                    owner = (mesh.edge_cols[e, 0] == col) & (mesh.edge_face[e, 0] == f)
                    sg = np.where(owner, s, p - s)
                    g[:, q] = ((e * L + lev) * nt + sg) * nt + t
                else:
                    k = lev + (1 if f == 5 else 0)
                    g[:, q] = NH + ((col * (L + 1) + k) * nt + s) * nt + t
    return g


# ---- the hybridised system ------------------------------------------------------------------
class HigherOrderHybrid:
    """Cell matrices, static condensation, S, B_lambda, recovery, Algorithm 1 at degree p, and
    Algorithm 2 with the lowest-order pressure multigrid as the coarse solve."""

    def __init__(self, hier, coeffs, p: int, omega=0.6, n_pre=1, n_post=2, mg=None):
        if coeffs.preset != 1:
            raise ValueError("the degree-p oracle covers the constant-coefficient Helmholtz preset")
        self.hier, self.coeffs, self.p = hier, coeffs, p
        self.mesh = mesh = hier.meshes[0]
        self.el = el = Element(p)
        self.omega, self.n_pre, self.n_post = omega, n_pre, n_post
        self.A, self.vol = cell_matrices(mesh, el, coeffs.sigma)
        self.Ainv = local_inverse(self.A)
        self.C = el.trace_coupling()
        nf = el.nfacet
        Cf = self.C[:nf]                                       # facet rows (the others are 0)
        self.S_K = np.einsum("ai,nab,bj->nij", Cf, self.Ainv[:, :nf, :nf], Cf)
        self.gid = trace_dof_ids(mesh, el)
        self.NH, self.NZ, self.T = trace_sizes(mesh, el)
        rows = np.broadcast_to(self.gid[:, :, None], self.S_K.shape).ravel()
        cols = np.broadcast_to(self.gid[:, None, :], self.S_K.shape).ravel()
        self.S = sp.coo_matrix((self.S_K.ravel(), (rows, cols)), shape=(self.T, self.T)).tocsr()
        # smoother blocks: each vertical facet's block of S and each column's S^zz
        self.D = self._smoother_matrix()
        self.Dlu = spla.splu(self.D.tocsc())
        # P: constant on each facet, the average of the adjacent cells' values
        count = np.zeros(self.T)
        np.add.at(count, self.gid, 1.0)
        cellsr = np.repeat(np.arange(mesh.ncell), el.nlam)
        self.P = sp.coo_matrix((1.0 / count[self.gid.ravel()], (self.gid.ravel(), cellsr)),
                               shape=(self.T, mesh.ncell)).tocsr()
        self.mg = mg if mg is not None else PressureMultigrid(hier, coeffs, 0.9, 1, 2, 3)
        one = np.ones(mesh.ncell)
        h1 = pressure_operator_times(self.mg.parts0, one)
        self.gamma = h1 / (self.P.T @ (self.S @ (self.P @ one)))

    def _smoother_matrix(self) -> sp.csr_matrix:
        """D of Algorithm 1: S restricted to the blocks of single vertical facets and of the
        horizontal facets of single columns (all couplings between two different blocks
        dropped)."""
        mesh, el = self.mesh, self.el
        nt2 = el.nt * el.nt
        block = np.empty(self.T, np.int64)
        block[:self.NH] = np.arange(self.NH) // nt2                       # one block per vertical facet
        block[self.NH:] = self.NH // nt2 + np.arange(self.NZ) // ((mesh.nlev + 1) * nt2)   # per column
        S = self.S.tocoo()
        keep = block[S.row] == block[S.col]
        return sp.coo_matrix((S.data[keep], (S.row[keep], S.col[keep])), shape=S.shape).tocsr()

    # -- Eq. hybrid-rhs and hybrid-recovery --------------------------------------------------
    def rhs(self, Ru: np.ndarray, Rpi: np.ndarray) -> np.ndarray:
        """B_lambda = sum_K C_K^T A_K^-1 R_K; Ru [C, nu], Rpi [C, npr]."""
        R = np.concatenate([Ru, Rpi], axis=1)
        Y = np.einsum("nij,nj->ni", self.Ainv, R)
        B = np.zeros(self.T)
        np.add.at(B, self.gid, Y[:, :self.el.nfacet] @ self.C[:self.el.nfacet])
        return B

    def reconstruct(self, lam, Ru, Rpi):
        """X_K = A_K^-1 (R_K - C_K lambda_K): velocity [C, nu] (outward facet fluxes first) and
        pressure [C, npr]."""
        R = np.concatenate([Ru, Rpi], axis=1)
        R[:, :self.el.nu] -= lam[self.gid] @ self.C.T
        X = np.einsum("nij,nj->ni", self.Ainv, R)
        return X[:, :self.el.nu], X[:, self.el.nu:]

    # -- Algorithm 1 and Algorithm 2 ---------------------------------------------------------
    def smooth(self, lam, b, nsweeps):
        for _ in range(nsweeps):
            lam = lam + self.omega * self.Dlu.solve(b - self.S @ lam)
        return lam

    def two_level(self, r):
        lam = self.smooth(np.zeros_like(r), r, self.n_pre)      # lines 1-2
        R = r - self.S @ lam                                    # line 3
        bbar = self.gamma * (self.P.T @ R)                      # lines 4-5
        dpi = self.mg.vcycle(bbar)                              # line 6
        lam = lam + self.P @ dpi                                # line 7
        return self.smooth(lam, r, self.n_post)                 # line 8

    def solve(self, Ru, Rpi, tol, maxit=300):
        B = self.rhs(Ru, Rpi)
        return bicgstab(lambda x: self.S @ x, B, self.two_level, tol, maxit)


# ---- the unhybridised mixed system (pin) ----------------------------------------------------
def facet_orientation(mesh, el: Element, cells=None) -> np.ndarray:
    """[n, nlam] sign of each local facet dof against the global orientation of the continuous
    RT_p dof: out of edge_cols[e][0] on vertical facets, upwards on horizontal ones."""
    s0 = fem.face_orientation(mesh, cells)                     # [n, 6]
    return np.repeat(s0, el.nt * el.nt, axis=1)


def mixed_solve(ho: HigherOrderHybrid, Ru, Rpi):
    """The continuous-RT_p / DG_p system (no hybridisation) assembled and solved directly:
    facet dofs shared between the two cells (global orientation), u.n = 0 on ground and lid,
    interior velocity dofs and DG_p pressure per cell. Returns (u_facet [T] in the trace
    numbering, 0 on ground and lid; u_interior [C, nu - nfacet]; Pi [C, npr])."""
    mesh, el, A = ho.mesh, ho.el, ho.A
    T, C, nu, npr, nf = ho.T, mesh.ncell, el.nu, el.npr, el.nfacet
    L, nt2 = mesh.nlev, el.nt * el.nt
    boundary = np.zeros(T, bool)
    for c in range(mesh.ncol):
        for k in (0, L):
            z0 = ho.NH + (c * (L + 1) + k) * nt2
            boundary[z0:z0 + nt2] = True
    interior = np.flatnonzero(~boundary)
    pos = -np.ones(T, np.int64)
    pos[interior] = np.arange(len(interior))
    nfi, nint = len(interior), nu - nf
    N = nfi + C * (nint + npr)
    # global index and sign of every local dof of every cell
    sg = facet_orientation(mesh, el)
    idx = np.zeros((C, nu + npr), np.int64)
    sgn = np.ones((C, nu + npr))
    idx[:, :nf] = pos[ho.gid]
    sgn[:, :nf] = sg
    base = nfi + np.arange(C)[:, None] * (nint + npr)
    idx[:, nf:] = base + np.arange(nint + npr)[None, :]
    R = np.concatenate([Ru, Rpi], axis=1)
    keep = idx >= 0
    rows, cols, vals = [], [], []
    rhs = np.zeros(N)
    for K in range(C):
        ok = np.flatnonzero(keep[K])
        I = idx[K, ok]
        s = sgn[K, ok]
        blk = A[K][np.ix_(ok, ok)] * s[:, None] * s[None, :]
        rows.append(np.repeat(I, len(I)))
        cols.append(np.tile(I, len(I)))
        vals.append(blk.ravel())
        np.add.at(rhs, I, s * R[K, ok])
    Mx = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(N, N)).tocsc()
    x = spla.spsolve(Mx, rhs)
    uf = np.zeros(T)
    uf[interior] = x[:nfi]
    rest = x[nfi:].reshape(C, nint + npr)
    return uf, rest[:, :nint], rest[:, nint:]


# ---- a smooth solution (pin of the convergence order) ---------------------------------------
def manufactured_rhs(ho: HigherOrderHybrid, pi_exact, f_exact, nq=None):
    """R_u = 0, R_Pi = int phi_j f (Gauss rule with p + 4 points per direction), and the L2 norm
    machinery: returns (Ru, Rpi, l2_error(Pi_dofs))."""
    mesh, el = ho.mesh, ho.el
    verts = fem.cell_vertices(mesh)
    qx, qw = gauss_legendre(nq or el.p + 4)
    C = mesh.ncell
    Rpi = np.zeros((C, el.npr))
    pts = []
    for a, xa in enumerate(qx):
        for b, xb in enumerate(qx):
            for c, xc in enumerate(qx):
                N, dN = fem.trilinear_shape(xa, xb, xc)
                x = N @ verts
                J = np.matmul(verts.transpose(0, 2, 1), dN)
                det = np.linalg.det(J)
                w = qw[a] * qw[b] * qw[c] * det
                phi = el.pressure(xa, xb, xc)
                Rpi += (w * f_exact(x))[:, None] * phi[None]
                pts.append((w, phi, pi_exact(x)))

    def l2_error(Pi):
        e2 = 0.0
        for w, phi, ex in pts:
            e2 += np.sum(w * (Pi @ phi - ex) ** 2)
        return np.sqrt(e2)
    return np.zeros((C, el.nu)), Rpi, l2_error
