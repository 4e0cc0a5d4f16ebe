"""Lowest-order compatible FE cell matrices, hybridisation and static condensation (FP64).

Oracle (test infrastructure only; see oracle/__init__.py).

Paper passages followed (arXiv 2210.11797):
* Sec. 2.1, Eqs. gh-u_elim..gh-pi_elim: the linear system after theta' elimination.
* Sec. 2.2, Eq. bilinear_forms: the forms m2, q22, g, d, m3, q32, m3^rho, m3^Pi; the
  quadrature statement (n = p+3 Gauss points per direction for volume terms, a one-point
  cell-centre rule for q32, m3^rho, m3^Pi).
* Eq. 2x2system: algebraic density elimination, B = Q32 + M3^rho M3^-1 D.
* Sec. 2.4, Eqs. gh-fem-hybrid .. hybrid-recovery: broken velocity, trace multipliers,
  S = C^T A^-1 K, B_lambda = C^T A^-1 R_X, X = A^-1 (R_X - K lambda).

Lowest order (p = 0): RT0 has one outward unit flux per face, DG0 one value per cell,
the trace space one value per facet.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

# 3-point Gauss-Legendre rule on [0,1] (n = p + 3 = 3 at p = 0).
_G = np.sqrt(15.0) / 10.0
GAUSS_X = np.array([0.5 - _G, 0.5, 0.5 + _G])
GAUSS_W = np.array([5.0, 8.0, 5.0]) / 18.0

# local face order: e0 (eta=0), e1 (xi=1), e2 (eta=1), e3 (xi=0), bottom (zeta=0), top (zeta=1)
BOTTOM, TOP = 4, 5


def rt0_reference_basis(xi: float, eta: float, zeta: float) -> np.ndarray:
    """[6,3] lowest-order Raviart-Thomas basis on the unit cube, each with unit OUTWARD
    flux through its own face, zero flux through the others and divergence 1."""
    return np.array([
        [0.0, eta - 1.0, 0.0],   # e0: eta = 0, outward normal -eta
        [xi, 0.0, 0.0],          # e1: xi = 1
        [0.0, eta, 0.0],         # e2: eta = 1
        [xi - 1.0, 0.0, 0.0],    # e3: xi = 0, outward normal -xi
        [0.0, 0.0, zeta - 1.0],  # bottom
        [0.0, 0.0, zeta],        # top
    ])


def trilinear_shape(xi, eta, zeta):
    """Values [8] and reference gradients [8,3] of the trilinear map's shape functions.
    Vertex v = a + 2b + 4c sits at (xi,eta,zeta) = (a,b,c)."""
    n = np.zeros(8)
    dn = np.zeros((8, 3))
    for v in range(8):
        a, b, c = v & 1, (v >> 1) & 1, (v >> 2) & 1
        fx, fy, fz = (xi if a else 1 - xi), (eta if b else 1 - eta), (zeta if c else 1 - zeta)
        gx, gy, gz = (1.0 if a else -1.0), (1.0 if b else -1.0), (1.0 if c else -1.0)
        n[v] = fx * fy * fz
        dn[v] = (gx * fy * fz, fx * gy * fz, fx * fy * gz)
    return n, dn


_CORNER_OF = {(0, 0): 0, (1, 0): 1, (1, 1): 2, (0, 1): 3}


def cell_vertices(mesh, cells=None) -> np.ndarray:
    """[n,8,3] physical vertices of the cells (c*nlev + k): the column corner times
    (R + z) on the sphere, (x, y, z) on the plane."""
    if cells is None:
        cells = np.arange(mesh.ncell)
    cells = np.asarray(cells)
    col, lev = np.divmod(cells, mesh.nlev)
    z = mesh.z_levels
    out = np.zeros((len(cells), 8, 3))
    for v in range(8):
        a, b, c = v & 1, (v >> 1) & 1, (v >> 2) & 1
        corner = mesh.corners[col, _CORNER_OF[(a, b)]]
        height = z[lev + c]
        if mesh.geometry == 1:
            out[:, v] = corner * (mesh.radius + height)[:, None]
        else:
            out[:, v] = corner
            out[:, v, 2] = height
    return out


def _vertical_unit(x: np.ndarray, geometry: int) -> np.ndarray:
    if geometry == 1:
        return x / np.linalg.norm(x, axis=-1, keepdims=True)
    r = np.zeros_like(x)
    r[..., 2] = 1.0
    return r


def local_mass(verts: np.ndarray, c22: np.ndarray, geometry: int, coriolis=None):
    """Velocity block of A_K and the volumes, by 3x3x3 Gauss quadrature (Sec. 2.2).

    M_K(f,g) = int_K [v_f.v_g + c22 (zhat.v_f)(zhat.v_g) + v_f.(c x v_g)] dx with the
    contravariant Piola map v = J vhat / det J; c22 is the vertical weight of -Q22 (the
    dimensionally inconsistent mu term of Eq. gh-u is dropped: buoyancy enters through -Q22
    only, whose weight tau_u tau_theta dt^2 N^2 makes 1 + c22 the paper's mu) and
    c = tau_u dt 2 Omega the Coriolis vector of Eq. gh-u
    (None: no rotation). Returns M [n,6,6], |K| (Gauss) [n], |K|_1 (one-point) [n] and
    (zhat . v_f) at the cell centre [n,6].
    """
    n = verts.shape[0]
    M = np.zeros((n, 6, 6))
    vol = np.zeros(n)
    for qi in range(3):
        for qj in range(3):
            for qk in range(3):
                xi, eta, zeta = GAUSS_X[qi], GAUSS_X[qj], GAUSS_X[qk]
                w = GAUSS_W[qi] * GAUSS_W[qj] * GAUSS_W[qk]
                N, dN = trilinear_shape(xi, eta, zeta)
                x = N @ verts                                   # [n,3]
                J = np.matmul(verts.transpose(0, 2, 1), dN)     # [n,3,3], J[:, i, d] = dx_i/dxi_d
                det = np.linalg.det(J)
                Jv = np.matmul(J, rt0_reference_basis(xi, eta, zeta).T)   # [n,3,6]: J vhat_f
                rv = np.matmul(_vertical_unit(x, geometry)[:, None, :], Jv)  # [n,1,6]
                M += (w / det)[:, None, None] * (
                    np.matmul(Jv.transpose(0, 2, 1), Jv)
                    + c22[:, None, None] * np.matmul(rv.transpose(0, 2, 1), rv))
                if coriolis is not None:
                    cxv = np.cross(np.asarray(coriolis, np.float64)[None, :, None], Jv, axis=1)   # c x (J vhat_g)
                    M += (w / det)[:, None, None] * np.matmul(Jv.transpose(0, 2, 1), cxv)
                vol += w * det
    N, dN = trilinear_shape(0.5, 0.5, 0.5)
    xc = N @ verts
    Jc = np.matmul(verts.transpose(0, 2, 1), dN)
    detc = np.linalg.det(Jc)
    Jv = np.matmul(Jc, rt0_reference_basis(0.5, 0.5, 0.5).T)
    zv_centre = np.matmul(_vertical_unit(xc, geometry)[:, None, :], Jv)[:, 0, :] / detc[:, None]
    return M, vol, detc, zv_centre


def other_column(mesh, col, face):
    """Column on the far side of vertical local face `face` of column `col`."""
    e = mesh.col_edges[col, face]
    c0, c1 = mesh.edge_cols[e, 0], mesh.edge_cols[e, 1]
    return np.where(c0 == col, c1, c0)


def cell_coefficients(mesh, bg, co, cells=None):
    """Per-cell ingredients of A_K (Eqs. bilinear_forms, 2x2system, hybrid-A).

    Returns a dict with
      M      [n,6,6]  velocity block (M2 - Q22 restricted to the cell)
      k      scalar   tau_u dt c_p  (1 for the Helmholtz preset)
      theta  [n,6]    single-valued theta* on each face (reading: mean of the two columns'
                      layer means on vertical faces, the level value on horizontal faces)
      b      [n,6]    pressure-row coupling (Q32 + M3^rho M3^-1 D) per face
      m      [n]      M3^Pi
      vol, vol1       Gauss and one-point volumes
    """
    if cells is None:
        cells = np.arange(mesh.ncell)
    cells = np.asarray(cells)
    col, lev = np.divmod(cells, mesh.nlev)
    verts = cell_vertices(mesh, cells)
    dz = mesh.z_levels[lev + 1] - mesh.z_levels[lev]
    th0, th1 = bg.theta_lev[col, lev], bg.theta_lev[col, lev + 1]
    pi0, pi1 = bg.exner_lev[col, lev], bg.exner_lev[col, lev + 1]
    if co.preset == 1:
        c22 = np.zeros(len(cells))
    else:
        # -Q22 weight: -tau_u tau_theta dt^2 c_p (d_z hatPi*)(d_z theta*), constant per cell
        c22 = -co.tau_u * co.tau_theta * co.dt ** 2 * co.cp * ((pi1 - pi0) / dz) * ((th1 - th0) / dz)
    omega = getattr(co, "omega", 0.0)
    # Coriolis (Eq. gh-u): tau_u dt 2 Omega, the rotation axis being the sphere's polar axis
    # (z of the Earth-centred frame) or the vertical of the plane (an f-plane)
    cor = None if (co.preset == 1 or omega == 0.0) else (0.0, 0.0, co.tau_u * co.dt * 2.0 * omega)
    M, vol, vol1, zv = local_mass(verts, c22, mesh.geometry, cor)
    theta = np.zeros((len(cells), 6))
    mean_own = 0.5 * (th0 + th1)
    for f in range(4):
        oc = other_column(mesh, col, f)
        mean_other = 0.5 * (bg.theta_lev[oc, lev] + bg.theta_lev[oc, lev + 1])
        theta[:, f] = 0.5 * (mean_own + mean_other)
    theta[:, BOTTOM], theta[:, TOP] = th0, th1
    if co.preset == 1:
        k = 1.0
        b = np.ones((len(cells), 6))
        m = co.sigma * vol1
        theta[:] = 1.0
    else:
        k = co.tau_u * co.dt * co.cp
        # q32 with the one-point rule: tau_theta dt |K|_1 (d_z theta*/theta*) (zhat.v_f)(x_c)
        dlogtheta = ((th1 - th0) / dz) / mean_own
        q = co.tau_theta * co.dt * (vol1 * dlogtheta)[:, None] * zv
        # M3^rho M3^-1 D: (|K|_1/rho*) (1/|K|) (tau_rho dt rho* 1^T); rho* cancels
        b = (co.tau_rho * co.dt * vol1 / vol)[:, None] + q
        m = (1.0 - co.kappa) / co.kappa * vol1 / bg.exner[col, lev]
    return dict(M=M, k=k, theta=theta, b=b, m=m, vol=vol, vol1=vol1, c22=c22)


def cell_system(mesh, bg, co, cells=None):
    """A_K [n,7,7] = [[M, G_K], [b^T, m]] with G_K = -k theta (Eq. hybrid-A), and the
    diagonal of K_K = k diag(theta) [n,6] (Eq. hybrid-K)."""
    cc = cell_coefficients(mesh, bg, co, cells)
    n = cc["M"].shape[0]
    A = np.zeros((n, 7, 7))
    A[:, :6, :6] = cc["M"]
    A[:, :6, 6] = -cc["k"] * cc["theta"]
    A[:, 6, :6] = cc["b"]
    A[:, 6, 6] = cc["m"]
    return A, cc["k"] * cc["theta"], cc


def trace_dof_ids(mesh, cells=None) -> np.ndarray:
    """[n,6] global trace dof of each local face: lambda^h at edge*L + k, lambda^z at
    nedge*L + c*(L+1) + k (bottom) and + k+1 (top)."""
    if cells is None:
        cells = np.arange(mesh.ncell)
    col, lev = np.divmod(np.asarray(cells), mesh.nlev)
    L, NH = mesh.nlev, mesh.n_trace_h
    g = np.zeros((len(col), 6), np.int64)
    for f in range(4):
        g[:, f] = mesh.col_edges[col, f].astype(np.int64) * L + lev
    g[:, BOTTOM] = NH + col * (L + 1) + lev
    g[:, TOP] = NH + col * (L + 1) + lev + 1
    return g


def local_inverse(A: np.ndarray) -> np.ndarray:
    """A_K^-1 [n,7,7] by block elimination of A_K = [[M, g], [b^T, m]] (the cell-local
    inversion of Sec. 2.4): with y = M^-1 g, z = M^-T b and the pressure Schur complement
    s = m - b.y,
        A^-1 = [[M^-1 + y z^T / s, -y / s], [-z^T / s, 1 / s]].
    M^-1 is taken from the symmetrically equilibrated velocity block diag(M)^-1/2 M
    diag(M)^-1/2. A_K's rows span ~20 orders of magnitude (|M| ~ 1e-11..1e-2, m ~ 1e13
    on the sphere), where partial pivoting on A_K itself loses up to 1e-12 relative
    accuracy; this form stays within a few ulps of the exact inverse."""
    M, g, b, m = A[:, :6, :6], A[:, :6, 6], A[:, 6, :6], A[:, 6, 6]
    d = 1.0 / np.sqrt(np.abs(np.diagonal(M, axis1=1, axis2=2)))
    Minv = d[:, :, None] * np.linalg.inv(M * d[:, :, None] * d[:, None, :]) * d[:, None, :]
    y = np.einsum("nij,nj->ni", Minv, g)
    z = np.einsum("nji,nj->ni", Minv, b)
    s = m - np.einsum("ni,ni->n", b, y)
    Ainv = np.empty_like(A)
    Ainv[:, :6, :6] = Minv + y[:, :, None] * z[:, None, :] / s[:, None, None]
    Ainv[:, :6, 6] = -y / s[:, None]
    Ainv[:, 6, :6] = -z / s[:, None]
    Ainv[:, 6, 6] = 1.0 / s
    return Ainv


def condense(A: np.ndarray, Kdiag: np.ndarray) -> np.ndarray:
    """Local Schur complement S_K = C_K^T A_K^-1 K_K with C_K = identity on the six faces
    (Eq. hybrid-S): the velocity rows of A_K^-1 times diag(K_K)."""
    return local_inverse(A)[:, :6, :6] * Kdiag[:, None, :]


def trace_row_sums(mesh, A: np.ndarray) -> np.ndarray:
    """S 1, the row sums of the trace operator, without cancellation.

    Since G_K = -K_K 1 (the volume and facet terms of g carry the same theta, Sec. 2.4),
    A_K [0; -1] = [K_K 1; -m_K], hence A_K^-1 [K_K 1; 0] = [0; -1] + m_K A_K^-1 e_p and
    S_K 1 = (A_K^-1)_uu K_K 1 = m_K (A_K^-1)_{u,p}. Summing S_K's rows entry by entry would
    cancel to ~1e-9 of the row scale on the sphere; this form does not."""
    contrib = A[:, 6, 6][:, None] * local_inverse(A)[:, :6, 6]
    out = np.zeros(mesh.n_trace)
    np.add.at(out, trace_dof_ids(mesh), contrib)
    return out


def assemble_trace_operator(mesh, S_K: np.ndarray) -> sp.csr_matrix:
    """S = sum over cells of S_K scattered to the cell's six trace dofs."""
    g = trace_dof_ids(mesh)
    rows = np.broadcast_to(g[:, :, None], S_K.shape).ravel()
    cols = np.broadcast_to(g[:, None, :], S_K.shape).ravel()
    T = mesh.n_trace
    return sp.coo_matrix((S_K.ravel(), (rows, cols)), shape=(T, T)).tocsr()


def trace_rhs(mesh, A: np.ndarray, Rub: np.ndarray, Rpi: np.ndarray) -> np.ndarray:
    """B_lambda = C^T A^-1 R_X (Eq. hybrid-rhs), R_X = (R_u^b, R_Pi) per cell."""
    R = np.concatenate([Rub, Rpi[:, None]], axis=1)
    Y = np.einsum("nij,nj->ni", local_inverse(A), R)
    B = np.zeros(mesh.n_trace)
    np.add.at(B, trace_dof_ids(mesh), Y[:, :6])
    return B


def reconstruct(mesh, A, Kdiag, lam, Rub, Rpi):
    """X_K = A_K^-1 (R_K - K_K lambda_K) (Eq. hybrid-recovery): broken u [C,6], Pi [C]."""
    R = np.concatenate([Rub - Kdiag * lam[trace_dof_ids(mesh)], Rpi[:, None]], axis=1)
    X = np.einsum("nij,nj->ni", local_inverse(A), R)
    return X[:, :6], X[:, 6]


def continuity_jump(mesh, ub: np.ndarray) -> np.ndarray:
    """C^T u^b: the sum of the outward fluxes of the cells sharing each facet."""
    J = np.zeros(mesh.n_trace)
    np.add.at(J, trace_dof_ids(mesh), ub)
    return J


def face_orientation(mesh, cells=None) -> np.ndarray:
    """[n,6] sign s_K(f) relating the cell's outward flux to the global orientation of the
    continuous W2 dof: vertical faces point out of edge_cols[e,0]; horizontal faces up."""
    if cells is None:
        cells = np.arange(mesh.ncell)
    col, _lev = np.divmod(np.asarray(cells), mesh.nlev)
    s = np.zeros((len(col), 6))
    for f in range(4):
        e = mesh.col_edges[col, f]
        s[:, f] = np.where((mesh.edge_cols[e, 0] == col) & (mesh.edge_face[e, 0] == f), 1.0, -1.0)
    s[:, BOTTOM], s[:, TOP] = -1.0, 1.0
    return s


def mixed_system(mesh, bg, co, Rub, Rpi):
    """The unhybridised 2x2 system (Eq. 2x2system) on continuous RT0 (interior faces only;
    u.n = 0 on the ground and lid), assembled densely for a direct solve.

    Unknowns: interior trace ids (the same numbering as lambda, boundary faces removed)
    followed by the cells. Returns (matrix, rhs, interior_ids)."""
    A, _Kd, _cc = cell_system(mesh, bg, co)
    g = trace_dof_ids(mesh)
    s = face_orientation(mesh)
    L = mesh.nlev
    T = mesh.n_trace
    is_boundary = np.zeros(T, bool)
    zc = np.arange(mesh.ncol) * (L + 1) + mesh.n_trace_h
    is_boundary[zc] = True
    is_boundary[zc + L] = True
    interior = np.flatnonzero(~is_boundary)
    pos = -np.ones(T, np.int64)
    pos[interior] = np.arange(len(interior))
    nf, C = len(interior), mesh.ncell
    Mx = np.zeros((nf + C, nf + C))
    rhs = np.zeros(nf + C)
    for K in range(C):
        for i in range(6):
            fi = pos[g[K, i]]
            if fi >= 0:
                rhs[fi] += s[K, i] * Rub[K, i]
                Mx[fi, nf + K] += s[K, i] * A[K, i, 6]          # G
                Mx[nf + K, fi] += s[K, i] * A[K, 6, i]          # B
                for j in range(6):
                    fj = pos[g[K, j]]
                    if fj >= 0:
                        Mx[fi, fj] += s[K, i] * s[K, j] * A[K, i, j]
        Mx[nf + K, nf + K] = A[K, 6, 6]
        rhs[nf + K] = Rpi[K]
    return Mx, rhs, interior
