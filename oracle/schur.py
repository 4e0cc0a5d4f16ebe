"""Configuration 1 of the paper (Sec. 2.3 and Sec. 3.2): BiCGStab on the unhybridised 2x2
system (Eq. 2x2system) preconditioned by the approximate Schur complement: the velocity
mass matrix replaced by its lumped diagonal, then Step 1 (Eq. pressure_rhs), Step 2 (the
pressure system, Eq. elliptic_pressure_system, by one multigrid V-cycle) and Step 3
(Eq. velocity_recovery).

Oracle (test infrastructure only; see oracle/__init__.py). FP64 numpy / scipy.sparse.

Unknowns: the continuous normal velocity on every facet in the trace numbering (T values;
the ground and lid facets carry u.n = 0 and get identity rows, which decouple them), then
the Exner increment on every cell (C values). The velocity of facet f is oriented as in
fem.face_orientation: out of edge_cols[e, 0] on vertical facets, upwards on horizontal ones.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import fem
from .nonnested import bicgstab
from .pressure_mg import PressureMultigrid


def boundary_facets(mesh) -> np.ndarray:
    """Trace ids of the ground and lid facets (u.n = 0 there)."""
    L = mesh.nlev
    zc = mesh.n_trace_h + np.arange(mesh.ncol) * (L + 1)
    return np.concatenate([zc, zc + L])


class MixedSolver:
    """The 2x2 operator, its right-hand side, the approximate Schur preconditioner and the
    BiCGStab solve of configuration 1."""

    def __init__(self, hier, coeffs, mg_omega=0.9, mg_npre=1, mg_npost=2, mg_ncoarse=3):
        self.mesh = mesh = hier.meshes[0]
        system = fem.cell_system(mesh, coeffs.levels[0], coeffs)
        A = system[0]
        self.A = A
        T, C = mesh.n_trace, mesh.ncell
        self.T, self.C = T, C
        g = fem.trace_dof_ids(mesh)
        s = fem.face_orientation(mesh)
        self.g, self.s = g, s
        interior = np.ones(T, bool)
        interior[boundary_facets(mesh)] = False
        self.interior = interior
        # velocity block: sum over cells of s_i s_j A_K(i, j), interior facets only
        cells = np.arange(C)
        rows, cols, vals = [], [], []
        for i in range(6):
            for j in range(6):
                ok = interior[g[:, i]] & interior[g[:, j]]
                rows.append(g[ok, i])
                cols.append(g[ok, j])
                vals.append(s[ok, i] * s[ok, j] * A[ok, i, j])
            ok = interior[g[:, i]]
            # velocity row f, pressure column K: s_i A_K(i, 6) (the G block)
            rows.append(g[ok, i])
            cols.append(T + cells[ok])
            vals.append(s[ok, i] * A[ok, i, 6])
            # pressure row K, velocity column f: s_i A_K(6, i) (the B block)
            rows.append(T + cells[ok])
            cols.append(g[ok, i])
            vals.append(s[ok, i] * A[ok, 6, i])
        rows.append(T + cells)
        cols.append(T + cells)
        vals.append(A[:, 6, 6])
        bnd = np.flatnonzero(~interior)
        rows.append(bnd)
        cols.append(bnd)
        vals.append(np.ones(len(bnd)))
        self.Mx = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                                shape=(T + C, T + C)).tocsr()
        self.mg = PressureMultigrid(hier, coeffs, mg_omega, mg_npre, mg_npost, mg_ncoarse, finest_system=system)
        self.Bg, self.inv_lump, self.Gg, self.m = self.mg.parts0

    def apply(self, x):
        return self.Mx @ x

    def rhs(self, Rub, Rpi):
        """(R_u, R_Pi): R_u on facet f sums s_K(f) R_u^b over the cells of f; 0 on the ground
        and lid."""
        Ru = np.zeros(self.T)
        np.add.at(Ru, self.g, self.s * Rub)
        Ru[~self.interior] = 0.0
        return np.concatenate([Ru, np.asarray(Rpi, np.float64)])

    def precond(self, r, pressure_solve=None):
        """Steps 1-3 with the lumped velocity mass; the pressure system by one V-cycle (or by
        `pressure_solve` when given)."""
        ru, rp = r[: self.T], r[self.T:]
        B = rp - self.Bg @ (self.inv_lump * ru)                       # Step 1
        pi = self.mg.vcycle(B) if pressure_solve is None else pressure_solve(B)   # Step 2
        u = self.inv_lump * (ru - self.Gg @ pi)                       # Step 3
        u[~self.interior] = ru[~self.interior]                        # identity rows
        return np.concatenate([u, pi])

    def solve(self, Rub, Rpi, tol, maxit=200):
        """Returns (u [T], Pi [C], history, status)."""
        b = self.rhs(Rub, Rpi)
        x, hist, status = bicgstab(self.apply, b, self.precond, tol, maxit)
        return x[: self.T], x[self.T:], hist, status
