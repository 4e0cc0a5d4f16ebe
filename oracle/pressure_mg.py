"""Pressure operator H and tensor-product pressure multigrid (FP64).

Oracle (test infrastructure only; see oracle/__init__.py).

Paper passages: Sec. 2.3 - the approximate Schur complement with the lumped velocity mass
matrix (Eq. 2x2system_approx), the pressure operator H = -B Mlump^-1 G + M3^Pi
(Eq. elliptic_pressure_system) and the column block-Jacobi smoother with H_z
(Eq. pressure_block_jacobi); Sec. 3.2 - 4 levels, 1 pre- and 2 post-smoothing steps,
omega_pressure = 0.9.

Readings (the paper defers these details to Maynard et al. 2020):
* lumping: Mlump_ff = sum over the cells K sharing f of |M_K(f,f)| + |M_K(f,f')|, f' the
  face opposite f in K (e0-e2, e1-e3, bottom-top). On boxes this is the absolute row sum,
  which gives the textbook 7-point finite-volume Helmholtz stencil; on cubed-sphere cells
  it leaves out the couplings between faces of different directions, which are artefacts
  of the non-orthogonal trilinear cells and, at aspect ratios of 10^3..10^4, outweigh the
  vertical mass entries by orders of magnitude;
* H_z = the diagonal of H plus its couplings inside one column (tridiagonal);
* coarse levels: 2x2 horizontal agglomeration, H rediscretised on the coarse mesh with the
  same background, restriction = sum over the four children, prolongation = injection;
* coarsest level: 3 block-Jacobi sweeps (the operator is well conditioned there).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import fem
from .smoother import thomas

OPPOSITE = (2, 3, 0, 1, 5, 4)   # e0-e2, e1-e3, bottom-top


def pressure_operator_parts(mesh, bg, co, system=None):
    """The factors of H = -B Mlump^-1 G + M3^Pi on continuous RT0 with u.n = 0 on ground and
    lid: (B [C x T], 1/Mlump [T] (0 on ground and lid faces), G [T x C], M3^Pi [C]).
    `system` may pass the (A, Kdiag, coefficients) of fem.cell_system for this mesh."""
    A, _Kd, cc = fem.cell_system(mesh, bg, co) if system is None else system
    g = fem.trace_dof_ids(mesh)
    s = fem.face_orientation(mesh)
    T, C, L = mesh.n_trace, mesh.ncell, mesh.nlev
    interior = np.ones(T, bool)
    zc = mesh.n_trace_h + np.arange(mesh.ncol) * (L + 1)
    interior[zc] = False
    interior[zc + L] = False
    # lumped mass: |diagonal| + |coupling to the opposite face|, summed over the two cells
    Mabs = np.abs(cc["M"])
    lump_cell = np.stack([Mabs[:, f, f] + Mabs[:, f, OPPOSITE[f]] for f in range(6)], axis=1)
    lump = np.zeros(T)
    np.add.at(lump, g, lump_cell)
    inv_lump = np.where(interior, 1.0 / np.where(interior, lump, 1.0), 0.0)
    cells = np.repeat(np.arange(C), 6)
    Bg = sp.coo_matrix(((s * A[:, 6, :6]).ravel(), (cells, g.ravel())), shape=(C, T)).tocsr()
    Gg = sp.coo_matrix(((s * A[:, :6, 6]).ravel(), (g.ravel(), cells)), shape=(T, C)).tocsr()
    return Bg, inv_lump, Gg, cc["m"]


def pressure_operator(mesh, bg, co, system=None) -> sp.csr_matrix:
    """H = -B Mlump^-1 G + M3^Pi (Eq. elliptic_pressure_system) as one sparse matrix."""
    Bg, inv_lump, Gg, m = pressure_operator_parts(mesh, bg, co, system)
    return (sp.diags(m) - Bg @ sp.diags(inv_lump) @ Gg).tocsr()


def pressure_operator_times(parts, x):
    """H x evaluated right to left through the factors, -B (Mlump^-1 (G x)) + M3^Pi x. For a
    constant x, G x vanishes exactly (the two cells of a facet contribute -k theta and
    +k theta), so H 1 = M3^Pi 1 without the cancellation of summing the rows of H."""
    Bg, inv_lump, Gg, m = parts
    return m * x - Bg @ (inv_lump * (Gg @ x))


def column_tridiagonal(mesh, H):
    """H_z: (sub, diag, sup) [ncol, L] of H restricted to each column."""
    L = mesh.nlev
    ids = np.arange(mesh.ncol)[:, None] * L + np.arange(L)[None, :]
    diag = np.asarray(H[ids.ravel(), ids.ravel()]).reshape(ids.shape)
    sub = np.zeros_like(diag)
    sup = np.zeros_like(diag)
    if L > 1:
        sub[:, 1:] = np.asarray(H[ids[:, 1:].ravel(), ids[:, :-1].ravel()]).reshape(mesh.ncol, L - 1)
        sup[:, :-1] = np.asarray(H[ids[:, :-1].ravel(), ids[:, 1:].ravel()]).reshape(mesh.ncol, L - 1)
    return sub, diag, sup


class PressureMultigrid:
    def __init__(self, hier, coeffs, omega=0.9, npre=1, npost=2, ncoarse=3, finest_system=None):
        self.hier = hier
        self.omega, self.npre, self.npost, self.ncoarse = omega, npre, npost, ncoarse
        self.H, self.Hz = [], []
        for l, (mesh, bg) in enumerate(zip(hier.meshes, coeffs.levels)):
            parts = pressure_operator_parts(mesh, bg, coeffs, finest_system if l == 0 else None)
            if l == 0:
                self.parts0 = parts
            Bg, inv_lump, Gg, m = parts
            H = (sp.diags(m) - Bg @ sp.diags(inv_lump) @ Gg).tocsr()
            self.H.append(H)
            self.Hz.append(column_tridiagonal(mesh, H))

    def block_jacobi(self, l, x, b):
        """x + omega H_z^-1 (b - H x) (Eq. pressure_block_jacobi)."""
        mesh = self.hier.meshes[l]
        r = (b - self.H[l] @ x).reshape(mesh.ncol, mesh.nlev)
        return x + self.omega * thomas(*self.Hz[l], r).ravel()

    def restrict(self, l, r):
        """Sum of the four horizontal children, level by level."""
        fine, coarse = self.hier.meshes[l], self.hier.meshes[l + 1]
        out = np.zeros((coarse.ncol, coarse.nlev))
        np.add.at(out, self.hier.parents[l], r.reshape(fine.ncol, fine.nlev))
        return out.ravel()

    def prolong(self, l, e):
        """Injection: every child takes its parent's value."""
        fine, coarse = self.hier.meshes[l], self.hier.meshes[l + 1]
        return e.reshape(coarse.ncol, coarse.nlev)[self.hier.parents[l]].ravel()

    def vcycle(self, b, l=0, x0=None):
        """One V-cycle for H_l x = b from a zero initial guess, or from x0 (the first
        smoothing sweep of level l then starts from x0)."""
        x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64)
        if l == self.hier.nmg - 1:
            for _ in range(self.ncoarse):
                x = self.block_jacobi(l, x, b)
            return x
        for _ in range(self.npre):
            x = self.block_jacobi(l, x, b)
        r = b - self.H[l] @ x
        x = x + self.prolong(l, self.vcycle(self.restrict(l, r), l + 1))
        for _ in range(self.npost):
            x = self.block_jacobi(l, x, b)
        return x
