"""Non-nested two-level preconditioner and the outer Krylov solve (FP64).

Oracle (test infrastructure only; see oracle/__init__.py).

Paper passages:
* Sec. 2.5 "Intergrid operators": P lambda = {{Pi}} (average of the two neighbouring
  cells), Restrict = P^T.
* Sec. 2.5 "Coarse level operator", Eq. scaling_matrix: Gamma_jj = (H 1)_j / (P^T S P 1)_j.
* Algorithm 2: the two-level cycle; Table solver_configurations: configurations 2, 3a,
  3b, 3c; Sec. 3.2: omega = 0.6, 1 pre- / 2 post-smoothing steps.
* Sec. 3.2: BiCGStab reducing the two-norm of the residual by the tolerance.

Readings: P on a boundary facet (one neighbour) takes the one-sided value, so its row of
P holds a single 1; BiCGStab is right-preconditioned, starts from zero and stops on the
unpreconditioned residual of its recurrence, ||r_i|| <= tol ||B_lambda||.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp

from . import fem
from .pressure_mg import PressureMultigrid, pressure_operator_times
from .smoother import LineSmoother


@dataclass
class OracleOptions:
    precond: str = "nonnested"   # "nonnested" (Alg. 2), "linesmooth" (config 2), "none"
    coarse: str = "vcycle"       # "vcycle" (3c), "exact" (3a: 1e-14), "approx" (3b: 1e-2)
    omega: float = 0.6
    n_pre: int = 1
    n_post: int = 2
    n_smooth: int = 1            # sweeps of the single-level preconditioner
    mg_omega: float = 0.9
    mg_npre: int = 1
    mg_npost: int = 2
    mg_ncoarse: int = 3


def prolongation(mesh) -> sp.csr_matrix:
    """P: W3 -> trace, lambda_f = average of the cells adjacent to f (1/2 each on interior
    facets, the single cell's value on ground and lid facets)."""
    g = fem.trace_dof_ids(mesh)
    count = np.zeros(mesh.n_trace)
    np.add.at(count, g, 1.0)
    cells = np.repeat(np.arange(mesh.ncell), 6)
    w = 1.0 / count[g.ravel()]
    return sp.coo_matrix((w, (g.ravel(), cells)), shape=(mesh.n_trace, mesh.ncell)).tocsr()


def bicgstab(apply_A, b, apply_M, tol, maxit, x0=None):
    """Right-preconditioned BiCGStab (van der Vorst 1992; Saad 2003 Alg. 7.7 with
    x = M^-1 y). Returns (x, history of ||r_i||/||b||, status)."""
    x = np.zeros_like(b) if x0 is None else x0.copy()
    r = b - apply_A(x) if x0 is not None else b.copy()
    rhat = r.copy()
    bnorm = np.linalg.norm(b)
    if bnorm == 0.0:
        return x, [0.0], "ok"
    hist = [np.linalg.norm(r) / bnorm]
    if hist[0] <= tol:
        return x, hist, "ok"
    rho_old = alpha = omega = 1.0
    v = np.zeros_like(b)
    p = np.zeros_like(b)
    for _ in range(maxit):
        rho = rhat @ r
        if rho == 0.0:
            return x, hist, "breakdown"
        beta = (rho / rho_old) * (alpha / omega)
        p = r + beta * (p - omega * v)
        phat = apply_M(p)
        v = apply_A(phat)
        rv = rhat @ v
        if rv == 0.0:
            return x, hist, "breakdown"
        alpha = rho / rv
        s = r - alpha * v
        shat = apply_M(s)
        t = apply_A(shat)
        tt = t @ t
        if tt == 0.0:
            return x + alpha * phat, hist, "breakdown"
        omega = (t @ s) / tt
        x = x + alpha * phat + omega * shat
        r = s - omega * t
        rho_old = rho
        hist.append(np.linalg.norm(r) / bnorm)
        if not np.isfinite(hist[-1]):
            return x, hist, "nonfinite"
        if hist[-1] <= tol:
            return x, hist, "ok"
    return x, hist, "not_converged"


class HybridSolver:
    """Static condensation, the non-nested preconditioner and BiCGStab on S lambda = B."""

    def __init__(self, hier, coeffs, opts: OracleOptions | None = None):
        self.hier, self.coeffs = hier, coeffs
        self.opts = opts or OracleOptions()
        self.mesh = mesh = hier.meshes[0]
        system = fem.cell_system(mesh, coeffs.levels[0], coeffs)
        self.A, self.Kdiag, _cc = system
        self.S_K = fem.condense(self.A, self.Kdiag)
        self.S = fem.assemble_trace_operator(mesh, self.S_K)
        self.smoother = LineSmoother(mesh, self.S)
        o = self.opts
        self.mg = PressureMultigrid(hier, coeffs, o.mg_omega, o.mg_npre, o.mg_npost, o.mg_ncoarse,
                                    finest_system=system)
        self.P = prolongation(mesh)
        # Gamma = (H 1) / (P^T S P 1); P 1 = 1, and H 1, S 1 are formed without cancellation
        one = np.ones(mesh.ncell)
        h1 = pressure_operator_times(self.mg.parts0, one)
        self.gamma = h1 / (self.P.T @ fem.trace_row_sums(mesh, self.A))

    # -- coarse solve (Alg. 2 line 6) -------------------------------------------------
    def coarse_solve(self, bbar):
        o = self.opts
        if o.coarse == "vcycle":
            return self.mg.vcycle(bbar)
        tol = 1e-14 if o.coarse == "exact" else 1e-2
        x, _h, _s = bicgstab(lambda y: self.mg.H[0] @ y, bbar, self.mg.vcycle, tol, 500)
        return x

    # -- preconditioners --------------------------------------------------------------
    def two_level(self, r):
        """Algorithm 2 applied to S z = r."""
        o = self.opts
        lam = np.zeros_like(r)                                       # line 1
        lam = self.smoother.smooth(lam, r, o.omega, o.n_pre)         # line 2
        R = r - self.S @ lam                                         # line 3
        b = self.P.T @ R                                             # line 4
        bbar = self.gamma * b                                        # line 5
        dpi = self.coarse_solve(bbar)                                # line 6
        lam = lam + self.P @ dpi                                     # line 7
        return self.smoother.smooth(lam, r, o.omega, o.n_post)       # line 8

    def precond(self, r):
        o = self.opts
        if o.precond == "nonnested":
            return self.two_level(r)
        if o.precond == "linesmooth":
            return self.smoother.smooth(np.zeros_like(r), r, o.omega, o.n_smooth)
        return r.copy()

    # -- whole solve ------------------------------------------------------------------
    def rhs(self, Rub, Rpi):
        return fem.trace_rhs(self.mesh, self.A, Rub, Rpi)

    def solve_trace(self, B, tol, maxit=200):
        return bicgstab(lambda x: self.S @ x, B, self.precond, tol, maxit)

    def solve(self, Rub, Rpi, tol, maxit=200):
        B = self.rhs(Rub, Rpi)
        lam, hist, status = self.solve_trace(B, tol, maxit)
        return lam, hist, status

    def reconstruct(self, lam, Rub, Rpi):
        return fem.reconstruct(self.mesh, self.A, self.Kdiag, lam, Rub, Rpi)
