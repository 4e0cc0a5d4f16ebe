"""Trace-space line smoother (Algorithm 1) and the Thomas algorithm (FP64).

Oracle (test infrastructure only; see oracle/__init__.py).

Paper passages: Sec. 2.5 "Trace space smoother" - the splitting lambda = (lambda^h,
lambda^z), the block structure of S with S^zz = blockdiag(S^zz_1 .. S^zz_ncol) of
per-column tridiagonals (Eq. banded_system), and Algorithm 1.

Reading: Algorithm 1 prints the updates as lambda <- lambda - omega * delta with
R = B - S lambda; that sign makes the iteration diverge, so the update is taken as
lambda <- lambda + omega * delta (standard damped block Jacobi).
"""
from __future__ import annotations

import numpy as np


def thomas(sub: np.ndarray, diag: np.ndarray, sup: np.ndarray, rhs: np.ndarray) -> np.ndarray:
    """Solve tridiagonal systems without pivoting, batched over the leading axis.
    Row i reads sub[:, i] x[i-1] + diag[:, i] x[i] + sup[:, i] x[i+1] = rhs[:, i]
    (sub[:, 0] and sup[:, -1] are ignored)."""
    n = diag.shape[1]
    c = np.zeros_like(diag)
    d = np.zeros_like(rhs)
    c[:, 0] = sup[:, 0] / diag[:, 0]
    d[:, 0] = rhs[:, 0] / diag[:, 0]
    for i in range(1, n):
        den = diag[:, i] - sub[:, i] * c[:, i - 1]
        c[:, i] = sup[:, i] / den if i < n - 1 else 0.0
        d[:, i] = (rhs[:, i] - sub[:, i] * d[:, i - 1]) / den
    x = np.zeros_like(rhs)
    x[:, n - 1] = d[:, n - 1]
    for i in range(n - 2, -1, -1):
        x[:, i] = d[:, i] - c[:, i] * x[:, i + 1]
    return x


def column_tridiagonals(mesh, S):
    """Extract S^zz_j for every column j: (sub, diag, sup), each [ncol, L+1]."""
    L1 = mesh.nlev + 1
    ids = mesh.n_trace_h + np.arange(mesh.ncol)[:, None] * L1 + np.arange(L1)[None, :]
    diag = np.asarray(S[ids.ravel(), ids.ravel()]).reshape(ids.shape)
    sub = np.zeros_like(diag)
    sup = np.zeros_like(diag)
    sub[:, 1:] = np.asarray(S[ids[:, 1:].ravel(), ids[:, :-1].ravel()]).reshape(mesh.ncol, L1 - 1)
    sup[:, :-1] = np.asarray(S[ids[:, :-1].ravel(), ids[:, 1:].ravel()]).reshape(mesh.ncol, L1 - 1)
    return sub, diag, sup


class LineSmoother:
    """Algorithm 1: n sweeps of block Jacobi on lambda^z (one tridiagonal per column) and
    point Jacobi on lambda^h, relaxation omega."""

    def __init__(self, mesh, S):
        self.mesh = mesh
        self.S = S
        self.sub, self.diag, self.sup = column_tridiagonals(mesh, S)
        self.diag_hh = S.diagonal()[: mesh.n_trace_h].copy()

    def sweep(self, lam: np.ndarray, B: np.ndarray, omega: float) -> np.ndarray:
        NH = self.mesh.n_trace_h
        R = B - self.S @ lam                                   # line 2
        Rz = R[NH:].reshape(self.mesh.ncol, self.mesh.nlev + 1)  # line 3
        dz = thomas(self.sub, self.diag, self.sup, Rz)         # line 5
        out = lam.copy()
        out[NH:] += omega * dz.ravel()                         # line 6 (+omega reading)
        out[:NH] += omega * R[:NH] / self.diag_hh              # line 8 (+omega reading)
        return out

    def smooth(self, lam: np.ndarray, B: np.ndarray, omega: float, nsweeps: int) -> np.ndarray:
        for _ in range(nsweeps):
            lam = self.sweep(lam, B, omega)
        return lam
