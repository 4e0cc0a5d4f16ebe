"""Pins of the configuration-1 oracle (approximate Schur complement solver, Sec. 2.3) on CPU:
the sparse 2x2 operator against the dense mixed system, Steps 1-3 with an exact pressure
solve against a dense solve of the lumped system (Eq. 2x2system_approx), and the converged
solution against the hybridised solve (both solve Eq. 2x2system)."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import fem
from oracle.nonnested import HybridSolver
from oracle.schur import MixedSolver, boundary_facets
from paper_2210_11797_gb300 import inputs as I


def _small(kind):
    if kind == "planar":
        return I.planar_helmholtz(n=4, nlev=3, nmg=2, seed=5)
    return I.cubed_sphere(2, 3, seed=6)


@pytest.mark.parametrize("kind", ["planar", "sphere"])
def test_sparse_operator_and_rhs_equal_the_dense_mixed_system(kind):
    w = _small(kind)
    ms = MixedSolver(w.hier, w.coeffs)
    dense, rhs, interior = fem.mixed_system(w.mesh, w.coeffs.levels[0], w.coeffs, w.Rub, w.Rpi)
    keep = np.concatenate([interior, ms.T + np.arange(ms.C)])
    got = ms.Mx.toarray()[np.ix_(keep, keep)]
    np.testing.assert_allclose(got, dense, rtol=1e-13, atol=1e-13 * np.abs(dense).max())
    b = ms.rhs(w.Rub, w.Rpi)
    np.testing.assert_allclose(b[keep], rhs, rtol=1e-13, atol=1e-13 * np.abs(rhs).max())
    # the ground and lid facets decouple: identity rows, no column entries from other rows
    bnd = boundary_facets(w.mesh)
    M = ms.Mx.toarray()
    np.testing.assert_array_equal(M[bnd][:, bnd], np.eye(len(bnd)))
    assert not np.any(np.delete(M, bnd, axis=0)[:, bnd])


@pytest.mark.parametrize("kind", ["planar", "sphere"])
def test_steps_1_to_3_with_an_exact_pressure_solve_invert_the_lumped_system(kind):
    """With H solved exactly, the preconditioner is the inverse of Eq. 2x2system_approx:
    [[Mlump, G], [B, M3^Pi]] with the lumped velocity mass on the interior facets."""
    w = _small(kind)
    ms = MixedSolver(w.hier, w.coeffs)
    T, C = ms.T, ms.C
    interior = ms.interior
    approx = np.zeros((T + C, T + C))
    lump = np.where(interior, 1.0 / np.where(interior, ms.inv_lump, 1.0), 1.0)
    approx[:T, :T] = np.diag(lump)
    G = ms.Gg.toarray()
    G[~interior] = 0.0
    B = ms.Bg.toarray()
    B[:, ~interior] = 0.0
    approx[:T, T:] = G
    approx[T:, :T] = B
    approx[T:, T:] = np.diag(ms.m)
    r = np.random.default_rng(3).standard_normal(T + C)
    r[:T][~interior] = 0.0
    H = ms.mg.H[0].tocsc()
    got = ms.precond(r, pressure_solve=lambda b: spla.spsolve(H, b))
    want = np.linalg.solve(approx, r)
    np.testing.assert_allclose(got, want, rtol=1e-9, atol=1e-11 * np.abs(want).max())


def test_configuration1_solution_equals_the_hybridised_solution():
    w = I.planar_helmholtz(n=8, nlev=4, nmg=2, seed=7)
    ms = MixedSolver(w.hier, w.coeffs)
    u, pi, hist, status = ms.solve(w.Rub, w.Rpi, 1e-12)
    assert status == "ok"
    hs = HybridSolver(w.hier, w.coeffs)
    lam, _h, st = hs.solve(w.Rub, w.Rpi, 1e-12)
    assert st == "ok"
    ub, pih = hs.reconstruct(lam, w.Rub, w.Rpi)
    np.testing.assert_allclose(pi, pih, rtol=1e-8, atol=1e-9 * np.abs(pih).max())
    # the broken velocity of the hybridised solution is continuous and equals s_K(f) u_f
    want = ms.s * u[ms.g]
    np.testing.assert_allclose(ub, want, rtol=1e-8, atol=1e-9 * np.abs(want).max())


@pytest.mark.parametrize("make", [lambda: I.planar_helmholtz(), lambda: I.cubed_sphere(6, 5, nmg=2, seed=4)])
def test_configuration1_converges_like_a_multigrid_solver(make):
    """Sanity of the method as the paper reports it (21 iterations to 1e-12 on C96): a
    handful of iterations per order of magnitude, not the hundreds of a single-level method."""
    w = make()
    ms = MixedSolver(w.hier, w.coeffs)
    _u, _pi, hist, status = ms.solve(w.Rub, w.Rpi, 1e-10, maxit=100)
    assert status == "ok" and len(hist) - 1 <= 40
