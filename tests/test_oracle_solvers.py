"""Pins of the oracle's smoother, pressure multigrid, coarse scaling and Krylov loop (CPU).

Closed forms (the 7-point finite-volume Helmholtz stencil, Gamma from Sherman-Morrison),
dense direct solves of the extracted column systems, and the convergence behaviour the
paper reports (Sec. 3.3, Appendix B) pin each step.
"""
import json
import os

import numpy as np
import pytest

from oracle import fem, nonnested, pressure_mg, smoother
from oracle.nonnested import HybridSolver, OracleOptions, bicgstab
from paper_2210_11797_gb300 import inputs as I

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_parameters.json")))


@pytest.fixture(scope="module")
def config1():
    w = I.planar_helmholtz()
    return w, HybridSolver(w.hier, w.coeffs)


def test_thomas_matches_dense_solve():
    rng = np.random.default_rng(1)
    n, m = 7, 31
    sub, sup = rng.standard_normal((n, m)), rng.standard_normal((n, m))
    diag = 4.0 + np.abs(rng.standard_normal((n, m)))
    rhs = rng.standard_normal((n, m))
    x = smoother.thomas(sub, diag, sup, rhs)
    for j in range(n):
        T = np.diag(diag[j]) + np.diag(sub[j, 1:], -1) + np.diag(sup[j, :-1], 1)
        np.testing.assert_allclose(x[j], np.linalg.solve(T, rhs[j]), rtol=1e-13, atol=1e-13)


def test_column_blocks_of_S_are_tridiagonal_and_match_dense(config1):
    """S^zz is block-diagonal with one tridiagonal per column (Sec. 2.5), and the Thomas
    solve of each extracted block equals a dense solve of the dense submatrix."""
    w, s = config1
    mesh = w.mesh
    S = s.S.toarray()
    NH, L1 = mesh.n_trace_h, mesh.nlev + 1
    for j in (0, 5, mesh.ncol - 1):
        ids = NH + j * L1 + np.arange(L1)
        blk = S[np.ix_(ids, ids)]
        assert np.abs(np.triu(blk, 2)).max() == 0.0 and np.abs(np.tril(blk, -2)).max() == 0.0
        r = np.random.default_rng(j).standard_normal(L1)
        sub, diag, sup = (a[j:j + 1] for a in (s.smoother.sub, s.smoother.diag, s.smoother.sup))
        x = smoother.thomas(sub, diag, sup, r[None])[0]
        np.testing.assert_allclose(x, np.linalg.solve(blk, r), rtol=1e-12)
    # other columns' z blocks do not couple
    z0 = NH + np.arange(L1)
    z1 = NH + L1 + np.arange(L1)
    assert np.abs(S[np.ix_(z0, z1)]).max() == 0.0


def test_line_sweep_formula_against_dense_algebra(config1):
    """One sweep of Algorithm 1 equals lambda + omega D^-1 (B - S lambda) with D the block
    diagonal [diag(S^hh), S^zz] formed densely (update sign +omega: Algorithm 1 prints a
    minus sign with R = B - S lambda, which diverges)."""
    w, s = config1
    mesh = w.mesh
    S = s.S.toarray()
    NH = mesh.n_trace_h
    D = np.zeros_like(S)
    D[np.arange(NH), np.arange(NH)] = np.diag(S)[:NH]
    L1 = mesh.nlev + 1
    for j in range(mesh.ncol):
        ids = NH + j * L1 + np.arange(L1)
        D[np.ix_(ids, ids)] = S[np.ix_(ids, ids)]
    rng = np.random.default_rng(3)
    lam, B = rng.standard_normal(mesh.n_trace), rng.standard_normal(mesh.n_trace)
    got = s.smoother.sweep(lam, B, 0.6)
    want = lam + 0.6 * np.linalg.solve(D, B - S @ lam)
    np.testing.assert_allclose(got, want, rtol=1e-11, atol=1e-11 * np.abs(want).max())


def test_pressure_operator_is_finite_volume_helmholtz(config1):
    """On boxes with the Helmholtz preset, H = sigma |K| + sum over interior faces of
    A_f / d_f on the diagonal and -A_f / d_f off it (7-point stencil)."""
    w, s = config1
    mesh = w.mesh
    H = s.mg.H[0].toarray()
    hx = hy = 1.0 / 16
    hz = 0.1 / 8
    L, n = mesh.nlev, 16
    ch, cz = hy * hz / hx, hx * hy / hz
    sig = w.coeffs.sigma * hx * hy * hz
    want = np.zeros_like(H)
    for c in range(mesh.ncol):
        i, j = c % n, c // n
        nbrs = [((i + 1) % n) + j * n, ((i - 1) % n) + j * n, i + ((j + 1) % n) * n, i + ((j - 1) % n) * n]
        for k in range(L):
            K = c * L + k
            want[K, K] += sig + 4 * ch
            for nb in nbrs:
                want[K, nb * L + k] -= ch
            if k > 0:
                want[K, K] += cz
                want[K, K - 1] -= cz
            if k < L - 1:
                want[K, K] += cz
                want[K, K + 1] -= cz
    np.testing.assert_allclose(H, want, rtol=0, atol=1e-12 * np.abs(want).max())


def test_gamma_closed_form_config1(config1):
    """Eq. scaling_matrix with H 1 = sigma |K| (G annihilates constants) and S 1 from the
    Sherman-Morrison S_K of each cell: per direction M^-1 1 = 6 A_d/h_d on both faces."""
    w, s = config1
    hx = hy = 1.0 / 16
    hz = 0.1 / 8
    L = w.mesh.nlev
    m = w.coeffs.sigma * hx * hy * hz
    minv1 = 6 * np.array([hx * hz / hy, hy * hz / hx, hx * hz / hy, hy * hz / hx, hx * hy / hz, hx * hy / hz])
    sk1 = minv1 * m / (m + minv1.sum())            # S_K 1 per local face
    # P^T S 1 per cell: an interior face has weight 1/2 and collects S_K 1 from both (equal)
    # cells; a ground or lid face has weight 1 and one cell. Either way each face adds sk1.
    want = np.full(L, m / sk1.sum())
    np.testing.assert_allclose(s.gamma.reshape(-1, L), np.broadcast_to(want, (w.mesh.ncol, L)), rtol=1e-12)


def test_restriction_is_transpose_of_prolongation(config1):
    w, s = config1
    mg = s.mg
    rng = np.random.default_rng(4)
    xf = rng.standard_normal(w.hier.meshes[0].ncell)
    xc = rng.standard_normal(w.hier.meshes[1].ncell)
    assert mg.restrict(0, xf) @ xc == pytest.approx(xf @ mg.prolong(0, xc), rel=1e-13)
    P = nonnested.prolongation(w.mesh)
    np.testing.assert_allclose(P @ np.ones(w.mesh.ncell), 1.0)   # averages of constants


def test_block_jacobi_sweep_solves_columns_exactly(config1):
    """x + omega H_z^-1 (b - H x) with H_z the dense column blocks of H."""
    w, s = config1
    mesh = w.mesh
    H = s.mg.H[0].toarray()
    L = mesh.nlev
    rng = np.random.default_rng(6)
    x, b = rng.standard_normal(mesh.ncell), rng.standard_normal(mesh.ncell)
    got = s.mg.block_jacobi(0, x, b)
    r = b - H @ x
    want = x.copy()
    for c in range(mesh.ncol):
        ids = c * L + np.arange(L)
        want[ids] += 0.9 * np.linalg.solve(H[np.ix_(ids, ids)], r[ids])
    np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-12 * np.abs(want).max())


def test_vcycle_contracts(config1):
    """The pressure V-cycle as a stationary iteration contracts the residual (<= 0.2 a cycle;
    the 8x8 coarsest level gets three block-Jacobi sweeps, not an exact solve)."""
    w, s = config1
    H = s.mg.H[0]
    b = np.random.default_rng(7).standard_normal(H.shape[0])
    x = np.zeros_like(b)
    prev = np.linalg.norm(b)
    for _ in range(4):
        x = x + s.mg.vcycle(b - H @ x)
        cur = np.linalg.norm(b - H @ x)
        assert cur < 0.2 * prev
        prev = cur


def test_bicgstab_exact_preconditioner_and_plain():
    rng = np.random.default_rng(8)
    n = 40
    Q = rng.standard_normal((n, n))
    A = Q @ Q.T + n * np.eye(n) + 0.3 * rng.standard_normal((n, n))
    b = rng.standard_normal(n)
    Ainv = np.linalg.inv(A)
    x, hist, st = bicgstab(lambda v: A @ v, b, lambda v: Ainv @ v, 1e-12, 10)
    assert st == "ok" and len(hist) == 2
    x, hist, st = bicgstab(lambda v: A @ v, b, lambda v: v, 1e-12, 200)
    assert st == "ok"
    np.testing.assert_allclose(x, np.linalg.solve(A, b), rtol=1e-9)


def test_config3c_converges_about_one_order_per_iteration(config1):
    """Sec. 3.3: textbook multigrid behaviour, ~1 order of residual reduction per iteration
    (16 iterations to 1e-12 on C96)."""
    w, s = config1
    s.opts = OracleOptions()
    lam, hist, st = s.solve(w.Rub, w.Rpi, 1e-10)
    assert st == "ok"
    its = len(hist) - 1
    assert its <= 12
    assert hist[-1] ** (1.0 / its) < 0.1 ** 0.8
    # converged answer solves the trace system
    B = s.rhs(w.Rub, w.Rpi)
    lam_direct = np.linalg.solve(s.S.toarray(), B)
    assert np.linalg.norm(lam - lam_direct) / np.linalg.norm(lam_direct) < 1e-8


def test_single_level_needs_many_more_iterations(config1):
    """Sec. 3.3: the line smoother alone (configuration 2) converges far more slowly."""
    w, s = config1
    B = s.rhs(w.Rub, w.Rpi)
    s.opts = OracleOptions()
    _l, h3c, _ = s.solve_trace(B, 1e-8)
    s.opts = OracleOptions(precond="linesmooth", n_smooth=1)
    _l, h2, st = s.solve_trace(B, 1e-8, 2000)
    s.opts = OracleOptions()
    assert len(h2) - 1 >= 3 * (len(h3c) - 1)


def test_exact_coarse_solve_barely_helps(config1):
    """Sec. 3.3: the convergence rate is virtually independent of the coarse solve (3a vs 3c)."""
    w, s = config1
    B = s.rhs(w.Rub, w.Rpi)
    s.opts = OracleOptions(coarse="exact")
    _l, h3a, _ = s.solve_trace(B, 1e-8)
    s.opts = OracleOptions()
    _l, h3c, _ = s.solve_trace(B, 1e-8)
    assert abs((len(h3a) - 1) - (len(h3c) - 1)) <= 2


def test_omega_above_point_eight_breaks_convergence(config1):
    """Appendix B: with two post-smoothing steps the method fails for omega > 0.8 while
    omega <= 0.7 is fine."""
    w, s = config1
    B = s.rhs(w.Rub, w.Rpi)
    s.opts = OracleOptions(omega=0.7)
    _l, hok, st_ok = s.solve_trace(B, 1e-8, 60)
    s.opts = OracleOptions(omega=1.2)
    _l, hbad, st_bad = s.solve_trace(B, 1e-8, 60)
    s.opts = OracleOptions()
    assert st_ok == "ok"
    assert st_bad != "ok" or len(hbad) > 3 * len(hok)


def test_cubed_sphere_physical_converges():
    """C12 x 30 stretched levels, isothermal background, Courant 8, 3 MG levels."""
    w = I.cubed_sphere(12, 30)
    s = HybridSolver(w.hier, w.coeffs)
    lam, hist, st = s.solve(w.Rub, w.Rpi, 1e-6)
    assert st == "ok" and len(hist) - 1 <= 15
    B = s.rhs(w.Rub, w.Rpi)
    assert np.linalg.norm(B - s.S @ lam) / np.linalg.norm(B) <= 1.01e-6


def test_paper_parameters_are_the_oracle_defaults():
    o = OracleOptions()
    assert o.omega == GOLDEN["omega_trace_smoother"]["value"]
    assert o.mg_omega == GOLDEN["omega_pressure"]["value"]
    assert (o.n_pre, o.n_post) == (GOLDEN["n_presmooth"]["value"], GOLDEN["n_postsmooth"]["value"])
    assert I.mg_levels_for(96) == GOLDEN["pressure_mg_levels"]["value"]
    assert len(fem.GAUSS_X) == GOLDEN["gauss_points_per_direction_p0"]["value"]
    assert 6 * 96 * 96 * 30 == GOLDEN["c96_cells"]["value"]


def test_pressure_operator_annihilates_constants_up_to_mass_term():
    """G 1 = 0 exactly on every interior facet (single-valued theta), so H 1 = M3^Pi 1 (the
    numerator of Gamma), while the plain row sums of H agree only up to their cancellation
    error. Ground and lid facets carry no velocity dof (inverse lumped mass 0)."""
    w = I.cubed_sphere(6, 8, nmg=1)
    s = HybridSolver(w.hier, w.coeffs)
    Bg, inv_lump, Gg, m = s.mg.parts0
    one = np.ones(w.mesh.ncell)
    assert np.all(inv_lump * (Gg @ one) == 0.0)
    assert np.array_equal(pressure_mg.pressure_operator_times(s.mg.parts0, one), m)
    H = s.mg.H[0]
    assert np.all(np.abs(H @ one - m) <= 1e-14 * (abs(H) @ one))


def test_vcycle_from_the_exact_solution_stays_there(config1):
    """Started from x0 = H^-1 b every residual is zero, so the V-cycle returns x0 (this pins
    the initial-guess form used by the learned coarse solve)."""
    import scipy.sparse.linalg as spla
    w, s = config1
    H = s.mg.H[0].tocsc()
    b = np.random.default_rng(9).standard_normal(H.shape[0])
    x0 = spla.spsolve(H, b)
    np.testing.assert_allclose(s.mg.vcycle(b, x0=x0), x0, rtol=1e-10, atol=1e-12 * np.abs(x0).max())
    # and from a zero guess it is the plain V-cycle
    np.testing.assert_array_equal(s.mg.vcycle(b, x0=np.zeros_like(b)), s.mg.vcycle(b))
