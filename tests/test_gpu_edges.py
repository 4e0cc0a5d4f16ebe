"""Edge cases of the CUDA path against the FP64 oracle: ragged sizes (column counts and level
counts that fill no launch shape evenly), a single layer, a single multigrid level, an odd
cubed-sphere panel, a non-isothermal, horizontally varying background, a rotating planet
(Coriolis: non-symmetric cell matrices), a zero right-hand
side, and the largest workload (C192 x 30, sampled rows). Tolerances as in test_gpu_parity:
whole solves converged to 1e-12 on both sides agree
to a relative 2-norm difference below 1e-9."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle import fem
from oracle.nonnested import HybridSolver
from paper_2210_11797_gb300 import inputs as I


def _cuda(a):
    return torch.as_tensor(np.ascontiguousarray(a, np.float64)).cuda()


def _np(t):
    return t.detach().cpu().numpy()


CASES = {
    "planar6x6x7": lambda: I.planar_helmholtz(n=6, nlev=7, nmg=2, seed=1),
    "planar8x8x1": lambda: I.planar_helmholtz(n=8, nlev=1, nmg=2, seed=2),
    "planar8x8x5_one_mg_level": lambda: I.planar_helmholtz(n=8, nlev=5, nmg=1, seed=3),
    "sphereC3L4": lambda: I.cubed_sphere(3, 4, seed=4),
    "sphereC10L9": lambda: I.cubed_sphere(10, 9, seed=5),
    # a general background: constant N over a latitude-dependent surface temperature
    "sphereC8L12_stratified": lambda: I.cubed_sphere(8, 12, seed=6, background="stratified"),
    # Coriolis (10x the Earth's rate): non-symmetric cell matrices and trace operator
    "sphereC8L12_rotating": lambda: I.cubed_sphere(8, 12, seed=7, omega=10 * I.EARTH_OMEGA),
}


@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("krylov", ["bicgstab", "fgmres"])
def test_small_and_ragged_solves_match_oracle(name, krylov):
    from paper_2210_11797_gb300.hmg import Solver
    w = CASES[name]()
    ora = HybridSolver(w.hier, w.coeffs)
    gpu = Solver(w.hier, w.coeffs, tol=1e-12, max_iter=400, krylov=krylov)
    gpu.autotune()
    lam, st = gpu.solve(_cuda(w.Rub.ravel()), _cuda(w.Rpi))
    assert st["status"] == "ok" and st["true_rel_residual"] < 1e-11
    ref, _hist, status = ora.solve(w.Rub, w.Rpi, 1e-12, maxit=400)
    assert status == "ok"
    assert np.linalg.norm(_np(lam) - ref) / np.linalg.norm(ref) < 1e-9
    # the host-buffer path gives the same lambda
    lam_h, st_h = gpu.solve_host(w.Rub.ravel(), w.Rpi)
    np.testing.assert_array_equal(lam_h, _np(lam))
    # and the recovered (u, Pi) satisfies the cell equations as the oracle's does
    ub, pi = gpu.reconstruct(lam, _cuda(w.Rub.ravel()), _cuda(w.Rpi))
    ub_o, pi_o = ora.reconstruct(ref, w.Rub, w.Rpi)
    assert np.linalg.norm(_np(pi) - pi_o.ravel()) <= 1e-8 * np.linalg.norm(pi_o)
    assert np.linalg.norm(_np(ub) - ub_o.ravel()) <= 1e-8 * np.linalg.norm(ub_o)
    gpu.close()


@pytest.mark.parametrize("krylov", ["bicgstab", "fgmres"])
@pytest.mark.parametrize("graph", [0, 1])
def test_zero_right_hand_side(krylov, graph):
    from paper_2210_11797_gb300.hmg import Solver
    w = I.planar_helmholtz()
    gpu = Solver(w.hier, w.coeffs, tol=1e-10, krylov=krylov, graph=graph)
    lam = _cuda(np.full(gpu.ntrace, 7.0))       # overwritten: the iteration starts from zero
    lam, st = gpu.solve(_cuda(np.zeros(6 * gpu.ncell)), _cuda(np.zeros(gpu.ncell)), lam)
    assert st["status"] == "ok" and st["iterations"] == 0
    assert not np.any(_np(lam))
    gpu.close()


def test_tolerance_one_and_zero_iterations():
    """tol >= 1 is met by lambda = 0 before any iteration; max_iter = 0 below it is reported."""
    from paper_2210_11797_gb300.hmg import Solver
    w = I.planar_helmholtz()
    gpu = Solver(w.hier, w.coeffs, tol=1.0)
    lam, st = gpu.solve(_cuda(w.Rub.ravel()), _cuda(w.Rpi))
    assert st["status"] == "ok" and st["iterations"] == 0 and not np.any(_np(lam))
    gpu.set_options(tol=1e-6, max_iter=0)
    _lam, st = gpu.solve(_cuda(w.Rub.ravel()), _cuda(w.Rpi), check=False)
    assert st["status"] == "not_converged" and st["iterations"] == 0
    gpu.close()


def test_largest_workload_c192_sampled_rows():
    """C192 x 30 (6.6M cells, 20.1M trace unknowns): sampled rows of S x against the
    oracle's cell matrices of the cells touching them, and the solve to 1e-6."""
    from paper_2210_11797_gb300.hmg import Solver
    w = I.cubed_sphere(192, 30)
    gpu = Solver(w.hier, w.coeffs, tol=1e-6)
    mesh, bg, co = w.mesh, w.coeffs.levels[0], w.coeffs
    rng = np.random.default_rng(11)
    L = mesh.nlev
    rows = np.unique(np.concatenate([rng.integers(0, mesh.n_trace_h, 200),
                                     rng.integers(mesh.n_trace_h, mesh.n_trace, 200),
                                     [0, mesh.n_trace_h - 1, mesh.n_trace_h, mesh.n_trace - 1]]))
    cells = []
    for r in rows:
        if r < mesh.n_trace_h:
            e, k = divmod(int(r), L)
            cells += [mesh.edge_cols[e, 0] * L + k, mesh.edge_cols[e, 1] * L + k]
        else:
            c, k = divmod(int(r) - mesh.n_trace_h, L + 1)
            if k < L:
                cells.append(c * L + k)
            if k > 0:
                cells.append(c * L + k - 1)
    cells = np.unique(cells)
    A, Kd, _cc = fem.cell_system(mesh, bg, co, cells=cells)
    SK = fem.condense(A, Kd)
    g = fem.trace_dof_ids(mesh, cells)
    x = rng.standard_normal(gpu.ntrace)
    y = _np(gpu.apply_trace(_cuda(x)))
    want, scale = np.zeros(len(rows)), np.zeros(len(rows))
    pos = {int(r): i for i, r in enumerate(rows)}
    for ci in range(len(cells)):
        for i in range(6):
            j = pos.get(int(g[ci, i]))
            if j is not None:
                want[j] += SK[ci, i] @ x[g[ci]]
                scale[j] += np.abs(SK[ci, i]) @ np.abs(x[g[ci]])
    assert np.all(np.abs(y[rows] - want) <= 1e-12 * scale)
    _lam, st = gpu.solve(_cuda(w.Rub.ravel()), _cuda(w.Rpi))
    assert st["status"] == "ok" and st["true_rel_residual"] <= 1.05e-6
    gpu.close()


@pytest.mark.parametrize("krylov", ["bicgstab", "fgmres"])
def test_warm_start_resumes_a_solve(krylov):
    """warm_start = 1 starts from the lambda passed in: resuming from a solution converged to
    1e-4 reaches 1e-10 in fewer iterations than from zero, with the same answer; the oracle's
    BiCGStab from the same start agrees; starting from the exact answer needs no iteration."""
    from paper_2210_11797_gb300.hmg import Solver
    w = I.cubed_sphere(6, 5, courant=8.0, nmg=2, seed=4)
    gpu = Solver(w.hier, w.coeffs, tol=1e-4, krylov=krylov)
    Rub, Rpi = _cuda(w.Rub.ravel()), _cuda(w.Rpi)
    lam0, _st = gpu.solve(Rub, Rpi)
    gpu.set_options(tol=1e-10)
    cold, st_cold = gpu.solve(Rub, Rpi)
    gpu.set_options(warm_start=1)
    warm = lam0.clone()
    warm, st_warm = gpu.solve(Rub, Rpi, warm)
    assert st_warm["status"] == "ok" and st_warm["iterations"] < st_cold["iterations"]
    assert st_warm["history"][0] < 1e-3                    # ||B - S lambda_0|| / ||B||
    assert np.linalg.norm(_np(warm) - _np(cold)) / np.linalg.norm(_np(cold)) < 1e-8
    if krylov == "bicgstab":
        ora = HybridSolver(w.hier, w.coeffs)
        from oracle.nonnested import bicgstab
        B = ora.rhs(w.Rub, w.Rpi)
        ref, hist, status = bicgstab(lambda v: ora.S @ v, B, ora.precond, 1e-10, 200, x0=_np(lam0))
        assert status == "ok" and abs(st_warm["iterations"] - (len(hist) - 1)) <= 1
        assert np.linalg.norm(_np(warm) - ref) / np.linalg.norm(ref) < 1e-9
    again, st_again = gpu.solve(Rub, Rpi, warm.clone())
    assert st_again["iterations"] <= 1
    gpu.close()


def test_async_stats_enqueue_the_solve_and_report_later():
    """async_stats = 1: hmg_solve only enqueues the graph-launched solve; hmg_solve_stats_get
    then gives the same stats as a synchronous solve (same lambda, iterations and history,
    bit for bit); nothing pending is NOT_READY; the host-buffer and host-driven solves stay
    synchronous."""
    from paper_2210_11797_gb300.hmg import HmgError, Solver
    w = I.cubed_sphere(12, 10, seed=3)
    gpu = Solver(w.hier, w.coeffs, tol=1e-8)
    Rub, Rpi = _cuda(w.Rub.ravel()), _cuda(w.Rpi)
    lam_s, st_s = gpu.solve(Rub, Rpi)
    gpu.set_options(async_stats=1)
    lam_a = torch.empty_like(lam_s)
    lam_a, st = gpu.solve(Rub, Rpi, lam_a)
    assert st is None
    st_a = gpu.solve_stats()
    assert st_a["status"] == "ok" and st_a["iterations"] == st_s["iterations"]
    np.testing.assert_array_equal(st_a["history"], st_s["history"])
    assert st_a["true_rel_residual"] == st_s["true_rel_residual"] and st_a["solve_ms"] > 0
    np.testing.assert_array_equal(_np(lam_a), _np(lam_s))
    with pytest.raises(HmgError):
        gpu.solve_stats()
    # two enqueued solves: the stats are the second's
    gpu.set_options(tol=1e-4)
    lam_a, st = gpu.solve(Rub, Rpi, lam_a)
    gpu.set_options(tol=1e-8)
    lam_a, st = gpu.solve(Rub, Rpi, lam_a)
    assert st is None and gpu.solve_stats()["iterations"] == st_s["iterations"]
    # host buffers and the host-driven loop ignore async_stats
    lam_h, st_h = gpu.solve_host(w.Rub.ravel(), w.Rpi)
    assert st_h["iterations"] == st_s["iterations"]
    gpu.set_options(graph=0)
    _l, st_g = gpu.solve(Rub, Rpi)
    assert st_g is not None and st_g["iterations"] == st_s["iterations"]
    gpu.close()


def test_autotune_after_a_captured_solve_changes_nothing_but_speed():
    """Block launch shapes change no arithmetic: a solve captured before hmg_autotune and the
    solve re-captured after it (autotune drops the old graph) give the same lambda bit for bit,
    unless the autotuner took the warp-per-column smoother (columns -1) on some level, whose scan
    changes the rounding order of the column solves only; resetting the shapes restores the
    first lambda bit for bit."""
    from paper_2210_11797_gb300.hmg import Solver
    w = I.cubed_sphere(16, 12, seed=12)
    gpu = Solver(w.hier, w.coeffs, tol=1e-8)
    Rub, Rpi = _cuda(w.Rub.ravel()), _cuda(w.Rpi)
    lam0, st0 = gpu.solve(Rub, Rpi)
    before = gpu.launch_shapes()
    gpu.autotune()
    lam1, st1 = gpu.solve(Rub, Rpi, torch.empty_like(lam0))
    assert st1["iterations"] == st0["iterations"]
    sw, mg = gpu.launch_shapes()
    assert sw[0] > 0 and all(c > 0 or c == -1 for c, _t in mg)   # tuned shapes are recorded
    if all(c > 0 for c, _t in mg):
        np.testing.assert_array_equal(_np(lam1), _np(lam0))
    else:
        assert np.linalg.norm(_np(lam1) - _np(lam0)) <= 1e-10 * np.linalg.norm(_np(lam0))
    gpu.set_launch_shapes(*before)                          # and can be reset
    lam2, _st = gpu.solve(Rub, Rpi, torch.empty_like(lam0))
    np.testing.assert_array_equal(_np(lam2), _np(lam0))
    gpu.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_tuned_shapes_carry_over_to_a_context_of_the_same_mesh(precision):
    """hmg_get_launch_shapes reports the shapes of the kernels the preconditioner runs (the FP32
    kernels' under precision mixed): applied to a second context of the same mesh and
    precision, they make the same launches, so its solve equals the tuned context's bit for bit."""
    from paper_2210_11797_gb300.hmg import Solver
    w = I.cubed_sphere(16, 12, seed=13)
    a = Solver(w.hier, w.coeffs, tol=1e-8, precision=precision)
    b = Solver(w.hier, w.coeffs, tol=1e-8, precision=precision)
    try:
        a.autotune()
        shapes = a.launch_shapes()
        b.set_launch_shapes(*shapes)
        assert b.launch_shapes() == shapes
        Rub, Rpi = _cuda(w.Rub.ravel()), _cuda(w.Rpi)
        lam_a, st_a = a.solve(Rub, Rpi)
        lam_b, st_b = b.solve(Rub, Rpi)
        assert st_a["status"] == st_b["status"] == "ok" and st_a["iterations"] == st_b["iterations"]
        np.testing.assert_array_equal(_np(lam_a), _np(lam_b))
    finally:
        a.close()
        b.close()


def test_tallest_columns_solve_and_one_more_layer_is_rejected():
    """The layer limit (2045: one column's three Thomas arrays fill a block's 48 KB of shared
    memory): a 4 x 4 x 2045 Helmholtz box solves (one column per block in the sweep and the
    smoother; the oracle's S certifies the residual), and 2046 layers are refused before
    anything runs on the device."""
    from paper_2210_11797_gb300.hmg import HmgError, Solver
    w = I.planar_helmholtz(n=4, nlev=2045, top=100.0, nmg=2, seed=9, tol=1e-8)
    gpu = Solver(w.hier, w.coeffs, tol=1e-8, max_iter=400)
    lam, st = gpu.solve(_cuda(w.Rub.ravel()), _cuda(w.Rpi))
    assert st["status"] == "ok" and st["true_rel_residual"] <= 1.05e-8
    ora = HybridSolver(w.hier, w.coeffs)
    B = ora.rhs(w.Rub, w.Rpi)
    assert np.linalg.norm(B - ora.S @ _np(lam)) / np.linalg.norm(B) <= 1.05e-8
    gpu.close()
    h = I.planar_hierarchy(4, 2046, 1.0, I.uniform_levels(2046, 100.0), 1)
    with pytest.raises(HmgError) as e:
        Solver(h, I.Coefficients([I.unit_background(h.meshes[0])], preset=1, sigma=1.0))
    assert e.value.status == 1
