"""The coarse levels of the pressure V-cycle (Sec. 2.3) as one cooperative launch (mg_fused = 1)
against one launch per smoothing sweep, restriction and injection (mg_fused = 0), and the
restriction / injection run inside the neighbouring sweep on small levels (mg_fuse_cells)
against separate kernels. All forms run the same arithmetic in the same order, so their
outputs agree bit for bit: the V-cycle in FP64 and FP32, the non-nested preconditioner, whole
solves (with and without the CUDA graph), and the mixed system with the Schur
preconditioner. The V-cycle is also checked against the oracle's."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle.nonnested import HybridSolver
from paper_2210_11797_gb300 import inputs as I


def _cuda(a):
    return torch.as_tensor(np.ascontiguousarray(a, np.float64)).cuda()


def _np(t):
    return t.detach().cpu().numpy()


CASES = {
    # 2 multigrid levels: the cooperative launch runs the coarsest sweeps alone
    "planar16_nmg2": lambda: I.planar_helmholtz(),
    "planar32x32x7_nmg4": lambda: I.planar_helmholtz(n=32, nlev=7, nmg=4, seed=2),
    "sphereC16L9": lambda: I.cubed_sphere(16, 9, seed=5),
    "sphereC24L30": lambda: I.cubed_sphere(24, 30, seed=6),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_fused_vcycle_is_bitwise_the_per_launch_vcycle(name):
    from paper_2210_11797_gb300.hmg import Solver
    w = CASES[name]()
    gpu = Solver(w.hier, w.coeffs, tol=1e-10, mg_fused=0)
    rng = np.random.default_rng(3)
    b = _cuda(rng.standard_normal(gpu.ncell))
    r = _cuda(rng.standard_normal(gpu.ntrace))
    ref_v, ref_z = _np(gpu.vcycle(b)), _np(gpu.precond(r))
    gpu.set_options(mg_fused=1)
    np.testing.assert_array_equal(_np(gpu.vcycle(b)), ref_v)
    np.testing.assert_array_equal(_np(gpu.precond(r)), ref_z)
    # and the V-cycle is the oracle's
    ora = HybridSolver(w.hier, w.coeffs)
    want = ora.mg.vcycle(_np(b))
    assert np.linalg.norm(ref_v - want) <= 1e-12 * np.linalg.norm(want)
    gpu.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("graph", [0, 1])
def test_fused_solve_is_bitwise_the_per_launch_solve(precision, graph):
    from paper_2210_11797_gb300.hmg import Solver
    w = I.cubed_sphere(24, 30, seed=8)
    Rub, Rpi = _cuda(w.Rub.ravel()), _cuda(w.Rpi)
    out = {}
    for fused in (0, 1):
        gpu = Solver(w.hier, w.coeffs, tol=1e-8, precision=precision, graph=graph, mg_fused=fused)
        lam, st = gpu.solve(Rub, Rpi)
        assert st["status"] == "ok"
        out[fused] = (_np(lam), st["iterations"], st["history"])
        gpu.close()
    np.testing.assert_array_equal(out[1][0], out[0][0])
    assert out[1][1] == out[0][1]
    np.testing.assert_array_equal(out[1][2], out[0][2])


def test_fused_schur_preconditioner_matches():
    """The mixed (u, Pi) system's approximate Schur preconditioner runs the same V-cycle."""
    from paper_2210_11797_gb300.hmg import Solver
    w = I.cubed_sphere(12, 10, seed=9)
    res = {}
    for fused in (0, 1):
        gpu = Solver(w.hier, w.coeffs, tol=1e-8, precond="schur", mg_fused=fused)
        r = _cuda(np.random.default_rng(4).standard_normal(gpu.ntrace + gpu.ncell))
        res[fused] = _np(gpu.precond(r))
        gpu.close()
    np.testing.assert_array_equal(res[1], res[0])


def test_fused_vcycle_with_tuned_launch_shapes():
    """Autotuned smoother shapes (columns per block) change nothing in the results."""
    from paper_2210_11797_gb300.hmg import Solver
    w = I.cubed_sphere(24, 12, seed=10, nmg=4)
    gpu = Solver(w.hier, w.coeffs, tol=1e-8, mg_fused=0, mg_twisted=0)
    b = _cuda(np.random.default_rng(5).standard_normal(gpu.ncell))
    ref = _np(gpu.vcycle(b))
    gpu.autotune()
    gpu.set_options(mg_fused=1)
    np.testing.assert_array_equal(_np(gpu.vcycle(b)), ref)
    gpu.close()


@pytest.mark.parametrize("name", sorted(CASES))
def test_restriction_and_injection_inside_the_sweeps_are_bitwise_the_separate_kernels(name):
    from paper_2210_11797_gb300.hmg import Solver
    w = CASES[name]()
    gpu = Solver(w.hier, w.coeffs, tol=1e-10, mg_fuse_cells=0)   # separate kernels everywhere
    rng = np.random.default_rng(6)
    b = _cuda(rng.standard_normal(gpu.ncell))
    r = _cuda(rng.standard_normal(gpu.ntrace))
    ref_v, ref_z = _np(gpu.vcycle(b)), _np(gpu.precond(r))
    gpu.set_options(mg_fuse_cells=1 << 30)                          # fused on every coarse level
    np.testing.assert_array_equal(_np(gpu.vcycle(b)), ref_v)
    np.testing.assert_array_equal(_np(gpu.precond(r)), ref_z)
    gpu.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_solves_with_and_without_the_fused_steps_agree_bitwise(precision):
    from paper_2210_11797_gb300.hmg import Solver
    w = I.cubed_sphere(24, 30, seed=11)
    Rub, Rpi = _cuda(w.Rub.ravel()), _cuda(w.Rpi)
    out = []
    for cells in (0, 1 << 30):
        gpu = Solver(w.hier, w.coeffs, tol=1e-8, precision=precision, mg_fuse_cells=cells)
        lam, st = gpu.solve(Rub, Rpi)
        assert st["status"] == "ok"
        out.append((_np(lam), st["iterations"]))
        gpu.close()
    np.testing.assert_array_equal(out[1][0], out[0][0])
    assert out[1][1] == out[0][1]


def test_fuse_threshold_must_not_be_negative():
    from paper_2210_11797_gb300.hmg import HmgError, Solver
    w = I.planar_helmholtz()
    gpu = Solver(w.hier, w.coeffs)
    with pytest.raises(HmgError):
        gpu.set_options(mg_fuse_cells=-1)
    gpu.close()


@pytest.mark.parametrize("name", sorted(CASES))
def test_twisted_column_solve_matches_the_oracle(name):
    """mg_twisted = 1: the two-lane twisted elimination of each column's H_z (rows from the
    top and from the bottom at once, the middle row last) rounds differently from the oracle's
    Thomas sweep but solves the same systems: the V-cycle agrees with the oracle's to 1e-12
    relative, and the fused and per-step forms still agree bit for bit."""
    from paper_2210_11797_gb300.hmg import Solver
    w = CASES[name]()
    gpu = Solver(w.hier, w.coeffs, tol=1e-10, mg_twisted=1)
    b = _cuda(np.random.default_rng(8).standard_normal(gpu.ncell))
    got = _np(gpu.vcycle(b))
    want = HybridSolver(w.hier, w.coeffs).mg.vcycle(_np(b))
    assert np.linalg.norm(got - want) <= 1e-12 * np.linalg.norm(want)
    gpu.set_options(mg_fused=1)
    np.testing.assert_array_equal(_np(gpu.vcycle(b)), got)
    gpu.set_options(mg_twisted=0, mg_fused=0)     # back to Thomas: the factors are rebuilt
    got0 = _np(gpu.vcycle(b))
    assert np.linalg.norm(got0 - want) <= 1e-12 * np.linalg.norm(want)
    gpu.close()


def test_autotune_may_pick_either_column_solve_and_keeps_the_solution():
    from paper_2210_11797_gb300.hmg import Solver
    w = I.cubed_sphere(24, 30, seed=13)
    Rub, Rpi = _cuda(w.Rub.ravel()), _cuda(w.Rpi)
    gpu = Solver(w.hier, w.coeffs, tol=1e-10)                # mg_twisted = 2 (default)
    lam0, st0 = gpu.solve(Rub, Rpi)
    gpu.autotune()
    lam1, st1 = gpu.solve(Rub, Rpi, torch.empty_like(lam0))
    assert st1["status"] == "ok" and abs(st1["iterations"] - st0["iterations"]) <= 1
    assert torch.linalg.norm(lam1 - lam0) <= 1e-8 * torch.linalg.norm(lam0)
    gpu.close()
