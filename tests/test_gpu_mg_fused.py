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
    """Autotuned block shapes (columns per block) change nothing in the results. (A level where
    the autotuner took the warp-per-column form, columns -1, is set back to the default block
    shape here: the cooperative coarse-level kernel runs the block form, and the warp form's
    scan has its own rounding order.)"""
    from paper_2210_11797_gb300.hmg import Solver
    w = I.cubed_sphere(24, 12, seed=10, nmg=4)
    gpu = Solver(w.hier, w.coeffs, tol=1e-8, mg_fused=0)
    b = _cuda(np.random.default_rng(5).standard_normal(gpu.ncell))
    ref = _np(gpu.vcycle(b))
    gpu.autotune()
    sw, mg = gpu.launch_shapes()
    gpu.set_launch_shapes(sw, [(c, t) if c > 0 else (0, 0) for c, t in mg])
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
