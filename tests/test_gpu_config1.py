"""Configuration 1 on the GPU (the unhybridised 2x2 system with the approximate Schur
complement preconditioner, Sec. 2.3) against its FP64 oracle (oracle/schur.py), through the
C ABI. Tolerances as for the hybridised path: a row of the operator (<= 13 products) within
1e-12 of |Mx| |x| row by row; one preconditioner application (Steps 1-3 around a V-cycle)
within 1e-11 of its max norm; whole solves converged to 1e-12 on both sides within 1e-9."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle.schur import MixedSolver
from paper_2210_11797_gb300 import inputs as I


def _cuda(a):
    return torch.as_tensor(np.ascontiguousarray(a, np.float64)).cuda()


def _np(t):
    return t.detach().cpu().numpy()


WORKLOADS = {
    "planar16": lambda: I.planar_helmholtz(),
    "sphereC6L5": lambda: I.cubed_sphere(6, 5, courant=8.0, nmg=2, seed=4),
    "sphereC12L30": lambda: I.cubed_sphere(12, 30),
    "sphereC6L5_rotating": lambda: I.cubed_sphere(6, 5, courant=8.0, nmg=2, seed=4, omega=10 * I.EARTH_OMEGA),
}
_CACHE = {}


def _pair(name):
    if name not in _CACHE:
        from paper_2210_11797_gb300.hmg import Solver
        w = WORKLOADS[name]()
        _CACHE[name] = (w, MixedSolver(w.hier, w.coeffs), Solver(w.hier, w.coeffs, tol=1e-12, precond="schur"))
    return _CACHE[name]


@pytest.mark.parametrize("name", sorted(WORKLOADS))
def test_mixed_operator_matches_oracle(name):
    _w, ms, gpu = _pair(name)
    x = np.random.default_rng(1).standard_normal(ms.T + ms.C)
    y = _np(gpu.apply_mixed(_cuda(x)))
    want = ms.Mx @ x
    scale = abs(ms.Mx) @ np.abs(x)
    assert np.all(np.abs(y - want) <= 1e-12 * scale)


@pytest.mark.parametrize("name", sorted(WORKLOADS))
def test_approximate_schur_preconditioner_matches_oracle(name):
    _w, ms, gpu = _pair(name)
    r = np.random.default_rng(2).standard_normal(ms.T + ms.C)
    z = _np(gpu.precond(_cuda(r)))
    want = ms.precond(r)
    assert np.abs(z - want).max() <= 1e-11 * np.abs(want).max()


@pytest.mark.parametrize("name", sorted(WORKLOADS))
def test_configuration1_solve_matches_oracle(name):
    """Both sides iterate to a recurrence residual of 1e-12. On the sphere BiCGStab on the 2x2
    system passes through residuals of ~5e3 ||B|| (the oracle's history shows the same), so the
    recomputed residual stalls near 4e-9 on both sides: the GPU's must match the oracle's
    within 10x, and the solutions agree to 1e-9 where the true residuals reach 1e-11 and to
    100x the true residual otherwise."""
    w, ms, gpu = _pair(name)
    u, pi, st = gpu.solve_mixed(_cuda(w.Rub.ravel()), _cuda(w.Rpi))
    uo, pio, hist, status = ms.solve(w.Rub, w.Rpi, 1e-12)
    # the spike amplifies rounding: the oracle itself takes 25 iterations on x86-64 and 27 on
    # aarch64 for C12 x 30, so the counts agree within 3
    assert status == "ok" and st["status"] == "ok" and abs(st["iterations"] - (len(hist) - 1)) <= 3
    xo = np.concatenate([uo, pio])
    b = ms.rhs(w.Rub, w.Rpi)
    true_o = np.linalg.norm(b - ms.Mx @ xo) / np.linalg.norm(b)
    assert st["true_rel_residual"] <= 10 * true_o + 1e-12, (st["true_rel_residual"], true_o)
    x = np.concatenate([_np(u), _np(pi)])
    err = np.linalg.norm(x - xo) / np.linalg.norm(xo)
    assert err < max(1e-9, 100 * max(true_o, st["true_rel_residual"])), (err, true_o)
    assert not np.any(_np(u)[_ground_lid(w.mesh)])      # u.n = 0 on the ground and the lid


def _ground_lid(mesh):
    L = mesh.nlev
    zc = mesh.n_trace_h + np.arange(mesh.ncol) * (L + 1)
    return np.concatenate([zc, zc + L])


def test_configuration1_and_3c_solve_the_same_mixed_system():
    """Both configurations solve Eq. 2x2system: the hybridised lambda, recovered to (u^b, Pi),
    gives the same Pi and a continuous u^b equal to s_K(f) u_f."""
    from paper_2210_11797_gb300.hmg import Solver
    w, ms, gpu1 = _pair("sphereC12L30")
    u, pi, _st = gpu1.solve_mixed(_cuda(w.Rub.ravel()), _cuda(w.Rpi))
    gpu3 = Solver(w.hier, w.coeffs, tol=1e-12)
    lam, _st3 = gpu3.solve(_cuda(w.Rub.ravel()), _cuda(w.Rpi))
    ub, pi3 = gpu3.reconstruct(lam, _cuda(w.Rub.ravel()), _cuda(w.Rpi))
    pi, pi3 = _np(pi), _np(pi3)
    assert np.linalg.norm(pi - pi3) / np.linalg.norm(pi3) < 1e-8
    want = ms.s * _np(u)[ms.g]
    assert np.linalg.norm(_np(ub).reshape(-1, 6) - want) / np.linalg.norm(want) < 1e-8
    gpu3.close()


def test_configuration1_graph_equals_host_loop():
    w, _ms, gpu = _pair("planar16")
    u1, pi1, st1 = gpu.solve_mixed(_cuda(w.Rub.ravel()), _cuda(w.Rpi))
    gpu.set_options(graph=0)
    try:
        u0, pi0, st0 = gpu.solve_mixed(_cuda(w.Rub.ravel()), _cuda(w.Rpi))
    finally:
        gpu.set_options(graph=1)
    assert st0["iterations"] == st1["iterations"]
    np.testing.assert_array_equal(_np(u0), _np(u1))
    np.testing.assert_array_equal(_np(pi0), _np(pi1))
