"""Pins of the oracle's network, its gradient, Adam and flexible GMRES (CPU only)."""
import numpy as np
import pytest

from oracle import learned as N
from paper_2210_11797_gb300 import inputs as I


def _brute_conv(W, x):
    ncol, cin, L = x.shape
    y = np.zeros((ncol, W.shape[0], L))
    for n in range(ncol):
        for o in range(W.shape[0]):
            for k in range(L):
                for i in range(cin):
                    for d in (-1, 0, 1):
                        if 0 <= k + d < L:
                            y[n, o, k] += W[o, i, d + 1] * x[n, i, k + d]
    return y


def test_conv1d_matches_brute_force():
    rng = np.random.default_rng(0)
    W, x = rng.standard_normal((4, 3, 3)), rng.standard_normal((2, 3, 7))
    np.testing.assert_allclose(N.conv1d(W, x), _brute_conv(W, x), rtol=1e-13, atol=1e-13)


def test_grid_neighbours_on_a_patch():
    edge, diag = N.grid_neighbours(3, 3)
    c = 4                                    # centre of a 3x3 patch
    assert sorted(edge[c]) == [1, 3, 5, 7] and sorted(diag[c]) == [0, 2, 6, 8]
    assert (edge[0] == [-1, 1, 3, -1]).all() and (diag[0] == [-1, 4, -1, -1]).all()


def test_mesh_neighbours_match_the_grid_inside_a_panel():
    m = I.planar_periodic_mesh(6, 2, 1.0, I.uniform_levels(2, 0.1))
    edge, diag = N.mesh_neighbours(m)
    col = lambda i, j: (j % 6) * 6 + (i % 6)
    c = col(2, 3)
    assert list(edge[c]) == [col(2, 2), col(3, 3), col(2, 4), col(1, 3)]
    # the mix is isotropic, so only the set of corner columns matters
    assert sorted(diag[c]) == sorted([col(3, 2), col(3, 4), col(1, 4), col(1, 2)])


def test_network_is_positively_homogeneous():
    p = N.init_params(1, ch=8)
    edge, diag = N.grid_neighbours(4, 4)
    x = np.random.default_rng(2).standard_normal((16, 6))
    np.testing.assert_allclose(N.forward(p, 3.5 * x, edge, diag), 3.5 * N.forward(p, x, edge, diag), rtol=1e-12)


def test_gradient_matches_central_differences():
    p = N.init_params(3, ch=6)
    edge, diag = N.grid_neighbours(3, 4)
    rng = np.random.default_rng(4)
    x, t = rng.standard_normal((12, 5)), rng.standard_normal((12, 5))
    loss, g = N.loss_and_grad(p, x, t, edge, diag)
    h = 1e-6
    for k in p:
        flat = p[k].reshape(-1)
        for idx in rng.choice(flat.size, size=min(6, flat.size), replace=False):
            save = flat[idx]
            flat[idx] = save + h
            lp, _ = N.loss_and_grad(p, x, t, edge, diag)
            flat[idx] = save - h
            lm, _ = N.loss_and_grad(p, x, t, edge, diag)
            flat[idx] = save
            fd = (lp - lm) / (2 * h)
            assert g[k].reshape(-1)[idx] == pytest.approx(fd, rel=1e-5, abs=1e-8)


def test_adam_first_step_is_signed_learning_rate():
    """With bias correction the first Adam step moves each weight by lr * g / (|g| + eps)."""
    p = {"w": np.array([1.0, -2.0, 3.0])}
    g = {"w": np.array([0.5, -4.0, 1e-3])}
    out = N.adam_step(dict(p), g, {}, lr=0.01)
    np.testing.assert_allclose(out["w"], p["w"] - 0.01 * np.sign(g["w"]), rtol=1e-6)


def test_fgmres_solves_and_is_flexible():
    rng = np.random.default_rng(5)
    n = 50
    A = rng.standard_normal((n, n)) + n * np.eye(n)
    b = rng.standard_normal(n)
    x, hist, st = N.fgmres(lambda v: A @ v, b, lambda v, k: v, 1e-12, restart=10, maxit=200)
    assert st == "ok"
    np.testing.assert_allclose(x, np.linalg.solve(A, b), rtol=1e-9)
    Ainv = np.linalg.inv(A)
    x, hist, st = N.fgmres(lambda v: A @ v, b, lambda v, k: Ainv @ v, 1e-12, restart=10)
    assert st == "ok" and len(hist) == 2          # exact preconditioner: one step
    # a preconditioner that changes every step (alternating scalings) still converges
    x, hist, st = N.fgmres(lambda v: A @ v, b, lambda v, k: v * (1.0 + (k % 2)), 1e-10, restart=20)
    assert st == "ok"
    np.testing.assert_allclose(x, np.linalg.solve(A, b), rtol=1e-7)
