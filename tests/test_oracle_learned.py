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


def test_bf16_rounding_matches_torch_and_ties_go_to_even():
    """round_bf16 against PyTorch's float32 -> bfloat16 conversion (round to nearest even) on
    values spread over the FP32 range, and against hand-made ties: 1 + 2^-8 lies halfway
    between 1 and 1 + 2^-7 and rounds to the even 1; 1 + 3 * 2^-8 rounds up to 1 + 2^-6."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(8)
    v = (rng.standard_normal(20000) * 10.0 ** rng.uniform(-30, 30, 20000)).astype(np.float32)
    ref = torch.from_numpy(v).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(N.round_bf16(v), ref)
    ties = np.array([1 + 2.0 ** -8, 1 + 3 * 2.0 ** -8, -(1 + 2.0 ** -8), 2.0 ** -7 * (1 + 2.0 ** -8)])
    np.testing.assert_array_equal(N.round_bf16(ties), [1.0, 1 + 2.0 ** -6, -1.0, 2.0 ** -7])


def test_bf16_forward_stores_rounded_values():
    """With BF16 storage every stored activation is a BF16 value and the output equals the FP64
    network applied to the rounded weights and input up to the rounding of the activations
    (relative effect of order 2^-8 per layer)."""
    p = N.init_params(2, ch=8)
    edge, diag = N.grid_neighbours(4, 3)
    x = np.random.default_rng(9).standard_normal((12, 7))
    y16, t = N.forward(p, x, edge, diag, keep=True, quant="bf16")
    for k in ("x", "h1", "h2", "h3"):
        np.testing.assert_array_equal(t[k], N.round_bf16(t[k]))
    for k in p:
        np.testing.assert_array_equal(t["W"][k], N.round_bf16(p[k]))
    y = N.forward({k: N.round_bf16(v) for k, v in p.items()}, N.round_bf16(x), edge, diag)
    assert np.linalg.norm(y16 - y) / np.linalg.norm(y) < 3 * 2.0 ** -8
    assert np.linalg.norm(y16 - y) > 0          # the activations were rounded


def test_bf16_gradient_matches_central_differences_of_the_rounded_network():
    """The BF16-storage gradient is the derivative of the loss with the activations held at
    their stored (rounded) values: in the last layer that is exact, so W3's gradient equals a
    central difference of the loss in W3 with h3 frozen (a linear layer, so the difference is
    exact up to FP64 rounding)."""
    p = N.init_params(5, ch=6)
    edge, diag = N.grid_neighbours(3, 3)
    rng = np.random.default_rng(10)
    x, tgt = rng.standard_normal((9, 5)), rng.standard_normal((9, 5))
    _loss, g = N.loss_and_grad(p, x, tgt, edge, diag, quant="bf16")
    _y, t = N.forward(p, x, edge, diag, keep=True, quant="bf16")
    W3 = t["W"]["W3"]
    denom = np.sum(tgt * tgt)

    def loss_w3(w):
        y = N.conv1d(w, t["h3"])[:, 0, :]
        return np.sum((y - tgt) ** 2) / denom
    h = 1e-5
    for idx in np.ndindex(W3.shape):
        wp, wm = W3.copy(), W3.copy()
        wp[idx] += h
        wm[idx] -= h
        fd = (loss_w3(wp) - loss_w3(wm)) / (2 * h)
        assert g["W3"][idx] == pytest.approx(fd, rel=1e-7, abs=1e-10)
    # and the full gradient with quant=None is the FP64 network's (the BF16 one differs)
    _l, g64 = N.loss_and_grad(p, x, tgt, edge, diag)
    assert not np.allclose(g64["W2"], g["W2"], rtol=1e-6)


def test_adam_three_steps_from_nonzero_moments_closed_form():
    """Three Adam steps continuing from step 4 with given moments, against the update written
    out from Kingma & Ba's definition for a scalar weight."""
    w0, m0, v0 = 0.7, 0.02, 3e-4
    gs = [0.1, -0.05, 0.2]
    lr, b1, b2, eps = 1e-3, 0.9, 0.999, 1e-8
    p = {"w": np.array([w0])}
    st = {"t": 4, "m_w": np.array([m0]), "v_w": np.array([v0])}
    w, m, v = w0, m0, v0
    for k, g in enumerate(gs):
        p = N.adam_step(p, {"w": np.array([g])}, st, lr=lr, b1=b1, b2=b2, eps=eps)
        t = 5 + k
        m = b1 * m + (1 - b1) * g
        v = b2 * v + (1 - b2) * g * g
        w = w - lr * (m / (1 - b1 ** t)) / (np.sqrt(v / (1 - b2 ** t)) + eps)
    assert p["w"][0] == pytest.approx(w, rel=1e-15)
    assert st["t"] == 7 and st["m_w"][0] == pytest.approx(m, rel=1e-15)
