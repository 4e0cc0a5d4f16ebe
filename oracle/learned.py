"""Learned coarse-level correction: the network, its gradient and Adam, and flexible GMRES.

Oracle (test infrastructure only; see oracle/__init__.py). FP64 numpy, plain loops over the
network's layers. The paper has no learned component: this is the growth axis of the hot
path that replaces (or seeds) the coarse solve of Algorithm 2 line 6 with a small network
f(bbar) ~ H^-1 bbar, inside a flexible Krylov method so that the answer is still judged by
the FP64 trace residual.

Network, per column over the levels (zero padding at the ground and the lid), bias-free so
f(a x) = a f(x) for a > 0:
    h1 = relu(conv1d(1 -> C, 3)(x))
    h2 = relu(conv1d(C -> C, 3)(h1))
    h3 = relu(w_c * h2 + w_e * sum(4 edge neighbours of h2) + w_d * sum(4 corner neighbours))
    y  = conv1d(C -> 1, 3)(h3)
conv1d(a -> b, 3): y[o, k] = sum_i sum_{d=-1..1} W[o, i, d+1] x[i, k+d].
The horizontal mix is depthwise (one (w_c, w_e, w_d) per channel) and isotropic.
Input and output are scaled by diag(H)^-1/2 around the network (a choice of this project:
the paper has no learned part; H's diagonal varies by orders of magnitude with height, and
the bias-free network is positively homogeneous, so the scaling gives it a dimensionless
problem), so the learned map is f_H(b) = D^-1/2 f(D^-1/2 b) with D = diag(H).

Flexible GMRES (Saad 2003 Alg. 9.6, restart m) allows the preconditioner to change between
steps (a network is not a fixed linear operator).

Storage precision: the network is specified with BF16 weights and activations and FP32
accumulation. `forward` and `loss_and_grad` take quant="bf16" to round, to the nearest BF16
value (ties to even), exactly the quantities that are stored in that format: the weights,
the input and the activations h1, h2, h3 after their ReLU. Everything else stays FP64, so
the result is the exact gradient of the network whose stored values are BF16; a BF16
implementation that accumulates in FP32 differs from it only by its FP32 roundings (and
the few stored values those move across a BF16 rounding boundary).
"""
from __future__ import annotations

import numpy as np

CHANNELS = 32


def init_params(seed: int = 0, ch: int = CHANNELS) -> dict:
    """He-style random initialisation from numpy's PCG64 (only used by the oracle's tests;
    the GPU path draws its own initial weights from SplitMix64 in inputs.py)."""
    rng = np.random.default_rng(seed)
    return {
        "W1": rng.standard_normal((ch, 1, 3)) * np.sqrt(2.0 / 3.0),
        "W2": rng.standard_normal((ch, ch, 3)) * np.sqrt(2.0 / (3.0 * ch)),
        "M": np.stack([np.ones(ch), 0.1 * np.ones(ch), 0.05 * np.ones(ch)], axis=1),  # (w_c, w_e, w_d)
        "W3": rng.standard_normal((1, ch, 3)) * np.sqrt(1.0 / (3.0 * ch)),
    }


def round_bf16(a) -> np.ndarray:
    """Round to the nearest BF16 value (8 significant bits, the exponent range of FP32), ties
    to even, returned in FP64. The value is first rounded to FP32 (the accumulation format),
    then the low 16 bits of its FP32 pattern are rounded away. Finite inputs only."""
    f = np.ascontiguousarray(a, np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def _storage(quant):
    if quant is None:
        return lambda a: a
    if quant == "bf16":
        return round_bf16
    raise ValueError(quant)


def conv1d(W: np.ndarray, x: np.ndarray) -> np.ndarray:
    """W [out, in, 3], x [ncol, in, L] -> [ncol, out, L], zero padding at both column ends."""
    ncol, cin, L = x.shape
    xp = np.zeros((ncol, cin, L + 2))
    xp[:, :, 1:-1] = x
    y = np.zeros((ncol, W.shape[0], L))
    for d in range(3):
        y += np.einsum("oi,nil->nol", W[:, :, d], xp[:, :, d:d + L])
    return y


def conv1d_backward(W: np.ndarray, x: np.ndarray, gy: np.ndarray):
    """Gradients of conv1d w.r.t. W and x given gy = dLoss/dy."""
    ncol, cin, L = x.shape
    xp = np.zeros((ncol, cin, L + 2))
    xp[:, :, 1:-1] = x
    gW = np.zeros_like(W)
    gxp = np.zeros_like(xp)
    for d in range(3):
        gW[:, :, d] = np.einsum("nol,nil->oi", gy, xp[:, :, d:d + L])
        gxp[:, :, d:d + L] += np.einsum("oi,nol->nil", W[:, :, d], gy)
    return gW, gxp[:, :, 1:-1]


def hmix(M: np.ndarray, h: np.ndarray, edge: np.ndarray, diag: np.ndarray) -> np.ndarray:
    """Depthwise 3x3 mix: M [ch, 3]; h [ncol, ch, L]; edge, diag [ncol, 4] neighbour column ids
    (-1 = none, i.e. zero padding)."""
    out = M[None, :, 0:1] * h
    for nb, wi in ((edge, 1), (diag, 2)):
        acc = np.zeros_like(h)
        for s in range(4):
            idx = nb[:, s]
            ok = idx >= 0
            acc[ok] += h[idx[ok]]
        out += M[None, :, wi:wi + 1] * acc
    return out


def hmix_backward(M, h, edge, diag, gout):
    gM = np.zeros_like(M)
    gM[:, 0] = np.einsum("ncl,ncl->c", gout, h)
    gh = M[None, :, 0:1] * gout
    for nb, wi in ((edge, 1), (diag, 2)):
        acc = np.zeros_like(h)
        for s in range(4):
            idx = nb[:, s]
            ok = idx >= 0
            acc[ok] += h[idx[ok]]
            # d/dh[idx] of M * h[idx] at column n: scatter gout[n] back to idx
            np.add.at(gh, idx[ok], M[None, :, wi:wi + 1] * gout[ok])
        gM[:, wi] = np.einsum("ncl,ncl->c", gout, acc)
    return gM, gh


def forward(params: dict, x: np.ndarray, edge: np.ndarray, diag: np.ndarray, keep: bool = False,
            quant=None):
    """x [ncol, L] -> y [ncol, L]. quant="bf16": weights, input and activations stored in
    BF16 (see the module docstring)."""
    q = _storage(quant)
    W = {k: q(v) for k, v in params.items()}
    x = q(x)
    a1 = conv1d(W["W1"], x[:, None, :])
    h1 = q(np.maximum(a1, 0.0))
    a2 = conv1d(W["W2"], h1)
    h2 = q(np.maximum(a2, 0.0))
    a3 = hmix(W["M"], h2, edge, diag)
    h3 = q(np.maximum(a3, 0.0))
    y = conv1d(W["W3"], h3)[:, 0, :]
    if keep:
        return y, dict(x=x, a1=a1, h1=h1, a2=a2, h2=h2, a3=a3, h3=h3, W=W)
    return y


def loss_and_grad(params, x, target, edge, diag, quant=None):
    """Relative squared error per sample summed: sum_s ||f(x_s) - t_s||^2 / ||t_s||^2 over the
    samples (the columns of one sample share a sample id in `sample`). Here one call is one
    sample: x, target [ncol, L]. With quant="bf16" the gradient is that of the network with
    BF16 storage, taken at the stored (rounded) weights and activations."""
    y, t = forward(params, x, edge, diag, keep=True, quant=quant)
    W = t["W"]
    denom = np.sum(target * target)
    r = y - target
    loss = np.sum(r * r) / denom
    gy = 2.0 * r / denom
    gW3, gh3 = conv1d_backward(W["W3"], t["h3"], gy[:, None, :])
    ga3 = gh3 * (t["a3"] > 0)
    gM, gh2 = hmix_backward(W["M"], t["h2"], edge, diag, ga3)
    ga2 = gh2 * (t["a2"] > 0)
    gW2, gh1 = conv1d_backward(W["W2"], t["h1"], ga2)
    ga1 = gh1 * (t["a1"] > 0)
    gW1, _gx = conv1d_backward(W["W1"], t["x"][:, None, :], ga1)
    return loss, {"W1": gW1, "W2": gW2, "M": gM, "W3": gW3}


def adam_step(params, grads, state, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """Kingma & Ba (2015) Adam with bias correction; state holds m, v and the step count."""
    state["t"] = state.get("t", 0) + 1
    t = state["t"]
    for k in params:
        m = state.setdefault("m_" + k, np.zeros_like(params[k]))
        v = state.setdefault("v_" + k, np.zeros_like(params[k]))
        g = grads[k]
        m[:] = b1 * m + (1 - b1) * g
        v[:] = b2 * v + (1 - b2) * g * g
        mhat = m / (1 - b1 ** t)
        vhat = v / (1 - b2 ** t)
        params[k] = params[k] - lr * mhat / (np.sqrt(vhat) + eps)
    return params


def grid_neighbours(nx: int, ny: int):
    """Edge and corner neighbours of an nx x ny patch of columns (c = j*nx + i), -1 outside."""
    ii, jj = np.meshgrid(np.arange(nx), np.arange(ny), indexing="xy")
    ii, jj = ii.ravel(), jj.ravel()

    def idx(di, dj):
        i2, j2 = ii + di, jj + dj
        ok = (i2 >= 0) & (i2 < nx) & (j2 >= 0) & (j2 < ny)
        return np.where(ok, j2 * nx + i2, -1)

    edge = np.stack([idx(0, -1), idx(1, 0), idx(0, 1), idx(-1, 0)], axis=1)
    diag = np.stack([idx(1, -1), idx(1, 1), idx(-1, 1), idx(-1, -1)], axis=1)
    return edge, diag


def mesh_neighbours(mesh):
    """Edge neighbours from the mesh tables and corner neighbours two steps away: across face
    f to n = nbr(c, f), then across the face of n that follows the shared one (shared + 1
    mod 4). On a structured panel this is the diagonal column."""
    col = np.arange(mesh.ncol)
    edge = np.zeros((mesh.ncol, 4), np.int64)
    nface = np.zeros((mesh.ncol, 4), np.int64)
    for f in range(4):
        e = mesh.col_edges[col, f]
        first = (mesh.edge_cols[e, 0] == col) & (mesh.edge_face[e, 0] == f)
        edge[:, f] = np.where(first, mesh.edge_cols[e, 1], mesh.edge_cols[e, 0])
        nface[:, f] = np.where(first, mesh.edge_face[e, 1], mesh.edge_face[e, 0])
    diag = np.zeros_like(edge)
    for f in range(4):
        n = edge[:, f]
        g = (nface[:, f] + 1) % 4
        e = mesh.col_edges[n, g]
        first = (mesh.edge_cols[e, 0] == n) & (mesh.edge_face[e, 0] == g)
        diag[:, f] = np.where(first, mesh.edge_cols[e, 1], mesh.edge_cols[e, 0])
    return edge, diag


def fgmres(apply_A, b, precond, tol, restart=30, maxit=300, on_step=None):
    """Right-preconditioned flexible GMRES(restart) from x = 0 with modified Gram-Schmidt and
    Givens rotations (Saad 2003 Alg. 9.6). precond(v, step) may change from step to step.
    Returns (x, history of ||r||/||b|| estimates, status)."""
    n = b.shape[0]
    x = np.zeros_like(b)
    bnorm = np.linalg.norm(b)
    if bnorm == 0.0:
        return x, [0.0], "ok"
    hist = [1.0]
    r = b.copy()
    step = 0
    while step < maxit:
        beta = np.linalg.norm(r)
        V = np.zeros((restart + 1, n))
        Z = np.zeros((restart, n))
        Hm = np.zeros((restart + 1, restart))
        cs, sn = np.zeros(restart), np.zeros(restart)
        g = np.zeros(restart + 1)
        g[0] = beta
        V[0] = r / beta
        j_done = 0
        for j in range(restart):
            Z[j] = precond(V[j], step)
            w = apply_A(Z[j])
            for i in range(j + 1):
                Hm[i, j] = w @ V[i]
                w = w - Hm[i, j] * V[i]
            Hm[j + 1, j] = np.linalg.norm(w)
            if Hm[j + 1, j] > 0:
                V[j + 1] = w / Hm[j + 1, j]
            for i in range(j):
                t = cs[i] * Hm[i, j] + sn[i] * Hm[i + 1, j]
                Hm[i + 1, j] = -sn[i] * Hm[i, j] + cs[i] * Hm[i + 1, j]
                Hm[i, j] = t
            den = np.hypot(Hm[j, j], Hm[j + 1, j])
            cs[j], sn[j] = Hm[j, j] / den, Hm[j + 1, j] / den
            Hm[j, j] = den
            Hm[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            step += 1
            j_done = j + 1
            rel = abs(g[j + 1]) / bnorm
            hist.append(rel)
            if on_step is not None:
                on_step(step, rel)
            if rel <= tol or step >= maxit:
                break
        y = np.linalg.solve(np.triu(Hm[:j_done, :j_done]), g[:j_done])
        x = x + Z[:j_done].T @ y
        r = b - apply_A(x)
        if hist[-1] <= tol:
            return x, hist, "ok"
    return x, hist, "not_converged"
