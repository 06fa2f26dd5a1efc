"""FP64 numpy restatement of the learned warm start's network (test infrastructure; see
oracle/__init__).  Not part of the paper: the network is an addition of this library.

Periodic 1D cross-correlation over the x positions (K taps, centred):
    Y[s, o, x] = b[o] + sum_{c, k} W[o, c, k] X[s, c, (x + k - K//2) mod n_x]
Network: conv(K) -> tanh -> conv(K) -> tanh -> conv(1).  Loss over outputs laid out
(sample, z, x) with the last z row (the surface) masked, e = Y - T:
    L = mean over entries of e^2 + lam ((e[z+1] - e[z])^2 + (e[x+1] - e[x])^2), x periodic.
Gradients by the chain rule written per layer; Adam (Kingma & Ba 2015, Algorithm 1) with
bias-corrected moments.  Input packing per node column: channels [eta/s_eta,
(eta - eta_prev)/s_deta, eta_x, one-hot of (x mod Q), p_prev(z)/s_p]; target (p - p_prev)/s_dp; guess
p_prev + s_dp * Y with the surface row unchanged.

Pins (tests/test_oracle_nn.py): the convolution against scipy.ndimage.correlate1d in wrap
mode and a brute-force loop; every gradient against central finite differences; the first
Adam step against its closed form lr * sign(g).
"""
import numpy as np


def shapes(C, H, NZ, K):
    return [("W1", (H, C, K)), ("b1", (H,)), ("W2", (H, H, K)), ("b2", (H,)), ("W3", (NZ, H, 1)), ("b3", (NZ,))]


def unflatten(flat, C, H, NZ, K):
    out, i = {}, 0
    for name, shp in shapes(C, H, NZ, K):
        n = int(np.prod(shp))
        out[name] = np.asarray(flat[i:i + n], dtype=np.float64).reshape(shp)
        i += n
    assert i == len(flat)
    return out


def flatten(d, C, H, NZ, K):
    return np.concatenate([d[name].reshape(-1) for name, _ in shapes(C, H, NZ, K)])


def shifted(X, off):
    """X[..., (x + off) mod n] for every x."""
    return np.roll(X, -off, axis=-1)


def conv(X, W, b):
    """Periodic cross-correlation, X (S, C, n), W (O, C, K) -> (S, O, n)."""
    O, C, K = W.shape
    Y = np.zeros((X.shape[0], O, X.shape[2]))
    for k in range(K):
        Y += np.einsum('oc,scx->sox', W[:, :, k], shifted(X, k - K // 2))
    return Y + b[None, :, None]


def conv_grads(X, W, dY):
    """(dX, dW, db) of the periodic cross-correlation for upstream gradient dY."""
    O, C, K = W.shape
    dX = np.zeros_like(X)
    dW = np.zeros_like(W)
    for k in range(K):
        off = k - K // 2
        dW[:, :, k] = np.einsum('sox,scx->oc', dY, shifted(X, off))
        dX += shifted(np.einsum('oc,sox->scx', W[:, :, k], dY), -off)
    return dX, dW, dY.sum(axis=(0, 2))


def forward(p, X):
    a1 = np.tanh(conv(X, p["W1"], p["b1"]))
    a2 = np.tanh(conv(a1, p["W2"], p["b2"]))
    y = conv(a2, p["W3"], p["b3"])
    return y, (X, a1, a2)


def loss(y, T, lam=0.0):
    """(L, dL/dy) of outputs y against targets T, both (S, NZ, n_x)."""
    e = y - T
    e[:, -1, :] = 0.0
    dz = np.diff(e, axis=1)
    dx = np.roll(e, -1, axis=2) - e
    val = (np.sum(e * e) + lam * (np.sum(dz * dz) + np.sum(dx * dx))) / e.size
    g = 2.0 * e
    g[:, :-1, :] -= 2.0 * lam * dz
    g[:, 1:, :] += 2.0 * lam * dz
    g -= 2.0 * lam * dx
    g += 2.0 * lam * np.roll(dx, 1, axis=2)
    g[:, -1, :] = 0.0
    return val, g / e.size


def loss_and_grads(p, X, T, lam=0.0):
    y, (X, a1, a2) = forward(p, X)
    loss_val, dy = loss(y, T, lam)
    da2, dW3, db3 = conv_grads(a2, p["W3"], dy)
    dz2 = da2 * (1.0 - a2 * a2)
    da1, dW2, db2 = conv_grads(a1, p["W2"], dz2)
    dz1 = da1 * (1.0 - a1 * a1)
    _, dW1, db1 = conv_grads(X, p["W1"], dz1)
    return loss_val, {"W1": dW1, "b1": db1, "W2": dW2, "b2": db2, "W3": dW3, "b3": db3}


def adam(p, g, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update at step t >= 1; returns (p, m, v)."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v


def pack(eta, eta_prev, etax, p_prev, NZ, Q, s_eta, s_deta, s_p):
    """Network input (NZ + 3 + Q, n_x) of one node-column state (p_prev z-fastest)."""
    eta, eta_prev, etax = (np.asarray(a, dtype=np.float64) for a in (eta, eta_prev, etax))
    NX = eta.shape[0]
    P = np.asarray(p_prev).reshape(NX, NZ).T
    onehot = (np.arange(NX)[None, :] % Q == np.arange(Q)[:, None]).astype(np.float64)
    return np.vstack([eta[None] / s_eta, (eta - eta_prev)[None] / s_deta, etax[None], onehot, P / s_p])


def target(p, p_prev, NZ, s_dp):
    NX = p.shape[0] // NZ
    return ((np.asarray(p) - np.asarray(p_prev)).reshape(NX, NZ).T) / s_dp


def guess(p_prev, y, NZ, s_dp):
    """p_prev + s_dp * y (y shaped (NZ, n_x)), surface row (last z) unchanged."""
    NX = p_prev.shape[0] // NZ
    d = (s_dp * np.asarray(y, dtype=np.float64)).T.copy()
    d[:, NZ - 1] = 0.0
    return np.asarray(p_prev) + d.reshape(-1)
