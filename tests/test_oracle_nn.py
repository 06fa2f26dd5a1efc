"""Pins of the warm-start network oracle (oracle/nn.py) against library routines, brute
force, finite differences and closed forms."""
import numpy as np
import pytest
import scipy.ndimage

from oracle import nn
from workloads.generators import normal


def _params(C, H, NZ, K, seed, scale=0.3):
    n = sum(int(np.prod(s)) for _, s in nn.shapes(C, H, NZ, K))
    return nn.unflatten(scale * normal(seed, n), C, H, NZ, K)


def test_conv_matches_scipy_wrap_correlation():
    X = normal(3, 2 * 3 * 11).reshape(2, 3, 11)
    W = normal(4, 4 * 3 * 5).reshape(4, 3, 5)
    b = normal(5, 4)
    Y = nn.conv(X, W, b)
    for s in range(2):
        for o in range(4):
            ref = b[o] + sum(scipy.ndimage.correlate1d(X[s, c], W[o, c], mode='wrap') for c in range(3))
            np.testing.assert_allclose(Y[s, o], ref, rtol=1e-13, atol=1e-13)


def test_conv_brute_force_loop():
    X = normal(6, 1 * 2 * 7).reshape(1, 2, 7)
    W = normal(7, 3 * 2 * 3).reshape(3, 2, 3)
    b = np.zeros(3)
    Y = nn.conv(X, W, b)
    for o in range(3):
        for x in range(7):
            ref = sum(W[o, c, k] * X[0, c, (x + k - 1) % 7] for c in range(2) for k in range(3))
            assert abs(Y[0, o, x] - ref) < 1e-13


@pytest.mark.parametrize("K,lam", [(1, 0.0), (3, 0.0), (5, 0.0), (3, 0.7)])
def test_gradients_match_finite_differences(K, lam):
    C, H, NZ, NX, S = 4, 5, 3, 7, 2
    p = _params(C, H, NZ, K, 11)
    X = normal(12, S * C * NX).reshape(S, C, NX)
    T = normal(13, S * NZ * NX).reshape(S, NZ, NX)
    _, g = nn.loss_and_grads(p, X, T, lam)
    flat = nn.flatten(p, C, H, NZ, K)
    gflat = nn.flatten(g, C, H, NZ, K)
    h = 1e-6
    for i in range(0, flat.size, max(1, flat.size // 60)):
        fp, fm = flat.copy(), flat.copy()
        fp[i] += h
        fm[i] -= h
        lp, _ = nn.loss_and_grads(nn.unflatten(fp, C, H, NZ, K), X, T, lam)
        lm, _ = nn.loss_and_grads(nn.unflatten(fm, C, H, NZ, K), X, T, lam)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - gflat[i]) <= 1e-7 * max(1.0, abs(fd)), (i, fd, gflat[i])


def test_loss_brute_force_and_special_cases():
    S, NZ, NX, lam = 2, 4, 5, 0.3
    y = normal(41, S * NZ * NX).reshape(S, NZ, NX)
    T = normal(42, S * NZ * NX).reshape(S, NZ, NX)
    ref = 0.0
    for s in range(S):
        for z in range(NZ - 1):  # the surface row is masked
            for x in range(NX):
                e = y[s, z, x] - T[s, z, x]
                ez = (y[s, z + 1, x] - T[s, z + 1, x]) if z + 1 < NZ - 1 else 0.0
                ex = y[s, z, (x + 1) % NX] - T[s, z, (x + 1) % NX]
                ref += e * e + lam * ((ez - e) ** 2 + (ex - e) ** 2)
        # the masked row still enters through the x-differences of nothing and the z-difference above
    ref /= S * NZ * NX
    val, g = nn.loss(y, T, lam)
    assert abs(val - ref) < 1e-13 * ref
    # lam = 0 is the mean squared error over rows below the surface (over all entries' count)
    val0, g0 = nn.loss(y, T, 0.0)
    e = (y - T)[:, :-1, :]
    assert abs(val0 - np.sum(e * e) / y.size) < 1e-14
    np.testing.assert_allclose(g0[:, :-1, :], 2 * e / y.size, rtol=1e-14)
    assert np.all(g0[:, -1, :] == 0) and np.all(g[:, -1, :] == 0)
    # a constant error has no difference terms
    c = np.full((1, 3, 4), 0.5)
    c[:, -1, :] = 0.0
    val_c, _ = nn.loss(c, np.zeros_like(c), 10.0)
    # only the z-difference into the masked surface row contributes
    assert abs(val_c - (8 * 0.25 + 10.0 * 4 * 0.25) / 12) < 1e-15


def test_input_gradient_matches_finite_differences():
    """The input-gradient branch of conv_grads (used between layers) on its own."""
    X = normal(21, 2 * 3 * 6).reshape(2, 3, 6)
    W = normal(22, 2 * 3 * 5).reshape(2, 3, 5)
    dY = normal(23, 2 * 2 * 6).reshape(2, 2, 6)
    dX, _, _ = nn.conv_grads(X, W, dY)
    f = lambda Xv: np.sum(dY * nn.conv(Xv, W, np.zeros(2)))
    for idx in [(0, 0, 0), (1, 2, 5), (0, 1, 3), (1, 0, 4)]:
        Xp, Xm = X.copy(), X.copy()
        Xp[idx] += 1e-6
        Xm[idx] -= 1e-6
        assert abs((f(Xp) - f(Xm)) / 2e-6 - dX[idx]) < 1e-8


def test_adam_first_step_is_signed_learning_rate():
    g = np.array([3.0, -2e-3, 0.5, -7.0])
    p0 = np.array([1.0, 2.0, 3.0, 4.0])
    p1, m, v = nn.adam(p0, g, np.zeros(4), np.zeros(4), 1, lr=0.01)
    np.testing.assert_allclose(p1, p0 - 0.01 * np.sign(g), rtol=0, atol=1e-7)
    # second step with the same gradient keeps the same step size
    p2, _, _ = nn.adam(p1, g, m, v, 2, lr=0.01)
    np.testing.assert_allclose(p2, p1 - 0.01 * np.sign(g), rtol=0, atol=1e-7)


def test_pack_target_guess_roundtrip():
    NX, NZ = 5, 4
    eta, eta_p = normal(31, NX), normal(35, NX)
    etax = normal(32, NX)
    pp = normal(33, NX * NZ)
    p = normal(34, NX * NZ)
    X = nn.pack(eta, eta_p, etax, pp, NZ, 2, 0.5, 0.25, 2.0)
    assert X.shape == (NZ + 5, NX)
    np.testing.assert_allclose(X[0], eta / 0.5)
    np.testing.assert_allclose(X[1], (eta - eta_p) / 0.25)
    np.testing.assert_allclose(X[2], etax)
    np.testing.assert_array_equal(X[3], [1, 0, 1, 0, 1])
    np.testing.assert_array_equal(X[4], [0, 1, 0, 1, 0])
    np.testing.assert_allclose(X[5 + 1, 3], pp[3 * NZ + 1] / 2.0)
    t = nn.target(p, pp, NZ, 0.1)
    g = nn.guess(pp, t, NZ, 0.1)
    top = np.arange(NX) * NZ + NZ - 1
    interior = np.setdiff1d(np.arange(NX * NZ), top)
    np.testing.assert_allclose(g[interior], p[interior], rtol=1e-14)
    np.testing.assert_array_equal(g[top], pp[top])
