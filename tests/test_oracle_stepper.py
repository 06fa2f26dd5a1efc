"""Pins of the oracle's wave-tank stepper (Sec. 2.1-2.2, Sec. 3, Eq. freesurf1)."""
import math

import numpy as np

from oracle import basis
from oracle.stepper import LSERK54_A, LSERK54_B, Tank, default_filter, filter_matrix, filter_response, lserk54


def test_gradient_exact_for_physical_linear_fields_on_curved_mesh():
    T = Tank(dict(cells_x=5, cells_z=3, order=5, x0=0.0, x1=3.0, h=1.0))
    m = T.m
    eta = 0.07 * np.cos(2 * np.pi * m.column_x() / 3.0) + 0.02 * np.sin(5 * m.column_x())
    X, Z = m.node_xz(eta)
    fx, fz = T.gradient(eta, 0.7 * X - 1.3 * Z + 0.2)
    np.testing.assert_allclose(fx, 0.7, atol=1e-11)
    np.testing.assert_allclose(fz, -1.3, atol=1e-11)


def test_slope_exact_on_polynomial_surface():
    T = Tank(dict(cells_x=4, cells_z=2, order=4, x0=0.0, x1=2.0, h=1.0))
    x = T.m.column_x()
    np.testing.assert_allclose(T.slope(0.1 * x - 0.02 * x ** 2), 0.1 - 0.04 * x, atol=1e-12)


def test_small_wave_keeps_linear_dispersion_over_one_period():
    """A small-amplitude progressive wave returns to its initial surface after one
    period of the linear dispersion relation omega^2 = g k tanh(k h)."""
    T = Tank(dict(cells_x=8, cells_z=2, order=6, x0=0.0, x1=2.0, h=1.0, periodic=True))
    amp, k = 1e-4, math.pi
    eta, u, w, om = T.linear_wave(amp, k)
    eta0 = eta.copy()
    steps = 100
    dt = 2 * math.pi / om / steps
    for _ in range(steps):
        eta, u, w, _ = T.step(eta, u, w, dt)
    assert np.max(np.abs(eta - eta0)) <= 2e-3 * amp
    # and half a period later the crest has become a trough
    for _ in range(steps // 2):
        eta, u, w, _ = T.step(eta, u, w, dt)
    assert np.max(np.abs(eta + eta0)) <= 3e-3 * amp


def test_filter_response_and_default_strength():
    P = 6
    Pc, alpha, beta = default_filter(P)
    S = filter_response(P, Pc, alpha, beta)
    assert Pc == 4 and beta == 8.0
    np.testing.assert_array_equal(S[:5], 1.0)
    assert abs(S[P] - 0.97) < 1e-15
    assert 0.97 < S[5] < 1.0
    # alpha = 0 is the identity
    np.testing.assert_allclose(filter_matrix(P, Pc, 0.0, beta), np.eye(P + 1), atol=1e-13)


def test_filter_scales_highest_mode_and_keeps_low_degree_polynomials():
    P = 5
    Pc, alpha, beta = default_filter(P)
    F = filter_matrix(P, Pc, alpha, beta)
    r, _ = basis.lgl_nodes_weights(P)
    V, _ = basis.vandermonde(P)
    np.testing.assert_allclose(F @ V[:, P], filter_response(P, Pc, alpha, beta)[P] * V[:, P], atol=1e-13)
    for deg in range(Pc + 1):
        np.testing.assert_allclose(F @ r ** deg, r ** deg, atol=1e-13)
    # on a mesh: fields polynomial of degree <= P_c in (x*, sigma) are unchanged, including
    # the averaging at shared nodes; the filtered surface likewise
    T = Tank(dict(cells_x=3, cells_z=2, order=P, x0=0.0, x1=3.0, h=1.0))
    x, sg = T.m.column_x(), T.m.row_sigma()
    X = np.repeat(x, T.m.NZ)
    S = np.tile(sg, T.m.NX)
    f = 0.3 + X ** 2 * S - 0.5 * X ** 3 + S ** 3
    np.testing.assert_allclose(T.filter_field(f, F), f, atol=1e-12)
    np.testing.assert_allclose(T.filter_surface(0.1 * x ** 3 - x, F), 0.1 * x ** 3 - x, atol=1e-12)


def test_filter_single_element_mode_product():
    """One element, no shared nodes: a product of Legendre modes i (x) j is scaled by S(i) S(j)."""
    P = 6
    Pc, alpha, beta = default_filter(P)
    S = filter_response(P, Pc, alpha, beta)
    T = Tank(dict(cells_x=1, cells_z=1, order=P, x0=0.0, x1=1.0, h=1.0))
    V, _ = basis.vandermonde(P)
    F = filter_matrix(P, Pc, alpha, beta)
    for i, j in [(6, 6), (5, 2), (0, 6), (3, 4)]:
        f = np.outer(V[:, i], V[:, j]).reshape(-1)   # node (ix, iz), z fastest
        np.testing.assert_allclose(T.filter_field(f, F), S[i] * S[j] * f, atol=1e-13)


def test_lserk54_is_fourth_order():
    """On y' = lam y one step multiplies by the stability polynomial R(z), z = lam dt: its
    Taylor coefficients up to z^4 are those of exp(z) (order four), the z^5 one is not 1/120
    (five stages, fourth order)."""
    zs = np.array([1e-2, 2e-2, -3e-2, 4e-2])
    R = np.array([lserk54(lambda y: (z * y[0],), [np.array([1.0])], 1.0)[0][0][0] for z in zs])
    taylor4 = 1 + zs + zs ** 2 / 2 + zs ** 3 / 6 + zs ** 4 / 24
    c5 = (R - taylor4) / zs ** 5
    np.testing.assert_allclose(c5, c5[0], rtol=2e-2)  # R is a degree-5 polynomial
    assert abs(c5[0] - 1 / 120) > 1e-4
    # exact polynomial coefficients from 5 points: degree 5 with the Taylor part up to z^4
    pts = np.array([0.1, 0.2, 0.3, 0.4, 0.5, 0.6])
    vals = [lserk54(lambda y: (z * y[0],), [np.array([1.0])], 1.0)[0][0][0] for z in pts]
    coef = np.polyfit(pts, vals, 5)[::-1]
    np.testing.assert_allclose(coef[:5], [1, 1, 1 / 2, 1 / 6, 1 / 24], atol=1e-9)
    assert len(LSERK54_A) == len(LSERK54_B) == 5 and LSERK54_A[0] == 0.0


def test_small_wave_keeps_linear_dispersion_with_lserk54():
    T = Tank(dict(cells_x=8, cells_z=2, order=6, x0=0.0, x1=2.0, h=1.0, periodic=True))
    amp, k = 1e-4, math.pi
    eta, u, w, om = T.linear_wave(amp, k)
    eta0 = eta.copy()
    steps = 60
    dt = 2 * math.pi / om / steps
    for _ in range(steps):
        eta, u, w, _ = T.step_lserk(eta, u, w, dt)
    assert np.max(np.abs(eta - eta0)) <= 3e-3 * amp


def test_mixed_stage_lserk_keeps_still_water_still():
    T = Tank(dict(cells_x=4, cells_z=2, order=4, x0=0.0, x1=2.0, h=1.0, periodic=True))
    z = np.zeros(T.m.NX), np.zeros(T.m.N), np.zeros(T.m.N)
    eta, u, w, ps = T.step_lserk_mixed(*z, 0.01)
    assert np.all(eta == 0.0) and np.all(u == 0.0) and np.all(w == 0.0)
    assert all(np.all(p == 0.0) for p in ps)


def test_small_wave_keeps_linear_dispersion_with_mixed_stage_lserk():
    """The paper's mixed-stage coupling (Sec. 3): a small wave returns after one linear
    period and is inverted half a period later."""
    T = Tank(dict(cells_x=8, cells_z=2, order=6, x0=0.0, x1=2.0, h=1.0, periodic=True))
    amp, k = 1e-4, math.pi
    eta, u, w, om = T.linear_wave(amp, k)
    eta0 = eta.copy()
    steps = 60
    dt = 2 * math.pi / om / steps
    for _ in range(steps):
        eta, u, w, _ = T.step_lserk_mixed(eta, u, w, dt)
    assert np.max(np.abs(eta - eta0)) <= 3e-3 * amp
    for _ in range(steps // 2):
        eta, u, w, _ = T.step_lserk_mixed(eta, u, w, dt)
    assert np.max(np.abs(eta + eta0)) <= 4e-3 * amp


def test_mixed_stage_stage_divergence_and_projection_agreement():
    """One mixed-stage LSERK step of a steep wave: after each stage the weak divergence on
    that stage's surface is the gradient-recovery error of the correction, far below that
    of u*; and the step agrees with the projection-form LSERK step (both consistent with
    the same equations) far below the wave's own change over the step."""
    T = Tank(dict(cells_x=8, cells_z=2, order=6, x0=0.0, x1=2.0, h=1.0, periodic=True))
    m = T.m
    amp, k = 0.03, math.pi
    eta, u, w, om = T.linear_wave(amp, k)
    dt = 2 * math.pi / om / 50
    free = ~m.dirichlet_mask()
    # first stage by hand: the divergence of u* and of u^(1) on the stage-1 surface
    rates = T.rates_without_dynamic_pressure(eta, u, w)
    b1 = LSERK54_B[0]
    eta1 = eta + b1 * dt * rates[0]
    us, ws = u + b1 * dt * rates[1], w + b1 * dt * rates[2]
    div_star = np.abs(m.rhs_divergence(eta1, us, ws)[free]).max()
    e1, u1, w1, ps = T.step_lserk_mixed(eta, u, w, dt)
    # replay the first stage of the step to get u^(1)
    px, pz = T.gradient(eta, ps[0])
    u_1, w_1 = us - b1 * dt * px / 999.70, ws - b1 * dt * pz / 999.70
    div_1 = np.abs(m.rhs_divergence(eta1, u_1, w_1)[free]).max()
    assert div_1 < 1e-2 * div_star, (div_1, div_star)
    e2, u2, w2, _ = T.step_lserk(eta, u, w, dt)
    change = np.abs(e2 - eta).max()
    assert np.abs(e1 - e2).max() < 1e-2 * change, (np.abs(e1 - e2).max(), change)


def test_gradient_exact_for_physical_linear_fields_over_sloped_bottom():
    """sigma_x = (h_x - sigma d_x) / d over a varying still-water depth (Sec. 2.2)."""
    import workloads as W
    bar = W.Bar(1.0, 0.6, 1.0, 2.0, 0.3, 0.2)
    T = Tank(dict(cells_x=6, cells_z=3, order=5, x0=0.0, x1=3.0, h=1.0, depth=bar))
    m = T.m
    eta = 0.05 * np.cos(2 * np.pi * m.column_x() / 3.0)
    X, Z = m.node_xz(eta)
    fx, fz = T.gradient(eta, 0.7 * X - 1.3 * Z + 0.2)
    np.testing.assert_allclose(fx, 0.7, atol=1e-10)
    np.testing.assert_allclose(fz, -1.3, atol=1e-10)


def test_still_water_over_bar_stays_still():
    import workloads as W
    wl = W.bar(8, 2, 4)
    T = Tank(dict(**wl.mesh_kwargs(), depth=wl.bathymetry))
    z = np.zeros(T.m.NX), np.zeros(T.m.N), np.zeros(T.m.N)
    eta, u, w, ps = T.step(*z, 0.01)
    assert np.all(eta == 0.0) and np.all(u == 0.0) and np.all(w == 0.0)
