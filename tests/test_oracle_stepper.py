"""Pins of the oracle's wave-tank stepper (Sec. 2.1-2.2, Sec. 3, Eq. freesurf1)."""
import math

import numpy as np

from oracle.stepper import Tank


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
