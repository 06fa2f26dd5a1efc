"""GPU parity of the wave-tank stepper kernels (gradient recovery, surface slope, forcing,
stage rates, RK4 combination) against the oracle stepper (oracle/stepper.py).

Tolerances: the gradient and slope kernels compute the same sums as the oracle in another
order, so they agree to 1e-11 of the field's gradient scale; a full RK4 step also goes
through the pressure solve (GPU residual 1e-12 against the oracle's direct solve), so the
state after a few steps agrees to 1e-9 relative."""
import math

import numpy as np
import pytest
import torch

import paper_2411_14977_gb300.pmg as pmg
from oracle.stepper import Tank, default_filter as oracle_default_filter, filter_matrix
from paper_2411_14977_gb300.stepper import WaveTank, default_filter
import workloads as W
from tests.gpu_helpers import n, t

pytestmark = pytest.mark.gpu


def wave_workload(cells_x, cells_z, order, periodic, L=2.0):
    s = W.Surface(0.05, 2 * np.pi / L)
    return W.Workload(f"wave_{cells_x}x{cells_z}_p{order}", cells_x, cells_z, order, 0.0, L, 1.0, periodic,
                      W.BASE_SEED + 91, s, "div", velocity=W.Velocity.random(W.BASE_SEED + 92))


@pytest.mark.parametrize("periodic", [True, False])
@pytest.mark.parametrize("order", [2, 5, 8])
def test_gradient_and_slope_match_oracle(periodic, order):
    w = wave_workload(8 if periodic else 6, 3, order, periodic)
    S = pmg.Solver(**w.mesh_kwargs())
    T = Tank(w.mesh_kwargs())
    xc, sr = S.node_coords()
    eta = 0.08 * np.cos(2 * np.pi * xc / 2.0) + 0.03 * np.sin(6 * np.pi * xc / 2.0)
    f = W.normal(W.BASE_SEED + 93, S.n)
    S.set_geometry(t(eta))
    fx, fz = S.gradient(t(f))
    ox, oz = T.gradient(eta, f)
    scale = max(np.abs(ox).max(), np.abs(oz).max())
    np.testing.assert_allclose(n(fx), ox, rtol=0, atol=1e-11 * scale)
    np.testing.assert_allclose(n(fz), oz, rtol=0, atol=1e-11 * scale)
    ex = S.surface_slope()
    np.testing.assert_allclose(n(ex), T.slope(eta), rtol=0, atol=1e-12 * np.abs(T.slope(eta)).max())


@pytest.mark.parametrize("periodic", [True, False])
@pytest.mark.parametrize("order", [3, 6, 10])
def test_filter_matches_oracle(periodic, order):
    w = wave_workload(8 if periodic else 5, 3, order, periodic)
    S = pmg.Solver(**w.mesh_kwargs())
    T = Tank(w.mesh_kwargs())
    flt = default_filter(order, strength=0.5, beta=4.0)
    assert np.allclose(flt, oracle_default_filter(order, strength=0.5, beta=4.0), rtol=1e-15)
    S.set_filter(*flt)
    F = filter_matrix(order, *flt)
    f = W.normal(W.BASE_SEED + 94, S.n)
    eta = W.normal(W.BASE_SEED + 95, S.NX)
    np.testing.assert_allclose(n(S.filter(t(f))), T.filter_field(f, F), rtol=0, atol=1e-13 * np.abs(f).max())
    np.testing.assert_allclose(n(S.filter(t(eta), surface=True)), T.filter_surface(eta, F), rtol=0,
                               atol=1e-13 * np.abs(eta).max())
    with pytest.raises(pmg.PmgError):
        x = t(f)
        S.filter(x, out=x)
    with pytest.raises(pmg.PmgError):
        S.set_filter(order + 1, -1.0, 8.0)


@pytest.mark.parametrize("periodic,cells,filtered,scheme", [(True, (8, 2, 6), False, "rk4"),
                                                             (False, (5, 2, 5), False, "rk4"),
                                                             (True, (8, 2, 6), True, "rk4"),
                                                             (True, (8, 2, 6), False, "lserk54"),
                                                             (False, (5, 2, 5), True, "lserk54"),
                                                             (True, (8, 2, 6), False, "lserk54_mixed"),
                                                             (False, (5, 2, 5), False, "lserk54_mixed"),
                                                             (True, (8, 3, 4), True, "lserk54_mixed")])
def test_steps_match_oracle(periodic, cells, filtered, scheme):
    w = wave_workload(*cells, periodic)
    amp, k = 0.03, 2 * np.pi / 2.0
    flt = default_filter(cells[2]) if filtered else None
    tank = WaveTank(w, tol=1e-12, filter=flt, scheme=scheme)
    om = tank.set_linear_wave(amp, k)
    dt = 2 * math.pi / om / 40
    tank.dt = dt
    T = Tank(w.mesh_kwargs())
    eta, u, wv, om2 = T.linear_wave(amp, k)
    assert abs(om - om2) < 1e-14
    np.testing.assert_allclose(n(tank.eta), eta, rtol=0, atol=1e-15)
    np.testing.assert_allclose(n(tank.u), u, rtol=0, atol=1e-13)
    np.testing.assert_allclose(n(tank.wv), wv, rtol=0, atol=1e-13)
    F = filter_matrix(cells[2], *flt) if filtered else None
    for _ in range(3):
        tank.step()
        eta, u, wv, ps = {"rk4": T.step, "lserk54": T.step_lserk, "lserk54_mixed": T.step_lserk_mixed}[scheme](
            eta, u, wv, dt)
        if filtered:
            eta, u, wv = T.filter_surface(eta, F), T.filter_field(u, F), T.filter_field(wv, F)
    torch.cuda.synchronize()
    for a, b in ((tank.eta, eta), (tank.u, u), (tank.wv, wv)):
        err = np.abs(n(a) - b).max() / np.abs(b).max()
        assert err <= 1e-9, err
    # the last stage's pressure too
    err = np.abs(n(tank.p) - ps[-1]).max() / np.abs(ps[-1]).max()
    assert err <= 1e-9, err
    assert all(i["status"] == 0 for i in tank.solve_infos)


def test_axpy_and_invalid_length():
    w = wave_workload(4, 2, 4, True)
    S = pmg.Solver(**w.mesh_kwargs())
    x = torch.ones(S.n, dtype=torch.float64, device="cuda")
    y = torch.full((S.n,), 2.0, dtype=torch.float64, device="cuda")
    out = torch.empty_like(x)
    S.axpy(0.5, x, y, out)
    assert torch.all(out == 2.5)
    st = pmg.load().pmg_axpy(S._h, -1, 0.5, pmg._ptr(x), pmg._ptr(y), pmg._ptr(out), pmg._stream())
    assert st == pmg.PMG_ERR_INVALID


def test_untrained_predictor_keeps_previous_pressure_and_answer():
    """A network whose last layer is zero returns p_prev bit for bit; the stepper with it
    takes the same path as without (same iterations, same state)."""
    from paper_2411_14977_gb300.warmstart import WarmStart
    w = wave_workload(8, 2, 6, True)
    runs = []
    for use in (False, True):
        tank = WaveTank(w, tol=1e-10)
        tank.set_linear_wave(0.03, 2 * np.pi / 2.0)
        if use:
            tank.predictor = WarmStart(tank.NX, tank.NZ, period=6, hidden=16, taps=5, seed=3, s_eta=0.03, s_deta=0.003,
                                       s_p=999.7 * 9.81 * 0.03, s_dp=30.0)
            g = tank.predictor.predict(tank.eta, tank.eta_p, tank.etax, tank.u)
            assert torch.equal(g, tank.u)
        for _ in range(2):
            tank.step()
        runs.append((n(tank.eta), [i["iterations"] for i in tank.solve_infos]))
    np.testing.assert_array_equal(runs[0][0], runs[1][0])
    assert runs[0][1] == runs[1][1]


@pytest.mark.parametrize("precision", [pmg.PMG_FP64, pmg.PMG_MIXED_FP32])
@pytest.mark.parametrize("outer", [pmg.PMG_GMRES, pmg.PMG_PDC])
def test_mixed_stage_stepper_outer_methods(precision, outer):
    """The mixed-stage coupling with either nonsymmetric outer method and precision gives
    the oracle's state after a few steps; CG is refused by the mixed-stage operator."""
    w = wave_workload(8, 2, 6, True)
    amp, k = 0.03, 2 * np.pi / 2.0
    tank = WaveTank(w, tol=1e-12, scheme="lserk54_mixed", precision=precision, outer=outer)
    om = tank.set_linear_wave(amp, k)
    dt = 2 * math.pi / om / 40
    tank.dt = dt
    T = Tank(w.mesh_kwargs())
    eta, u, wv, _ = T.linear_wave(amp, k)
    for _ in range(2):
        tank.step()
        eta, u, wv, ps = T.step_lserk_mixed(eta, u, wv, dt)
    torch.cuda.synchronize()
    for a, b in ((tank.eta, eta), (tank.u, u), (tank.wv, wv)):
        assert np.abs(n(a) - b).max() / np.abs(b).max() <= 1e-9
    assert all(i["status"] == 0 for i in tank.solve_infos)
    with pytest.raises(pmg.PmgError):
        WaveTank(w, dt=0.01, scheme="lserk54_mixed", outer=pmg.PMG_PCG).step()


def test_gradient_over_bar_matches_oracle():
    w = W.bar(10, 2, 5)
    S = pmg.Solver(**w.mesh_kwargs())
    xc, sr = S.node_coords()
    F = w.fields(xc, sr)
    S.set_bathymetry(t(F["h"]))
    S.set_geometry(t(F["eta"]))
    T = Tank(dict(**w.mesh_kwargs(), depth=F["h"]))
    rng = np.random.default_rng(41)
    f = rng.standard_normal(T.m.N)
    fx, fz = S.gradient(t(f))
    rx, rz = T.gradient(F["eta"], f)
    sc = max(np.abs(rx).max(), np.abs(rz).max())
    assert np.abs(n(fx) - rx).max() <= 1e-11 * sc and np.abs(n(fz) - rz).max() <= 1e-11 * sc
    S.close()


@pytest.mark.parametrize("scheme", ["rk4", "lserk54"])
def test_steps_over_bar_match_oracle(scheme):
    """A surface hump on the bar's up-slope (Sec. 6 geometry) stepped by the projection
    schemes over the varying depth: GPU against the oracle after three steps."""
    w = W.bar(10, 2, 5)
    dt = 0.02
    tank = WaveTank(w, tol=1e-12, scheme=scheme, dt=dt)
    xc = tank.xc
    eta0 = 0.01 * np.exp(-((xc - 14.0) / 2.0) ** 2)
    zero = np.zeros(tank.N)
    tank.set_state(eta0, zero, zero)
    T = Tank(dict(**w.mesh_kwargs(), depth=w.depth(xc)))
    eta, u, wv = eta0.copy(), zero.copy(), zero.copy()
    for _ in range(3):
        tank.step()
        eta, u, wv, ps = {"rk4": T.step, "lserk54": T.step_lserk}[scheme](eta, u, wv, dt)
    torch.cuda.synchronize()
    for a, b in ((tank.eta, eta), (tank.u, u), (tank.wv, wv)):
        err = np.abs(n(a) - b).max() / np.abs(b).max()
        assert err <= 1e-9, err
    assert all(i["status"] == 0 for i in tank.solve_infos)


def test_mixed_stage_coupling_refuses_varying_depth():
    with pytest.raises(pmg.PmgError):
        tank = WaveTank(W.bar(6, 2, 4), dt=0.02, scheme="lserk54_mixed")
        tank.step()
