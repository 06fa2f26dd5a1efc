"""GPU parity of the warm-start network kernels (forward, backward, Adam, packing)
against the FP64 oracle (oracle/nn.py), and the gain test on a small wave tank.

FP32 tolerances: forward outputs within 1e-5 of the output scale (unit roundoff 6e-8
times contraction depths of a few hundred); gradients per layer within 1e-4 relative in
the 2-norm (the backward pass adds two more contractions and the tanh derivative)."""
import math

import numpy as np
import pytest
import torch

from oracle import nn
from paper_2411_14977_gb300.pmg import load
from paper_2411_14977_gb300.warmstart import WarmStart
import workloads as W
from tests.gpu_helpers import n, t

pytestmark = pytest.mark.gpu

DIMS = [  # (X, NZ, H, K, S): tile-ragged positions and channels
    (70, 13, 24, 5, 3),
    (17, 4, 8, 3, 1),
    (130, 9, 65, 1, 2),
]


def _setup(X, NZ, H, K, S, seed):
    ws = WarmStart(X, NZ, period=1, hidden=H, taps=K, max_batch=max(S, 1), seed=seed)
    C = NZ + 4
    flat = 0.3 * W.normal(seed, ws.n_params)
    ws.set_params(torch.from_numpy(flat))
    Xin = W.normal(seed + 1, S * C * X).reshape(S, C, X)
    T = W.normal(seed + 2, S * NZ * X).reshape(S, NZ, X)
    return ws, nn.unflatten(flat.astype(np.float32).astype(np.float64), C, H, NZ, K), Xin, T


@pytest.mark.parametrize("dims", DIMS)
def test_forward_matches_oracle(dims):
    X, NZ, H, K, S = dims
    ws, p, Xin, _ = _setup(*dims, seed=W.BASE_SEED + 100)
    Xf = Xin.astype(np.float32)
    y = n(ws.forward(t(Xf.reshape(S, -1), torch.float32))).reshape(S, NZ, X)
    ref, _ = nn.forward(p, Xf.astype(np.float64))
    assert np.abs(y - ref).max() <= 1e-5 * np.abs(ref).max()


@pytest.mark.parametrize("lam", [0.0, 0.5])
@pytest.mark.parametrize("dims", DIMS)
def test_gradients_match_oracle(dims, lam):
    X, NZ, H, K, S = dims
    ws, p, Xin, T = _setup(*dims, seed=W.BASE_SEED + 110)
    load().pmg_ws_set_roughness(ws._w, lam)
    Xf, Tf = Xin.astype(np.float32), T.astype(np.float32)
    loss, g = ws.gradients(t(Xf.reshape(S, -1), torch.float32), t(Tf.reshape(S, -1), torch.float32))
    ref_loss, ref = nn.loss_and_grads(p, Xf.astype(np.float64), Tf.astype(np.float64), lam)
    assert abs(loss - ref_loss) <= 1e-5 * ref_loss
    C = NZ + 4
    got = nn.unflatten(n(g), C, H, NZ, K)
    for name, _ in nn.shapes(C, H, NZ, K):
        e = np.linalg.norm(got[name] - ref[name]) / np.linalg.norm(ref[name])
        assert e <= 1e-4, (name, e)


def test_adam_step_matches_oracle():
    X, NZ, H, K, S = DIMS[0]
    ws, p, Xin, T = _setup(X, NZ, H, K, S, seed=W.BASE_SEED + 120)
    C = NZ + 4
    Xf, Tf = Xin.astype(np.float32), T.astype(np.float32)
    flat0 = nn.flatten(p, C, H, NZ, K)
    lr = 1e-3
    p_cur, m, v = flat0.copy(), np.zeros_like(flat0), np.zeros_like(flat0)
    for step in (1, 2):
        ws.train_step(t(Xf.reshape(S, -1), torch.float32), t(Tf.reshape(S, -1), torch.float32), lr)
        _, g = nn.loss_and_grads(nn.unflatten(p_cur, C, H, NZ, K), Xf.astype(np.float64), Tf.astype(np.float64))
        gflat = nn.flatten(g, C, H, NZ, K)
        p_cur, m, v = nn.adam(p_cur, gflat, m, v, step, lr)
        got = n(ws.get_params())
        # |update| <= lr by Adam's bound; where the gradient is not tiny the FP32 update
        # agrees with the FP64 one to 1e-3 relative
        big = np.abs(gflat) > 1e-3 * np.sqrt(np.mean(gflat ** 2))
        d_got, d_ref = got - flat0, p_cur - flat0
        assert np.all(np.abs(d_got) <= step * lr * (1 + 1e-3) + 1e-6 * np.abs(flat0))
        np.testing.assert_allclose(d_got[big], d_ref[big], rtol=0, atol=1e-3 * step * lr + 1e-6 * np.abs(flat0[big]).max())


SC = dict(s_eta=0.04, s_deta=0.004, s_p=390.0, s_dp=20.0)


def test_pack_target_predict_match_oracle(tmp_path):
    NX, NZ = 37, 7
    ws = WarmStart(NX, NZ, period=4, hidden=12, taps=3, seed=9, **SC)
    eta, etax = 0.04 * W.normal(1, NX), 0.1 * W.normal(2, NX)
    eta_p = eta + 0.004 * W.normal(6, NX)
    pp, p = 390.0 * W.normal(3, NX * NZ), 390.0 * W.normal(4, NX * NZ)
    got = n(ws.pack(t(eta), t(eta_p), t(etax), t(pp))).reshape(NZ + 7, NX)
    ref = nn.pack(eta, eta_p, etax, pp, NZ, 4, SC["s_eta"], SC["s_deta"], SC["s_p"])
    np.testing.assert_allclose(got, ref, rtol=1e-7, atol=0)
    got_t = n(ws.target(t(p), t(pp))).reshape(NZ, NX)
    np.testing.assert_allclose(got_t, nn.target(p, pp, NZ, SC["s_dp"]), rtol=1e-7, atol=1e-30)
    # untrained network (zero last layer): the guess is p_prev exactly
    assert torch.equal(ws.predict(t(eta), t(eta_p), t(etax), t(pp)), t(pp))
    # random parameters: guess = p_prev + s_dp * net(input)
    flat = 0.3 * W.normal(5, ws.n_params)
    ws.set_params(torch.from_numpy(flat))
    prm = nn.unflatten(flat.astype(np.float32).astype(np.float64), NZ + 7, 12, NZ, 3)
    y, _ = nn.forward(prm, ref.astype(np.float32).astype(np.float64)[None])
    g_ref = nn.guess(pp, y[0], NZ, SC["s_dp"])
    g = n(ws.predict(t(eta), t(eta_p), t(etax), t(pp)))
    assert np.abs(g - g_ref).max() <= 1e-5 * SC["s_dp"] * np.abs(y).max()
    # save / load round trip
    ws.save(tmp_path / "w.bin")
    ws2 = WarmStart(NX, NZ, period=4, hidden=12, taps=3, seed=10, **SC)
    ws2.load(tmp_path / "w.bin")
    assert torch.equal(ws2.get_params(), ws.get_params())
    ws3 = WarmStart(NX, NZ, period=4, hidden=13, taps=3, seed=10, **SC)
    with pytest.raises(Exception):
        ws3.load(tmp_path / "w.bin")


def wave_scales(amp, om, dt):
    """Input / output scales of a wave of amplitude amp and frequency om stepped by dt."""
    from paper_2411_14977_gb300.stepper import G, RHO
    return dict(s_eta=amp, s_deta=amp * om * dt, s_p=RHO * G * amp, s_dp=RHO * G * amp * om * dt)


def test_warm_start_no_regression_against_previous_pressure():
    """Train on recorded stage solves of a small periodic wave tank, then continue from the
    same state with and without the network.  What this asserts: the network fits the
    pressure change far better than the previous pressure does (L2 loss down by 100x),
    and with the residual fallback the learned warm start causes NO REGRESSION -- the
    solves never take more iterations than from the previous pressure, and the state is
    the same to the solve tolerance.  It does not assert a gain: on these workloads the
    fallback rejects the network's guesses (their residual is above the previous
    pressure's), so the iteration counts are equal; the counts and the residual ratio are
    printed."""
    from paper_2411_14977_gb300.stepper import WaveTank
    L, amp = 4.0, 0.04
    w = W.Workload("gain_32x2_p6", 32, 2, 6, 0.0, L, 1.0, True, W.BASE_SEED + 130, W.Surface(amp, 2 * np.pi / L),
                   "div", velocity=W.Velocity.random(W.BASE_SEED + 131))
    tank = WaveTank(w, tol=1e-10, record=True)
    om = tank.set_linear_wave(amp, 2 * np.pi / L)
    tank.dt = 2 * math.pi / om / 60
    for _ in range(30):
        tank.step()
    ws = WarmStart(tank.NX, tank.NZ, period=6, hidden=32, taps=5, max_batch=32, seed=4, roughness=10.0,
                   **wave_scales(amp, om, tank.dt))
    hist = ws.fit(tank.samples[4:], epochs=150, batch=16, lr=2e-3)
    state = [x.clone() for x in (tank.eta, tank.u, tank.wv, tank.p, tank.eta_p)]
    res = []
    for pred in (None, ws):
        for x, x0 in zip((tank.eta, tank.u, tank.wv, tank.p, tank.eta_p), state):
            x.copy_(x0)
        tank.predictor, tank.record = pred, False
        tank.solve_infos, tank.guess_log = [], []
        for _ in range(8):
            tank.step()
        res.append((n(tank.eta), sum(i["iterations"] for i in tank.solve_infos), list(tank.guess_log)))
    (eta_a, it_a, _), (eta_b, it_b, log) = res
    print("loss", hist[0], hist[-1], "iterations", it_a, it_b,
          "median residual ratio", float(np.median([r_nn / r_prev for r_prev, r_nn in log])))
    assert hist[-1] < 0.01 * hist[0]
    assert 0 < len(log) <= 32
    assert np.abs(eta_a - eta_b).max() <= 1e-6 * amp
    assert it_b <= it_a, (it_b, it_a)
