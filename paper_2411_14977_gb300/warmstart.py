"""Learned initial guess for the pressure solve of the wave-tank stepper.

Successive Runge-Kutta stages solve nearly the same Poisson problem, so the previous
stage's pressure is already a good initial guess; a small periodic 1D convolutional
network over the node columns learns the remaining change from the surface, its change
since the previous solve, its slope and the previous pressure.
The network, its backward pass and the Adam optimiser are the library's FP32 kernels
(pmg_ws_* in include/pmg.h); this module marshals arguments and batches training
samples.  The solve that follows always iterates to the requested residual, so the
predictor can only change how many iterations it takes, never the pressure it returns.
"""
import ctypes

import torch

from . import pmg
from .pmg import _check, _ptr, _stream, load


class WarmStart:
    def __init__(self, n_cols, col_len, period=1, hidden=128, taps=5, max_batch=64, seed=1, s_eta=1.0, s_deta=1.0,
                 s_p=1.0, s_dp=1.0, roughness=0.0):
        self.X, self.NZ, self.Q, self.H, self.K = n_cols, col_len, period, hidden, taps
        self.C = col_len + 3 + period
        self.max_batch = max_batch
        self.scales = (s_eta, s_deta, s_p, s_dp)
        h = ctypes.c_void_p()
        _check(load().pmg_ws_create(n_cols, col_len, period, hidden, taps, max_batch, seed, float(s_eta), float(s_deta),
                                    float(s_p), float(s_dp), ctypes.byref(h)))
        self._w = h
        _check(load().pmg_ws_set_roughness(self._w, float(roughness)))
        n = ctypes.c_int64()
        _check(load().pmg_ws_num_params(self._w, ctypes.byref(n)))
        self.n_params = n.value
        self.adam_steps = 0

    def close(self):
        if getattr(self, "_w", None):
            load().pmg_ws_destroy(self._w)
            self._w = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- parameters
    def get_params(self):
        out = torch.empty(self.n_params, dtype=torch.float32)
        _check(load().pmg_ws_get_params(self._w, ctypes.c_void_p(out.data_ptr())))
        return out

    def set_params(self, flat):
        flat = flat.detach().to(torch.float32).contiguous().cpu()
        if flat.numel() != self.n_params:
            raise ValueError("parameter count mismatch")
        _check(load().pmg_ws_set_params(self._w, ctypes.c_void_p(flat.data_ptr())))

    def layer_shapes(self):
        X, C, H, K, NZ = self.X, self.C, self.H, self.K, self.NZ
        return [("W1", (H, C, K)), ("b1", (H,)), ("W2", (H, H, K)), ("b2", (H,)), ("W3", (NZ, H, 1)), ("b3", (NZ,))]

    def save(self, path):
        _check(load().pmg_ws_save(self._w, str(path).encode()))

    def load(self, path):
        _check(load().pmg_ws_load(self._w, str(path).encode()))

    # ---- data
    def pack(self, eta, eta_prev, etax, p_prev, out=None):
        out = torch.empty(self.C * self.X, dtype=torch.float32, device=eta.device) if out is None else out
        _check(load().pmg_ws_pack(self._w, _ptr(eta), _ptr(eta_prev), _ptr(etax), _ptr(p_prev),
                                  _ptr(out, torch.float32), _stream()))
        return out

    def target(self, p, p_prev, out=None):
        out = torch.empty(self.NZ * self.X, dtype=torch.float32, device=p.device) if out is None else out
        _check(load().pmg_ws_target(self._w, _ptr(p), _ptr(p_prev), _ptr(out, torch.float32), _stream()))
        return out

    def forward(self, inputs):
        """inputs (S, C*X) float32 -> outputs (S, NZ*X) float32."""
        S = inputs.shape[0]
        out = torch.empty(S, self.NZ * self.X, dtype=torch.float32, device=inputs.device)
        _check(load().pmg_ws_forward(self._w, _ptr(inputs, torch.float32), S, _ptr(out, torch.float32), _stream()))
        return out

    def predict(self, eta, eta_prev, etax, p_prev, out=None):
        out = torch.empty_like(p_prev) if out is None else out
        _check(load().pmg_ws_predict(self._w, _ptr(eta), _ptr(eta_prev), _ptr(etax), _ptr(p_prev), _ptr(out),
                                     _stream()))
        return out

    def gradients(self, inputs, targets):
        """(loss, flat gradient) of the mean-squared error of a batch (one forward+backward)."""
        S = inputs.shape[0]
        g = torch.empty(self.n_params, dtype=torch.float32, device=inputs.device)
        loss = ctypes.c_double()
        _check(load().pmg_ws_gradients(self._w, _ptr(inputs, torch.float32), _ptr(targets, torch.float32), S,
                                       _ptr(g, torch.float32), ctypes.byref(loss), _stream()))
        return loss.value, g

    def train_step(self, inputs, targets, lr=1e-3):
        S = inputs.shape[0]
        loss = ctypes.c_double()
        _check(load().pmg_ws_train_step(self._w, _ptr(inputs, torch.float32), _ptr(targets, torch.float32), S,
                                        float(lr), ctypes.byref(loss), _stream()))
        self.adam_steps += 1
        return loss.value

    def dataset(self, samples):
        """Stack (eta, eta_prev, eta_x, p_prev, p) samples into (inputs, targets) on the device."""
        ins = torch.stack([self.pack(e, ep, ex, pp) for e, ep, ex, pp, _ in samples])
        tgs = torch.stack([self.target(p, pp) for _, _, _, pp, p in samples])
        return ins, tgs

    def fit(self, samples, epochs=200, batch=32, lr=1e-3, seed=0):
        """Adam over shuffled mini-batches; returns the loss history (one value per step)."""
        ins, tgs = self.dataset(samples)
        gen = torch.Generator().manual_seed(seed)
        hist = []
        n = ins.shape[0]
        batch = min(batch, self.max_batch, n)
        for _ in range(epochs):
            perm = torch.randperm(n, generator=gen).to(ins.device)
            for i in range(0, n - batch + 1, batch):
                idx = perm[i:i + batch]
                hist.append(self.train_step(ins[idx].contiguous(), tgs[idx].contiguous(), lr))
        return hist
