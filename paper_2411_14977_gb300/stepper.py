"""Wave-tank time stepper around the pressure solve (the workload that runs one
Poisson solve per Runge-Kutta stage).

Inviscid sigma-transformed INSE in the projection reading: per stage, with the static
pressure folded in (p = p_D + rho g (eta - z), Sec. 2.1),
    F      = -(u . grad) u - g eta_x e_x
    Delta p_D = rho div F,  p_D = 0 on the surface, d p_D/dn = rho n.F elsewhere
    du/dt  = F - grad p_D / rho + sigma eta_t du/dz        (at fixed sigma, Sec. 2.2)
    eta_t  = w - u eta_x                                   (kinematic condition, Eq. freesurf1)
advanced by the classical fourth-order Runge-Kutta method (four solves per step) or the
paper's LSERK(5,4) (five), optionally followed by the modal exponential cut-off filter of
eta, u and w (Sec. "Spectral Filtering").

scheme="lserk54_mixed" is the paper's own mixed-stage pressure-velocity coupling (Sec. 3,
Eq. rkforc1 to Eq. bcpdneu): stage k advances eta by the kinematic condition, forms u* of
Eq. rkforc1 with every force except the dynamic pressure, solves the mixed-stage Poisson
problem  int grad^k v . grad^(k-1) p = rho/(beta_k dt) int grad^k v . u*  (nonsymmetric:
outer PDC or GMRES) and sets u^(k) = u* - (beta_k dt/rho) grad^(k-1) p.  All
arithmetic runs in the library's kernels; this module orders the calls.  Each solve is
warm-started from the previous stage's pressure, optionally corrected by a learned
predictor (paper_2411_14977_gb300.warmstart).
"""
import math

import numpy as np
import torch

from . import pmg

G = 9.81
RHO = 999.70


# Five-stage fourth-order 2N-storage Runge-Kutta of Carpenter & Kennedy (1994), the
# paper's time integrator (Sec. 3): K <- a_k K + dt f(y), y <- y + b_k K.
LSERK_A = (0.0, -567301805773.0 / 1357537059087.0, -2404267990393.0 / 2016746695238.0,
           -3550918686646.0 / 2091501179385.0, -1275806237668.0 / 842570457699.0)
LSERK_B = (1432997174477.0 / 9575080441755.0, 5161836677717.0 / 13612068292357.0,
           1720146321549.0 / 2090206949498.0, 3134564353537.0 / 4481467310338.0,
           2277821191437.0 / 14882151754819.0)


def default_filter(P, strength=0.97, beta=8.0):
    """(cutoff, alpha, beta): modes above P - 2 damped, the highest by the factor `strength`."""
    cutoff = max(P - 2, 0)
    return cutoff, math.log(strength) / ((P - cutoff) / (P + 1 - cutoff)) ** beta, beta


class WaveTank:
    def __init__(self, workload, dt=None, device="cuda", predictor=None, record=False, guess_policy="residual",
                 filter=None, filter_stages=False, scheme="rk4", guess_smooth=None, **solver_opts):
        if scheme not in ("rk4", "lserk54", "lserk54_mixed"):
            raise ValueError("scheme: rk4, lserk54 or lserk54_mixed")
        self.scheme = scheme
        self.w = workload
        if scheme == "lserk54_mixed":
            solver_opts.setdefault("outer", pmg.PMG_GMRES)  # the mixed-stage operator is nonsymmetric
        self.S = pmg.Solver(**workload.mesh_kwargs(), **solver_opts)
        S = self.S
        self.dev = torch.device(device)
        self.xc, self.sr = S.node_coords()
        if workload.bathymetry is not None:  # varying still-water depth (projection schemes)
            self.depth = torch.as_tensor(workload.depth(self.xc), dtype=torch.float64, device=self.dev)
            S.set_bathymetry(self.depth)
        f64 = dict(dtype=torch.float64, device=self.dev)
        self.N, self.NX, self.NZ = S.n, S.NX, S.NZ
        z = lambda n=None: torch.zeros(self.N if n is None else n, **f64)
        self.eta, self.u, self.wv = z(self.NX), z(), z()
        self.p = z()                        # last stage's dynamic pressure (warm start)
        self.eta_p = z(self.NX)             # the surface that pressure was solved on
        self.pD = z()                       # p_D = 0 on the surface
        self.buf = {k: z() for k in ("ux", "uz", "wx", "wz", "Fu", "Fw", "b", "px", "pz", "zero", "us", "ws")}
        self.eta_km1 = z(self.NX)           # stage-(k-1) surface of the mixed-stage coupling
        self.etax = z(self.NX)
        self.k = [(z(self.NX), z(), z()) for _ in range(4)]
        self.ys = (z(self.NX), z(), z())
        self.acc = (z(self.NX), z(), z())
        self.dt = dt
        self.predictor = predictor
        # "residual": use the network's guess only where its residual is smaller than that
        # of the previous pressure; after `probe_after` rejections in a row the network is
        # consulted only on every `probe_every`-th solve until it wins again (its checks
        # cost two operator applications); "always": use it unconditionally
        self.guess_policy = guess_policy
        self.probe_after, self.probe_every = 8, 16
        self._rejected = 0
        self._skipped = 0
        # guess_smooth = (cutoff, alpha, beta): the predictor's change of the pressure is
        # passed through this per-element modal low-pass (pmg_filter on a second handle of
        # the same mesh) before it is used, so that no node-scale roughness reaches x0
        self.S_smooth = None
        if guess_smooth is not None:
            self.S_smooth = pmg.Solver(**workload.mesh_kwargs())
            self.S_smooth.set_filter(*guess_smooth)
        self.record = record
        self.samples = []                   # (eta, eta_prev, eta_x, p_prev, p) per solve when recording
        self.solve_infos = []
        self.guess_log = []                 # (residual of p_prev, residual of the network's guess)
        self.t = 0.0
        # spectral filter after every step: None, or (cutoff, alpha, beta)
        self.filter = filter
        self.filter_stages = filter_stages     # also filter every intermediate stage state
        if filter is not None:
            S.set_filter(*filter)
            self.ftmp = (z(self.NX), z(), z())

    def set_state(self, eta, u, w):
        """Initial surface (NX) and velocities (N), any array-likes."""
        for dst, src in ((self.eta, eta), (self.u, u), (self.wv, w)):
            dst.copy_(torch.as_tensor(np.asarray(src, dtype=np.float64)))
        self.eta_p.copy_(self.eta)

    def set_linear_wave(self, amp, k):
        """Linear-theory progressive wave eta = a cos(kx) with its velocity field."""
        h = self.w.h
        om = math.sqrt(G * k * math.tanh(k * h))
        X = np.repeat(self.xc, self.NZ)
        eta0 = amp * np.cos(k * self.xc)
        Z = (self.sr[None, :] * (eta0 + h)[:, None] - h).reshape(-1)
        u = amp * om * np.cosh(k * (Z + h)) / np.sinh(k * h) * np.cos(k * X)
        w = amp * om * np.sinh(k * (Z + h)) / np.sinh(k * h) * np.sin(k * X)
        self.eta.copy_(torch.from_numpy(eta0))
        self.eta_p.copy_(self.eta)
        self.u.copy_(torch.from_numpy(u))
        self.wv.copy_(torch.from_numpy(w))
        if self.dt is None:
            self.dt = 2 * math.pi / om / 100.0
        return om

    def _forces(self, eta, u, w):
        """Velocity gradients, surface slope and the forcing F on the surface eta."""
        S, B = self.S, self.buf
        S.set_geometry(eta)
        S.gradient(u, B["ux"], B["uz"])
        S.gradient(w, B["wx"], B["wz"])
        S.surface_slope(self.etax)
        S.forcing(u, w, B["ux"], B["uz"], B["wx"], B["wz"], self.etax, G, B["Fu"], B["Fw"])

    def smooth_change(self, p, p_prev):
        """p_prev + F(p - p_prev) with the guess low-pass F (guess_smooth)."""
        d = p - p_prev
        out = torch.empty_like(d)
        self.S_smooth.filter(d, out)
        return p_prev + out

    def _predict(self, eta):
        guess = self.predictor.predict(eta, self.eta_p, self.etax, self.p)
        return guess if self.S_smooth is None else self.smooth_change(guess, self.p)

    def _solve(self, eta):
        """Pressure solve of the right-hand side in buf["b"] on the operator set last, from the
        previous pressure or the predictor's guess; the result replaces self.p."""
        S, B = self.S, self.buf
        x0 = self.p
        if self.predictor is not None:
            # keep the network's guess only where its residual beats the previous pressure
            if self.guess_policy == "always":
                x0 = self._predict(eta)
            elif self._rejected < self.probe_after or self._skipped + 1 >= self.probe_every:
                self._skipped = 0
                guess = self._predict(eta)
                r_nn = S.residual_norm(B["b"], self.pD, guess)
                r_prev = S.residual_norm(B["b"], self.pD, self.p)
                self.guess_log.append((r_prev, r_nn))
                if r_nn < r_prev:
                    x0 = guess
                    self._rejected = 0
                else:
                    self._rejected += 1
            else:
                self._skipped += 1
        prev = (self.eta_p.clone(), self.p.clone()) if self.record else None
        _, info = S.solve(B["b"], self.pD, x0=x0, out=self.p)
        self.eta_p.copy_(eta)
        self.solve_infos.append(info)
        if self.record:
            self.samples.append((eta.clone(), prev[0], self.etax.clone(), prev[1], self.p.clone()))

    def rates(self, eta, u, w, out):
        S, B = self.S, self.buf
        deta, du, dw = out
        self._forces(eta, u, w)
        S.assemble_rhs_div(B["Fu"], B["Fw"], RHO, out=B["b"])
        self._solve(eta)
        S.gradient(self.p, B["px"], B["pz"])
        S.stage_rates(u, w, B["uz"], B["wz"], B["Fu"], B["Fw"], B["px"], B["pz"], self.etax, RHO, du, dw, deta)

    def step(self):
        """One time step: classical RK4 (four pressure solves) or LSERK(5,4) (five, projection
        or mixed-stage coupling)."""
        if self.scheme == "lserk54":
            return self._step_lserk()
        if self.scheme == "lserk54_mixed":
            return self._step_lserk_mixed()
        S, dt = self.S, self.dt
        y = (self.eta, self.u, self.wv)
        cs = (0.5, 0.5, 1.0)
        wts = (1.0, 2.0, 2.0, 1.0)
        for a in self.acc:
            a.zero_()
        cur = y
        for s in range(4):
            self.rates(*cur, self.k[s])
            for a, kk in zip(self.acc, self.k[s]):
                S.axpy(wts[s] * dt / 6.0, kk, a, a)
            if s < 3:
                for ys, yy, kk in zip(self.ys, y, self.k[s]):
                    S.axpy(cs[s] * dt, kk, yy, ys)
                if self.filter is not None and self.filter_stages:
                    self._filter(self.ys)
                cur = self.ys
        for yy, a in zip(y, self.acc):
            S.axpy(1.0, a, yy, yy)
        if self.filter is not None:
            self._filter(y)
        self.t += dt

    def _step_lserk(self):
        S, dt = self.S, self.dt
        y = (self.eta, self.u, self.wv)
        K, kk = self.acc, self.k[0]
        for a, b in zip(LSERK_A, LSERK_B):
            self.rates(*y, kk)
            for Kv, r in zip(K, kk):
                if a == 0.0:
                    Kv.zero_()
                else:
                    S.axpy(a - 1.0, Kv, Kv, Kv)  # K <- a K
                S.axpy(dt, r, Kv, Kv)            # K <- K + dt f
            for yy, Kv in zip(y, K):
                S.axpy(b, Kv, yy, yy)            # y <- y + b K
        if self.filter is not None:
            self._filter(y)
        self.t += dt

    def _step_lserk_mixed(self):
        S, B, dt = self.S, self.buf, self.dt
        K, r = self.acc, self.k[0]
        for a, b in zip(LSERK_A, LSERK_B):
            self.eta_km1.copy_(self.eta)
            # f(q^(k-1)) without the dynamic pressure, on the stage-(k-1) surface
            self._forces(self.eta, self.u, self.wv)
            S.stage_rates(self.u, self.wv, B["uz"], B["wz"], B["Fu"], B["Fw"], B["zero"], B["zero"], self.etax, RHO,
                          r[1], r[2], r[0])
            for Kv, rv in zip(K, r):
                if a == 0.0:
                    Kv.zero_()
                else:
                    S.axpy(a - 1.0, Kv, Kv, Kv)      # K <- a K
                S.axpy(dt, rv, Kv, Kv)               # K <- K + dt f
            S.axpy(b, K[0], self.eta, self.eta)      # eta^(k)
            S.axpy(b, K[1], self.u, B["us"])         # u* = u^(k-1) + b K
            S.axpy(b, K[2], self.wv, B["ws"])
            # int grad^k v . grad^(k-1) p = rho/(b dt) int grad^k v . u*
            S.set_geometry_mixed(self.eta, self.eta_km1)
            S.assemble_rhs_div(B["us"], B["ws"], RHO / (b * dt), out=B["b"])
            self._solve(self.eta)
            # K <- K - dt grad^(k-1) p / rho;  u^(k) = u^(k-1) + b K
            S.set_geometry(self.eta_km1)
            S.gradient(self.p, B["px"], B["pz"])
            S.axpy(-dt / RHO, B["px"], K[1], K[1])
            S.axpy(-dt / RHO, B["pz"], K[2], K[2])
            S.axpy(b, K[1], self.u, self.u)
            S.axpy(b, K[2], self.wv, self.wv)
        if self.filter is not None:
            self._filter((self.eta, self.u, self.wv))
        self.t += dt

    def _filter(self, state):
        for i, (yy, tmp) in enumerate(zip(state, self.ftmp)):
            self.S.filter(yy, tmp, surface=(i == 0))
            yy.copy_(tmp)
