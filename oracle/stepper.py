"""Wave-tank time stepper, FP64 numpy (test infrastructure; see oracle/__init__).

Inviscid sigma-transformed INSE (Sec. 2.1-2.2) in the projection reading: per stage
    F = -(u . grad) u - g eta_x e_x                    (p = p_D + rho g (eta - z))
    Delta p_D = rho div F, p_D = 0 on the surface, d p_D/dn = rho n.F elsewhere
    du/dt|sigma = F - grad p_D / rho + sigma eta_t du/dz,   eta_t = w - u eta_x  (Eq. freesurf1)
with nodal gradients by the lumped-mass L2 projection (element-local derivatives of the
isoparametric map, mean over the elements of a node) and classical RK4.  The pressure is
the exact solution of the discrete system (sparse LU).

Spectral filter (Sec. "Spectral Filtering"): per element, F = V diag(S) V^{-1} with the
exponential cut-off S(i) = 1 for i <= P_c, exp(alpha ((i - P_c)/(P + 1 - P_c))^beta) above,
applied as F (x) F to u, w and as F to eta, followed by the mean at shared nodes.

Time stepping: classical RK4, or the paper's five-stage fourth-order low-storage scheme
(LSERK(5,4), Carpenter & Kennedy 1994), with the projection above per stage or with the
paper's mixed-stage pressure-velocity coupling (Sec. 3, Eq. rkforc1 to Eq. bcpdneu): stage k
advances eta by the kinematic condition, forms the velocity u* of Eq. rkforc1 with every
force except the dynamic pressure, solves the mixed-stage Poisson problem
    int_{Omega^k} grad^k v . grad^(k-1) p = rho / (beta_k dt) int_{Omega^k} grad^k v . u*
(the weak form of Eq. poissonp; its boundary terms are the Neumann data of Eq. bcpdneu),
and sets u^(k) = u* - (beta_k dt / rho) grad^(k-1) p, the dynamic-pressure force of
f(q^(k-1)) taken on the stage-(k-1) surface.

Pins (tests/test_oracle_stepper.py): exact gradients of physical linear functions on a
curved mesh; a small-amplitude wave keeps the linear dispersion relation over a period;
the filter keeps polynomials of degree <= P_c, scales mode P by S(P), and is the
identity for alpha = 0; LSERK(5,4) has order four on y' = lambda y (stability polynomial
matches exp to z^4) and keeps the dispersion relation like RK4; the mixed-stage coupling
keeps still water still, keeps the dispersion relation, removes the stage-k divergence of
u* down to the gradient-recovery error, and tracks the projection-form LSERK.
"""
import math

import numpy as np

from . import basis
from .sem import Mesh, solve_direct

G = 9.81
RHO = 999.70


# Five-stage fourth-order 2N-storage Runge-Kutta (Carpenter & Kennedy 1994), the scheme of
# the paper's time stepping (Sec. 3): K <- a_k K + dt f(y), y <- y + b_k K.
LSERK54_A = (0.0, -567301805773.0 / 1357537059087.0, -2404267990393.0 / 2016746695238.0,
             -3550918686646.0 / 2091501179385.0, -1275806237668.0 / 842570457699.0)
LSERK54_B = (1432997174477.0 / 9575080441755.0, 5161836677717.0 / 13612068292357.0,
             1720146321549.0 / 2090206949498.0, 3134564353537.0 / 4481467310338.0,
             2277821191437.0 / 14882151754819.0)


def lserk54(f, y, dt):
    """One LSERK(5,4) step of y' = f(y) for a list of arrays y; returns (y_new, stage extras):
    f returns (rates..., extra) with one rate per component of y."""
    K = [np.zeros_like(v) for v in y]
    y = [np.array(v, dtype=np.float64, copy=True) for v in y]
    extras = []
    for a, b in zip(LSERK54_A, LSERK54_B):
        out = f(y)
        rates, extra = out[:len(y)], out[len(y):]
        K = [a * Kv + dt * r for Kv, r in zip(K, rates)]
        y = [v + b * Kv for v, Kv in zip(y, K)]
        extras.append(extra)
    return y, extras


def filter_response(P, cutoff, alpha, beta):
    """S(i), i = 0..P: the exponential cut-off of the modal coefficients."""
    i = np.arange(P + 1, dtype=np.float64)
    S = np.ones(P + 1)
    hi = i > cutoff
    S[hi] = np.exp(alpha * ((i[hi] - cutoff) / (P + 1 - cutoff)) ** beta)
    return S


def filter_matrix(P, cutoff, alpha, beta):
    """Nodal filter V diag(S) V^{-1} at the LGL nodes of order P."""
    V, _ = basis.vandermonde(P)
    return V @ np.diag(filter_response(P, cutoff, alpha, beta)) @ np.linalg.inv(V)


def default_filter(P, strength=0.97, beta=8.0):
    """(P_c, alpha, beta) with P_c = P - 2 and S(P) = strength."""
    cutoff = max(P - 2, 0)
    return cutoff, math.log(strength) / ((P - cutoff) / (P + 1 - cutoff)) ** beta, beta


class Tank:
    def __init__(self, mesh_kwargs):
        self.m = Mesh(**mesh_kwargs)

    def gradient(self, eta, f):
        """Nodal (f_x, f_z): element derivatives through the metric, averaged per node."""
        m = self.m
        rx, rz, sx, sz, J = m.element_metrics(eta)
        fe = m.gather(f).reshape(-1, m.P + 1, m.P + 1)
        fr = np.einsum('im,emj->eij', m.D, fe)
        fs = np.einsum('jm,eim->eij', m.D, fe)
        fx = rx * fr + sx * fs
        fz = rz * fr + sz * fs
        cnt = m.scatter(np.ones_like(fx.reshape(fx.shape[0], -1)))
        return m.scatter(fx.reshape(fx.shape[0], -1)) / cnt, m.scatter(fz.reshape(fz.shape[0], -1)) / cnt

    def slope(self, eta):
        """eta_x per node column: mean of the element derivatives of the surface polynomial."""
        m = self.m
        P = m.P
        acc = np.zeros(m.NX)
        cnt = np.zeros(m.NX)
        for ex in range(m.Nx):
            cols = ex * P + np.arange(P + 1)
            if m.periodic:
                cols = cols % m.NX
            d = (m.D @ eta[cols]) * (2.0 / m.dx)
            np.add.at(acc, cols, d)
            np.add.at(cnt, cols, 1.0)
        return acc / cnt

    def filter_field(self, f, F):
        """Element-wise F (x) F on a nodal field, then the mean at shared nodes."""
        m = self.m
        fe = m.gather(f).reshape(-1, m.P + 1, m.P + 1)
        fe = np.einsum('im,jq,emq->eij', F, F, fe).reshape(fe.shape[0], -1)
        cnt = m.scatter(np.ones_like(fe))
        return m.scatter(fe) / cnt

    def filter_surface(self, eta, F):
        """Element-wise F on the surface elevation, then the mean at shared columns."""
        m = self.m
        acc = np.zeros(m.NX)
        cnt = np.zeros(m.NX)
        for ex in range(m.Nx):
            cols = ex * m.P + np.arange(m.P + 1)
            if m.periodic:
                cols = cols % m.NX
            np.add.at(acc, cols, F @ np.asarray(eta)[cols])
            np.add.at(cnt, cols, 1.0)
        return acc / cnt

    def rates_without_dynamic_pressure(self, eta, u, w):
        """(eta_t, du, dw) of the sigma-frame equations with every force except grad p_D."""
        m = self.m
        ux, uz = self.gradient(eta, u)
        wx, wz = self.gradient(eta, w)
        etax = self.slope(eta)
        ex_node = np.repeat(etax, m.NZ)
        Fu = -(u * ux + w * uz) - G * ex_node
        Fw = -(u * wx + w * wz)
        top = np.arange(m.NX) * m.NZ + m.NZ - 1
        eta_t = w[top] - u[top] * etax
        sig = np.tile(m.row_sigma(), m.NX)
        et_node = np.repeat(eta_t, m.NZ)
        return eta_t, Fu + sig * et_node * uz, Fw + sig * et_node * wz

    def step_lserk_mixed(self, eta, u, w, dt):
        """LSERK(5,4) with the mixed-stage coupling of Sec. 3 (five nonsymmetric solves);
        returns the new state and the stage pressures."""
        m = self.m
        dmask = m.dirichlet_mask()
        y = [np.array(v, dtype=np.float64, copy=True) for v in (eta, u, w)]
        K = [np.zeros_like(v) for v in y]
        ps = []
        for a, b in zip(LSERK54_A, LSERK54_B):
            eta0, u0, w0 = y
            rates = self.rates_without_dynamic_pressure(eta0, u0, w0)
            K = [a * Kv + dt * r for Kv, r in zip(K, rates)]
            eta1 = eta0 + b * K[0]
            us, ws = u0 + b * K[1], w0 + b * K[2]
            rhs = m.rhs_divergence(eta1, us, ws, scale=RHO / (b * dt))
            p = solve_direct(m.assemble_mixed(eta1, eta0), rhs, np.zeros(m.N), dmask)
            px, pz = self.gradient(eta0, p)
            K[1] = K[1] - dt * px / RHO
            K[2] = K[2] - dt * pz / RHO
            y = [eta1, u0 + b * K[1], w0 + b * K[2]]
            ps.append(p)
        return y[0], y[1], y[2], ps

    def rates(self, eta, u, w):
        m = self.m
        ux, uz = self.gradient(eta, u)
        wx, wz = self.gradient(eta, w)
        etax = self.slope(eta)
        ex_node = np.repeat(etax, m.NZ)
        Fu = -(u * ux + w * uz) - G * ex_node
        Fw = -(u * wx + w * wz)
        b = m.rhs_divergence(eta, Fu, Fw, scale=RHO)
        p = solve_direct(m.assemble(eta), b, np.zeros(m.N), m.dirichlet_mask())
        px, pz = self.gradient(eta, p)
        top = np.arange(m.NX) * m.NZ + m.NZ - 1
        eta_t = w[top] - u[top] * etax
        sig = np.tile(m.row_sigma(), m.NX)
        et_node = np.repeat(eta_t, m.NZ)
        du = Fu - px / RHO + sig * et_node * uz
        dw = Fw - pz / RHO + sig * et_node * wz
        return eta_t, du, dw, p

    def step(self, eta, u, w, dt):
        """Classical RK4; returns the new state and the four stage pressures."""
        k1 = self.rates(eta, u, w)
        k2 = self.rates(eta + 0.5 * dt * k1[0], u + 0.5 * dt * k1[1], w + 0.5 * dt * k1[2])
        k3 = self.rates(eta + 0.5 * dt * k2[0], u + 0.5 * dt * k2[1], w + 0.5 * dt * k2[2])
        k4 = self.rates(eta + dt * k3[0], u + dt * k3[1], w + dt * k3[2])
        comb = lambda i: (k1[i] + 2 * k2[i] + 2 * k3[i] + k4[i]) * (dt / 6.0)
        return eta + comb(0), u + comb(1), w + comb(2), [k1[3], k2[3], k3[3], k4[3]]

    def step_lserk(self, eta, u, w, dt):
        """LSERK(5,4) step (five pressure solves); returns the new state and the stage pressures."""
        (eta, u, w), extras = lserk54(lambda y: self.rates(*y), [eta, u, w], dt)
        return eta, u, w, [e[0] for e in extras]

    def linear_wave(self, amp, k):
        """Linear-theory progressive wave eta = a cos(kx): (eta, u, w, omega)."""
        m = self.m
        om = math.sqrt(G * k * math.tanh(k * m.h))
        eta = amp * np.cos(k * m.column_x())
        X, Z = m.node_xz(eta)
        u = amp * om * np.cosh(k * (Z + m.h)) / np.sinh(k * m.h) * np.cos(k * X)
        w = amp * om * np.sinh(k * (Z + m.h)) / np.sinh(k * m.h) * np.sin(k * X)
        return eta, u, w, om
