"""Workload descriptors and closed-form input fields.

Random numbers: SplitMix64 (Steele, Lea, Flood 2014; counter form: the i-th draw of
stream s is mix(s + (i+1) * 0x9E3779B97F4A7C15)) mapped to doubles in [0, 1) by the
top 53 bits, and standard normals by the Box-Muller transform.  Base seed 20241122,
plus the workload id and the problem index.

Fields follow the wave-tank shapes of the paper's experiments (sigma-mapped tank,
few elements in depth, kh of order 1, steepness of a few percent).
"""
import math
from dataclasses import dataclass, field

import numpy as np

BASE_SEED = 20241122
_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed, n, offset=0):
    """n consecutive SplitMix64 outputs of stream `seed`, as uint64."""
    i = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
    with np.errstate(over='ignore'):
        z = np.uint64(seed) + i * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed, n, offset=0):
    """Doubles in [0, 1) from the top 53 bits."""
    return (splitmix64(seed, n, offset) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def normal(seed, n, offset=0):
    """Standard normals by Box-Muller on consecutive uniform pairs."""
    u = uniform(seed, 2 * n, 2 * offset)
    u1 = 1.0 - u[0::2]                       # (0, 1]
    u2 = u[1::2]
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)


# ---------------------------------------------------------------------------------
# Closed-form fields
# ---------------------------------------------------------------------------------
@dataclass
class Surface:
    """eta(x) = amp cos(k x) + noise_amp * xi(x); xi = unit-RMS sum of Fourier modes
    on [x0, x0 + L] with N(0,1) coefficients damped by exp(-(m/m0)^2)."""
    amp: float = 0.0
    k: float = 0.0
    noise_amp: float = 0.0
    L: float = 1.0
    x0: float = 0.0
    a: np.ndarray = field(default_factory=lambda: np.zeros(0))
    b: np.ndarray = field(default_factory=lambda: np.zeros(0))

    @staticmethod
    def smoothed(amp, k, noise_amp, L, x0, seed, modes=64, m0=40.0):
        c = normal(seed, 2 * modes)
        m = np.arange(1, modes + 1)
        damp = np.exp(-(m / m0) ** 2)
        a, b = c[:modes] * damp, c[modes:] * damp
        rms = math.sqrt(0.5 * float(np.sum(a * a + b * b)))
        return Surface(amp, k, noise_amp, L, x0, a / rms, b / rms)

    def __call__(self, x):
        x = np.asarray(x, float)
        out = self.amp * np.cos(self.k * x)
        if self.a.size and self.noise_amp:
            m = np.arange(1, self.a.size + 1)
            ph = 2.0 * np.pi * np.outer(x - self.x0, m) / self.L
            out = out + self.noise_amp * (np.cos(ph) @ self.a + np.sin(ph) @ self.b)
        return out


@dataclass
class Velocity:
    """u = sum_m (A_m, B_m)/|kappa_m|^2 cos(kappa_m . (x, z) + phi_m)."""
    kx: np.ndarray
    kz: np.ndarray
    A: np.ndarray
    B: np.ndarray
    phi: np.ndarray

    @staticmethod
    def random(seed, modes=16, kmin=2 * np.pi / 20, kmax=2 * np.pi / 0.5):
        u = uniform(seed, 3 * modes)
        g = normal(seed + 7, 2 * modes)
        kmag = kmin + (kmax - kmin) * u[:modes]
        th = 2.0 * np.pi * u[modes:2 * modes]
        return Velocity(kmag * np.cos(th), kmag * np.sin(th), g[:modes], g[modes:],
                        2.0 * np.pi * u[2 * modes:])

    def __call__(self, x, z):
        x, z = np.asarray(x, float), np.asarray(z, float)
        k2 = self.kx ** 2 + self.kz ** 2
        arg = np.outer(x, self.kx) + np.outer(z, self.kz) + self.phi
        c = np.cos(arg)
        return c @ (self.A / k2), c @ (self.B / k2)


@dataclass
class Harmonic:
    """p = cos(k (x + xs)) cosh(k (z + zs)): harmonic, with its gradient."""
    k: float
    xs: float = 0.0
    zs: float = 1.0

    def __call__(self, x, z):
        return np.cos(self.k * (np.asarray(x) + self.xs)) * np.cosh(self.k * (np.asarray(z) + self.zs))

    def grad(self, x, z):
        x, z = np.asarray(x, float), np.asarray(z, float)
        px = -self.k * np.sin(self.k * (x + self.xs)) * np.cosh(self.k * (z + self.zs))
        pz = self.k * np.cos(self.k * (x + self.xs)) * np.sinh(self.k * (z + self.zs))
        return px, pz


@dataclass
class Bar:
    """Still-water depth of a submerged bar: depth h0 off the bar, hc over its crest, the
    crest between x_a and x_b, smooth tanh ramps of widths w_a (up-slope) and w_b
    (down-slope):  h(x) = h0 - (h0 - hc) (tanh((x - x_a)/w_a) - tanh((x - x_b)/w_b)) / 2.
    A synthetic stand-in with the features of a bar experiment (shoaling up-slope, shallow
    crest, steeper down-slope); with its derivative for Neumann data."""
    h0: float
    hc: float
    x_a: float
    x_b: float
    w_a: float
    w_b: float

    def __call__(self, x):
        x = np.asarray(x, float)
        s = 0.5 * (np.tanh((x - self.x_a) / self.w_a) - np.tanh((x - self.x_b) / self.w_b))
        return self.h0 - (self.h0 - self.hc) * s

    def slope(self, x):
        x = np.asarray(x, float)
        ds = 0.5 * (1.0 / (self.w_a * np.cosh((x - self.x_a) / self.w_a) ** 2)
                    - 1.0 / (self.w_b * np.cosh((x - self.x_b) / self.w_b) ** 2))
        return -(self.h0 - self.hc) * ds


# ---------------------------------------------------------------------------------
# Workloads
# ---------------------------------------------------------------------------------
@dataclass
class Workload:
    name: str
    cells_x: int
    cells_z: int
    order: int
    x0: float
    x1: float
    h: float
    periodic: bool
    seed: int
    surface: Surface
    rhs: str                          # 'div' (weak divergence of u) or 'source' (-M f + Neumann)
    velocity: Velocity = None
    pressure: Harmonic = None
    noise_sd: float = 0.0
    bathymetry: Bar = None            # still-water depth h(x); None: the constant h
    order_z: int = None               # order along sigma; None: order

    def mesh_kwargs(self):
        d = dict(cells_x=self.cells_x, cells_z=self.cells_z, order=self.order,
                 x0=self.x0, x1=self.x1, h=self.h, periodic=self.periodic)
        if self.order_z is not None and self.order_z != self.order:
            d["order_z"] = self.order_z
        return d

    def depth(self, x_cols):
        """Still-water depth at the node columns."""
        x_cols = np.asarray(x_cols, float)
        return self.bathymetry(x_cols) if self.bathymetry is not None else np.full(x_cols.size, self.h)

    def fields(self, x_cols, sig_rows):
        """Input arrays at the nodes given by their column x* and row sigma.

        Returns eta (NX), and per global node g = ix*NZ + iz: u, w (for 'div'), f, pD;
        per boundary: g_bottom (NX), g_left / g_right (NZ) outward normal derivatives.
        """
        x_cols, sig_rows = np.asarray(x_cols, float), np.asarray(sig_rows, float)
        NX, NZ = x_cols.size, sig_rows.size
        eta = self.surface(x_cols)
        hc = self.depth(x_cols)
        d = eta + hc
        X = np.repeat(x_cols, NZ)
        Z = (sig_rows[None, :] * d[:, None] - hc[:, None]).reshape(-1)
        out = dict(eta=eta, X=X, Z=Z, h=hc)
        top = np.arange(NX) * NZ + NZ - 1
        pD = np.zeros(NX * NZ)
        if self.rhs == 'div':
            u, w = self.velocity(X, Z)
            out.update(u=u, w=w)
        else:
            f = np.zeros(NX * NZ)
            if self.noise_sd:
                f = self.noise_sd * normal(self.seed + 1, NX * NZ)
            out['f'] = f
        gb, gl, gr = np.zeros(NX), np.zeros(NZ), np.zeros(NZ)
        if self.pressure is not None:
            pD[top] = self.pressure(x_cols, eta)
            px, pz = self.pressure.grad(x_cols, -hc)
            if self.bathymetry is None:
                gb = -pz                                              # n = (0, -1)
            else:                                                     # n = -(h_x, 1)/|.|
                hx = self.bathymetry.slope(x_cols)
                gb = -(hx * px + pz) / np.sqrt(1.0 + hx * hx)
            zl = sig_rows * (eta[0] + hc[0]) - hc[0]
            gl = -self.pressure.grad(np.full(NZ, self.x0), zl)[0]      # n = (-1, 0)
            zr = sig_rows * (eta[-1] + hc[-1]) - hc[-1]
            gr = self.pressure.grad(np.full(NZ, self.x1), zr)[0]       # n = (+1, 0)
        out.update(pD=pD, g_bottom=gb, g_left=gl, g_right=gr)
        return out


def config1(noise=True):
    """16 x 4 quads on [0,10] x [-1,0], P = 4, flat; manufactured p = cos(kx)cosh(k(z+1))."""
    k = 2 * np.pi / 10
    return Workload('cfg1_p4_16x4', 16, 4, 4, 0.0, 10.0, 1.0, False, BASE_SEED + 1,
                    Surface(), 'source', pressure=Harmonic(k, 0.0, 1.0),
                    noise_sd=1e-3 if noise else 0.0)


def _tank(name, cells_x, cells_z, order, seed, L=200.0, h=1.0):
    s = Surface.smoothed(0.05, 2 * np.pi / 10, 0.01, L, 0.0, seed)
    return Workload(name, cells_x, cells_z, order, 0.0, L, h, False, seed, s, 'div',
                    velocity=Velocity.random(seed + 3))


def config2():
    """512 x 32 quads on [0,200] x [-1, eta], P = 6, curved surface, divergence RHS."""
    return _tank('cfg2_p6_512x32', 512, 32, 6, BASE_SEED + 2)


def config3():
    """Config 2's tank at P = 8 (1,052,929 nodes)."""
    return _tank('cfg3_p8_512x32', 512, 32, 8, BASE_SEED + 3)


def tank(cells_x, cells_z, order, seed=BASE_SEED + 2, L=None, h=1.0):
    """Config 2's problem family on a smaller mesh (cell width 200/512 kept unless L given)."""
    L = 0.390625 * cells_x if L is None else L
    return _tank(f'tank_p{order}_{cells_x}x{cells_z}', cells_x, cells_z, order, seed, L, h)


def config4(n=64):
    """64 independent problems: N_x ~ U{64..1024}, N_z ~ U{8..32}, P ~ U{4..8},
    h ~ U[0.5, 2], L = 0.390625 N_x; surface as config 2 scaled by h; RHS as config 1
    (manufactured harmonic Dirichlet data, exact nonzero wall flux, N(0,1e-3^2) noise)."""
    out = []
    for j in range(n):
        seed = BASE_SEED + 4 + 1000 * (j + 1)
        u = uniform(seed, 4)
        Nx = 64 + int(u[0] * 961)
        Nz = 8 + int(u[1] * 25)
        P = 4 + int(u[2] * 5)
        h = 0.5 + 1.5 * u[3]
        L = 0.390625 * Nx
        s = Surface.smoothed(0.05 * h, 2 * np.pi / 10, 0.01 * h, L, 0.0, seed)
        k = 2 * np.pi / 10
        out.append(Workload(f'cfg4_{j}', Nx, Nz, P, 0.0, L, h, False, seed, s, 'source',
                            pressure=Harmonic(k, 0.0, h), noise_sd=1e-3))
    return out


def config5():
    """Periodic tank [0,20] x [-1, eta], 256 x 16, P = 6, eta0 = 0.05 cos(pi x)."""
    s = Surface(0.05, np.pi)
    return Workload('cfg5_p6_256x16_periodic', 256, 16, 6, 0.0, 20.0, 1.0, True,
                    BASE_SEED + 5, s, 'div', velocity=Velocity.random(BASE_SEED + 8))


def paper_shape():
    """Sec. 6.3 shape: P = 8, N_x = 102, N_z = 2, 17 waves of kh = 1, H/L = 0.0301."""
    k = 1.0
    L = 17 * 2 * np.pi
    s = Surface(0.5 * 0.0301 * 2 * np.pi, k)
    return Workload('paper_p8_102x2', 102, 2, 8, 0.0, L, 1.0, False, BASE_SEED + 6, s, 'div',
                    velocity=Velocity.random(BASE_SEED + 9))


def paper_scaling(cells_x, order, ppw=48.0, order_z=None):
    """Sec. 6.3 scaling family: N_z = 2, waves of kh = 1 and H/L = 0.0301 at about `ppw`
    points per wavelength along x (the domain grows with the node count); the vertical
    order is `order_z` (the paper's P_z = 8) or, when None, the horizontal one."""
    k = 1.0
    L = cells_x * order * 2 * np.pi / ppw
    s = Surface(0.5 * 0.0301 * 2 * np.pi, k)
    tag = f'p{order}' if order_z in (None, order) else f'p{order}z{order_z}'
    return Workload(f'paper_scaling_{tag}_{cells_x}x2', cells_x, 2, order, 0.0, L, 1.0, False,
                    BASE_SEED + 6, s, 'div', velocity=Velocity.random(BASE_SEED + 9), order_z=order_z)


def bar(cells_x=100, cells_z=2, order=8, rhs='div'):
    """Wave tank over a submerged bar (the shape of the paper's bar experiment, Sec. 6:
    P = 8, N_x = 100, N_z = 2 there): depth 0.4 (kh = 0.67 at the paper's wavelength
    3.74), a synthetic smooth bar (crest depth 0.1, up-slope ramp width 2, down-slope
    ramp width 1, crest from x = 12 to 20) on [0, 36], waves of height 0.02 and length
    3.74.  rhs='div': weak divergence of a random velocity field; 'source': manufactured
    harmonic pressure with its exact Neumann data on the sloped bottom and the walls."""
    L = 36.0
    h0 = 0.4
    bathy = Bar(h0, 0.1, 12.0, 20.0, 2.0, 1.0)
    s = Surface(0.01, 2 * np.pi / 3.74)
    seed = BASE_SEED + 10
    name = f'bar_p{order}_{cells_x}x{cells_z}'
    if rhs == 'div':
        return Workload(name, cells_x, cells_z, order, 0.0, L, h0, False, seed, s, 'div',
                        velocity=Velocity.random(seed + 3), bathymetry=bathy)
    return Workload(name, cells_x, cells_z, order, 0.0, L, h0, False, seed, s, 'source',
                    pressure=Harmonic(2 * np.pi / 3.74, 0.0, h0), bathymetry=bathy)


def by_name(name):
    return {'cfg1': config1, 'cfg2': config2, 'cfg3': config3, 'cfg5': config5,
            'paper': paper_shape}[name]()
