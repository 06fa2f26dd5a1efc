"""Geometric p-multigrid preconditioned Krylov solve, FP64, assembled matrices.

Test infrastructure only (see ``oracle/__init__``).

Paper passages followed (Sec. 5):
  * level hierarchy: same mesh, orders P_{n-1} = ceil((P_n + 1)/2)          (Sec. 5.1)
    (iterated down to 2, then order 1 appended: the rule's fixed point is 2); with
    different horizontal and vertical orders, semi-coarsening of the higher one until
    they match (`basis.semi_coarsening_sequence`)
  * each level re-discretised on the same cells ("geometric" p-MG), either on
    the actual geometry or on the flat, linearised geometry eta = 0 that makes
    the preconditioner time-constant                                        (Sec. 5, Sec. 5.4)
    (with a varying still-water depth h(x) the flat level operator keeps each node
    column's depth, evaluated at the level's nodes, and drops the bottom-slope terms:
    `Mesh.element_stiffness_separable`)
  * prolongation = interpolation of the coarse polynomial at the fine nodes,
    I = Phi V^{-1} per element; restriction R = P^T                        (Sec. 5.2)
  * additive Schwarz smoother  x <- x - S^{-1}(A x - b),
    S^{-1} = W sum_i R_i^T (R_i A R_i^T)^{-1} R_i,  W = (sum_i R_i R_i^T)^{-1},
    subdomain = element block plus `overlap` node lines of the neighbours   (Sec. 5.3)
    with damping omega; post-smoothing uses the adjoint S^{-T} (W on the right)
    so that the V-cycle is a symmetric preconditioner for CG.  The overlap is the
    user's choice (the paper leaves it open); on a level of order p it is capped at
    floor((p-1)/2) lines so that the overlap lines of two neighbouring subdomains
    never meet (order 2 runs without overlap)
  * V-cycle                                                               (Sec. 5, Fig. V-cycle)
  * outer methods: PCG, flexible CG, and preconditioned defect correction
    x <- x + B (b - A x)                                                  (Sec. 5.4)

The coarsest level (order 1) is solved exactly by a sparse LU (library primitive).

Parity status: the V-cycle's quality is pinned to the PDC-MG iteration counts the paper
prints in Table 1 (Sec. 6, within one: the right-hand side is synthetic), and tests pin
its symmetry and positivity, exact-solve limits, the flat iteration counts in N_x and P
claimed in Sec. 6.3, and flexible GMRES's minimal residual against defect correction.
The level geometry (`Hierarchy._eta_at_level`: the surface and the still-water depth at
each level's nodes) is pinned by polynomial exactness: piecewise polynomials of degree
<= P must come out at the level's LGL nodes exactly as numpy.polynomial evaluates them.
"""
import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import basis
from .sem import Mesh, lifted_system


class Level:
    def __init__(self, mesh, A, overlap, overlap_z=None):
        self.mesh = mesh
        self.dmask = mesh.dirichlet_mask()
        self.free = np.flatnonzero(~self.dmask)
        self.A = sp.csr_matrix(A)[self.free][:, self.free]      # A_FF of this level
        self.pos = -np.ones(mesh.N, dtype=np.int64)             # global -> free index
        self.pos[self.free] = np.arange(self.free.size)
        self.overlap = overlap
        self.overlap_z = overlap if overlap_z is None else overlap_z
        self.blocks = None
        self.W = None

    def build_schwarz(self):
        """Subdomains R_i (element nodes + overlap lines, free nodes only), the dense
        Cholesky factors of R_i A R_i^T, and W = (sum R_i R_i^T)^{-1} (Sec. 5.3)."""
        m, o, oz = self.mesh, self.overlap, self.overlap_z
        P, Pz = m.P, m.Pz
        blocks = []
        count = np.zeros(self.free.size)
        for ex in range(m.Nx):
            xs = np.arange(ex * P - o, ex * P + P + o + 1)
            if m.periodic:
                xs = np.unique(xs % m.NX)
            else:
                xs = xs[(xs >= 0) & (xs < m.NX)]
            for ez in range(m.Nz):
                zs = np.arange(ez * Pz - oz, ez * Pz + Pz + oz + 1)
                zs = zs[(zs >= 0) & (zs < m.NZ - 1)]                  # drop the Dirichlet row
                g = (xs[:, None] * m.NZ + zs[None, :]).reshape(-1)
                idx = self.pos[g]
                assert np.all(idx >= 0)
                Ai = self.A[idx][:, idx].toarray()
                blocks.append((idx, sla.cho_factor(Ai)))
                count[idx] += 1.0
        self.blocks = blocks
        self.W = 1.0 / count

    def schwarz(self, r):
        """sum_i R_i^T (R_i A R_i^T)^{-1} R_i r."""
        out = np.zeros_like(r)
        for idx, c in self.blocks:
            out[idx] += sla.cho_solve(c, r[idx])
        return out


class Hierarchy:
    """p-multigrid hierarchy on free nodes.

    geometry: 'flat' (eta = 0 for every level: the paper's time-constant
    preconditioner) or 'actual' (each level re-discretised on eta interpolated to
    the level's nodes).
    """

    def __init__(self, mesh, eta, orders=None, overlap=1, nu=2, omega=1.0, geometry='flat', coarse_geometry=None):
        """orders: x-orders of the levels (equal orders in both directions), or (p_x, p_z)
        pairs; default: the coarsening rule, with semi-coarsening when P_z != P.
        coarse_geometry: geometry of the coarsest level ('flat' or 'actual'; default: as
        `geometry`).  With geometry='actual' and coarse_geometry='flat' the order-1 level
        keeps the still-water operator, whose exact solve is separable."""
        if orders is None:
            pairs = (basis.semi_coarsening_sequence(mesh.P, mesh.Pz) if mesh.Pz != mesh.P
                     else [(p, p) for p in basis.coarsening_sequence(mesh.P)])
        else:
            pairs = [tuple(o) if np.ndim(o) else (int(o), int(o)) for o in orders]
        assert pairs[0] == (mesh.P, mesh.Pz)
        self.pairs = pairs
        self.orders = [px for px, _ in pairs]
        self.orders_z = [pz for _, pz in pairs]
        self.nu, self.omega = nu, omega
        self.levels = []
        self.P = []                      # prolongations level l+1 -> l on free nodes
        eta = np.asarray(eta, float)
        coarse_geometry = geometry if coarse_geometry is None else coarse_geometry
        for l, (p, pz) in enumerate(self.pairs):
            geo_l = coarse_geometry if l == len(self.pairs) - 1 else geometry
            ml = Mesh(mesh.Nx, mesh.Nz, p, mesh.x0, mesh.x1, mesh.h, mesh.periodic, order_z=pz)
            if mesh.variable_depth:
                probe = ml
                h_l = self._eta_at_level(mesh, mesh.hcol, probe)
                ml = Mesh(mesh.Nx, mesh.Nz, p, mesh.x0, mesh.x1, mesh.h, mesh.periodic, depth=h_l, order_z=pz)
            if geo_l == 'flat':
                if mesh.variable_depth:
                    A_l = ml.assemble_separable(ml.hcol)
                else:
                    A_l = ml.assemble(np.zeros(ml.NX))
            else:
                A_l = ml.assemble(self._eta_at_level(mesh, eta, ml))
            lev = Level(ml, A_l, min(overlap, (p - 1) // 2), min(overlap, (pz - 1) // 2))
            if l < len(self.orders) - 1:
                lev.build_schwarz()
            self.levels.append(lev)
        for l in range(len(self.orders) - 1):
            self.P.append(self._prolongation(self.levels[l], self.levels[l + 1]))
        c = self.levels[-1]
        self.coarse_lu = spla.splu(sp.csc_matrix(c.A))

    @staticmethod
    def _eta_at_level(fine, eta, ml):
        """Evaluate the fine-level surface polynomial of each cell at the level's nodes."""
        I = basis.transfer_1d(fine.P, ml.P) if ml.P != fine.P else np.eye(fine.P + 1)
        # I maps order-P nodal values to order-p nodes when p < P (evaluation of the fine
        # polynomial at the coarse nodes): Phi^{p-nodes} V_P^{-1}.
        out = np.zeros(ml.NX)
        for ex in range(fine.Nx):
            cf = (ex * fine.P + np.arange(fine.P + 1)) % fine.NX if fine.periodic else ex * fine.P + np.arange(fine.P + 1)
            cc = (ex * ml.P + np.arange(ml.P + 1)) % ml.NX if ml.periodic else ex * ml.P + np.arange(ml.P + 1)
            out[cc] = I @ eta[cf]
        return out

    @staticmethod
    def _prolongation(fine, coarse):
        """P = D_f^{-1} Q_f^T (J (x) J)_blk Q_c restricted to free nodes (Sec. 5.2).

        J = transfer_1d(p_c, p_f): coarse modal expansion evaluated at fine nodes.
        D_f = multiplicity of each fine global node (element copies agree, so this
        averages identical values).
        """
        mf, mc = fine.mesh, coarse.mesh
        Jx = basis.transfer_1d(mc.P, mf.P) if mc.P != mf.P else np.eye(mf.P + 1)
        Jz = basis.transfer_1d(mc.Pz, mf.Pz) if mc.Pz != mf.Pz else np.eye(mf.Pz + 1)
        B = np.kron(Jx, Jz)                                     # (nf_x nf_z, nc_x nc_z)
        E = mf.Nx * mf.Nz
        rows = np.repeat(mf.e2g[:, :, None], B.shape[1], axis=2).reshape(-1)
        cols = np.repeat(mc.e2g[:, None, :], B.shape[0], axis=1).reshape(-1)
        vals = np.tile(B.reshape(-1), E)
        S = sp.coo_matrix((vals, (rows, cols)), shape=(mf.N, mc.N)).tocsr()
        mult = np.bincount(mf.e2g.reshape(-1), minlength=mf.N).astype(float)
        Pg = sp.diags(1.0 / mult) @ S
        return sp.csr_matrix(Pg[fine.free][:, coarse.free])

    # --- smoothing and V-cycle ------------------------------------------------------
    def smooth(self, l, b, x, post):
        lev = self.levels[l]
        for _ in range(self.nu):
            r = b - lev.A @ x
            if post:
                x = x + self.omega * lev.schwarz(lev.W * r)
            else:
                x = x + self.omega * lev.W * lev.schwarz(r)
        return x

    def vcycle(self, b, l=0):
        """One V-cycle for A_l x = b from x = 0: pre-smooth, restrict the residual,
        recurse, prolong the correction, post-smooth.  Coarsest level: exact solve."""
        if l == len(self.levels) - 1:
            return self.coarse_lu.solve(b)
        lev = self.levels[l]
        x = self.smooth(l, b, np.zeros_like(b), post=False)
        r = b - lev.A @ x
        rc = self.P[l].T @ r
        x = x + self.P[l] @ self.vcycle(rc, l + 1)
        return self.smooth(l, b, x, post=True)


def pcg(A, b, prec, x0=None, tol=1e-10, maxit=500):
    """Preconditioned CG; stops when ||r||_2 / ||b||_2 <= tol (recursive residual).
    Returns (x, iterations, relres history)."""
    x = np.zeros_like(b) if x0 is None else np.array(x0, float, copy=True)
    nb = np.linalg.norm(b)
    if nb == 0.0:
        return np.zeros_like(b), 0, [0.0]
    r = b - A @ x
    hist = [np.linalg.norm(r) / nb]
    if hist[-1] <= tol:
        return x, 0, hist
    z = prec(r)
    p = z.copy()
    rz = r @ z
    for k in range(1, maxit + 1):
        Ap = A @ p
        alpha = rz / (p @ Ap)
        x = x + alpha * p
        r = r - alpha * Ap
        hist.append(np.linalg.norm(r) / nb)
        if hist[-1] <= tol:
            return x, k, hist
        z = prec(r)
        rz_new = r @ z
        p = z + (rz_new / rz) * p
        rz = rz_new
    return x, maxit, hist


def fcg(A, b, prec, x0=None, tol=1e-10, maxit=500):
    """Flexible CG with the Polak-Ribiere beta = <z_k, r_k - r_{k-1}> / <z_{k-1}, r_{k-1}>."""
    x = np.zeros_like(b) if x0 is None else np.array(x0, float, copy=True)
    nb = np.linalg.norm(b)
    if nb == 0.0:
        return np.zeros_like(b), 0, [0.0]
    r = b - A @ x
    hist = [np.linalg.norm(r) / nb]
    if hist[-1] <= tol:
        return x, 0, hist
    z = prec(r)
    p = z.copy()
    rz = r @ z
    for k in range(1, maxit + 1):
        Ap = A @ p
        alpha = rz / (p @ Ap)
        x = x + alpha * p
        r_old = r
        r = r - alpha * Ap
        hist.append(np.linalg.norm(r) / nb)
        if hist[-1] <= tol:
            return x, k, hist
        z = prec(r)
        beta = (z @ (r - r_old)) / rz
        rz = r @ z
        p = z + beta * p
    return x, maxit, hist


def pdc(A, b, prec, x0=None, tol=1e-10, maxit=500):
    """Preconditioned defect correction x <- x + B (b - A x) (Sec. 5.4)."""
    x = np.zeros_like(b) if x0 is None else np.array(x0, float, copy=True)
    nb = np.linalg.norm(b)
    if nb == 0.0:
        return np.zeros_like(b), 0, [0.0]
    hist = []
    for k in range(0, maxit + 1):
        r = b - A @ x
        hist.append(np.linalg.norm(r) / nb)
        if hist[-1] <= tol:
            return x, k, hist
        x = x + prec(r)
    return x, maxit, hist


def fgmres(A, b, prec, x0=None, tol=1e-10, maxit=500, restart=30):
    """Flexible GMRES(restart) with right preconditioning (Saad 1993): Arnoldi by modified
    Gram-Schmidt on z_j = prec(v_j), the least-squares problem by Givens rotations, and
    x = x0 + Z y at the end of a cycle.  Stops when the residual estimate |g_{j+1}| <=
    tol ||b|| (checked against the true residual at each restart).  Returns (x,
    iterations, relres history)."""
    x = np.zeros_like(b) if x0 is None else np.array(x0, float, copy=True)
    nb = np.linalg.norm(b)
    if nb == 0.0:
        return np.zeros_like(b), 0, [0.0]
    r = b - A @ x
    hist = [np.linalg.norm(r) / nb]
    its = 0
    while hist[-1] > tol and its < maxit:
        beta = np.linalg.norm(r)
        m = min(restart, maxit - its)
        V = np.zeros((m + 1, b.size))
        Z = np.zeros((m, b.size))
        H = np.zeros((m + 1, m))
        cs, sn = np.zeros(m), np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        V[0] = r / beta
        k = 0
        for j in range(m):
            Z[j] = prec(V[j])
            w = A @ Z[j]
            for i in range(j + 1):
                H[i, j] = w @ V[i]
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            if H[j + 1, j] > 0:
                V[j + 1] = w / H[j + 1, j]
            for i in range(j):  # earlier rotations on the new column
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            den = np.hypot(H[j, j], H[j + 1, j])
            cs[j], sn[j] = H[j, j] / den, H[j + 1, j] / den
            H[j, j] = den
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            its += 1
            k = j + 1
            hist.append(abs(g[j + 1]) / nb)
            if hist[-1] <= tol:
                break
        y = np.linalg.solve(np.triu(H[:k, :k]), g[:k])
        x = x + Z[:k].T @ y
        r = b - A @ x
        hist[-1] = np.linalg.norm(r) / nb
    return x, its, hist


def solve(mesh, eta, b, p_dirichlet, hier=None, method='pcg', x0=None, tol=1e-10, maxit=500,
          eta_prev=None, **hier_kw):
    """Full solve on the actual geometry: Dirichlet lifting, then the preconditioned
    Krylov method on A_FF with one V-cycle of `hier` as the preconditioner.  With
    eta_prev the operator is the mixed-stage one (stage k = eta, stage k-1 = eta_prev).
    Returns (p full-length, iterations, history, hierarchy)."""
    A = mesh.assemble(eta) if eta_prev is None else mesh.assemble_mixed(eta, eta_prev)
    dmask = mesh.dirichlet_mask()
    AFF, bt, free = lifted_system(A, b, p_dirichlet, dmask)
    if hier is None:
        hier = Hierarchy(mesh, eta, **hier_kw)
    x0f = None if x0 is None else np.asarray(x0, float)[free]
    f = {'pcg': pcg, 'fcg': fcg, 'pdc': pdc, 'gmres': fgmres}[method]
    xf, its, hist = f(AFF, bt, hier.vcycle, x0=x0f, tol=tol, maxit=maxit)
    p = np.array(p_dirichlet, float, copy=True)
    p[free] = xf
    return p, its, hist, hier
