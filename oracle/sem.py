"""Sigma-mapped quadrilateral SEM discretisation of the pressure-Poisson problem, FP64.

Test infrastructure only (see ``oracle/__init__``).

Problem (the same-geometry symmetric reading of the paper's pressure-Poisson BVP):
find p_h in V_P, p_h = p_D on the free surface (Sec. 3.2, p_D = 0 condition), with
    a(N_i, p_h) = l(N_i)  for every free node i,
    a(v, p) = int_Omega grad v . grad p dOmega                                (Sec. 4.2)
    l(v)    = -int_Omega v f dOmega + int_{Gamma_N} v g dGamma                 (Neumann, Sec. 3.2)
pulled back to the sigma-domain by the vertical map sigma = (z + h(x))/d, d = eta + h(x)
(Sec. 2.2, Eq. sigtrans: h(x) is the still-water depth, constant unless a per-column
depth is given), on a structured mesh of N_x x N_z quads (Sec. 4.3) with LGL nodes.

Node numbering (shared by the CUDA path's ABI, defined there independently):
    g = ix * NZ + iz,  ix in [0, NX), iz in [0, NZ),  NZ = N_z P_z + 1,
    NX = N_x P + 1 (walls) or N_x P (periodic in x).  iz = NZ - 1 is the free surface.
The vertical order P_z defaults to the horizontal order P (Sec. 5.1 allows them to differ).

Quadrature: LGL collocation at the (P+1)^2 element nodes for stiffness, mass and
load; the element matrices are formed densely from that definition:
    K_e = Gx^T diag(w J) Gx + Gz^T diag(w J) Gz,  Gx = R_x Dr + S_x Ds, ...
where (r_x, s_x, r_z, s_z) and J come from the isoparametric map of the nodal
coordinates (x*, z = sigma d(x) - h) (Sec. 4.3, D_x = R_x D_r).

Pins (tests/test_oracle_operator.py): flat element factors equal |J| D^T M D with the
exact mass of Sec. 4.3; exactness of a(N_i, l) for physical linear l against boundary
fluxes on a curved mesh; symmetry; SPD of A_FF; pure-Neumann A 1 = 0; spectral
convergence to harmonic closed forms; brute-force dense solves; with a varying depth
(tests/test_oracle_bathymetry.py) the same identities with the bottom-slope fluxes, the
reduction to the constant-depth mesh, and the separable level operator of
`assemble_separable` against its Kronecker-sum form.
"""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import basis


class Mesh:
    """Structured sigma-domain mesh: [x0, x1] x [0, 1] split into cells_x x cells_z quads."""

    def __init__(self, cells_x, cells_z, order, x0=0.0, x1=1.0, h=1.0, periodic=False, depth=None, order_z=None):
        """order: polynomial order along x (P); order_z: along sigma (P_z, default P).
        h: constant still-water depth; depth: optional still-water depth h(x) per node
        column (array of NX values, or a function of x evaluated at the node columns),
        which then replaces h everywhere."""
        order_z = order if order_z is None else order_z
        if cells_x < 1 or cells_z < 1 or order < 1 or order_z < 1:
            raise ValueError("bad mesh")
        self.Nx, self.Nz, self.P, self.Pz = int(cells_x), int(cells_z), int(order), int(order_z)
        self.x0, self.x1, self.h = float(x0), float(x1), float(h)
        self.periodic = bool(periodic)
        P, Pz = self.P, self.Pz
        self.NX = self.Nx * P + (0 if self.periodic else 1)
        self.NZ = self.Nz * Pz + 1
        self.N = self.NX * self.NZ
        self.dx = (self.x1 - self.x0) / self.Nx
        self.dsig = 1.0 / self.Nz
        self.r, self.w = basis.lgl_nodes_weights(P)
        self.D = basis.diff_matrix(P)
        self.rz, self.wz = basis.lgl_nodes_weights(Pz)
        self.Dz = basis.diff_matrix(Pz)
        nx, nz = P + 1, Pz + 1
        # element -> global node map, element e = ex * Nz + ez, local node a = i * (Pz + 1) + j
        ex = np.arange(self.Nx)[:, None, None, None]
        ez = np.arange(self.Nz)[None, :, None, None]
        i = np.arange(nx)[None, None, :, None]
        j = np.arange(nz)[None, None, None, :]
        ix = (ex * P + i) % self.NX if self.periodic else ex * P + i
        iz = ez * Pz + j
        self.e2g = (ix * self.NZ + iz).reshape(self.Nx * self.Nz, nx * nz)
        self.ecol = np.repeat(np.arange(self.Nx), self.Nz)
        self.erow = np.tile(np.arange(self.Nz), self.Nx)
        self.variable_depth = depth is not None
        if depth is None:
            self.hcol = np.full(self.NX, self.h)
        else:
            hc = depth(self.column_x()) if callable(depth) else depth
            self.hcol = np.array(hc, dtype=float).reshape(-1)
            if self.hcol.size != self.NX:
                raise ValueError("depth needs one value per node column")
        if not np.all(self.hcol > 0.0):
            raise ValueError("still-water depth must be positive")

    # --- node coordinates -------------------------------------------------------
    def column_x(self):
        """x* of every node column ix."""
        P = self.P
        ix = np.arange(self.NX)
        ex, i = ix // P, ix % P
        return self.x0 + (ex + (self.r[i] + 1.0) / 2.0) * self.dx

    def row_sigma(self):
        """sigma of every node row iz (0 at the bottom, 1 at the free surface)."""
        Pz = self.Pz
        iz = np.arange(self.NZ)
        ez, j = np.minimum(iz // Pz, self.Nz - 1), iz - np.minimum(iz // Pz, self.Nz - 1) * Pz
        return (ez + (self.rz[j] + 1.0) / 2.0) * self.dsig

    def node_xz(self, eta):
        """Physical (x, z) of every global node for surface elevation eta (per column)."""
        x = self.column_x()
        s = self.row_sigma()
        d = np.asarray(eta, float) + self.hcol
        X = np.repeat(x, self.NZ)
        Z = (s[None, :] * d[:, None] - self.hcol[:, None]).reshape(-1)
        return X, Z

    def dirichlet_mask(self):
        m = np.zeros(self.N, bool)
        m[np.arange(self.NX) * self.NZ + self.NZ - 1] = True
        return m

    # --- element geometry (isoparametric) ---------------------------------------
    def element_coords(self, eta):
        """Nodal (x, z) per element, shape (E, n, n): x* from the element's own cell,
        z = sigma d(x) - h(x) with d = eta + h sampled at the element's node columns."""
        P, n, nz = self.P, self.P + 1, self.Pz + 1
        eta = np.asarray(eta, float)
        xe = self.x0 + (self.ecol[:, None] + (self.r[None, :] + 1.0) / 2.0) * self.dx  # (E, n)
        sig = (self.erow[:, None] + (self.rz[None, :] + 1.0) / 2.0) * self.dsig         # (E, nz)
        cols = self.ecol[:, None] * P + np.arange(n)[None, :]
        if self.periodic:
            cols = cols % self.NX
        hc = self.hcol[cols]                                                              # (E, n)
        d = eta[cols] + hc
        X = np.repeat(xe[:, :, None], nz, axis=2)
        Z = sig[:, None, :] * d[:, :, None] - hc[:, :, None]
        return X, Z

    def element_metrics(self, eta):
        """Per element-local node: (r_x, r_z, s_x, s_z, J) of the isoparametric map.

        x_r = D x along r, x_s = x D^T along s (same for z); J = x_r z_s - x_s z_r;
        r_x = z_s/J, r_z = -x_s/J, s_x = -z_r/J, s_z = x_r/J.
        """
        X, Z = self.element_coords(eta)
        D, Dz = self.D, self.Dz
        xr = np.einsum('im,emj->eij', D, X)
        xs = np.einsum('jm,eim->eij', Dz, X)
        zr = np.einsum('im,emj->eij', D, Z)
        zs = np.einsum('jm,eim->eij', Dz, Z)
        J = xr * zs - xs * zr
        if np.any(J <= 0):
            raise ValueError("non-positive Jacobian: eta <= -h somewhere")
        return zs / J, -xs / J, -zr / J, xr / J, J

    def ref_gradients(self):
        """(Gr, Gs): derivatives of the element basis at the element nodes, (n^2, n^2).

        Gr[(qa,qb),(i,j)] = D[qa,i] delta(qb,j);  Gs[(qa,qb),(i,j)] = delta(qa,i) D_z[qb,j].
        """
        return np.kron(self.D, np.eye(self.Pz + 1)), np.kron(np.eye(self.P + 1), self.Dz)

    def quad_weights(self):
        """Tensor LGL weights w_i w_j at local node (i, j), flattened."""
        return np.outer(self.w, self.wz).reshape(-1)

    def element_stiffness(self, eta, elems=None):
        """Dense K_e = Gx^T diag(w J) Gx + Gz^T diag(w J) Gz for the selected elements."""
        rx, rz, sx, sz, J = self.element_metrics(eta)
        if elems is not None:
            rx, rz, sx, sz, J = rx[elems], rz[elems], sx[elems], sz[elems], J[elems]
        E = rx.shape[0]
        nn = (self.P + 1) * (self.Pz + 1)
        Gr, Gs = self.ref_gradients()
        wJ = self.quad_weights()[None, :] * J.reshape(E, nn)
        Gx = rx.reshape(E, nn, 1) * Gr[None] + sx.reshape(E, nn, 1) * Gs[None]
        Gz = rz.reshape(E, nn, 1) * Gr[None] + sz.reshape(E, nn, 1) * Gs[None]
        return (np.einsum('eqa,eq,eqb->eab', Gx, wJ, Gx)
                + np.einsum('eqa,eq,eqb->eab', Gz, wJ, Gz))

    def element_stiffness_mixed(self, eta_k, eta_km1, elems=None):
        """Mixed-stage element matrices (Sec. 3, the mixed-stage Laplace operator) in the
        conservative weak form a(v, p) = int_{Omega^k} grad^k v . grad^(k-1) p: the test
        gradient with the stage-k map, the trial gradient with the stage-(k-1) map, the
        measure of stage k.  Nonsymmetric unless the two surfaces coincide."""
        rx, rz, sx, sz, J = self.element_metrics(eta_k)
        qx, qz, tx, tz, _ = self.element_metrics(eta_km1)
        if elems is not None:
            rx, rz, sx, sz, J = rx[elems], rz[elems], sx[elems], sz[elems], J[elems]
            qx, qz, tx, tz = qx[elems], qz[elems], tx[elems], tz[elems]
        E = rx.shape[0]
        nn = (self.P + 1) * (self.Pz + 1)
        Gr, Gs = self.ref_gradients()
        wJ = self.quad_weights()[None, :] * J.reshape(E, nn)
        Vx = rx.reshape(E, nn, 1) * Gr[None] + sx.reshape(E, nn, 1) * Gs[None]
        Vz = rz.reshape(E, nn, 1) * Gr[None] + sz.reshape(E, nn, 1) * Gs[None]
        Px = qx.reshape(E, nn, 1) * Gr[None] + tx.reshape(E, nn, 1) * Gs[None]
        Pz = qz.reshape(E, nn, 1) * Gr[None] + tz.reshape(E, nn, 1) * Gs[None]
        return (np.einsum('eqa,eq,eqb->eab', Vx, wJ, Px)
                + np.einsum('eqa,eq,eqb->eab', Vz, wJ, Pz))

    def assemble_mixed(self, eta_k, eta_km1, chunk=2048):
        """Global mixed-stage matrix sum_e Q_e^T K_e Q_e (rows: stage-k test functions)."""
        E = self.Nx * self.Nz
        A = sp.csr_matrix((self.N, self.N))
        for s in range(0, E, chunk):
            el = np.arange(s, min(E, s + chunk))
            K = self.element_stiffness_mixed(eta_k, eta_km1, el)
            g = self.e2g[el]
            rows = np.repeat(g[:, :, None], g.shape[1], axis=2).reshape(-1)
            cols = np.repeat(g[:, None, :], g.shape[1], axis=1).reshape(-1)
            A = A + sp.coo_matrix((K.reshape(-1), (rows, cols)), shape=(self.N, self.N)).tocsr()
        A.sum_duplicates()
        return A

    def assemble(self, eta, chunk=2048):
        """Global stiffness A = sum_e Q_e^T K_e Q_e (Sec. 4.2 global = sum of local), CSR."""
        E = self.Nx * self.Nz
        A = sp.csr_matrix((self.N, self.N))
        for s in range(0, E, chunk):
            el = np.arange(s, min(E, s + chunk))
            K = self.element_stiffness(eta, el)
            g = self.e2g[el]
            rows = np.repeat(g[:, :, None], g.shape[1], axis=2).reshape(-1)
            cols = np.repeat(g[:, None, :], g.shape[1], axis=1).reshape(-1)
            A = A + sp.coo_matrix((K.reshape(-1), (rows, cols)), shape=(self.N, self.N)).tocsr()
        A.sum_duplicates()
        return A

    def element_stiffness_separable(self, depth, elems=None):
        """Element matrices of the still-water (eta = 0) operator with the bottom-slope
        terms dropped: each node column keeps its own depth d_i = depth[column], the
        metric loses its cross term, so
            G_rr = w_i w_j d_i dsig/dx,  G_rs = 0,  G_ss = w_i w_j (dx/dsig) / d_i,
            K_e = Dr^T diag(G_rr) Dr + Ds^T diag(G_ss) Ds.
        With a constant depth this is the flat operator exactly (the sigma-map of a flat
        bottom has no cross term); with a varying depth it is the time-constant level
        operator of the p-multigrid preconditioner (a reading: the slope terms are what
        would make it non-separable)."""
        depth = np.asarray(depth, float)
        P, n = self.P, self.P + 1
        el = np.arange(self.Nx * self.Nz) if elems is None else np.asarray(elems)
        cols = self.ecol[el][:, None] * P + np.arange(n)[None, :]
        if self.periodic:
            cols = cols % self.NX
        dcol = depth[cols]                                                     # (E, n): d_i
        nz = self.Pz + 1
        W = self.quad_weights().reshape(n, nz)                                 # w_i w_j
        grr = (W[None] * dcol[:, :, None] * (self.dsig / self.dx)).reshape(len(el), n * nz)
        gss = (W[None] / dcol[:, :, None] * (self.dx / self.dsig)).reshape(len(el), n * nz)
        Gr, Gs = self.ref_gradients()
        return (np.einsum('qa,eq,qb->eab', Gr, grr, Gr) + np.einsum('qa,eq,qb->eab', Gs, gss, Gs))

    def assemble_separable(self, depth):
        """Global sum of `element_stiffness_separable` (CSR)."""
        K = self.element_stiffness_separable(depth)
        g = self.e2g
        rows = np.repeat(g[:, :, None], g.shape[1], axis=2).reshape(-1)
        cols = np.repeat(g[:, None, :], g.shape[1], axis=1).reshape(-1)
        A = sp.coo_matrix((K.reshape(-1), (rows, cols)), shape=(self.N, self.N)).tocsr()
        A.sum_duplicates()
        return A

    # --- load vectors -------------------------------------------------------------
    def scatter(self, local):
        """sum_e Q_e^T local_e for local arrays of shape (E, n^2)."""
        out = np.zeros(self.N)
        np.add.at(out, self.e2g.reshape(-1), local.reshape(-1))
        return out

    def gather(self, glob):
        return np.asarray(glob)[self.e2g]

    def rhs_source(self, eta, f, g_bottom=None, g_left=None, g_right=None):
        """l(N_i) = -sum_q w_q J_q N_i f_q + Neumann edge terms (LGL collocation).

        g_bottom: d p/d n on the bottom (per node column, n outward);
        g_left / g_right: on the walls x = x0 / x = x1 (per node row).  The edge
        quadrature uses the physical arc length |d(x,z)/d xi| of the mapped edge.
        Entries at Dirichlet nodes are set to zero.
        """
        rx, rz, sx, sz, J = self.element_metrics(eta)
        E, n, P, nz, Pz = J.shape[0], self.P + 1, self.P, self.Pz + 1, self.Pz
        wJ = self.quad_weights()[None, :] * J.reshape(E, n * nz)
        b = -self.scatter(wJ * self.gather(f))
        X, Z = self.element_coords(eta)
        D = self.D
        if g_bottom is not None:
            g_bottom = np.asarray(g_bottom, float)
            for ex in range(self.Nx):
                e = ex * self.Nz
                xr = D @ X[e, :, 0]
                zr = D @ Z[e, :, 0]
                ds = np.sqrt(xr ** 2 + zr ** 2)
                for i in range(n):
                    ix = (ex * P + i) % self.NX
                    b[ix * self.NZ] += self.w[i] * ds[i] * g_bottom[ix]
        if not self.periodic:
            for side, gw in ((0, g_left), (1, g_right)):
                if gw is None:
                    continue
                gw = np.asarray(gw, float)
                ex = 0 if side == 0 else self.Nx - 1
                i = 0 if side == 0 else P
                ix = ex * P + i
                for ez in range(self.Nz):
                    e = ex * self.Nz + ez
                    xs = self.Dz @ X[e, i, :]
                    zs = self.Dz @ Z[e, i, :]
                    ds = np.sqrt(xs ** 2 + zs ** 2)
                    for j in range(nz):
                        iz = ez * Pz + j
                        b[ix * self.NZ + iz] += self.wz[j] * ds[j] * gw[iz]
        b[self.dirichlet_mask()] = 0.0
        return b

    def rhs_divergence(self, eta, u, w, scale=1.0):
        """l(N_i) = scale * int grad N_i . (u, w) dOmega (weak divergence, LGL collocation).

        For the projection reading of the pressure step this carries the Neumann data
        n.u on walls and bottom implicitly.  Entries at Dirichlet nodes are zero.
        """
        rx, rz, sx, sz, J = self.element_metrics(eta)
        E, nn = J.shape[0], (self.P + 1) * (self.Pz + 1)
        Gr, Gs = self.ref_gradients()
        wJ = self.quad_weights()[None, :] * J.reshape(E, nn)
        Gx = rx.reshape(E, nn, 1) * Gr[None] + sx.reshape(E, nn, 1) * Gs[None]
        Gz = rz.reshape(E, nn, 1) * Gr[None] + sz.reshape(E, nn, 1) * Gs[None]
        ue, we = self.gather(u), self.gather(w)
        loc = (np.einsum('eqa,eq->ea', Gx, wJ * ue) + np.einsum('eqa,eq->ea', Gz, wJ * we))
        b = scale * self.scatter(loc)
        b[self.dirichlet_mask()] = 0.0
        return b


def lifted_system(A, b, p_dirichlet, dmask):
    """(A_FF, b_F - A_FD p_D, free index): the Dirichlet-lifted free-node system."""
    free = np.flatnonzero(~dmask)
    dir_ = np.flatnonzero(dmask)
    A = sp.csr_matrix(A)
    AFF = A[free][:, free]
    bt = np.asarray(b, float)[free] - A[free][:, dir_] @ np.asarray(p_dirichlet, float)[dir_]
    return AFF, bt, free


def apply_masked(A, x, dmask):
    """y = A_FF x_F on free rows, y_D = x_D: the operator as the CUDA ABI exposes it."""
    x = np.asarray(x, float)
    xf = np.where(dmask, 0.0, x)
    y = A @ xf
    return np.where(dmask, x, y)


def solve_direct(A, b, p_dirichlet, dmask):
    """Exact solution by a sparse LU of A_FF (library primitive); full-length vector."""
    AFF, bt, free = lifted_system(A, b, p_dirichlet, dmask)
    p = np.array(p_dirichlet, float, copy=True)
    p[free] = spla.splu(sp.csc_matrix(AFF)).solve(bt)
    return p


def solve_dense(A, b, p_dirichlet, dmask):
    """Brute force: dense Cholesky of A_FF (small meshes only)."""
    import scipy.linalg as sla
    AFF, bt, free = lifted_system(A, b, p_dirichlet, dmask)
    c = sla.cho_factor(AFF.toarray())
    p = np.array(p_dirichlet, float, copy=True)
    p[free] = sla.cho_solve(c, bt)
    return p


def relative_residual(A, b, p, dmask):
    """||b~_F - A_FF p_F||_2 / ||b~_F||_2 with b~ = b - A_FD p_D."""
    AFF, bt, free = lifted_system(A, b, p, dmask)
    r = bt - AFF @ np.asarray(p, float)[free]
    nb = np.linalg.norm(bt)
    return np.linalg.norm(r) / (nb if nb > 0 else 1.0)
