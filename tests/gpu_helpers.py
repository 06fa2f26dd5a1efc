"""Shared setup of the GPU parity tests: a workload on both sides (CUDA path through the
C ABI, oracle on the CPU) from the same seeded generator."""
import numpy as np
import torch

import paper_2411_14977_gb300.pmg as pmg
from oracle import mg
from oracle.sem import Mesh

DEV = torch.device("cuda:0")


def t(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device=DEV)


def n(x):
    return x.detach().double().cpu().numpy()


class Case:
    """Solver + oracle mesh + fields for one workload."""

    def __init__(self, w, **opts):
        self.w = w
        self.S = pmg.Solver(**w.mesh_kwargs(), **opts)
        self.m = Mesh(**w.mesh_kwargs())
        xc, sr = self.S.node_coords()
        np.testing.assert_allclose(xc, self.m.column_x(), rtol=0, atol=1e-13 * max(1.0, abs(w.x1)))
        np.testing.assert_allclose(sr, self.m.row_sigma(), rtol=0, atol=1e-15)
        self.F = w.fields(xc, sr)
        self.eta = self.F["eta"]
        if w.bathymetry is not None:
            # both sides get the same nodal depths
            self.m = Mesh(**w.mesh_kwargs(), depth=self.F["h"])
            self.S.set_bathymetry(t(self.F["h"]))
        self.S.set_geometry(t(self.eta))
        self.opts = self.S.opts

    def rhs_oracle(self):
        F = self.F
        if self.w.rhs == "div":
            return self.m.rhs_divergence(self.eta, F["u"], F["w"])
        return self.m.rhs_source(self.eta, F["f"], F["g_bottom"], F["g_left"], F["g_right"])

    def rhs_gpu(self):
        F = self.F
        if self.w.rhs == "div":
            return self.S.assemble_rhs_div(t(F["u"]), t(F["w"]))
        per = self.w.periodic
        return self.S.assemble_rhs(t(F["f"]), t(F["g_bottom"]), None if per else t(F["g_left"]),
                                   None if per else t(F["g_right"]))

    def hierarchy(self, geometry="flat"):
        o = self.opts
        return mg.Hierarchy(self.m, self.eta, overlap=o.overlap, nu=o.nu, omega=o.omega, geometry=geometry)
