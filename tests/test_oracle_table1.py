"""Pins of the oracle's multigrid quality on the paper's Table 1 case (Sec. 6, P = 8,
N_x = 102, N_z = 2, kh = 1, H/L = 0.0301, the mixed-stage operator of Sec. 3), against
the iteration counts the paper prints (tests/golden/table1_mg_iterations.txt) and against
the minimal-residual property that ties GMRES to defect correction; and the synthetic
Table 1 case and scaling-study family are the discretisations Sec. 6 states."""
import os

import numpy as np
import pytest

from oracle import mg
from oracle.sem import Mesh
from oracle.stepper import G
import workloads as W

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "table1_mg_iterations.txt")


def golden_rows():
    rows = []
    for line in open(GOLDEN):
        line = line.strip()
        if line and not line.startswith("#"):
            tol, pdc, gm = line.split()
            rows.append((float(tol), int(pdc), int(gm)))
    return rows


_case = {}


def table1_case():
    """The Table 1 shape with a seeded divergence right-hand side; stage k is a linear wave
    of the case's steepness and stage k-1 the same wave one time step (T/100) earlier."""
    if not _case:
        w = W.paper_shape()
        m = Mesh(**w.mesh_kwargs())
        F = w.fields(m.column_x(), m.row_sigma())
        b = m.rhs_divergence(F["eta"], F["u"], F["w"])
        x = m.column_x()
        k, h = w.surface.k, w.h
        omega = np.sqrt(G * k * np.tanh(k * h))
        shift = (omega / k) * (2 * np.pi / omega / 100)
        eta_k = w.surface.amp * np.cos(k * x)
        eta_km1 = w.surface.amp * np.cos(k * (x + shift))
        H = mg.Hierarchy(m, eta_k, overlap=1, nu=2, omega=0.8)
        _case.update(m=m, b=b, pD=F["pD"], eta_k=eta_k, eta_km1=eta_km1, H=H)
    return _case


def test_case_is_the_table1_discretisation():
    """Sec. 6 describes the Table 1 case as P = 8, N_x = 102, N_z = 2, seventeen waves of
    kh = 1 with H/L = 0.0301, about 48 points per wavelength: the workload is that case."""
    w = W.paper_shape()
    assert (w.order, w.cells_x, w.cells_z, w.h, w.periodic) == (8, 102, 2, 1.0, False)
    k = w.surface.k
    wavelength = 2 * np.pi / k
    assert abs(k * w.h - 1.0) < 1e-15
    np.testing.assert_allclose((w.x1 - w.x0) / wavelength, 17.0, rtol=1e-14)
    np.testing.assert_allclose(2 * w.surface.amp / wavelength, 0.0301, rtol=1e-14)
    assert abs(w.cells_x * w.order / 17.0 - 48.0) < 0.1


@pytest.mark.parametrize("cells_x,order", [(25, 8), (200, 8), (800, 8), (200, 2), (200, 10)])
def test_scaling_family_keeps_the_paper_resolution(cells_x, order):
    """Sec. 6's scaling study: N_z = 2, P_z = 8, waves of kh = 1 and H/L = 0.0301 at about
    48 points per wavelength whatever N_x or P_x."""
    w = W.paper_scaling(cells_x, order, order_z=8)
    assert (w.cells_z, w.order_z, w.h) == (2, 8, 1.0)
    wavelength = 2 * np.pi / w.surface.k
    assert abs(w.surface.k * w.h - 1.0) < 1e-15
    np.testing.assert_allclose(2 * w.surface.amp / wavelength, 0.0301, rtol=1e-14)
    np.testing.assert_allclose(cells_x * order / ((w.x1 - w.x0) / wavelength), 48.0, rtol=1e-12)


def test_golden_file_is_the_printed_table():
    assert golden_rows() == [(1e-4, 3, 1), (1e-6, 5, 3), (1e-8, 8, 4)]


@pytest.mark.parametrize("tol,pdc_paper,_gm", golden_rows())
def test_pdc_mg_iterations_match_table1(tol, pdc_paper, _gm):
    """p-MG-accelerated defect correction on the mixed-stage operator needs the paper's
    iteration count within one (the right-hand side is synthetic, the smoother's overlap,
    sweeps and damping are this implementation's reading)."""
    c = table1_case()
    _, its, hist, _ = mg.solve(c["m"], c["eta_k"], c["b"], c["pD"], hier=c["H"], method="pdc", tol=tol,
                               eta_prev=c["eta_km1"])
    assert hist[-1] <= tol
    assert abs(its - pdc_paper) <= 1, (its, pdc_paper)


def test_gmres_residual_never_above_defect_correction():
    """With the same fixed linear preconditioner B (one V-cycle), the k-th defect-correction
    iterate lies in x0 + B K_k(AB, r0), the space GMRES minimises the residual over; so the
    k-th GMRES residual is at most the k-th PDC residual, at every step of the first cycle."""
    c = table1_case()
    _, _, h_pdc, _ = mg.solve(c["m"], c["eta_k"], c["b"], c["pD"], hier=c["H"], method="pdc", tol=1e-9,
                              eta_prev=c["eta_km1"])
    _, _, h_gm, _ = mg.solve(c["m"], c["eta_k"], c["b"], c["pD"], hier=c["H"], method="gmres", tol=1e-9,
                             eta_prev=c["eta_km1"])
    n = min(len(h_pdc), len(h_gm))
    assert n >= 6
    for k in range(n):
        assert h_gm[k] <= h_pdc[k] * (1 + 1e-8) + 1e-15, (k, h_gm[k], h_pdc[k])
    # and strictly fewer or equal iterations at every printed tolerance
    for tol, _, _ in golden_rows():
        assert min(i for i, v in enumerate(h_gm) if v <= tol) <= min(i for i, v in enumerate(h_pdc) if v <= tol)
