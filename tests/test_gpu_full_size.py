"""Config 2 at its full size (512 x 32 quads, P = 6, 593,089 nodes) in the launch
configuration the bench times (mixed precision, autotuned kernels, double-float outer
operator), checked where the oracle can follow it:

* sampled outputs: a node's row of the operator and its load-vector entry involve only the
  elements that contain it, and an element's geometry only the surface at its own node
  columns (the sigma map of Sec. 2.2 is element-local).  So for a sampled element column
  the oracle assembles a slice of the tank -- that column and its neighbours, with the same
  surface, velocities and iterate -- and its rows at the column's nodes are the full
  tank's rows.  Checked: the outer operator (1e-12 of the summand scale, the FP64 bound),
  the FP32 operator (2e-5), the divergence load vector, and the true residual of the
  timed solve at those nodes;
* properties that hold at any size: the operator symmetric and positive on the free nodes,
  the FP32 V-cycle symmetric to FP32 rounding.
The sampled columns include both walls and their neighbours."""
import numpy as np
import pytest
import torch

import paper_2411_14977_gb300.pmg as pmg
import workloads as W
from oracle.sem import Mesh, apply_masked
from tests.gpu_helpers import n, t

pytestmark = pytest.mark.gpu

SAMPLED = [0, 1, 137, 255, 256, 400, 510, 511]
_state = {}


def full():
    if "S" not in _state:
        w = W.config2()
        S = pmg.Solver(**w.mesh_kwargs(), precision=pmg.PMG_MIXED_FP32)
        xc, sr = S.node_coords()
        F = w.fields(xc, sr)
        S.set_geometry(t(F["eta"]))
        S.autotune()
        _state.update(S=S, w=w, F=F, xc=xc)
    return _state["S"], _state["w"], _state["F"]


def slice_of(w, F, e, S):
    """Oracle mesh of element columns e-1 .. e+1 (clipped at the walls), the slice's node
    columns in the full tank, and the local node columns of element e."""
    P, Nx, NZ = w.order, w.cells_x, S.NZ
    e0, e1 = max(e - 1, 0), min(e + 1, Nx - 1)
    dx = (w.x1 - w.x0) / Nx
    m = Mesh(e1 - e0 + 1, w.cells_z, P, x0=w.x0 + e0 * dx, x1=w.x0 + (e1 + 1) * dx, h=w.h)
    cols = np.arange(e0 * P, (e1 + 1) * P + 1)
    own = np.arange((e - e0) * P, (e - e0) * P + P + 1)
    np.testing.assert_allclose(m.column_x(), _state["xc"][cols], rtol=0, atol=1e-12)
    return m, cols, own, NZ


def take(v, cols, NZ):
    return np.asarray(v).reshape(-1, NZ)[cols].reshape(-1)


def test_full_size_operator_rows_match_oracle_slices():
    S, w, F = full()
    rng = np.random.default_rng(21)
    x = rng.standard_normal(S.n)
    y = n(S.apply(t(x)))
    y32 = n(S.apply_f32(t(x, torch.float32)))
    x32 = x.astype(np.float32).astype(np.float64)
    for e in SAMPLED:
        m, cols, own, NZ = slice_of(w, F, e, S)
        A = m.assemble(F["eta"][cols])
        xs = take(x, cols, NZ)
        ref = apply_masked(A, xs, m.dirichlet_mask()).reshape(-1, NZ)[own]
        sc = np.max(np.abs(A) @ np.abs(np.where(m.dirichlet_mask(), 0, xs)))
        got = take(y, cols, NZ).reshape(-1, NZ)[own]
        assert np.max(np.abs(got - ref)) <= 1e-12 * sc, (e, np.max(np.abs(got - ref)) / sc)
        xs32 = take(x32, cols, NZ)
        ref32 = apply_masked(A, xs32, m.dirichlet_mask()).reshape(-1, NZ)[own]
        got32 = take(y32, cols, NZ).reshape(-1, NZ)[own]
        assert np.max(np.abs(got32 - ref32)) <= 2e-5 * sc, e


def test_full_size_load_vector_and_solve_residual_at_sampled_columns():
    S, w, F = full()
    b = S.assemble_rhs_div(t(F["u"]), t(F["w"]))
    pD = t(F["pD"])
    p, info = S.solve(b, pD)
    assert info["status"] == pmg.PMG_OK and info["rel_residual"] <= 1e-10
    bn, pn = n(b), n(p)
    # ||b~|| over the free nodes: the residual of x = 0 with the surface row set to p_D
    bnorm = S.residual_norm(b, pD, torch.zeros_like(b))
    for e in SAMPLED:
        m, cols, own, NZ = slice_of(w, F, e, S)
        eta = F["eta"][cols]
        A = m.assemble(eta)
        us, ws = take(F["u"], cols, NZ), take(F["w"], cols, NZ)
        bref = m.rhs_divergence(eta, us, ws).reshape(-1, NZ)[own]
        bgot = take(bn, cols, NZ).reshape(-1, NZ)[own]
        assert np.max(np.abs(bgot - bref)) <= 1e-12 * max(1.0, np.max(np.abs(bref))), e
        # true residual b - A p at the column's free nodes (p carries p_D on the surface row)
        ps = take(pn, cols, NZ)
        r = (take(bn, cols, NZ) - A @ ps).reshape(-1, NZ)[own][:, :-1]
        assert np.max(np.abs(r)) <= 1e-10 * bnorm, (e, np.max(np.abs(r)) / bnorm)


def test_full_size_operator_symmetric_positive_and_vcycle_symmetric():
    S, w, F = full()
    rng = np.random.default_rng(22)
    mask = np.zeros((S.NX, S.NZ), bool)
    mask[:, -1] = True
    mask = mask.reshape(-1)
    x = np.where(mask, 0.0, rng.standard_normal(S.n))
    y = np.where(mask, 0.0, rng.standard_normal(S.n))
    Ax, Ay = n(S.apply(t(x))), n(S.apply(t(y)))
    xAy, yAx = x @ np.where(mask, 0.0, Ay), y @ np.where(mask, 0.0, Ax)
    assert abs(xAy - yAx) <= 1e-12 * (np.abs(x) @ np.abs(Ay) + np.abs(y) @ np.abs(Ax))
    assert x @ np.where(mask, 0.0, Ax) > 0 and y @ np.where(mask, 0.0, Ay) > 0
    zx = n(S.vcycle(t(x, torch.float32)))
    zy = n(S.vcycle(t(y, torch.float32)))
    yBx, xBy = y @ np.where(mask, 0.0, zx), x @ np.where(mask, 0.0, zy)
    assert abs(yBx - xBy) <= 1e-5 * (np.abs(y) @ np.abs(zx) + np.abs(x) @ np.abs(zy))
    assert x @ np.where(mask, 0.0, zx) > 0
