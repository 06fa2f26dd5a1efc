"""Batched solves (independent problems of uneven size and order, concurrent
device-side loops) and the CTA-size autotuner, against the CPU oracle."""
import numpy as np
import pytest
import torch

import paper_2411_14977_gb300.pmg as pmg
import workloads as W
from oracle.sem import Mesh, solve_direct
from tests.gpu_helpers import n, t

pytestmark = pytest.mark.gpu


def small_config4(k=5):
    """Config 4's problem family (harmonic Dirichlet data, exact wall flux, noise, depth
    h and surface per problem) on meshes small enough for the oracle's direct solve."""
    out = []
    for j, (nx, nz, P, h) in enumerate([(9, 3, 4, 0.7), (14, 2, 5, 1.6), (6, 4, 6, 1.0), (11, 2, 7, 0.5),
                                        (5, 3, 8, 1.9)][:k]):
        seed = W.BASE_SEED + 4 + 1000 * (j + 1)
        L = 0.390625 * nx
        s = W.Surface.smoothed(0.05 * h, 2 * np.pi / 10, 0.01 * h, L, 0.0, seed)
        out.append(W.Workload(f"small4_{j}", nx, nz, P, 0.0, L, h, False, seed, s, "source",
                              pressure=W.Harmonic(2 * np.pi / 10, 0.0, h), noise_sd=1e-3))
    return out


def uneven_batch():
    """Config 4's family with every order 4..8, column depths 1..5 cells, a periodic tank,
    and element-column counts from 1 to 17: uneven work per problem and per level."""
    out = small_config4()
    for j, (nx, nz, P, h, per) in enumerate([(1, 2, 5, 1.2, False), (8, 5, 4, 0.8, True), (17, 1, 6, 1.4, False),
                                               (4, 2, 8, 0.6, True), (3, 3, 7, 1.1, False)]):
        seed = W.BASE_SEED + 4 + 1000 * (j + 11)
        L = 0.390625 * nx
        if per:
            s = W.Surface(0.03 * h, 2 * np.pi / L)
        else:
            s = W.Surface.smoothed(0.05 * h, 2 * np.pi / 10, 0.01 * h, L, 0.0, seed)
        out.append(W.Workload(f"uneven_{j}", nx, nz, P, 0.0, L, h, per, seed, s, "source",
                              pressure=None if per else W.Harmonic(2 * np.pi / 10, 0.0, h), noise_sd=1e-3))
    return out


def _inputs(ws, B):
    bs, pds, refs = [], [], []
    for w, S in zip(ws, B.members):
        xc, sr = S.node_coords()
        F = w.fields(xc, sr)
        S.set_geometry(t(F["eta"]))
        per = w.periodic
        b = S.assemble_rhs(t(F["f"]), t(F["g_bottom"]), None if per else t(F["g_left"]),
                           None if per else t(F["g_right"]))
        bs.append(b)
        pds.append(t(F["pD"]))
        m = Mesh(**w.mesh_kwargs())
        bo = m.rhs_source(F["eta"], F["f"], F["g_bottom"], None if per else F["g_left"],
                          None if per else F["g_right"])
        refs.append(solve_direct(m.assemble(F["eta"]), bo, F["pD"], m.dirichlet_mask()))
    return bs, pds, refs


def test_batched_graph_uneven_orders_against_oracle():
    """The single graph of batched launches (mixed precision): ten problems of orders 4..8,
    1..17 element columns, 1..5 element rows, walls and a periodic tank, all against the
    oracle's direct solves; two calls in a row give the same bits; a zero right-hand side
    and a non-finite one finish at once with their own status, the others unaffected."""
    ws = uneven_batch()
    B = pmg.Batch([w.mesh_kwargs() for w in ws], tol=1e-12, precision=pmg.PMG_MIXED_FP32)
    assert B.info()["batched"] == 1
    bs, pds, refs = _inputs(ws, B)
    outs, infos = B.solve(bs, pds)
    assert B.info()["launches"] > 0
    for o, ref, info in zip(outs, refs, infos):
        assert info["status"] == 0 and info["rel_residual"] <= 1e-12, info
        assert info["iterations"] > 0
        assert np.linalg.norm(n(o) - ref) <= 1e-10 * np.linalg.norm(ref)
    outs2, infos2 = B.solve(bs, pds)
    for o, o2, i1, i2 in zip(outs, outs2, infos, infos2):
        assert torch.equal(o, o2) and i1["iterations"] == i2["iterations"]
    # the host-driven loop (profiling aid) runs the same launches: the same bits
    B.set_path(1)
    outs_e, infos_e = B.solve(bs, pds)
    B.set_path(0)
    for o, o2, i1, i2 in zip(outs, outs_e, infos, infos_e):
        assert torch.equal(o, o2) and i1["iterations"] == i2["iterations"]
    # the per-problem loops reach the same pressures (their own kernels: not the same bits)
    B.set_path(2)
    assert B.info()["batched"] == 0
    outs_s, infos_s = B.solve(bs, pds)
    B.set_path(0)
    for o, ref, info in zip(outs_s, refs, infos_s):
        assert info["status"] == 0 and np.linalg.norm(n(o) - ref) <= 1e-10 * np.linalg.norm(ref)
    bz = [b.clone() for b in bs]
    bz[2].zero_()
    pz = [p.clone() for p in pds]
    pz[2].zero_()
    bz[5][3] = float("nan")
    outs3, infos3 = B.solve(bz, pz, raise_on_error=False)
    assert infos3[2]["status"] == 0 and infos3[2]["iterations"] == 0 and torch.count_nonzero(outs3[2]) == 0
    assert infos3[5]["status"] == pmg.PMG_ERR_NONFINITE
    for k in (0, 1, 3, 4, 6, 7, 8, 9):
        assert infos3[k]["status"] == 0
        assert np.linalg.norm(n(outs3[k]) - refs[k]) <= 1e-10 * np.linalg.norm(refs[k])


def test_batched_graph_iteration_cap():
    """A cap of two outer iterations: every problem stops with PMG_ERR_NOT_CONVERGED, two
    iterations, a finite residual below the start."""
    ws = small_config4(3)
    B = pmg.Batch([w.mesh_kwargs() for w in ws], tol=1e-12, max_iter=2, precision=pmg.PMG_MIXED_FP32)
    bs, pds, _ = _inputs(ws, B)
    _, infos = B.solve(bs, pds, raise_on_error=False)
    for info in infos:
        assert info["status"] == pmg.PMG_ERR_NOT_CONVERGED and info["iterations"] == 2, info
        assert 0 < info["rel_residual"] < 1


@pytest.mark.parametrize("precision", [pmg.PMG_FP64, pmg.PMG_MIXED_FP32])
def test_batch_matches_oracle_and_single_solves(precision):
    ws = small_config4()
    B = pmg.Batch([w.mesh_kwargs() for w in ws], tol=1e-12, precision=precision)
    assert B.info()["batched"] == (1 if precision == pmg.PMG_MIXED_FP32 else 0)
    bs, pds, refs, singles = [], [], [], []
    for w, S in zip(ws, B.members):
        xc, sr = S.node_coords()
        F = w.fields(xc, sr)
        S.set_geometry(t(F["eta"]))
        b = S.assemble_rhs(t(F["f"]), t(F["g_bottom"]), t(F["g_left"]), t(F["g_right"]))
        bs.append(b)
        pds.append(t(F["pD"]))
        m = Mesh(**w.mesh_kwargs())
        bo = m.rhs_source(F["eta"], F["f"], F["g_bottom"], F["g_left"], F["g_right"])
        refs.append(solve_direct(m.assemble(F["eta"]), bo, F["pD"], m.dirichlet_mask()))
        single = pmg.Solver(**w.mesh_kwargs(), tol=1e-12, precision=precision)
        single.set_geometry(t(F["eta"]))
        singles.append(single.solve(b, pds[-1])[0])
    outs, infos = B.solve(bs, pds)
    for o, ref, sgl, info in zip(outs, refs, singles, infos):
        assert info["status"] == 0 and info["rel_residual"] <= 1e-12, info
        assert np.linalg.norm(n(o) - ref) <= 1e-10 * np.linalg.norm(ref)
        assert torch.allclose(o, sgl, rtol=0, atol=1e-10 * torch.max(torch.abs(sgl)).item())


@pytest.mark.parametrize("fuse", [0, -1])
def test_autotune_keeps_results(fuse):
    """CTA sizes, the level-operator kernel and (fuse -1) the fused level residuals picked
    by timing leave the answer unchanged."""
    w = W.tank(16, 4, 6)
    S = pmg.Solver(**w.mesh_kwargs(), tol=1e-11, precision=pmg.PMG_MIXED_FP32, fuse_residual=fuse)
    xc, sr = S.node_coords()
    F = w.fields(xc, sr)
    S.set_geometry(t(F["eta"]))
    b = S.assemble_rhs_div(t(F["u"]), t(F["w"]))
    p1, i1 = S.solve(b, t(F["pD"]))
    S.autotune()
    p2, i2 = S.solve(b, t(F["pD"]))
    assert i2["rel_residual"] <= 1e-11
    assert torch.allclose(p1, p2, rtol=0, atol=1e-9 * torch.max(torch.abs(p1)).item())
