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


@pytest.mark.parametrize("precision", [pmg.PMG_FP64, pmg.PMG_MIXED_FP32])
def test_batch_matches_oracle_and_single_solves(precision):
    ws = small_config4()
    B = pmg.Batch([w.mesh_kwargs() for w in ws], tol=1e-12, precision=precision)
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
