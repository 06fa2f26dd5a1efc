"""pmg_apply_noalloc against pmg_apply.

pmg_apply_noalloc serves callers that may not allocate device memory (a host framework
that owns every device allocation, a fixed pool, code inside a stream capture); it keeps
its working data in a static device array of the library instead of a handle.  This file
is collected last so that a run stopping at the first failure has run every other test.
"""
import numpy as np
import pytest
import torch

import paper_2411_14977_gb300.pmg as pmg
import workloads as W

pytestmark = pytest.mark.gpu


def _reference(w, x):
    """The existing entry point: a handle, its geometry, pmg_apply."""
    S = pmg.Solver(**w.mesh_kwargs())
    xc, sr = S.node_coords()
    eta = torch.as_tensor(w.fields(xc, sr)["eta"], dtype=torch.float64, device="cuda")
    S.set_geometry(eta)
    y = S.apply(x)
    torch.cuda.synchronize()
    return eta, y, S


def test_noalloc_apply_matches_handle_apply_twice():
    rng = np.random.default_rng(11)
    cases = [W.tank(12, 3, 6), W.tank(7, 2, 8)]        # two calls in a row, different meshes
    for w in cases:
        S0 = pmg.Solver(**w.mesh_kwargs())
        x = torch.as_tensor(rng.standard_normal(S0.n), dtype=torch.float64, device="cuda")
        eta, yref, S = _reference(w, x)
        y = torch.full_like(x, float("nan"))
        pmg.apply_noalloc(w.mesh_kwargs(), eta, x, y)
        torch.cuda.synchronize()
        scale = torch.max(torch.abs(yref)).item()
        assert torch.max(torch.abs(y - yref)).item() <= 1e-12 * scale


def test_noalloc_rejects_oversized_mesh():
    big = dict(cells_x=4096, cells_z=32, order=8, x0=0.0, x1=1600.0, h=1.0)
    t = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(pmg.PmgError) as e:
        pmg.apply_noalloc(big, t, t, t)
    assert e.value.status == pmg.PMG_ERR_INVALID and "static scratch" in str(e.value)
