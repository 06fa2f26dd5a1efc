"""pmg_apply_noalloc against pmg_apply.

pmg_apply_noalloc serves callers that may not allocate device memory (a host framework
that owns every device allocation, a fixed pool, code inside a stream capture); it keeps
its working data in a static device array of the library instead of a handle.  This file
is collected last so that a run stopping at the first failure has run every other test.
"""
import dataclasses

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


# two calls in a row on walled meshes, then a periodic one (its last slab edge wraps to
# the first: a different edge path in the kernel)
CASES = [W.tank(12, 3, 6), W.tank(7, 2, 8), dataclasses.replace(W.tank(8, 3, 6), periodic=True)]


def test_noalloc_apply_matches_handle_apply_twice():
    rng = np.random.default_rng(11)
    for w in CASES:
        S0 = pmg.Solver(**w.mesh_kwargs())
        x = torch.as_tensor(rng.standard_normal(S0.n), dtype=torch.float64, device="cuda")
        eta, yref, S = _reference(w, x)
        y = torch.full_like(x, float("nan"))
        pmg.apply_noalloc(w.mesh_kwargs(), eta, x, y)
        torch.cuda.synchronize()
        scale = torch.max(torch.abs(yref)).item()
        assert torch.max(torch.abs(y - yref)).item() <= 1e-12 * scale


def test_noalloc_bad_depth_gives_nan():
    # eta <= -h somewhere: the handle path returns PMG_ERR_INVALID; the allocation-free
    # call reads nothing back and reports it as NaN in every entry of y
    w = W.tank(8, 2, 6)
    S0 = pmg.Solver(**w.mesh_kwargs())
    xc, sr = S0.node_coords()
    eta = np.array(w.fields(xc, sr)["eta"])
    eta[len(eta) // 2] = -2.0 * w.h
    x = torch.ones(S0.n, dtype=torch.float64, device="cuda")
    y = torch.zeros_like(x)
    pmg.apply_noalloc(w.mesh_kwargs(), torch.as_tensor(eta, device="cuda"), x, y)
    torch.cuda.synchronize()
    assert torch.isnan(y).all()
    # the next call on a good surface is unaffected
    eta_ok = torch.as_tensor(w.fields(xc, sr)["eta"], dtype=torch.float64, device="cuda")
    _, yref, _ = _reference(w, x)
    pmg.apply_noalloc(w.mesh_kwargs(), eta_ok, x, y)
    torch.cuda.synchronize()
    assert torch.max(torch.abs(y - yref)).item() <= 1e-12 * torch.max(torch.abs(yref)).item()


def test_noalloc_rejects_oversized_or_invalid_mesh():
    big = dict(cells_x=4096, cells_z=32, order=8, x0=0.0, x1=1600.0, h=1.0)
    t = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(pmg.PmgError) as e:
        pmg.apply_noalloc(big, t, t, t)
    assert e.value.status == pmg.PMG_ERR_INVALID and "static scratch" in str(e.value)
    # the mesh rules of pmg_create: cells_z <= 64, a power-of-two periodic cells_x
    for bad in (dict(cells_x=4, cells_z=65, order=2), dict(cells_x=6, cells_z=2, order=4, periodic=True)):
        with pytest.raises(pmg.PmgError) as e:
            pmg.apply_noalloc(dict(bad, x0=0.0, x1=1.0, h=1.0), t, t, t)
        assert e.value.status == pmg.PMG_ERR_INVALID
