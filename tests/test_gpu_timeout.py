"""The bounded device-side wait: the z-split Schwarz sweep waits on an mbarrier for its TMA
slab copies, and gives up after the handle's wait limit (pmg_set_wait_limit).  With a
limit of zero cycles every sweep gives up at once: each CTA raises the handle's timeout
flag, waits for its own copies in flight and returns, and pmg_solve reports
PMG_ERR_TIMEOUT.  No GPU fault is involved: the copies always land, and the handle is
usable again once the limit is restored."""
import numpy as np
import pytest

import paper_2411_14977_gb300.pmg as pmg
import workloads as W
from oracle.sem import solve_direct
from tests.gpu_helpers import Case, n, t

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("sweep", [1, 3096])
def test_wait_limit_zero_reports_timeout_and_recovers(sweep):
    c = Case(W.tank(8, 3, 6), precision=pmg.PMG_MIXED_FP32, tol=1e-11, max_iter=40, sweep_kernel=sweep)
    b, pD = c.rhs_gpu(), t(c.F["pD"])
    c.S.set_wait_limit(0)
    with pytest.raises(pmg.PmgError) as e:
        c.S.solve(b, pD)
    assert e.value.status == pmg.PMG_ERR_TIMEOUT
    # the flag is reported once; with the default limit restored the same handle solves
    c.S.set_wait_limit(-1)
    p, info = c.S.solve(b, pD)
    assert info["status"] == pmg.PMG_OK and info["rel_residual"] <= 1e-11
    pref = solve_direct(c.m.assemble(c.eta), c.rhs_oracle(), c.F["pD"], c.m.dirichlet_mask())
    assert np.linalg.norm(n(p) - pref) <= 1e-9 * np.linalg.norm(pref)
