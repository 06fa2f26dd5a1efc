"""The launch-configuration query (pmg_level_kernels) reports a valid configuration for
every level: the creation defaults, each forced level-operator family, and after the
autotuner's choice."""
import pytest

import paper_2411_14977_gb300.pmg as pmg
import workloads as W

from gpu_helpers import Case

pytestmark = pytest.mark.gpu


def _tile_ok(code):
    ext, zt = (code // 100) % 100, code % 100
    return code // 10000 == 1 and ext in (8, 16, 32) and zt in (4, 8) and (ext * zt) % 32 == 0 and ext * zt <= 256


def _valid_flat(code):
    return 32 <= code <= 512 or -256 <= code <= -32 or _tile_ok(code)


@pytest.mark.parametrize("flat", [-1, 0, 1, 2, 13204])
def test_level_kernels_valid(flat):
    c = Case(W.tank(12, 3, 6), precision=pmg.PMG_MIXED_FP32, flat_kernel=flat)
    S = c.S
    before = [S.level_kernels(l) for l in range(S.nlevels)]
    if flat == 1:
        assert all(k["flat32"] < 0 for k in before)
    if flat == 2:
        assert all(k["flat32"] == 11608 for k in before)
    if flat == 13204:
        assert all(k["flat32"] == 13204 for k in before)
    S.autotune()
    after = [S.level_kernels(l) for l in range(S.nlevels)]
    for k in after:
        assert _valid_flat(k["flat32"]), k
    if flat == 0:
        assert all(k["flat32"] > 0 for k in after)
    if flat in (2, 13204):
        assert all(_tile_ok(k["flat32"]) for k in after)   # constant depth, orders <= 8
    with pytest.raises(pmg.PmgError):
        S.level_kernels(S.nlevels)
