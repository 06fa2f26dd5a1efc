"""Seeded input generators: SplitMix64 against its published first outputs for seed 0,
Box-Muller moments, and determinism of the workload fields."""
import numpy as np

import workloads as W


def test_splitmix64_reference_outputs():
    got = [int(v) for v in W.splitmix64(0, 3)]
    assert got == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_normal_moments_and_determinism():
    z = W.normal(W.BASE_SEED, 200000)
    assert abs(z.mean()) < 0.01 and abs(z.std() - 1) < 0.01
    np.testing.assert_array_equal(z[:10], W.normal(W.BASE_SEED, 10))
    np.testing.assert_array_equal(z[5:10], W.normal(W.BASE_SEED, 5, offset=5))


def test_surface_unit_rms_noise():
    s = W.Surface.smoothed(0.0, 0.0, 1.0, 200.0, 0.0, 11)
    x = np.linspace(0, 200, 200001)[:-1]
    assert abs(np.sqrt(np.mean(s(x) ** 2)) - 1.0) < 1e-3


def test_config4_ranges():
    ps = W.config4()
    assert len(ps) == 64
    for w in ps:
        assert 64 <= w.cells_x <= 1024 and 8 <= w.cells_z <= 32 and 4 <= w.order <= 8
        assert 0.5 <= w.h <= 2.0
