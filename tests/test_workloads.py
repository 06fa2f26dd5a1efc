"""Seeded input generators: SplitMix64 against its published first outputs for seed 0,
Box-Muller moments, determinism of the workload fields, and each configuration's stated
mesh, order, domain, surface and node count."""
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


def _nodes(w):
    NX = w.cells_x * w.order + (0 if w.periodic else 1)
    return NX * (w.cells_z * (w.order_z or w.order) + 1)


def test_config_recipes():
    """Every configuration is the stated mesh, order, domain, surface and size."""
    c1 = W.config1()
    assert (c1.cells_x, c1.cells_z, c1.order, c1.x0, c1.x1, c1.h, c1.periodic) == (16, 4, 4, 0.0, 10.0, 1.0, False)
    assert c1.rhs == "source" and c1.noise_sd == 1e-3 and c1.surface.amp == 0.0 and _nodes(c1) == 1105
    np.testing.assert_allclose(c1.pressure.k, 2 * np.pi / 10, rtol=1e-15)
    for w, P, n in ((W.config2(), 6, 593089), (W.config3(), 8, 1052929)):
        assert (w.cells_x, w.cells_z, w.order, w.x0, w.x1, w.h, w.periodic) == (512, 32, P, 0.0, 200.0, 1.0, False)
        assert w.rhs == "div" and _nodes(w) == n
        assert (w.surface.amp, w.surface.noise_amp) == (0.05, 0.01)
        np.testing.assert_allclose(w.surface.k, 2 * np.pi / 10, rtol=1e-15)
    c5 = W.config5()
    assert (c5.cells_x, c5.cells_z, c5.order, c5.x0, c5.x1, c5.periodic) == (256, 16, 6, 0.0, 20.0, True)
    assert (c5.surface.amp, c5.surface.k) == (0.05, np.pi) and _nodes(c5) == 148992
