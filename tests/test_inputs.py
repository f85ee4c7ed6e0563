"""The seeded input generators terminate and are well formed on every box
shape the tests and the benchmark use, including one-cell axes."""
import numpy as np
import pytest

import rpk_inputs as I

T0 = 0.2948964908710633


@pytest.mark.parametrize("dims", [(1, 1, 1), (2, 1, 1), (3, 2, 1), (1, 5, 1), (150, 3, 2),
                                  (129, 1, 1), (5, 4, 3), (24, 16, 8), (32, 32, 32)])
def test_generators_on_all_shapes(dims):
    nx, ny, nz = dims
    n = 2 * nx * ny * nz
    for f in (I.random_smooth(nx, ny, nz, T0), I.fourier_modes(nx, ny, nz, T0)[0],
              I.uniform(nx, ny, nz, T0)):
        assert f["rho"].shape == (n,) and f["u"].shape == (3, n)
        assert np.all(f["rho"] > 0) and np.all(f["T"] > 0) and np.all(f["R"] > 0)
        assert np.all(np.isfinite(f["u"]))


def test_mode_count_and_determinism():
    f1, m1 = I.fourier_modes(16, 8, 4, T0)
    f2, m2 = I.fourier_modes(16, 8, 4, T0)
    assert len(m1) == 8
    np.testing.assert_array_equal(f1["rho"], f2["rho"])
    _, m = I.fourier_modes(2, 1, 1, T0, nmax=2)
    assert len(m) == 2
    _, m = I.fourier_modes(1, 1, 1, T0)
    assert m == []


def test_tile_is_periodic_copy():
    f, _ = I.fourier_modes(4, 3, 2, T0)
    g = I.tile(f, 4, 3, 2, (2, 3, 2))
    a = g["u"].reshape(3, 2, 4, 9, 8)
    assert np.array_equal(a[..., :4], a[..., 4:])
    assert np.array_equal(a[:, :, :2], a[:, :, 2:])
