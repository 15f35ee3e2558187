"""The seeded synthetic inputs: deterministic, of the requested size, and with
the structure their recipes state (Sec. 3.2 test sets, Sec. 3.5 galaxy)."""
import numpy as np
import pytest

from paper_2002_04894_gb300 import inputs


@pytest.mark.parametrize("kind", sorted(inputs.DISTRIBUTIONS))
@pytest.mark.parametrize("n", [1, 999, 20000])
def test_deterministic_and_sized(kind, n):
    a = inputs.points(kind, n, seed=3)
    b = inputs.points(kind, n, seed=3)
    assert a.shape == (n, 3) and a.dtype == np.float64
    np.testing.assert_array_equal(a, b)
    assert np.isfinite(a).all()
    if n > 1:
        assert not np.array_equal(a, inputs.points(kind, n, seed=4))


def test_galaxy_is_a_thin_multiscale_disc():
    x = inputs.points("galaxy", 200_000, seed=0) - 0.5
    r = np.hypot(x[:, 0], x[:, 1])
    # disc: the vertical spread is a small fraction of the in-plane one
    assert x[:, 2].std() < 0.1 * np.abs(x[:, :2]).std()
    # ring: few points inside the inner radius (6000 of 18000 pc, less the
    # spread of the refinement spheroids)
    r_in = 6000.0 / (2.2 * 18000.0)
    assert np.mean(r < 0.6 * r_in) < 0.01
    # clumped: counts in 200 x 200 columns over the plane are overdispersed
    # (variance / mean over occupied columns is ~1 for a Poisson cloud)
    h, _, _ = np.histogram2d(x[:, 0] + 0.5, x[:, 1] + 0.5, bins=200, range=[[0, 1], [0, 1]])
    h = h[h > 0]
    assert h.var() / h.mean() > 5


def test_galaxy_generations_keep_the_seed_ring_for_small_n():
    x = inputs.points("galaxy", 5000, seed=1) - 0.5
    r = np.hypot(x[:, 0], x[:, 1]) * 2.2 * 18000.0
    assert r.min() >= 6000.0 * 0.99 and r.max() <= 18000.0 * 1.01
