"""The device reciprocal of the pivots (Newton-Raphson from the hardware
approximation, used by the Gauss-Jordan decoupling and the block ILU(0) and
block-Jacobi inverses) against the device's own 1.0 / x: within one unit in the
last place over the whole normal range, both signs, and exactly the division's
result for zero, infinities, NaN and subnormals (which take the division)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def check():
    from paper_1811_11992_gb300 import build
    build.build()
    from paper_1811_11992_gb300.isc import check_reciprocal
    return check_reciprocal


def _ulps(a, b):
    ia = a.view(np.int64)
    ib = b.view(np.int64)
    return np.abs(ia - ib)


def test_normal_range_within_one_ulp(check):
    rng = np.random.default_rng(11)
    mant = rng.uniform(1.0, 2.0, 200_000)
    expo = rng.integers(-1021, 1023, 200_000)
    x = np.ldexp(mant, expo) * rng.choice([-1.0, 1.0], 200_000)
    # pivots of the workloads' decoupled blocks span a few decades around 1
    x = np.concatenate([x, rng.uniform(-1e3, 1e3, 50_000), 1.0 + np.arange(-50, 50) * 2.0 ** -52])
    x = x[x != 0.0]
    y, z = check(x)
    assert np.all(np.isfinite(y))
    u = _ulps(y, z)
    assert u.max() <= 1, (u.max(), x[np.argmax(u)])
    assert np.mean(u == 0) > 0.9         # nearly always the correctly rounded quotient


def test_special_values_take_the_division(check):
    tiny = np.nextafter(0.0, 1.0)
    x = np.array([0.0, -0.0, np.inf, -np.inf, np.nan, tiny, -tiny, 1e-310, 2.2250738585072014e-308,
                  1.7976931348623157e308, -1.7976931348623157e308])
    y, z = check(x)
    same = (y.view(np.int64) == z.view(np.int64)) | (np.isnan(y) & np.isnan(z))
    assert np.all(same[:8]), (x[:8], y[:8], z[:8])
    assert np.all(_ulps(y[8:], z[8:]) <= 1)     # smallest normal and the largest finite values
