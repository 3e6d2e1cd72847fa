"""The device reciprocal used for 1/|det E| and 1/det M, and the device square
root used for the face areas (Newton iterations from single-precision seeds),
against the correctly rounded IEEE results computed on the host: at most one
ulp away in their fast ranges, the IEEE result itself outside them."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ph():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2509_11133_gb300 as ph
    from paper_2509_11133_gb300 import build
    build.build()
    ph.load()
    return ph


def ulps(a, b):
    """Distance in ulps between two positive doubles."""
    return np.abs(a.view(np.int64) - b.view(np.int64))


def test_fast_range_within_one_ulp(ph):
    rng = np.random.default_rng(0)
    e = rng.uniform(-1019.5, 1020.5, 4_000_000)
    x = np.ldexp(rng.uniform(1.0, 2.0, e.size), np.floor(e).astype(int))
    # mantissa extremes and powers of two
    x = np.concatenate([x, 2.0 ** np.arange(-1020, 1021), np.nextafter(2.0 ** np.arange(-1019, 1021), 0),
                        np.nextafter(2.0 ** np.arange(-1020, 1020), np.inf), [1.0, 3.0, 7.0, 1 / 3]])
    y = ph.ph_rcp(torch.as_tensor(x, device="cuda")).cpu().numpy()
    ref = 1.0 / x
    d = ulps(y, ref)
    assert d.max() <= 1
    assert (d == 0).mean() > 0.9            # mostly the rounded quotient itself


def test_outside_fast_range_is_ieee(ph):
    tiny = np.array([5e-324, 2.2250738585072014e-308, 2.0 ** -1021, np.nextafter(2.0 ** -1020, 0)])
    huge = np.array([2.0 ** 1021, 1.7976931348623157e308, np.nextafter(2.0 ** 1021, np.inf)])
    special = np.array([0.0, -0.0, -1.0, -2.5e-300, np.inf, -np.inf, np.nan])
    x = np.concatenate([tiny, huge, special])
    y = ph.ph_rcp(torch.as_tensor(x, device="cuda")).cpu().numpy()
    with np.errstate(divide="ignore", over="ignore"):
        ref = 1.0 / x
    # the device may flush subnormal results of the IEEE divide differently
    # from the host in no case: both are correctly rounded
    same = (y.view(np.int64) == ref.view(np.int64)) | (np.isnan(y) & np.isnan(ref))
    assert same.all(), (x[~same], y[~same], ref[~same])


def test_half_sqrt_fast_range_within_one_ulp(ph):
    rng = np.random.default_rng(1)
    e = rng.uniform(-960.0, 960.0, 4_000_000)
    x = np.ldexp(rng.uniform(1.0, 2.0, e.size), np.floor(e).astype(int))
    p2 = 2.0 ** np.arange(-960, 960)
    # powers of two (both exponent parities), their neighbours, perfect squares,
    # mantissas next to 1, 2 and 4 after the exponent split, typical face sizes
    sq = np.arange(1, 5000, dtype=np.float64) ** 2
    x = np.concatenate([sq, x, p2, np.nextafter(p2[1:], 0), np.nextafter(p2, np.inf), sq * 2.0 ** -80,
                        np.nextafter(sq, np.inf), rng.uniform(1e-16, 1e-2, 200_000)])
    y = ph.ph_half_sqrt(torch.as_tensor(x, device="cuda")).cpu().numpy()
    ref = 0.5 * np.sqrt(x)
    d = ulps(y, ref)
    assert d.max() <= 1
    assert (d == 0).mean() > 0.99           # almost always the rounded root itself
    assert (y[:sq.size] == np.arange(1, 5000) / 2).all()  # exact roots are found exactly


def test_half_sqrt_outside_fast_range_is_ieee(ph):
    x = np.array([0.0, -0.0, 5e-324, 2.2250738585072014e-308, 2.0 ** -961, np.nextafter(2.0 ** -960, 0),
                  2.0 ** 960, 1.7976931348623157e308, np.inf, -1.0, -np.inf, np.nan])
    y = ph.ph_half_sqrt(torch.as_tensor(x, device="cuda")).cpu().numpy()
    with np.errstate(invalid="ignore"):
        ref = 0.5 * np.sqrt(x)
    same = (y.view(np.int64) == ref.view(np.int64)) | (np.isnan(y) & np.isnan(ref))
    assert same.all(), (x[~same], y[~same], ref[~same])
