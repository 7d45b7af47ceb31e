"""The integer-pipe precision conversions of the mixed-precision path
(mg_convert_f64_to_f32 / mg_convert_f32_to_f64) against the hardware
conversions that torch performs on the same device: identical bits for every
non-NaN input, NaN for NaN."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1910_12979_gb300 import native as N  # noqa: E402

DEV = "cuda:0"


def _f64_cases(rng):
    """Random bit patterns (every exponent, NaN, infinity, subnormals) plus
    doubles placed exactly on, just below and just above the midpoint between
    two neighbouring floats (the ties-to-even cases), zeros and range ends."""
    raw = rng.integers(0, 2 ** 64, size=200_000, dtype=np.uint64).view(np.float64)
    with np.errstate(over="ignore"):
        f = (rng.normal(size=50_000) * 2.0 ** rng.integers(-140, 128, size=50_000)).astype(np.float32)
    f = f[np.isfinite(f)].astype(np.float64)      # exact floats, held as doubles
    bits = f.view(np.uint64)
    half = np.uint64(1 << 28)                      # half a float ulp in the double's fraction
    ties = np.concatenate([bits + half, bits + half - np.uint64(1), bits + half + np.uint64(1)]).view(np.float64)
    fmax, fmin = float(np.finfo(np.float32).max), float(np.finfo(np.float32).tiny)
    edge = np.array([0.0, -0.0, 1.0, -1.0, fmax, -fmax, fmin, -fmin, fmin / 2, fmax * (1 + 2 ** -25),
                     fmax * (1 + 2 ** -24), fmax * (1 - 2 ** -26), np.inf, -np.inf, np.nan, 5e-324, 1e300, -1e-300])
    return np.concatenate([raw, ties, edge])


def test_f64_to_f32_matches_hardware_rounding():
    x = torch.from_numpy(_f64_cases(np.random.default_rng(11))).to(DEV)
    y = torch.empty(x.numel(), dtype=torch.float32, device=DEV)
    N.mg_convert_f64_to_f32(x.data_ptr(), y.data_ptr(), x.numel(), None)
    ref = x.float()
    torch.cuda.synchronize()
    nan = torch.isnan(ref)
    assert torch.equal(torch.isnan(y), nan)
    assert torch.equal(y[~nan].view(torch.int32), ref[~nan].view(torch.int32))


def test_f32_to_f64_exact():
    rng = np.random.default_rng(12)
    raw = rng.integers(0, 2 ** 32, size=300_000, dtype=np.uint64).astype(np.uint32).view(np.float32)
    edge = np.array([0.0, -0.0, np.inf, -np.inf, np.nan, 1e-45, -1e-45, 1.1754942e-38, 3.4028235e38],
                    dtype=np.float32)
    x = torch.from_numpy(np.concatenate([raw, edge])).to(DEV)
    y = torch.empty(x.numel(), dtype=torch.float64, device=DEV)
    N.mg_convert_f32_to_f64(x.data_ptr(), y.data_ptr(), x.numel(), None)
    ref = x.double()
    torch.cuda.synchronize()
    nan = torch.isnan(ref)
    assert torch.equal(torch.isnan(y), nan)
    assert torch.equal(y[~nan].view(torch.int64), ref[~nan].view(torch.int64))


def test_convert_rejects_null():
    with pytest.raises(N.MGError):
        N.mg_convert_f64_to_f32(None, None, 4, None)
    N.mg_convert_f32_to_f64(None, None, 0, None)   # nothing to do


def test_reciprocal_within_one_ulp():
    """mg_reciprocal_f64 (Newton's method from a binary32 estimate) against the
    correctly rounded quotient: at most one ulp away over every exponent, and
    exact IEEE results for zeros, infinities, NaN and the range ends."""
    rng = np.random.default_rng(13)
    mant = rng.uniform(1.0, 2.0, size=400_000)
    x = mant * 2.0 ** rng.integers(-1022, 1023, size=mant.size) * rng.choice([-1.0, 1.0], size=mant.size)
    edge = np.array([0.0, -0.0, np.inf, -np.inf, np.nan, 1.0, 2.0 ** -125, 2.0 ** 126, 2.0 ** 126 * (1 - 2 ** -53),
                     2.0 ** -125 * (1 - 2 ** -53), 5e-324, 1.7976931348623157e308, 3.0, 7.0, 0.1])
    xt = torch.from_numpy(np.concatenate([x, edge])).to(DEV)
    y = torch.empty_like(xt)
    N.mg_reciprocal_f64(xt.data_ptr(), y.data_ptr(), xt.numel(), None)
    ref = 1.0 / xt
    torch.cuda.synchronize()
    nan = torch.isnan(ref)
    assert torch.equal(torch.isnan(y), nan)
    yi, ri = y[~nan].view(torch.int64), ref[~nan].view(torch.int64)
    assert int((yi - ri).abs().max()) <= 1   # same sign, neighbouring bit patterns


@pytest.mark.parametrize("shift", [-60, -13, 0, 7, 100])
def test_f64_to_f32_pow2_matches_scaled_hardware_rounding(shift):
    """The FP64 residual kernels fold their power-of-two scale into the
    conversion: the result must equal converting the exactly scaled double."""
    x = torch.from_numpy(_f64_cases(np.random.default_rng(1000 + shift))).to(DEV)
    y = torch.empty(x.numel(), dtype=torch.float32, device=DEV)
    N.mg_convert_f64_to_f32_pow2(x.data_ptr(), y.data_ptr(), x.numel(), shift, None)
    ref = (x * 2.0 ** shift).float()
    torch.cuda.synchronize()
    nan = torch.isnan(ref)
    assert torch.equal(torch.isnan(y), nan)
    assert torch.equal(y[~nan].view(torch.int32), ref[~nan].view(torch.int32))
    with pytest.raises(N.MGError):
        N.mg_convert_f64_to_f32_pow2(x.data_ptr(), y.data_ptr(), x.numel(), 2000, None)
