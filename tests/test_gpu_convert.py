"""The FP64 <-> FP32 conversions of the mixed-precision kernels (integer operations on the
IEEE-754 bit patterns) against IEEE-754 conversion (numpy, round to nearest even).

FP64 -> FP32 must equal the IEEE result bit for bit wherever that result is a normal float or
an infinity, except at exact halfway points (there it rounds away from zero); results in the
subnormal range are signed zeros, NaNs become infinities. FP32 -> FP64 is exact for normal
floats, infinities and NaNs; subnormals become signed zeros.
"""
import numpy as np
import pytest
import torch

from paper_2004_02276_gb300 import binding

pytestmark = pytest.mark.gpu

FLT_MIN = np.float32(np.finfo(np.float32).tiny)


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__

    __graft_entry__.build()
    torch.cuda.set_device(0)


def d2f_gpu(x):
    y = binding.convert(torch.from_numpy(np.ascontiguousarray(x)).cuda())
    torch.cuda.synchronize()
    return y.cpu().numpy()


def f2d_gpu(x):
    y = binding.convert(torch.from_numpy(np.ascontiguousarray(x)).cuda())
    torch.cuda.synchronize()
    return y.cpu().numpy()


def bits32(a):
    return np.asarray(a, dtype=np.float32).view(np.uint32)


def test_f64_to_f32_random():
    rng = np.random.default_rng(0)
    n = 1 << 22
    # magnitudes from 2^-160 to 2^140 (below the subnormal range to beyond FLT_MAX), both signs,
    # full 52-bit mantissas
    e = rng.integers(-160, 141, n)
    m = rng.integers(0, 1 << 52, n, dtype=np.int64)
    x = np.ldexp(1.0 + m / 2.0**52, e) * np.where(rng.random(n) < 0.5, -1.0, 1.0)
    got = d2f_gpu(x)
    with np.errstate(over="ignore"):
        ref = x.astype(np.float32)
    normal = np.isfinite(ref) & (np.abs(ref) >= FLT_MIN)
    assert normal.sum() > n // 2
    # exact halfway points are measure-zero among random mantissas: bitwise equal
    assert np.array_equal(bits32(got[normal]), bits32(ref[normal]))
    over = np.isinf(ref)
    assert over.sum() > 0 and np.array_equal(bits32(got[over]), bits32(ref[over]))
    tiny = np.abs(ref) < FLT_MIN
    assert tiny.sum() > 0
    assert np.all(got[tiny] == 0.0) and np.array_equal(np.signbit(got[tiny]), np.signbit(x[tiny]))


def test_f64_to_f32_edges():
    fmax = float(np.finfo(np.float32).max)
    ulp1 = 2.0**-23
    x = np.array([
        0.0, -0.0, 1.0, -1.0, 0.1, -3.5, fmax, -fmax,
        float(FLT_MIN), -float(FLT_MIN),
        float(FLT_MIN) * (1 - 2.0**-25),       # rounds up to FLT_MIN
        float(FLT_MIN) * (1 - 2.0**-22),       # rounds to a subnormal in IEEE: zero here
        1.0 + ulp1 / 2,                        # halfway: away from zero -> 1 + ulp (IEEE even: 1)
        -(1.0 + ulp1 / 2),
        1.0 + 3 * ulp1 / 2,                    # halfway with odd neighbour: both give 1 + 2 ulp
        1.0 + ulp1 / 2 + 2.0**-50,             # just above halfway
        1.0 + ulp1 / 2 - 2.0**-50,             # just below halfway
        2.0 - 2.0**-30,                        # mantissa carry into the exponent -> 2.0
        fmax + 2.0**103,                       # halfway above FLT_MAX -> inf (both rules)
        1e300, -1e300, 1e-300, -1e-300, np.inf, -np.inf, np.nan,
    ])
    got = d2f_gpu(x)
    want = np.array([
        0.0, -0.0, 1.0, -1.0, np.float32(0.1), -3.5, fmax, -fmax,
        FLT_MIN, -FLT_MIN, FLT_MIN, 0.0,
        1.0 + ulp1, -(1.0 + ulp1), 1.0 + 2 * ulp1, 1.0 + ulp1, 1.0, 2.0,
        np.inf, np.inf, -np.inf, 0.0, -0.0, np.inf, -np.inf, np.inf,
    ], dtype=np.float32)
    assert np.array_equal(bits32(got), bits32(want)), (got, want)


def test_f32_to_f64_all_exponents():
    rng = np.random.default_rng(1)
    b = rng.integers(0, 1 << 32, 1 << 22, dtype=np.uint64).astype(np.uint32)
    b[:4] = [0x00000000, 0x80000000, 0x7F800000, 0xFF800000]  # +-0, +-inf
    b[4:6] = [0x7FC00001, 0xFFA00000]  # NaNs
    x = b.view(np.float32)
    got = f2d_gpu(x)
    with np.errstate(invalid="ignore"):  # the NaN inputs
        ref = x.astype(np.float64)
    sub = (b & 0x7F800000) == 0
    nan = np.isnan(ref)
    rest = ~sub & ~nan
    assert np.array_equal(got[rest].view(np.uint64), ref[rest].view(np.uint64))
    assert np.all(np.isnan(got[nan]))
    assert np.all(got[sub] == 0.0) and np.array_equal(np.signbit(got[sub]), np.signbit(x[sub]))


def test_convert_argument_errors():
    x = torch.zeros(4, dtype=torch.float64, device="cuda")
    lib = binding.lib()
    assert lib.strm_convert_f64_f32(binding._ptr(x), None, 4, None) == -1  # STRM_EINVAL
    assert lib.strm_convert_f32_f64(None, binding._ptr(x), -1, None) == -1  # STRM_EINVAL
    assert lib.strm_convert_f64_f32(None, None, 0, None) == 0
