"""The stochastic rounding of half storage against its definition.

The half-storage step keeps g and l as weight-shifted halves, rounded
stochastically so that the small per-step changes of conduction and of the
potential survive on average (the stored value is unbiased).  The library
performs that rounding with the GPU's conversion instruction; these tests
call it through the C ABI (`lbm_round_half_sr`) and compare each result bit
for bit with the definition written out here in exact float64 arithmetic,
and check the unbiasedness it exists for."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2410_06657_gb300 import lbm  # noqa: E402

pytestmark = pytest.mark.gpu

HALF_MAX = 65504.0


def definition(v: np.ndarray, r: np.ndarray) -> np.ndarray:
    """Half bits of v rounded with the 13 random bits r & 0x1fff."""
    r13 = (r.astype(np.uint32) & 0x1FFF).astype(np.float64)
    a = np.abs(v.astype(np.float64))
    out = np.zeros(v.shape, dtype=np.float64)
    nan = np.isnan(a)
    big = ~nan & (a >= 2.0 ** -14)
    # normal half range: spacing s = 2^(e - 10) at |v| in [2^e, 2^(e+1))
    e = np.floor(np.log2(np.where(big, a, 1.0)))
    s = np.exp2(e - 10)
    t = np.where(big, a, 0.0) / s
    q = np.floor(t)
    d = (t - q) * 8192.0                       # the 13 dropped bits, an integer
    up = (d + r13) >= 8192.0
    out = np.where(big, (q + up) * s, out)
    # subnormal half range: |v| + r 2^-37 in single precision, truncated
    small = ~nan & ~big
    x = (np.where(small, a, 0.0) + r13 * 2.0 ** -37).astype(np.float32).astype(np.float64)
    out = np.where(small, np.floor(x / 2.0 ** -24) * 2.0 ** -24, out)
    out = np.minimum(out, HALF_MAX)
    out = np.copysign(out, v.astype(np.float64))
    out = np.where(nan, np.nan, out)
    return out.astype(np.float16).view(np.uint16)


def run(v: np.ndarray, r: np.ndarray) -> np.ndarray:
    dv = torch.from_numpy(v.astype(np.float32)).cuda()
    dr = torch.from_numpy(r.astype(np.uint32).view(np.int32)).cuda()
    out = lbm.round_half_sr(dv, dr)
    torch.cuda.synchronize()
    return out.cpu().numpy().view(np.uint16)


def magnitudes(rng, n, lo_exp, hi_exp):
    """Floats with uniformly drawn exponents in [lo_exp, hi_exp] and random
    mantissas and signs (biased exponents of the float format)."""
    exp = rng.integers(lo_exp, hi_exp + 1, n).astype(np.uint32)
    bits = (rng.integers(0, 2, n).astype(np.uint32) << 31) | (exp << 23) | \
        rng.integers(0, 1 << 23, n).astype(np.uint32)
    return bits.view(np.float32)


@pytest.mark.parametrize("name,lo,hi", [
    ("normal halves", 113, 141),          # 2^-14 .. 2^15
    ("subnormal halves", 103, 112),       # 2^-24 .. 2^-14
    ("below the smallest half", 1, 102),  # normal floats under 2^-24
    ("float subnormals", 0, 0),
    ("beyond the half range", 142, 150),  # 2^15 .. 2^24 (from 65504 up)
])
def test_rounding_matches_its_definition(name, lo, hi):
    rng = np.random.default_rng(2410066 + lo)
    n = 1 << 18
    v = magnitudes(rng, n, lo, hi)
    r = rng.integers(0, 1 << 32, n, dtype=np.uint64).astype(np.uint32)
    got, want = run(v, r), definition(v, r)
    bad = np.nonzero(got != want)[0]
    assert bad.size == 0, f"{name}: {bad.size} of {n} differ, first v={v[bad[0]]!r} r={r[bad[0]] & 0x1fff}: " \
                          f"{got[bad[0]]:#06x} against {want[bad[0]]:#06x}"


def test_exact_values_zero_and_nan_pass_through():
    vals = np.array([0.0, -0.0, 1.0, -2.5, 65504.0, -65504.0, 2.0 ** -24, 3 * 2.0 ** -24, 2.0 ** -14,
                     np.float32(np.nan)], dtype=np.float32)
    for r in (0, 1, 0x1FFF, 0xFFFFFFFF):
        rr = np.full(vals.size, r, dtype=np.uint32)
        got = run(vals, rr)
        want = vals.astype(np.float16).view(np.uint16)
        assert np.array_equal(got[:-1], want[:-1])
        assert np.isnan(got[-1:].view(np.float16)[0])


def test_rounding_is_unbiased_over_the_random_bits():
    """Over all 8192 values of the random bits the mean of the rounded
    normal-range value is the input itself, exactly; in the subnormal range
    it is the input to within the 2^-37 resolution of the random bits."""
    rng = np.random.default_rng(2410067)
    for lo, hi, tol in ((113, 141, 0.0), (103, 112, 2.0 ** -37)):
        k = 48
        v = np.repeat(magnitudes(rng, k, lo, hi), 8192)
        r = np.tile(np.arange(8192, dtype=np.uint32), k)
        got = run(v, r).view(np.float16).astype(np.float64).reshape(k, 8192)
        mean = got.sum(axis=1) / 8192.0
        err = np.abs(mean - v[::8192].astype(np.float64))
        assert err.max() <= tol, (lo, err.max())


def test_long_ragged_array_is_rounded_element_for_element():
    """More elements than the launch has threads (the grid-stride loop goes
    round more than once) and a count that is no multiple of the block."""
    rng = np.random.default_rng(2410068)
    n = 1_000_003
    v = magnitudes(rng, n, 100, 145)
    r = rng.integers(0, 1 << 32, n, dtype=np.uint64).astype(np.uint32)
    got, want = run(v, r), definition(v, r)
    assert np.array_equal(got, want)
    assert np.array_equal(run(v[:1], r[:1]), want[:1])
