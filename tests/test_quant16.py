"""The exact FP64 -> 16-bit rounding helper used by the 16-bit factor tests,
pinned against numpy's own IEEE half conversion and against the definition of
BF16 (a float32 whose low 16 bits are zero)."""

import numpy as np

from quant16 import bf16, fp16, round_to_format


def _samples():
    rng = np.random.Generator(np.random.PCG64(5))
    v = rng.uniform(-1, 1, 200000) * 2.0 ** rng.integers(-30, 1, 200000)
    # exact ties of the FP16 grid (odd multiples of half an ulp) and tiny values
    k = rng.integers(1024, 2048, 2000)
    ties = (2 * k + 1) * 2.0 ** -12
    sub = rng.integers(0, 4096, 2000) * 2.0 ** -26
    return np.concatenate([v, ties, -ties, sub, [0.0, -0.0, 1.0, -1.0]])


def test_fp16_rounding_matches_numpy_half():
    v = _samples()
    ref = v.astype(np.float16).astype(np.float64)
    assert np.array_equal(fp16(v), ref)


def test_bf16_rounding_is_nearest_even_float32_with_zero_low_half():
    v = _samples()
    q = bf16(v)
    bits = q.astype(np.float32).view(np.uint32)
    assert np.all(q.astype(np.float32).astype(np.float64) == q)
    assert np.all(bits & 0xFFFF == 0)
    # neighbours one bf16 step away are never closer
    up = (bits.astype(np.uint64) + 0x10000).astype(np.uint32).view(np.float32).astype(np.float64)
    dn = (bits.astype(np.int64) - 0x10000).clip(0).astype(np.uint32).view(np.float32).astype(np.float64)
    nz = np.abs(q) > 0
    assert np.all(np.abs(q - v) <= np.abs(up - v))
    assert np.all(np.abs(q - v)[nz] <= np.abs(dn - v)[nz])
    # ties go to the even neighbour
    t = np.array([1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, 0.5 + 2.0 ** -9])
    assert np.array_equal(bf16(t), np.array([1.0, 1.0 + 4 * 2.0 ** -8, 0.5]))


def test_half_ulp_bound():
    v = _samples()
    for mant, emin, f in ((10, -14, fp16), (7, -126, bf16)):
        a = np.abs(v[np.abs(v) <= 1.0])
        assert np.all(np.abs(f(a) - a) <= 2.0 ** -(mant + 2) + 2.0 ** (emin - mant - 1))
        assert np.array_equal(f(a), round_to_format(a, mant, emin))
