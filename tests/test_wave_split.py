"""The wave encoding of the tensor-core sweep, restated in numpy (CPU): the
tile's incident waves w are scaled by sc = 2^(13 - E), E the exponent of the
largest |w|, and entered as two 16-bit numbers hi = rn(sc w), lo = rn(sc w -
hi) (FP32 difference).  This checks the precision the kernel's design relies
on: hi + lo carries sc w to about 2^-22 (FP16) or 2^-16 (BF16) of the largest
wave, far below the 2^-11 / 2^-8 rounding of the stored reflection matrices.
It also checks that sc and 1 / sc are normal and exact inverses for every
exponent, including an all-zero tile and non-finite waves.
"""
import numpy as np
import pytest


def scale_pair(amax):
    """sc and 1/sc for the largest |w| (float32), as bit patterns: biased
    exponent e of amax, se = clamp(267 - e, 1, 253)."""
    e = (np.float32(amax).view(np.uint32) >> np.uint32(23)) & np.uint32(0xFF)
    se = int(min(max(267 - int(e), 1), 253))
    sc = np.uint32(se << 23).view(np.float32)
    isc = np.uint32((254 - se) << 23).view(np.float32)
    return sc, isc


def to_bf16(x):
    """Round float32 to bfloat16 (nearest, ties to even), returned as float32."""
    u = np.asarray(x, np.float32).view(np.uint32).astype(np.uint64)
    r = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return r.astype(np.uint32).view(np.float32)


def to_fp16(x):
    return np.asarray(x, np.float32).astype(np.float16).astype(np.float32)


@pytest.mark.parametrize("fmt,bits", [("fp16", 22), ("bf16", 16)])
def test_hi_lo_pair_carries_the_scaled_waves(fmt, bits):
    rnd = to_fp16 if fmt == "fp16" else to_bf16
    rng = np.random.default_rng(7)
    for trial in range(200):
        # one tile's waves: random signs, magnitudes over up to 12 decades,
        # the overall scale anywhere from 1e-30 to 1e30
        n = 126
        mag = 10.0 ** rng.uniform(-12 * rng.random(), 0, n) * 10.0 ** rng.uniform(-30, 30)
        w = (rng.choice([-1.0, 1.0], n) * mag).astype(np.float32)
        amax = np.abs(w).max()
        sc, isc = scale_pair(amax)
        x = w * sc  # exact: a power of two, no overflow or underflow here
        assert np.array_equal(x * isc, w)
        assert np.abs(x).max() < 2.0 ** 14 and np.abs(x).max() >= 2.0 ** 13
        hi = rnd(x)
        lo = rnd((x - hi).astype(np.float32))
        err = np.abs(hi.astype(np.float64) + lo - x.astype(np.float64)).max()
        assert err <= 2.0 ** -bits * np.abs(x).max(), (trial, err / np.abs(x).max())
        # and in the FP16 range: no half overflows
        assert np.isfinite(hi).all() and np.isfinite(lo).all()


def test_scale_and_inverse_are_exact_for_every_exponent():
    for e in range(0, 256):
        amax = np.uint32(e << 23).view(np.float32)  # 2^(e-127), or 0 / inf for e = 0 / 255
        sc, isc = scale_pair(amax)
        assert sc * isc == np.float32(1.0)
        assert np.isfinite(sc) and np.isfinite(isc) and sc > 0 and isc > 0
        # both normal numbers
        assert sc >= np.finfo(np.float32).tiny and isc >= np.finfo(np.float32).tiny


def test_all_zero_and_non_finite_tiles():
    sc, isc = scale_pair(np.float32(0.0))
    assert sc == np.float32(2.0 ** 126) and isc == np.float32(2.0 ** -126)
    # a NaN or an infinite wave keeps a finite scale, so it propagates to the
    # products (and the residual) as NaN / inf instead of being scaled away
    for bad in (np.float32(np.inf), np.float32(np.nan)):
        sc, isc = scale_pair(bad)
        assert np.isfinite(sc) and sc * isc == np.float32(1.0)
        assert not np.isfinite(to_fp16(np.float32(bad) * sc))
