"""The split operand representations of the tensor-core paths, emulated on the CPU: a float32
value x becomes hi + lo with hi = RN16(x) and lo = RN16(x - hi) in a 16-bit type, and the
product is taken as hi*hi + hi*lo + lo*hi (lo*lo dropped).

bf16 pieces (8 significant bits each) leave a relative representation error of about 2^-16,
fp16 pieces (11 bits each) about 2^-22, provided both pieces stay in fp16's normal range --
which is what the split-FP16 path's power-of-two operand scale (default 2^12) is for: exit
waves of unit norm give residuals |psi - mu| <= 2, scaled to <= 8192 (nearly eight times
inside 65504), while
residual pieces of components down to ~1e-4 stay normal.  These are the bounds quoted for the
two precisions; the tensor core's FP32 accumulation then adds its own error on top."""
import numpy as np


def rn_bf16(x):
    """Round float32 to the nearest bf16 (ties to even), returned as float32."""
    b = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return r.astype(np.uint32).view(np.float32)


def split(x, kind, scale=1.0):
    x = np.asarray(x, dtype=np.float32) * np.float32(scale)
    if kind == "bf16":
        hi = rn_bf16(x)
        lo = rn_bf16(x - hi)
    else:
        hi = x.astype(np.float16).astype(np.float32)
        lo = (x - hi).astype(np.float16).astype(np.float32)
    return hi, lo


def test_bf16_rounding_matches_nearest_even():
    # 1 + 2^-8 is a tie between 1 and 1 + 2^-7: ties to even -> 1; just above rounds up
    assert rn_bf16(np.float32(1 + 2 ** -8)) == 1.0
    assert rn_bf16(np.float32(1 + 2 ** -8 + 2 ** -20)) == np.float32(1 + 2 ** -7)
    assert rn_bf16(np.float32(3.0)) == 3.0


def test_representation_error_of_the_pieces():
    """Components over three decades (1e-3 .. 2, the scaled residuals 4 .. 8192 on the fp16
    path): each split carries its bound relative to the component itself."""
    rng = np.random.default_rng(0)
    mag = np.exp(rng.uniform(np.log(1e-3), np.log(2.0), 200000))
    x = (mag * rng.choice([-1.0, 1.0], 200000)).astype(np.float32)
    for kind, bound, s in (("bf16", 2.0 ** -16, 1.0), ("fp16", 2.0 ** -22, 2.0 ** 12)):
        hi, lo = split(x, kind, scale=s)
        rel = np.abs((hi.astype(np.float64) + lo) / s - x) / np.abs(x)
        assert rel.max() <= bound, (kind, rel.max())
        # and it is not much better than that: the bound is the right order
        assert rel.max() >= bound / 8, (kind, rel.max())


def test_three_product_split_against_exact_products():
    """a: a scaled residual component (1e-3 .. 2), b: a twiddle (|b| <= 1, split unscaled).
    The error of hi*hi + hi*lo + lo*hi is bounded relative to |a| * max|b| = |a|: twiddle
    pieces below fp16's normal range keep an absolute resolution of 2^-24 or better."""
    rng = np.random.default_rng(1)
    a = (np.exp(rng.uniform(np.log(1e-3), np.log(2.0), 100000)) * rng.choice([-1.0, 1.0], 100000)).astype(np.float32)
    b = rng.uniform(-1, 1, 100000).astype(np.float32)
    exact = a.astype(np.float64) * b
    for kind, bound, s in (("bf16", 2.0 ** -15, 1.0), ("fp16", 2.0 ** -21, 2.0 ** 12)):
        ah, al = split(a, kind, s)
        bh, bl = split(b, kind)
        p = (ah.astype(np.float64) * bh + ah.astype(np.float64) * bl + al.astype(np.float64) * bh) / s
        err = np.abs(p - exact) / np.abs(a.astype(np.float64))
        assert err.max() <= bound, (kind, err.max())


def test_default_fp16_scale_keeps_unit_norm_residuals_in_range_and_normal():
    s = 2.0 ** 12
    big = np.float32(2.0)                                  # |psi - mu| <= 2 for unit-norm exit waves
    assert float(big) * s * 7 <= 65504 < float(big) * s * 8   # nearly eight times inside the fp16 range
    small = np.float32(1e-4)
    hi, lo = split(small, "fp16", s)
    assert abs(float(hi)) >= 2.0 ** -14                     # hi normal
    # the residual piece of a 1e-4 component is still represented to ~2^-11 of itself
    rel = abs((float(hi) + float(lo)) / s - float(small)) / float(small)
    assert rel <= 2.0 ** -20
    # without the scale the same component loses its residual piece to fp16 subnormals
    hi0, lo0 = split(small, "fp16", 1.0)
    rel0 = abs((float(hi0) + float(lo0)) - float(small)) / float(small)
    assert rel0 > 100 * rel
