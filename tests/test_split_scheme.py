"""The split-precision number scheme, checked in NumPy (CPU).

The tensor-core path stores every FP64 operand block as x * s = hi + lo,
hi and lo FP16 and s a power of two per block with |x * s| <= 2^14, and
forms a product from lo.hi + hi.lo + hi.hi with FP32 accumulation.  These
tests pin the accuracy claims of that scheme on random blocks, independent
of the kernels: each pair carries ~22 significant bits for elements near the
block's largest, an absolute accuracy of about 2^-39 of the largest for tiny
ones, and a dot product of length K is accurate to a few 2^-24 relative.
"""
import numpy as np


def pow2_scale(m):
    """Power of two s with m * s <= 2^14 (m = f 2^e, f in [0.5, 1))."""
    if not m > 0:
        return 1.0
    _, e = np.frexp(m)
    return float(np.ldexp(1.0, 14 - int(e)))


def split(x):
    s = pow2_scale(np.max(np.abs(x)))
    y = x * s
    hi = y.astype(np.float16)
    lo = (y - hi.astype(np.float64)).astype(np.float16)
    return hi, lo, s


def test_scale_keeps_fp16_in_range():
    rng = np.random.default_rng(0)
    for mag in (1e-30, 1e-8, 1.0, 3.7, 1e8, 1e30):
        x = rng.standard_normal(1000) * mag
        hi, lo, s = split(x)
        assert np.all(np.isfinite(hi)) and np.all(np.isfinite(lo))
        assert np.max(np.abs(x * s)) <= 2.0 ** 14
        assert np.max(np.abs(x * s)) > 2.0 ** 13     # the full FP16 range is used


def test_pair_carries_22_bits_near_the_block_max():
    rng = np.random.default_rng(1)
    x = rng.uniform(0.5, 1.0, 20000) * rng.choice([-1, 1], 20000)
    hi, lo, s = split(x)
    back = (hi.astype(np.float64) + lo.astype(np.float64)) / s
    rel = np.abs(back - x) / np.abs(x)
    assert rel.max() <= 2.0 ** -21


def test_tiny_elements_keep_absolute_accuracy():
    rng = np.random.default_rng(2)
    x = rng.standard_normal(20000) * 1e-9
    x[0] = 1.0                       # the block's largest element
    hi, lo, s = split(x)
    back = (hi.astype(np.float64) + lo.astype(np.float64)) / s
    assert np.max(np.abs(back - x)) <= 2.0 ** -38


def test_three_product_dot_with_fp32_accumulation():
    rng = np.random.default_rng(3)
    for K in (16, 256, 4096):
        a = rng.standard_normal((64, K))
        b = rng.standard_normal((K, 8))
        ah, al, sa = split(a)
        bh, bl, sb = split(b)
        f = lambda u: u.astype(np.float32)
        # FP32 accumulation of the three FP16 x FP16 products (each exact in FP32)
        acc = f(al) @ f(bh) + f(ah) @ f(bl) + f(ah) @ f(bh)
        got = acc.astype(np.float64) / (sa * sb)
        exact = a @ b
        rel = np.linalg.norm(got - exact) / np.linalg.norm(exact)
        assert rel <= 64 * 2.0 ** -24 * np.sqrt(K / 16), (K, rel)
        # leaving out one cross term is visibly worse: all three are needed
        worse = (f(ah) @ f(bh) + f(ah) @ f(bl)).astype(np.float64) / (sa * sb)
        assert np.linalg.norm(worse - exact) / np.linalg.norm(exact) > 10 * rel
