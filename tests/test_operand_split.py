"""The arithmetic of the two operand splits of the mixed path's tensor-core updates, restated in numpy and checked
against the error bounds the library documents (GP_OPT_SPLIT_F16). Each FP32 entry x of L becomes a pair
(hi, lo) and a product x y is taken as hi_x hi_y + hi_x lo_y + lo_x hi_y (the lo lo term is dropped):
  FP16 pair (of x scaled below 2^13): hi = x rounded to FP16, lo = x - hi rounded to FP16;
  TF32 pair: hi = x truncated to TF32 (the low 13 mantissa bits dropped, as the TF32 MMAs read an FP32 operand),
             lo = x - hi rounded to TF32 (to nearest, ties away from zero).
Both pairs hold x to within 2^-22 of its magnitude (the FP16 pair with an absolute floor of 2^-25 below 2^-3, its
low part then being subnormal); the dropped lo lo term is at most 2^-22 of |x y| with the rounded FP16 high part
against 2^-20 with the truncated TF32 one."""
import numpy as np


def _sample(n=400_000, lo_exp=-40, hi_exp=13, seed=0):
    rng = np.random.default_rng(seed)
    e = rng.uniform(lo_exp, hi_exp, size=n)
    x = (np.sign(rng.standard_normal(n)) * np.exp2(e)).astype(np.float32)
    return x[(np.abs(x) < 2.0 ** 13) & (x != 0)]


def _f16_pair(x):
    hi = x.astype(np.float16)
    r = (x - hi.astype(np.float32)).astype(np.float32)
    return hi.astype(np.float64), r.astype(np.float16).astype(np.float64), r


def _tf32_pair(x):
    hi = (x.view(np.uint32) & np.uint32(0xFFFFE000)).view(np.float32)
    r = (x - hi).astype(np.float32)
    u = r.view(np.uint32).astype(np.uint64)
    lo = (((u + 0x1000) & 0xFFFFE000).astype(np.uint32)).view(np.float32)   # ties away from zero (cvt.rna)
    return hi.astype(np.float64), lo.astype(np.float64), r


def test_remainders_are_exact_in_fp32():
    x = _sample()
    for pair in (_f16_pair, _tf32_pair):
        hi, _, r = pair(x)
        assert np.array_equal(x.astype(np.float64) - hi, r.astype(np.float64))


def test_fp16_pair_error_bound():
    x = _sample()
    hi, lo, _ = _f16_pair(x)
    err = np.abs(x.astype(np.float64) - hi - lo)
    assert np.all(err <= np.maximum(2.0 ** -22 * np.abs(x.astype(np.float64)), 2.0 ** -25))
    big = np.abs(x) >= 0.125
    assert np.all(err[big] <= 2.0 ** -22 * np.abs(x[big].astype(np.float64)))


def test_tf32_pair_error_bound():
    x = _sample(lo_exp=-100)
    hi, lo, _ = _tf32_pair(x)
    err = np.abs(x.astype(np.float64) - hi - lo)
    assert np.all(err <= 2.0 ** -22 * np.abs(x.astype(np.float64)))


def test_dropped_low_product():
    x = _sample(lo_exp=-3)   # the FP16 pair's normal range
    for pair, bound in ((_f16_pair, 2.0 ** -22), (_tf32_pair, 2.0 ** -20)):
        hi, lo, _ = pair(x)
        assert np.all(np.abs(lo) <= bound ** 0.5 * np.abs(x.astype(np.float64)))   # |lo| <= 2^-11 |x| or 2^-10 |x|
    hi16, lo16, _ = _f16_pair(x)
    hit, lot, _ = _tf32_pair(x)
    # the truncated high part leaves larger low parts: on average about twice the FP16 pair's
    assert np.mean(np.abs(lot)) > 1.5 * np.mean(np.abs(lo16))


def test_three_product_dot_products():
    """Dot products of length 2048 (a group's K) through each split, with the products and sums in FP64 so that
    only the split shows: both stay within a few 2^-22 of the exact dot product's scale."""
    rng = np.random.default_rng(5)
    a = (rng.standard_normal((64, 2048)) * 100).astype(np.float32)
    b = (rng.standard_normal((64, 2048)) * 100).astype(np.float32)
    exact = a.astype(np.float64) @ b.astype(np.float64).T
    scale = np.abs(a.astype(np.float64)) @ np.abs(b.astype(np.float64)).T
    for pair in (_f16_pair, _tf32_pair):
        ha, la, _ = pair(a.ravel())
        hb, lb, _ = pair(b.ravel())
        ha, la, hb, lb = (v.reshape(64, 2048) for v in (ha, la, hb, lb))
        got = ha @ hb.T + ha @ lb.T + la @ hb.T
        assert np.max(np.abs(got - exact) / scale) <= 4 * 2.0 ** -22
