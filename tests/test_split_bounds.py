"""The error claims behind the product tolerances of the tensor-core passes
(CPU only, exact arithmetic in numpy; no library code involved).

* Scaled FP16x3: a value scaled by a power of two into FP16's range, split
  into hi (the scaled value with its low 13 mantissa bits cleared: exact in
  FP16) and lo (the remainder rounded to FP16), is within 2^-21 of itself,
  relative, plus 2^-24 of the scaled unit where the parts underflow FP16's
  normal range; three products hi*hi + hi*lo + lo*hi are within 2^-19 |a||p|
  (the dropped lo*lo, up to 2^-20, and the two roundings of the lo parts,
  2^-21 each) plus the underflow terms, and 2^-20 alone is not enough.
* E4M3: a row scaled by the power of two that brings its max to at most 448
  and rounded to nearest E4M3 (saturating) is within 2^-4 of itself,
  relative, in E4M3's normal range, and within 2^-10 (half the smallest
  subnormal step, 2^-9) of the scaled unit below it.
* 3xTF32: the three TF32 products are within 2^-19 |a||p| whether the tensor
  core truncates or rounds the low part of a.
The tolerances of tests/test_gpu_tc.py are built from these bounds."""
import numpy as np
import pytest


def trunc13(x):
    """x (float32) with its low 13 mantissa bits cleared."""
    b = np.asarray(x, np.float32).view(np.uint32) & np.uint32(0xFFFFE000)
    return b.view(np.float32)


def split_f16(x):
    """The hi / lo FP16 parts of float32 x (already scaled)."""
    hi = trunc13(x)
    lo = (x - hi).astype(np.float16)  # the remainder is exact in FP32, then rounded
    return hi, lo


def pow2_scale_into(amax, top_exp=14):
    """The power of two s with amax * s in [2^(top_exp - 1), 2^top_exp)."""
    e = int(np.floor(np.log2(amax)))
    return np.float32(2.0 ** (top_exp - 1 - e))


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_fp16_split_of_scaled_values(seed):
    rng = np.random.default_rng(seed)
    # a wide spread of magnitudes, as in rows of very different scale
    a = (rng.standard_normal(200000) * np.exp2(rng.integers(-30, 8, size=200000))).astype(np.float32)
    s = pow2_scale_into(float(np.abs(a).max()))
    x = (a * s).astype(np.float32)  # exact: a power of two
    assert np.abs(x).max() < 2.0 ** 14
    hi, lo = split_f16(x)
    # hi is exact in FP16 wherever it is in FP16's normal range
    hin = np.abs(hi) >= 2.0 ** -14
    assert np.array_equal(hi[hin].astype(np.float16).astype(np.float32), hi[hin])
    err = np.abs(x.astype(np.float64) - hi.astype(np.float16).astype(np.float64) - lo.astype(np.float64))
    bound = 2.0 ** -21 * np.abs(x.astype(np.float64)) + 2.0 ** -24
    assert np.all(err <= bound), float(np.max(err / bound))
    # and the bound is nearly attained (the reading is not loose by a factor)
    big = np.abs(x) > 1.0
    assert np.max(err[big] / np.abs(x[big])) > 2.0 ** -23


@pytest.mark.parametrize("seed", [3, 4])
def test_fp16x3_products(seed):
    rng = np.random.default_rng(seed)
    a = (rng.standard_normal(100000) * np.exp2(rng.integers(-6, 6, size=100000))).astype(np.float32)
    p = rng.standard_normal(100000).astype(np.float32)
    sa, sp = pow2_scale_into(float(np.abs(a).max())), pow2_scale_into(float(np.abs(p).max()))
    ah, al = split_f16((a * sa).astype(np.float32))
    ph, pl = split_f16((p * sp).astype(np.float32))
    ah, al, ph, pl = (v.astype(np.float16).astype(np.float64) for v in (ah, al, ph, pl))
    # each of the three products is exact in FP32 (11 x 11 significant bits)
    approx = (ah * ph + ah * pl + al * ph) / (float(sa) * float(sp))
    exact = a.astype(np.float64) * p.astype(np.float64)
    # below FP16's normal range each part's rounding adds at most 2^-25, so a
    # scaled operand x = hi + lo is within 2^-21 |x| + 2^-24; over the product,
    # 2^-24 (|x| + |y|) in scaled units, divided back by the scales
    xs = np.abs(a.astype(np.float64)) * float(sa)
    ys = np.abs(p.astype(np.float64)) * float(sp)
    under = 2.0 ** -24 * (xs + ys + 2.0 ** -20) / (float(sa) * float(sp))
    assert np.all(np.abs(approx - exact) <= 2.0 ** -19 * np.abs(exact) + under)
    # away from underflow the error passes 2^-20 |a||p| (so 2^-19 is the bound to use)
    big = np.abs(exact) > 1e-3 * np.abs(exact).max()
    rel = np.abs(approx - exact)[big] / np.abs(exact)[big]
    assert rel.max() > 2.0 ** -20


def rna_tf32(x):
    """float32 x rounded to TF32 (10 explicit mantissa bits), ties away from
    zero (the cvt.rna rule): add half of the dropped range, then clear it."""
    b = np.asarray(x, np.float32).view(np.uint32).astype(np.uint64)
    return ((b + 0x1000) & 0xFFFFE000).astype(np.uint32).view(np.float32)


@pytest.mark.parametrize("lo_rule", ["truncate", "round"])
def test_3xtf32_products(lo_rule):
    """a_hi = a with 13 bits cleared, a_lo = a - a_hi (exact), taken by the
    tensor core as TF32 either truncated or rounded; the panel split by
    round-to-nearest TF32 twice; a_hi p_hi + a_hi p_lo + a_lo p_hi is within
    2^-19 |a||p| whichever rule the tensor core applies to a_lo."""
    rng = np.random.default_rng(7)
    a = (rng.standard_normal(100000) * np.exp2(rng.integers(-20, 20, size=100000))).astype(np.float32)
    p = (rng.standard_normal(100000) * np.exp2(rng.integers(-20, 20, size=100000))).astype(np.float32)
    ah = trunc13(a)
    al = (a - ah).astype(np.float32)
    al = trunc13(al) if lo_rule == "truncate" else rna_tf32(al)
    ph = rna_tf32(p)
    pl = rna_tf32((p - ph).astype(np.float32))
    f = lambda v: v.astype(np.float64)
    approx = f(ah) * f(ph) + f(ah) * f(pl) + f(al) * f(ph)
    exact = f(a) * f(p)
    assert np.all(np.abs(approx - exact) <= 2.0 ** -19 * np.abs(exact))


def e4m3_round(x):
    """Round float64 x to the nearest E4M3 value (ties to even), saturating at
    +-448: sign, 4 exponent bits (bias 7), 3 mantissa bits, subnormals
    below 2^-6 in steps of 2^-9."""
    x = np.asarray(x, np.float64)
    ax = np.minimum(np.abs(x), 448.0)
    e = np.floor(np.log2(np.maximum(ax, 2.0 ** -6)))
    step = 2.0 ** (e - 3)
    q = np.round(ax / step) * step  # numpy rounds half to even
    return np.sign(x) * np.minimum(q, 448.0)


def test_e4m3_rounding_table():
    """The rounding rule on hand-picked points: the grid near 1, a tie to
    even, saturation, the subnormal step."""
    pts = np.array([1.0, 1.0625, 1.1, 1.1875, 448.0, 460.0, 1e6, 2.0 ** -9, 3 * 2.0 ** -10, -2.5])
    want = np.array([1.0, 1.0, 1.125, 1.25, 448.0, 448.0, 448.0, 2.0 ** -9, 2.0 ** -8, -2.5])
    np.testing.assert_array_equal(e4m3_round(pts), want)


@pytest.mark.parametrize("seed", [5, 6])
def test_e4m3_row_scaling_error(seed):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((400, 300)) * np.exp2(rng.integers(-12, 12, size=(400, 1)))
    mx = np.abs(A).max(axis=1, keepdims=True)
    e = np.ceil(np.log2(mx / 448.0))  # the smallest power of two with max / 2^e <= 448
    X = A / 2.0 ** e
    assert np.all(np.abs(X).max(axis=1) <= 448.0) and np.all(np.abs(X).max(axis=1) > 224.0)
    Q = e4m3_round(X)
    err = np.abs(Q - X)
    normal = np.abs(X) >= 2.0 ** -6
    assert np.all(err[normal] <= 2.0 ** -4 * np.abs(X[normal]))
    assert np.all(err[~normal] <= 2.0 ** -10 + 1e-300)
    assert np.max(err[normal] / np.abs(X[normal])) > 2.0 ** -5  # nearly attained
