"""CPU check of the arithmetic the mixed-precision path is built on: float-pair
numbers (hi + lo in two FP32), their split from FP64, the error-free multiply-add,
and the cut of a float pair into BF16 slices whose products the tensor cores
accumulate exactly per slice order.

Each FP32 operation is written out as the exact rational result rounded once to
FP32 (round to nearest, ties to even), which is what the GPU's __fadd_rn,
__fmul_rn and __fmaf_rn do, so the error bounds checked here are the kernels'
and not those of a different evaluation order.  Nothing here is shared with the
CUDA sources or the oracle."""
import math
from fractions import Fraction

import numpy as np

F = Fraction


def r32(q):
    """Round a rational to the nearest FP32 value (ties to even), as a Fraction."""
    q = F(q)
    if q == 0:
        return F(0)
    s = -1 if q < 0 else 1
    a = abs(q)
    e = math.floor(math.log2(a.numerator) - math.log2(a.denominator))
    while F(2) ** e > a:
        e -= 1
    while F(2) ** (e + 1) <= a:
        e += 1
    e = max(e, -126)                  # subnormal range shares the last exponent
    ulp = F(2) ** (e - 23)
    n, rem = divmod(a, ulp)
    if rem > ulp / 2 or (rem == ulp / 2 and n % 2 == 1):
        n += 1
    return s * n * ulp


def fadd(a, b):
    return r32(F(a) + F(b))


def fmul(a, b):
    return r32(F(a) * F(b))


def fma(a, b, c):
    return r32(F(a) * F(b) + F(c))


def is_f32(q):
    return r32(q) == q


def sig_bits(q):
    """Number of significant bits of a dyadic rational."""
    q = abs(F(q))
    if q == 0:
        return 0
    n, d = q.numerator, q.denominator
    while n % 2 == 0:
        n //= 2
    return n.bit_length()


# ---- float pairs ----------------------------------------------------------------------

def split(x):
    """FP64 -> (hi, lo): hi = leading 24 significand bits (truncated), lo = the
    next 23, both exact (the integer construction of the split)."""
    x = F(x)
    if x == 0:
        return F(0), F(0)
    s = -1 if x < 0 else 1
    a = abs(x)
    e = math.floor(math.log2(a))
    while F(2) ** e > a:
        e -= 1
    while F(2) ** (e + 1) <= a:
        e += 1
    hi = (a / F(2) ** (e - 23)).__floor__() * F(2) ** (e - 23)
    lo = ((a - hi) / F(2) ** (e - 46)).__floor__() * F(2) ** (e - 46)
    return s * hi, s * lo


def two_sum(a, b):
    s = fadd(a, b)
    bb = fadd(s, -a)
    return s, fadd(fadd(a, -fadd(s, -bb)), fadd(b, -bb))


def mac(h, l, a, b):
    """(h, l) += a b as the error-free multiply-add of the float-pair kernels."""
    p = fmul(a[0], b[0])
    e = fma(a[0], b[0], -p)
    e = fma(a[0], b[1], e)
    e = fma(a[1], b[0], e)
    s, t = two_sum(h, p)
    return s, fadd(l, fadd(t, e))


def test_split_bounds():
    rng = np.random.default_rng(1)
    xs = list(rng.normal(size=300) * 10.0 ** rng.integers(-20, 20, size=300)) + [1.0, -3.0]
    for x in xs:
        hi, lo = split(float(x))
        assert is_f32(hi) and is_f32(lo)
        assert sig_bits(hi) <= 24 and sig_bits(lo) <= 23
        assert abs(F(float(x)) - hi - lo) < F(2) ** -46 * abs(F(float(x)))
        assert abs(lo) < F(2) ** -23 * abs(hi)


def test_two_sum_is_error_free():
    rng = np.random.default_rng(2)
    for _ in range(300):
        a = r32(F(float(rng.normal() * 10.0 ** rng.integers(-6, 6))))
        b = r32(F(float(rng.normal() * 10.0 ** rng.integers(-6, 6))))
        s, t = two_sum(a, b)
        assert s + t == a + b and s == fadd(a, b)


def test_float_pair_dot_product():
    """K float-pair multiply-adds carry the dot product to about K ulp of the
    high part's 2^-47 relative precision: far below the 1e-9 relative the
    energy needs."""
    rng = np.random.default_rng(3)
    for K in (16, 128):
        xs = [split(float(v)) for v in rng.normal(size=K)]
        ys = [split(float(v)) for v in rng.normal(size=K)]
        h = l = F(0)
        for x, y in zip(xs, ys):
            h, l = mac(h, l, x, y)
        exact = sum((x[0] + x[1]) * (y[0] + y[1]) for x, y in zip(xs, ys))
        scale = sum(abs((x[0] + x[1]) * (y[0] + y[1])) for x, y in zip(xs, ys))
        assert abs(h + l - exact) <= 2 * K * F(2) ** -47 * scale


# ---- BF16 slices --------------------------------------------------------------------------

C = [F(12582912), F(49152), F(192), F(3, 4)]  # 1.5 * 2^(23 - 8k)


def slices(x, sc, ns=4):
    """The slicing of the tensor-core passes: x sc = r0 + ... + r_{ns-1} + small."""
    r = [fadd(fma(x[0], sc, C[0]), -C[0])]
    u = fma(x[1], sc, fma(x[0], sc, -r[0]))
    for k in range(1, ns):
        if k > 1:
            u = fadd(u, -r[k - 1])
        r.append(fadd(fadd(u, C[k]), -C[k]))
    return r


def _random_pairs(rng, n):
    out = []
    for _ in range(n):
        v = float(rng.uniform(-1, 1) * 2.0 ** rng.integers(-3, 4))
        out.append(split(v))
    return out


def _scale_for(x):
    """Power of two with |x sc| <= 128 (the per-row / per-function exponent)."""
    a = abs(x[0] + x[1])
    if a == 0:
        return F(1)
    e = math.floor(math.log2(a)) + 1
    return F(2) ** (7 - e)


def test_slices_are_bf16_bounded_and_reconstruct():
    rng = np.random.default_rng(4)
    for x in _random_pairs(rng, 400):
        sc = _scale_for(x)
        r = slices(x, sc)
        for k, rk in enumerate(r):
            assert sig_bits(rk) <= 8                              # exact in BF16
            assert (rk / F(2) ** (-8 * k)).denominator == 1       # multiple of 2^-8k
            assert abs(rk) <= 128 * F(2) ** (-8 * k)
        err = abs((x[0] + x[1]) * sc - sum(r))
        assert err <= F(2) ** -24                                 # of a value up to 128


def test_per_order_accumulation_is_exact_in_fp32():
    """Products of slices of orders i and j are integers times 2^-8(i+j) below
    2^14 of that unit, so an FP32 accumulator of one order over 128 K steps of
    up to four products never rounds."""
    rng = np.random.default_rng(5)
    K = 128
    X = [slices(x, _scale_for(x)) for x in _random_pairs(rng, K)]
    W = [slices(w, _scale_for(w)) for w in _random_pairs(rng, K)]
    for order in range(4):
        acc = F(0)
        exact = F(0)
        for xs, ws in zip(X, W):
            for i in range(order + 1):
                p = fmul(ws[i], xs[order - i])
                assert p == ws[i] * xs[order - i]                 # the product is exact
                acc = fadd(acc, p)
                exact += ws[i] * xs[order - i]
        assert acc == exact
        assert abs(exact) < F(2) ** 24 * F(2) ** (-8 * order)


def test_three_slices_and_orders_up_to_three():
    """The V pass keeps three slices of each operand and the slice products of
    orders 0..3 (eight per K step).  Per term, the operands' cut at three slices
    costs up to 2^-24 of each (the remainder below 2^-16 of values up to 128),
    while the one dropped product (order 4, W2 X2) is below 2^-32 of the term's
    scale: the pass is as accurate as its three-slice operands."""
    rng = np.random.default_rng(6)
    K = 64
    xs, ws = _random_pairs(rng, K), _random_pairs(rng, K)
    sx = [_scale_for(x) for x in xs]
    sw = [_scale_for(w) for w in ws]
    X = [slices(x, s, 3) for x, s in zip(xs, sx)]
    W = [slices(w, s, 3) for w, s in zip(ws, sw)]
    for t in range(K):
        wv, xv = (ws[t][0] + ws[t][1]) * sw[t], (xs[t][0] + xs[t][1]) * sx[t]
        assert abs(sum(W[t]) - wv) <= F(2) ** -17 and abs(sum(X[t]) - xv) <= F(2) ** -17
        dropped = W[t][2] * X[t][2]
        assert abs(dropped) <= F(2) ** -18                       # 2^-32 of 128 * 128
    kept = sum(W[t][i] * X[t][j] for t in range(K) for i in range(3) for j in range(3)
               if i + j <= 3)
    full3 = sum(sum(W[t]) * sum(X[t]) for t in range(K))
    assert abs(kept - full3) <= K * F(2) ** -18
    exact = sum(((w[0] + w[1]) * a) * ((x[0] + x[1]) * b)
                for w, x, a, b in zip(ws, xs, sw, sx))
    assert abs(kept - exact) <= K * (2 * 128 * F(2) ** -17 + F(2) ** -18)


def dot_sub(a, b, c, d):
    """a b - c d with one renormalization, as the FFT passes' butterflies form
    their complex products: TwoSum of the two rounded products, their exact
    errors and the cross terms gathered in the low part."""
    p, q = fmul(a[0], b[0]), fmul(c[0], d[0])
    ep, eq = fma(a[0], b[0], -p), fma(c[0], d[0], -q)
    s, t = two_sum(p, -q)
    e = fadd(t, fadd(ep, -eq))
    e = fma(a[0], b[1], fma(a[1], b[0], e))
    e = fma(-c[0], d[1], fma(-c[1], d[0], e))
    h = fadd(s, e)
    return h, fadd(e, -fadd(h, -s))


def test_float_pair_dot_sub():
    """The butterfly product a b - c d keeps about 2^-44 of |a b| + |c d| when the
    TwoSum sees the two rounded products (the float-pair FFT's accuracy rests on
    this step)."""
    rng = np.random.default_rng(7)
    for _ in range(500):
        a, b, c, d = [split(float(rng.normal() * 2.0 ** rng.integers(-4, 4))) for _ in range(4)]
        A, B, Cc, D = [x[0] + x[1] for x in (a, b, c, d)]
        h, l = dot_sub(a, b, c, d)
        assert abs(h + l - (A * B - Cc * D)) <= F(2) ** -43 * (abs(A * B) + abs(Cc * D))


def test_ql_reciprocal_square_root():
    """The QL sweeps' 1/sqrt (kpoint.cu, ql_rsqrt): a single-precision seed
    with any relative error up to 2^-21, refined by two Newton-Raphson steps
    y <- y (3 - x y^2) / 2 in FP64, is within 2 ulp of 1/sqrt(x) over the
    range it is used on, [1e-30, 1e30]."""
    rng = np.random.default_rng(0)
    x = np.exp(rng.uniform(np.log(1e-30), np.log(1e30), 200000))
    y = (1.0 / np.sqrt(x.astype(np.float32))).astype(np.float64)
    y = y * (1.0 + rng.uniform(-2.0 ** -21, 2.0 ** -21, x.size))
    for _ in range(2):
        y = y * (1.5 - (0.5 * x) * (y * y))
    rel = np.abs(y - 1.0 / np.sqrt(x)) * np.sqrt(x)
    assert rel.max() < 2.0 * 2.0 ** -52


# ---- five slices: the tensor-core products of the dense chains --------------------------

C5 = [F(3, 2) * F(2) ** (23 - 8 * k) for k in range(5)]  # 1.5 * 2^(23 - 8k)


def slices5(x, sc):
    """The cut of the dense chains' products: the high part alone gives the
    slices of orders 0 and 1 (exact remainders), the low part joins the
    remainder once (the one rounding), then orders 2, 3 and 4."""
    r = [fadd(fma(x[0], sc, C5[0]), -C5[0])]
    u = fma(x[0], sc, -r[0])
    r.append(fadd(fadd(u, C5[1]), -C5[1]))
    u = fma(x[1], sc, fadd(u, -r[1]))
    for k in (2, 3, 4):
        r.append(fadd(fadd(u, C5[k]), -C5[k]))
        u = fadd(u, -r[k])
    return r


def _row_scale(row):
    """2^(8 - e) with e = floor(log2 max|hi|) + 2: every |x sc| below 128."""
    b = max(abs(x[0]) for x in row)
    return F(2) ** (8 - (math.floor(math.log2(b)) + 2))


def _five_slice_dot(a, b):
    """sum_k a_k b_k as the tensor-core product forms it over one chunk of K:
    slices of both operands, orders 0, 1, 2 in one FP32 sum each, orders 3 and
    4 together in a fourth, orders >= 5 dropped.  Returns the four sums, their
    exact values, the scales and the slices."""
    sa, sb = _row_scale(a), _row_scale(b)
    A = [slices5(x, sa) for x in a]
    B = [slices5(y, sb) for y in b]
    acc, exact = [F(0)] * 4, [F(0)] * 4
    for ra, rb in zip(A, B):
        for i in range(5):
            for j in range(5 - i):
                p = ra[i] * rb[j]
                assert fmul(ra[i], rb[j]) == p        # BF16 x BF16 is exact in FP32
                q = min(i + j, 3)
                acc[q] = fadd(acc[q], p)
                exact[q] += p
    return acc, exact, sa, sb, A, B


def test_five_slices_bf16_and_reconstruct():
    """Each slice is exact in BF16, a multiple of 2^-8k with a numerator of at
    most 129, and the five carry x sc to 2^-32 (x sc below 128)."""
    rng = np.random.default_rng(21)
    row = [split(float(v)) for v in rng.uniform(-1, 1, 400) * 2.0 ** rng.integers(-9, 3, 400)]
    sc = _row_scale(row)
    for x in row:
        assert abs((x[0] + x[1]) * sc) < 128
        r = slices5(x, sc)
        for k, rk in enumerate(r):
            assert sig_bits(rk) <= 8
            num = rk * F(2) ** (8 * k)
            assert num.denominator == 1 and abs(num) <= 129
        assert abs((x[0] + x[1]) * sc - sum(r)) <= F(2) ** -32


def test_five_slice_orders_exact_over_a_chunk_and_the_product_bound():
    """Over a chunk of 21 K steps (336 elements) the sums of orders 0, 1 and 2
    never round: at most three products per element of at most 129^2 units
    each, 3 x 336 x 129^2 < 2^24.  The chunk's dot product, in the units of the
    scaled operands (|a sc|, |b sc| < 128), is within K 2^-23 + K^2 2^-32 of
    the exact one: per element the dropped orders >= 5 (at most
    129^2 (4 2^-40 + 3 2^-48 + ...) < 2^-23.9) and the slices' cut (2^-32 of
    each operand, times the other one), and the FP32 sum of orders 3 and 4,
    each addition within 2^-24 of a partial sum of at most K 2^-7.9.  For
    operands whose entries are comparable to their maxima the error is about
    2^-39 of sum |a b| or less (checked at 2^-38)."""
    assert 3 * 336 * 129 ** 2 < 2 ** 24
    rng = np.random.default_rng(22)
    K = 336
    for spread in (9, 0):  # entries over 2^9 below the maximum, or comparable to it
        a = [split(float(v)) for v in rng.uniform(-1, 1, K) * 2.0 ** rng.integers(-spread, 1, K)]
        b = [split(float(v)) for v in rng.uniform(-1, 1, K) * 2.0 ** rng.integers(-spread, 1, K)]
        acc, exact, sa, sb, _, _ = _five_slice_dot(a, b)
        for q in range(3):
            assert acc[q] == exact[q]
        got = acc[0] + acc[1] + acc[2] + acc[3]
        true = sum((x[0] + x[1]) * sa * (y[0] + y[1]) * sb for x, y in zip(a, b))
        assert abs(got - true) <= K * F(2) ** -23 + K * K * F(2) ** -32
        if spread == 0:
            mag = sum(abs((x[0] + x[1]) * sa * (y[0] + y[1]) * sb) for x, y in zip(a, b))
            assert abs(got - true) <= F(2) ** -38 * mag
