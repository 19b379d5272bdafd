"""Host checks of the float arithmetic the complex128 kernels rely on.

The complex128 spread and interpolation run on the FP32 pipe.  Two of their building blocks make
claims that follow from IEEE single-precision rounding and can be checked exactly on the CPU by
emulating each float operation (every product, sum and fused multiply-add rounded once to the
nearest float, ties to even) with rational arithmetic:

  * the spread's split of a double-float product a b into three 32-bit fixed-point words,
    v ~ x2 2^42 + x1 2^21 + x0, each word obtained by adding 1.5 2^23 to a float below 2^22 and
    reading the bit pattern: the words' sum is a b to within one unit or |a b| 2^-46, and each word
    stays inside the bounds that keep a 512-point chunk's sums inside int32
    (|x2| <= 2^10, |x1| <= 2^20 + 2^9, |x0| <= 2^21 for |a b| <= 2^52);
  * the double-float exponential e^x of the kernel evaluation (Eq. (ES)), x in [-60, 0] (the
    kernels need x >= -2 beta >= -74; below -60 the values are under 1e-26): its relative error
    stays below 2^-46.  Its constants (ln 2 in three parts, the Taylor
    coefficients) are read from the kernel source, so the check follows the shipped code.

Both emulations follow the operation sequence of paper_1808_06736_gb300/csrc/spread_dw.cuh
(dw_split) and csrc/df.cuh (df_exp_neg) step by step.  Two more checks cover the complex64
path: the spread's rounding of each contribution to an integer by one FMA (spread_interp.cuh,
Fixed<float>), and the binning's fold of a coordinate to (cell, fraction) with an FMA error term
(binsort.cu, fold), accurate to 1e-7 cells.
"""
import os
import random
import re
from decimal import Decimal, getcontext
from fractions import Fraction as F

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
DF_SRC = os.path.join(ROOT, "paper_1808_06736_gb300", "csrc", "df.cuh")


def rnd(x) -> float:
    """The float32 nearest to the rational x (ties to even), as a Python float."""
    x = F(x)
    if x == 0:
        return 0.0
    s = -1 if x < 0 else 1
    a = abs(x)
    e = a.numerator.bit_length() - a.denominator.bit_length()
    if F(2) ** e > a:
        e -= 1
    if F(2) ** (e + 1) <= a:
        e += 1
    e = max(e, -126)
    q = F(2) ** (e - 23)
    n = a / q
    fl = n.numerator // n.denominator
    rem = n - fl
    if rem > F(1, 2) or (rem == F(1, 2) and fl % 2 == 1):
        fl += 1
    return float(s * fl * q)


def fma(a, b, c):
    return rnd(F(a) * F(b) + F(c))


def mul(a, b):
    return rnd(F(a) * F(b))


def add(a, b):
    return rnd(F(a) + F(b))


def sub(a, b):
    return rnd(F(a) - F(b))


def bits(x: float) -> int:
    return int(np.array([x], dtype=np.float32).view(np.int32)[0])


M = 12582912.0  # 1.5 2^23
B = 0x4B400000


def dw_split(ah, al, bh, bl):
    ph = mul(ah, bh)
    e = fma(ah, bh, -ph)
    e = fma(ah, bl, e)
    e = fma(al, bh, e)
    t2 = fma(ph, 2.0 ** -42, M)
    r2 = add(ph, fma(t2, -2.0 ** 42, M * 2.0 ** 42))
    t1 = fma(r2, 2.0 ** -21, M)
    r1 = add(r2, fma(t1, -2.0 ** 21, M * 2.0 ** 21))
    te = fma(e, 2.0 ** -21, M)
    re = add(e, fma(te, -2.0 ** 21, M * 2.0 ** 21))
    t0 = add(add(r1, re), M)
    return bits(t2) - B, bits(t1) + bits(te) - 2 * B, bits(t0) - B


def float_pair(x: float):
    h = rnd(F(x))
    return h, rnd(F(x) - F(h))


def test_word_split_reconstructs_the_product_and_keeps_its_bounds():
    rng = random.Random(11)
    for it in range(3000):
        k = 2.0 ** rng.uniform(30, 52)
        a = rng.uniform(-1, 1) * k * (10 ** rng.uniform(-9, 0) if it % 3 == 0 else 1.0)
        b = rng.uniform(0, 1)
        ah, al = float_pair(a)
        bh, bl = float_pair(b)
        x2, x1, x0 = dw_split(ah, al, bh, bl)
        exact = (F(ah) + F(al)) * (F(bh) + F(bl))
        v = x2 * 2 ** 42 + x1 * 2 ** 21 + x0
        assert abs(F(v) - exact) <= max(F(1), abs(exact) * F(2) ** -46), (a, b, x2, x1, x0)
        assert abs(x2) <= 2 ** 10 and abs(x1) <= 2 ** 20 + 2 ** 9 and abs(x0) <= 2 ** 21


def test_word_split_of_exact_integers_is_exact():
    """Products that are integers of at most 24 bits come out exactly, in every word position."""
    rng = random.Random(12)
    for _ in range(500):
        n = rng.randint(-(2 ** 24) + 1, 2 ** 24 - 1)
        sh = rng.choice([0, 5, 21, 28, 42 - 23])
        a = float(n * 2 ** sh)
        x2, x1, x0 = dw_split(a, 0.0, 1.0, 0.0)
        assert x2 * 2 ** 42 + x1 * 2 ** 21 + x0 == n * 2 ** sh


def _df_constants():
    src = open(DF_SRC).read()
    body = src[src.index("DF df_exp_neg(DF x)"):]
    body = body[: body.index("\n}\n")]

    def lit(t: str) -> float:  # a float literal of the source, rounded to float32 as the compiler does
        t = t.strip().rstrip("f")
        return rnd(F(float.fromhex(t) if "0x" in t else float(t)))

    c = {name: lit(re.search(r"%s = ([^;]+);" % name, body).group(1)) for name in ("LN2_HI", "LN2_MID", "LN2_LO")}
    c["LOG2E"] = lit(re.search(r"__fmul_rn\(x\.hi, ([^)]+)\)", body).group(1))
    c["fh"] = [lit(v) for v in re.search(r"fh\[8\] = \{([^}]+)\}", body).group(1).split(",")]
    c["fl"] = [lit(v) for v in re.search(r"fl\[8\] = \{([^}]+)\}", body).group(1).split(",")]
    c["t12"] = lit(re.search(r"float t = ([^;]+);", body).group(1))
    c["tail"] = [lit(v) for v in re.findall(r"t = __fmaf_rn\(t, r\.hi, ([^)]+)\);", body)]
    return c


def two_sum(a, b):
    s = add(a, b)
    v = sub(s, a)
    return s, add(sub(a, sub(s, v)), sub(b, v))


def quick(a, b):
    s = add(a, b)
    return s, sub(b, sub(s, a))


def df_exp_neg(xh, xl, c):
    k = float(np.rint(mul(xh, c["LOG2E"])))
    a = fma(-k, c["LN2_HI"], xh)
    s1h, s1l = two_sum(a, xl)
    s2h, s2l = two_sum(s1h, -mul(k, c["LN2_MID"]))
    rh, rl = quick(s2h, add(add(s1l, s2l), mul(-k, c["LN2_LO"])))
    t = c["t12"]
    for coef in c["tail"]:
        t = fma(t, rh, coef)
    yh, yl = t, 0.0
    for j in range(7, -1, -1):
        p = mul(rh, yh)
        e = fma(rh, yh, -p)
        e = fma(rh, yl, e)
        e = fma(rl, yh, e)
        sh = add(c["fh"][j], p)
        err = sub(p, sub(sh, c["fh"][j]))
        yh, yl = sh, add(err, add(e, c["fl"][j]))
    yh, yl = quick(yh, yl)
    sc = 2.0 ** int(k)
    return mul(yh, sc), mul(yl, sc)


def test_double_float_exponential_relative_error():
    c = _df_constants()
    assert len(c["fh"]) == 8 and len(c["fl"]) == 8 and len(c["tail"]) == 4
    getcontext().prec = 50
    rng = random.Random(13)
    worst = 0.0
    for it in range(600):
        x = -rng.uniform(0, 60) if it % 2 else -rng.uniform(0, 1)
        xh = rnd(F(x))
        xl = rnd(F(rng.uniform(-1, 1)) * F(float(np.spacing(np.float32(xh)))) / 2)
        yh, yl = df_exp_neg(xh, xl, c)
        xe = Decimal(xh) + Decimal(xl)
        ex = xe.exp()
        rel = abs((Decimal(yh) + Decimal(yl)) - ex) / ex
        worst = max(worst, float(rel))
    assert worst < 2.0 ** -46, worst


def test_complex64_fixed_point_rounding():
    """The complex64 spread's contribution: the bit pattern of fma(a, b, 1.5 2^23) minus that of
    1.5 2^23 is a b rounded to the nearest integer, for |a b| below 2^22 (ties to even)."""
    rng = random.Random(14)
    for _ in range(3000):
        a = rnd(F(rng.uniform(-1, 1) * 2.0 ** rng.uniform(0, 22)))
        b = rnd(F(rng.uniform(0, 1)))
        ex = F(a) * F(b)
        if abs(ex) >= 2 ** 22:
            continue
        v = bits(fma(a, b, M)) - B
        fl = ex.numerator // ex.denominator
        rem = ex - fl
        want = fl + (1 if rem > F(1, 2) or (rem == F(1, 2) and fl % 2 == 1) else 0)
        assert v == want, (a, b, v, want)


def _fold(x, s_hi, s_lo, n):
    """The complex64 fold of binsort.cu: u = x n / (2 pi) as (cell in [0, n), frac in [0, 1))."""
    p = mul(x, s_hi)
    e = fma(x, s_hi, -p)
    corr = fma(x, s_lo, e)
    fl = float(np.floor(p))
    fr = add(sub(p, fl), corr)  # p - fl is exact
    i = int(fl)
    if fr < 0.0:
        fr = add(fr, 1.0)
        i -= 1
    if fr >= 1.0:
        fr = sub(fr, 1.0)
        i += 1
    return i % n, fr


def test_fold_fraction_accuracy():
    """The fold forms x n / (2 pi) in float with an FMA error term and a two-float split of
    n / (2 pi); the fraction it gives is within 1e-7 cells of the exact value for |x| <= 3 pi
    (a plain float product is off by up to 2^-24 |u|, ~6e-5 cells at u ~ 1000)."""
    mpmath = __import__("pytest").importorskip("mpmath")
    mpmath.mp.prec = 120
    rng = random.Random(15)
    for n in (27, 512, 2048, 4096):
        s = mpmath.mpf(n) / (2 * mpmath.pi)
        s_hi = rnd(F(float(s)))  # the host's (float)(double)(n / 2 pi), as make_fold_const forms it
        s_lo = rnd(F(float(s - mpmath.mpf(s_hi))))
        worst = 0.0
        for it in range(400):
            x = rnd(F(rng.uniform(-3, 3) * 3.141592653589793))
            cell, fr = _fold(x, s_hi, s_lo, n)
            assert 0 <= cell < n and 0.0 <= fr < 1.0
            u = mpmath.mpf(x) * s
            u = u - n * mpmath.floor(u / n)  # in [0, n)
            d = abs((cell + mpmath.mpf(fr)) - u)
            d = min(d, n - d)  # u near n folds to near 0
            worst = max(worst, float(d))
        assert worst < 1e-7, (n, worst)
