"""The packed double-float multiply-add of the staged SpMV rounds like the scalar one.

The staged SpMV accumulates q = K p in double-float (an unevaluated sum hi + lo of two FP32
numbers). Its scalar multiply-add forms p = v*ph, the exact product error pe = fma(v, ph, -p),
TwoSum(hi, p) and the low-word update. The packed form applies the same steps to two accumulators
per instruction with the sm_100-family FP32-pair instructions, which offer add, sub, mul and fma but
no negation, so it forms -p as v*(-ph) and p - bb as -((-p) + bb). Both flips are exact under IEEE
round-to-nearest-even (rounding is symmetric in sign), so every accumulator must come out bit for bit
as in the scalar form. This test emulates both sequences on the host in FP32 (numpy for +, -, *; an
exactly rounded FMA from rational arithmetic) on operands spread over many binades, with
cancellations and zeros, and compares the bits. It checks the algebra the kernel relies on; the GPU
parity tests check the kernel against the oracle.
"""
from fractions import Fraction

import numpy as np

F = np.float32


def _round_f32(x: Fraction) -> np.float32:
    """x rounded to the nearest FP32 value, ties to even (x within the normal FP32 range)."""
    c = F(float(x))                     # float(x) is correctly rounded to FP64; fix a double rounding below
    cands = [c, np.nextafter(c, F(np.inf)), np.nextafter(c, F(-np.inf))]

    def key(v):
        return (abs(Fraction(float(v)) - x), int(np.array(v, dtype=F).view(np.uint32)) & 1)
    return min(cands, key=key)


def fma32(a, b, c) -> np.float32:
    """FP32 fused multiply-add, rounded once (signed zeros as IEEE 754 specifies for RN)."""
    a, b, c = F(a), F(b), F(c)
    exact = Fraction(float(a)) * Fraction(float(b)) + Fraction(float(c))
    if exact == 0:
        prod_neg = np.signbit(a) != np.signbit(b)
        if float(a) * float(b) == 0.0 and float(c) == 0.0 and prod_neg == bool(np.signbit(c)):
            return F(-0.0) if prod_neg else F(0.0)
        return F(0.0)
    return _round_f32(exact)


def scalar_step(hi, lo, v, ph, pl):
    p = F(v * ph)
    pe = fma32(v, ph, -p)
    s = F(hi + p)
    bb = F(s - hi)
    e = F(F(hi - F(s - bb)) + F(p - bb))
    lo = F(lo + F(e + pe))
    return s, fma32(v, pl, lo)


def packed_step(hi, lo, v, ph, pl):
    nph = F(ph * F(-1.0))
    npr = F(v * nph)                    # -p
    pe = fma32(v, ph, npr)
    s = F(hi - npr)
    bb = F(s - hi)
    t2 = F(hi - F(s - bb))
    e = F(t2 - F(npr + bb))
    lo = F(lo + F(e + pe))
    return s, fma32(v, pl, lo)


def _bits(x):
    return int(np.array(x, dtype=F).view(np.uint32))


def _cases(n, seed):
    rng = np.random.default_rng(seed)
    for i in range(n):
        sgn = lambda: F(1.0) if rng.random() < 0.5 else F(-1.0)  # noqa: E731
        hi = F(sgn() * F(2.0) ** int(rng.integers(-12, 12)) * F(rng.uniform(1, 2)))
        lo = F(hi * F(2.0 ** -25) * F(rng.uniform(-1, 1)))
        v = F(sgn() * F(2.0) ** int(rng.integers(-15, 15)) * F(rng.uniform(1, 2)))
        ph = F(sgn() * F(2.0) ** int(rng.integers(-15, 15)) * F(rng.uniform(1, 2)))
        if i % 5 == 0:                  # v*ph close to -hi: cancellation in TwoSum
            ph = F(-hi / v * F(1 + rng.uniform(-1e-6, 1e-6)))
        if i % 17 == 0:
            hi, lo = F(0.0), F(0.0)
        if i % 23 == 0:
            ph = F(0.0) if rng.random() < 0.5 else F(-0.0)
        pl = F(ph * F(2.0 ** -25) * F(rng.uniform(-1, 1)))
        yield hi, lo, v, ph, pl


def test_fma_emulation_is_correctly_rounded():
    # products of two FP32 values are exact in FP64, so fma(a, b, 0) is the product rounded once
    rng = np.random.default_rng(5)
    for _ in range(500):
        a, b = F(rng.standard_normal()), F(rng.standard_normal())
        assert _bits(fma32(a, b, F(0.0))) == _bits(F(a * b))
    # a case where rounding the FP64 sum to FP32 rounds twice: 1 + 2^-24 + 2^-60 must round up
    x = Fraction(1) + Fraction(1, 2 ** 24) + Fraction(1, 2 ** 60)
    assert _round_f32(x) == np.nextafter(F(1.0), F(2.0))
    assert F(float(x)) == F(1.0)        # the naive double rounding gets it wrong


def test_packed_step_equals_scalar_step_bitwise():
    n_diff = 0
    for hi, lo, v, ph, pl in _cases(3000, 11):
        a = scalar_step(hi, lo, v, ph, pl)
        b = packed_step(hi, lo, v, ph, pl)
        n_diff += (_bits(a[0]) != _bits(b[0])) or (_bits(a[1]) != _bits(b[1]))
    assert n_diff == 0


def test_packed_chain_equals_scalar_chain_bitwise():
    """A row's worth of multiply-adds (81 products) accumulated both ways, from the same start."""
    rng = np.random.default_rng(3)
    for _ in range(40):
        vs = [F(x) for x in rng.standard_normal(81)]
        phs = [F(x) for x in rng.standard_normal(81) * 10.0 ** rng.integers(-3, 3)]
        pls = [F(p * F(2.0 ** -25) * F(rng.uniform(-1, 1))) for p in phs]
        h1 = l1 = h2 = l2 = F(0.0)
        for v, ph, pl in zip(vs, phs, pls):
            h1, l1 = scalar_step(h1, l1, v, ph, pl)
            h2, l2 = packed_step(h2, l2, v, ph, pl)
        assert (_bits(h1), _bits(l1)) == (_bits(h2), _bits(l2))


def test_a_wrong_sign_flip_is_detected():
    """The comparison is sensitive: forming p - bb as (-p) + bb (a dropped negation) differs."""
    def wrong(hi, lo, v, ph, pl):
        npr = F(v * F(ph * F(-1.0)))
        pe = fma32(v, ph, npr)
        s = F(hi - npr)
        bb = F(s - hi)
        e = F(F(hi - F(s - bb)) + F(npr + bb))
        lo = F(lo + F(e + pe))
        return s, fma32(v, pl, lo)
    n_diff = sum(_bits(scalar_step(*c)[1]) != _bits(wrong(*c)[1]) for c in _cases(300, 2))
    assert n_diff > 0
