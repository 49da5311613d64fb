"""The identities the kernels' path tracking rests on, checked on CPU.

For one output, the sequential loop of Algorithm 1 (ascending k, strict "<")
walks candidates c_0, c_1, ... from an initial value and records the k of each
strict improvement; P is the last one.  The kernels get the same k in other
ways:
  * lazy recovery (phase 4, phase 1): the first k whose candidate equals the
    final value, when that value is below the initial one;
  * eager per-pair tracking (phase 4 early rounds, batched): a three-input
    min folds the candidates of k-pairs (2p, 2p+1); the pair p of the last
    strict decrease is kept, and inside it the lower k is taken if its
    candidate equals the final value, else the upper one;
  * eager per-chunk tracking (FP32 phase 4 early rounds, batched 64-block
    eager): two k-pairs (four k) are folded per step; the chunk of the last
    strict decrease is kept, and inside it the first k whose candidate
    equals the final value is taken.
FP64 pass 1 tests "x below ru(d)" for a float x and a double d; that equals
"x below d" (a float below d is below the smallest float >= d).  The FP64
path's float bounds bracket every exact sum (lower bounds added rounding down,
upper bounds rounding up), which is what lets it skip or confirm candidates.
"""
import math
import random
import struct

import numpy as np
import pytest


def sequential(init, cands):
    d, last = init, -1
    for k, c in enumerate(cands):
        if c < d:
            d, last = c, k
    return d, last


def lazy(init, cands):
    g = min([init] + list(cands))
    if not g < init:
        return g, -1
    return g, next(k for k, c in enumerate(cands) if c == g)


def eager_pairs(init, cands):
    cs = list(cands) + ([math.inf] if len(cands) % 2 else [])
    acc, kp = init, -1
    for p in range(len(cs) // 2):
        m = min(acc, cs[2 * p], cs[2 * p + 1])
        if m < acc:
            kp = p
        acc = m
    if kp < 0:
        return acc, -1
    return acc, 2 * kp if cs[2 * kp] == acc else 2 * kp + 1


def eager_chunks(init, cands, chunk=4):
    cs = list(cands) + [math.inf] * (-len(cands) % chunk)
    acc, kc = init, -1
    for c in range(len(cs) // chunk):
        m = min([acc] + cs[chunk * c:chunk * c + chunk])
        if m < acc:
            kc = c
        acc = m
    if kc < 0:
        return acc, -1
    return acc, next(chunk * kc + q for q in range(chunk) if cs[chunk * kc + q] == acc)


def _cases(seed, count):
    rng = random.Random(seed)
    for _ in range(count):
        n = rng.randint(0, 40)
        kind = rng.choice(["int", "small", "real"])
        if kind == "int":      # many ties
            cands = [float(rng.randint(0, 6)) for _ in range(n)]
            init = float(rng.randint(0, 8))
        elif kind == "small":  # few distinct values and +inf
            cands = [rng.choice([1.0, 2.0, 3.0, math.inf]) for _ in range(n)]
            init = rng.choice([2.0, 5.0, math.inf])
        else:
            cands = [rng.uniform(0, 10) for _ in range(n)]
            init = rng.choice([rng.uniform(0, 10), math.inf])
        yield init, cands


@pytest.mark.parametrize("seed", range(4))
def test_lazy_and_eager_pairs_give_the_sequential_path_entry(seed):
    for init, cands in _cases(seed, 3000):
        want = sequential(init, cands)
        assert lazy(init, cands) == want, (init, cands)
        assert eager_pairs(init, cands) == want, (init, cands)


def _f32(x):
    return struct.unpack("<f", struct.pack("<f", x))[0]


def _ru32(d):
    """Smallest float >= d (numpy rounding to float32 then one step up if below)."""
    f = np.float32(d)
    if float(f) < d:
        f = np.nextafter(f, np.float32(np.inf))
    return float(f)


def test_float_below_double_equals_float_below_its_upper_float_bound():
    rng = random.Random(5)
    vals = [0.0, -0.0, 1.0, -1.0, 1e-40, 3e38, math.inf, -math.inf]
    for _ in range(20000):
        d = rng.choice([rng.uniform(-1e6, 1e6), rng.uniform(-1, 1) * 1e-30, rng.uniform(0, 100)])
        x = _f32(d + rng.choice([0.0, 1e-9, -1e-9, 1.0, -1.0]) * rng.random())
        vals.append(d)
        assert (x < _ru32(d)) == (x < d), (x, d)
    for d in vals:
        for x in (_f32(d) if math.isfinite(d) else d, 0.0, 1.0, -1.0):
            if math.isnan(x) or math.isnan(d):
                continue
            assert (x < _ru32(d)) == (x < d), (x, d)


@pytest.mark.parametrize("seed", range(4))
def test_eager_chunks_give_the_sequential_path_entry(seed):
    """Four-candidate chunks (two k-pairs) with the last strictly decreasing
    chunk kept: the first k inside it that reaches the final value is the
    sequential loop's last improvement."""
    for init, cands in _cases(100 + seed, 3000):
        assert eager_chunks(init, cands) == sequential(init, cands)


# --------------------------------------------------------------- FP64 interval bounds
def _down32(x):
    """Largest float32 <= x (x a Fraction or +-inf)."""
    from fractions import Fraction
    if x in (math.inf, -math.inf):
        return np.float32(x)
    f = np.float32(float(x))
    if math.isinf(f) and f < 0:  # below every finite float
        return f
    while (math.isinf(f) and f > 0) or (math.isfinite(f) and Fraction(float(f)) > x):
        f = np.nextafter(f, np.float32(-np.inf))
    if math.isinf(f):  # stepped below the most negative float
        return f
    while True:
        g = np.nextafter(f, np.float32(np.inf))
        if math.isinf(g) or Fraction(float(g)) > x:
            return f
        f = g


def _up32(x):
    """Smallest float32 >= x (x a Fraction)."""
    return -_down32(-x)


@pytest.mark.parametrize("seed", range(2))
def test_fp64_interval_sums_bracket_the_exact_sum(seed):
    """Each FP64 value is carried as float bounds [rd(d), ru(d)].  The main
    loop adds lower bounds rounding down, the confirmation adds upper bounds
    rounding up; the exact sum always lies between, so (a) "lower sum >= ru(old)"
    proves no FP64 candidate beats old, and (b) equal bounds prove the sum exact."""
    from fractions import Fraction
    rng = random.Random(seed)
    for _ in range(4000):
        a = rng.choice([rng.uniform(0, 1e3), rng.uniform(0, 1) * 2.0 ** rng.randint(-60, 60),
                        float(rng.randint(1, 1 << 30)), rng.uniform(0, 1e3) + 2.0 ** -40])
        b = rng.choice([rng.uniform(0, 1e3), rng.uniform(0, 1) * 2.0 ** rng.randint(-60, 60),
                        float(rng.randint(1, 1 << 30))])
        A, B = Fraction(a), Fraction(b)
        la, ha, lb, hb = _down32(A), _up32(A), _down32(B), _up32(B)
        lo = _down32(Fraction(float(la)) + Fraction(float(lb)))   # add.rm of the lower bounds
        hi = _up32(Fraction(float(ha)) + Fraction(float(hb)))   # add.rp of the upper bounds
        exact = A + B
        assert Fraction(float(lo)) <= exact <= Fraction(float(hi)), (a, b)
        if lo == hi:
            assert exact == Fraction(float(lo))
        old = rng.choice([a + b, (a + b) * (1 + 1e-12), (a + b) * (1 - 1e-12), rng.uniform(0, 2e3)])
        if float(lo) >= float(_up32(Fraction(old))):
            assert not (a + b < old), (a, b, old)     # the filter never drops an improvement
