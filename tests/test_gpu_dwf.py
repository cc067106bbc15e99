"""The double-word float arithmetic of the mixed-precision M2M / L2L shifts
above the leaf level (a value = unevaluated sum of two floats), held to its
error bounds against exact rational arithmetic.

Each input is first rounded to a double-word float (h = fl32(x),
l = fl32(x - h)); the bounds then apply to the operation on the rounded
inputs xr, yr, with u = 2^-24:
  * sum: |got - (xr + yr)| <= 4 u^2 (|xr| + |yr|)  (an absolute bound: there
    is none relative to the result when xr and yr cancel);
  * product: |got - xr yr| <= 4 u^2 |xr yr|;
  * multiply-add x y + x: within the product's bound plus the sum's.
The tests also check that the low word carries information a float cannot:
sums and products whose exact value needs 40-48 bits come back to 2^-46.
"""
import ctypes
from fractions import Fraction

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

U2 = 2.0 ** -48


@pytest.fixture(scope="module")
def lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2305_17867_gb300 import _lib

    return _lib.load()


def run(lib, op, x, y):
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.ascontiguousarray(y, dtype=np.float64)
    out = np.empty_like(x)
    p = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    assert lib.fmm_selftest_dw(op, x.size, p(x), p(y), p(out)) == 0
    return out


def dw_round(x):
    h = x.astype(np.float32)
    lo = (x - h.astype(np.float64)).astype(np.float32)
    return h.astype(np.float64) + lo.astype(np.float64)  # exact: <= 49 bits


def operands(n, seed):
    rng = np.random.default_rng(seed)
    mag = np.exp2(rng.uniform(-30, 30, n))
    x = rng.choice([-1.0, 1.0], n) * mag * rng.uniform(1, 2, n)
    y = rng.choice([-1.0, 1.0], n) * np.exp2(rng.uniform(-30, 30, n)) * rng.uniform(1, 2, n)
    # a quarter of the pairs nearly cancel: y = -x (1 + tiny)
    k = n // 4
    y[:k] = -x[:k] * (1.0 + rng.uniform(-1e-9, 1e-9, k))
    return x, y


@pytest.mark.parametrize("op", [0, 1, 2])
def test_error_bounds_exact(lib, op):
    x, y = operands(4000, 11 + op)
    got = run(lib, op, x, y)
    xr, yr = dw_round(x), dw_round(y)
    worst = 0.0
    for a, b, g in zip(xr, yr, got):
        fa, fb = Fraction(a), Fraction(b)
        if op == 0:
            exact, bound = fa + fb, 4 * U2 * (abs(fa) + abs(fb))
        elif op == 1:
            exact, bound = fa * fb, 4 * U2 * abs(fa * fb)
        else:
            exact = fa * fb + fa
            bound = 4 * U2 * abs(fa * fb) * (1 + 4 * U2) + 4 * U2 * (abs(fa * fb) + abs(fa))
        err = abs(Fraction(g) - exact)
        assert err <= bound, (op, a, b, g, float(err), float(bound))
        if bound:
            worst = max(worst, float(err / bound))
    print(f"op {op}: worst error / bound = {worst:.3f}")


def test_low_word_carries_the_bits_a_float_drops(lib):
    # exact values needing ~40-48 significant bits
    x = np.array([1.0 + 2.0 ** -30, 3.0, 1.0 + 2.0 ** -20, 7.0 / 3.0])
    y = np.array([2.0 ** -40, 2.0 ** -35, 1.0 - 2.0 ** -31, 1.0 / 7.0])
    s = run(lib, 0, x, y)
    pr = run(lib, 1, x, y)
    xr, yr = dw_round(x), dw_round(y)
    for i in range(x.size):
        es = Fraction(xr[i]) + Fraction(yr[i])
        ep = Fraction(xr[i]) * Fraction(yr[i])
        assert abs(Fraction(s[i]) - es) <= abs(es) * 2.0 ** -46
        assert abs(Fraction(pr[i]) - ep) <= abs(ep) * 2.0 ** -46
        # a float result would be off by far more
        assert abs(Fraction(float(np.float32(es))) - es) > abs(es) * 2.0 ** -40 or i == 3


def test_rounding_keeps_48_bits(lib):
    rng = np.random.default_rng(5)
    x = rng.normal(size=10000)
    got = run(lib, 0, x, np.zeros_like(x))  # x + 0: the round trip alone
    rel = np.abs(got - x) / np.abs(x)
    assert rel.max() <= 2.0 ** -47
